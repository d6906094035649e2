"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This package draws random numbers and lays them out; it holds none of the
method's arithmetic (no projection, blending, loss or gradient).
"""
from .scenes import (  # noqa: F401
    Scene, make_scene, make_tiny_scene, make_records, make_conics, make_point_cloud, param_layout, CONFIG_NAMES,
)
