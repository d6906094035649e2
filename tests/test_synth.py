"""The seeded workload generator: shapes and the properties the workloads are meant to
have (CPU; visibility from the oracle's projection)."""
import numpy as np

from oracle import oracle as O
from synth import make_scene


def test_window8_visible_counts_are_uneven_20k_to_150k():
    sc = make_scene(4)
    assert (sc.views, sc.n, sc.width, sc.height) == (8, 200_000, 640, 480)
    pre = O.preprocess(sc.params, sc.n, 3, sc.cams, sc.width, sc.height, 16)
    vis = (pre["radius"].reshape(sc.views, -1) > 0).sum(1)
    assert vis.min() < 25_000 and vis.max() > 145_000
    assert np.all(np.diff(vis) < 0)          # one view after another sees less of the room


def test_workload_shapes():
    for cfg, shape in {1: (1, 2000, 160, 120, 0), 2: (1, 100_000, 1200, 680, 3), 3: (1, 5000, 320, 240, 1),
                       5: (16, 300_000, 1200, 680, 3)}.items():
        sc = make_scene(cfg)
        assert (sc.views, sc.n, sc.width, sc.height, sc.sh_degree) == shape
        assert sc.params.dtype == np.float32 and sc.params.size == O.lr_per_element(sc.n, sc.sh_degree, [1] * 6).size
