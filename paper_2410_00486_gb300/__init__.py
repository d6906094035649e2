"""GB300-native (sm_103a) differentiable 3D Gaussian Splatting mapping iteration of
CaRtGS (arXiv 2410.00486): C-ABI library libcgs (include/cgs.h) plus a thin Python
binding.  Every compute step runs in the library's CUDA kernels; there is no CPU
fallback."""
from . import _native  # noqa: F401
from ._native import Scheduler, CgsError  # noqa: F401


def __getattr__(name):
    if name in ("MappingWindow", "LR_DEFAULT"):
        from . import window
        return getattr(window, name)
    if name in ("RasterizeWindow", "RenderWindow"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
