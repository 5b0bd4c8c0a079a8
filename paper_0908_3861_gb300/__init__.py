"""GB300-native adaptive elliptical filtering with box splines.

The filter of Chaudhury, Munoz-Barrutia and Unser (four-direction box splines,
Sec. 4-7): a global pre-integration by running sums and a per-pixel affine
finite-difference mesh, as hand-written CUDA kernels for sm_103a behind the C
ABI of include/abf.h (libabf.so).  ``_abf`` binds that ABI one to one;
``AdaptiveFilter`` adds buffer allocation with PyTorch; ``AdaptiveFilter1D``
does the same for the 1-D scale-adaptive B-spline filter of Sec. 3.
"""
from . import _abf
from ._abf import AbfError

__all__ = ["_abf", "AbfError", "AdaptiveFilter", "AdaptiveFilter1D", "Batch", "Server", "make_desc",
           "estimate_ellipses", "ellipse_product_bound"]


def __getattr__(name):
    if name in ("AdaptiveFilter", "AdaptiveFilter1D", "Batch", "Server", "make_desc", "estimate_ellipses",
                "ellipse_product_bound"):
        from . import filter as _f
        return getattr(_f, name)
    raise AttributeError(name)
