"""GB300-native event-camera renderer: Monte Carlo path tracing with
per-pixel log-luminance statistics and Student t-test early stopping
(arXiv 2408.07996).

The compute path is the CUDA library `_build/libmcev.so` (C ABI in
include/mcev.h); this package is its argument-marshalling layer.
"""
from ._lib import (  # noqa: F401
    MEAN_ONLY,
    ONE_TAILED,
    SE_PAPER,
    SE_WELCH,
    TWO_TAILED,
    UNIFORM,
    McevError,
    library_path,
    load,
)


def Renderer(*args, **kwargs):  # noqa: N802 - factory keeps torch import lazy
    from .api import Renderer as _R
    return _R(*args, **kwargs)
