"""GB300-native iterative Marchenko synthesis.

The hot loop (contraction of Eq. (1) per frequency, inverse transform, time
reversal, theta mute, Neumann accumulation of Algorithm 1, forward transform)
runs in hand-written sm_103a CUDA kernels behind the C ABI of
include/marchenko.h.  ``binding`` mirrors that ABI name for name; ``api.Plan``
wraps it with PyTorch-allocated workspace and streams.
"""

from ._native import (  # noqa: F401
    MK_F_ALL,
    MK_F_F1M,
    MK_F_F1P,
    MK_F_F2P,
    MK_F_G,
    MK_F_GMINUS,
    MK_F_GPLUS,
    MK_F_N,
    MK_F_PMIN,
    MK_FLAG_TIMING,
    MK_R_C64,
    MK_R_CBF16,
    MK_R_CF16,
    MK_R_SPLIT_BF16,
    MK_R_SPLIT3_BF16,
    MK_R_SPLIT_F16,
)


def __getattr__(name):
    # torch is imported lazily so that the ABI declarations load without it
    if name in ("Plan", "Desc"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
