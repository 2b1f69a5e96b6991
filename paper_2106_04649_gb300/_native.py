"""ctypes declarations of the C ABI in include/marchenko.h.

Loading fails loudly when libmarchenko.so has not been built: there is no
fallback implementation of any step.
"""

from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmarchenko.so")

MK_OK, MK_ERR_ARG, MK_ERR_STATE, MK_ERR_OOM, MK_ERR_CUDA, MK_ERR_TIMEOUT, MK_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = ["MK_OK", "MK_ERR_ARG", "MK_ERR_STATE", "MK_ERR_OOM", "MK_ERR_CUDA", "MK_ERR_TIMEOUT",
                "MK_ERR_UNSUPPORTED"]
MK_R_C64, MK_R_CBF16, MK_R_CF16, MK_R_SPLIT_BF16, MK_R_SPLIT3_BF16, MK_R_SPLIT_F16 = range(6)
MK_F_N, MK_F_F1P, MK_F_F1M, MK_F_F2P, MK_F_PMIN, MK_F_G, MK_F_GMINUS, MK_F_GPLUS = (1 << i for i in range(8))
MK_F_ALL = 0xFF
MK_FLAG_TIMING = 1
MK_FLAG_GRAPH = 2
MK_FLAG_STREAM_R = 4
MK_FLAG_AUTOTUNE = 8
MK_SRC_HOST = 0
MK_SRC_DEVICE = 1
MK_SRC_HOST_ASYNC = 2


class MkDesc(ctypes.Structure):
    _fields_ = [
        ("nsrc", ctypes.c_int32),
        ("nrec", ctypes.c_int32),
        ("nt", ctypes.c_int32),
        ("nfocal", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("fmax_hz", ctypes.c_double),
        ("rprec", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("row_begin", ctypes.c_int32),
        ("row_count", ctypes.c_int32),
    ]


class MkStats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_uint64),
        ("contract_launches", ctypes.c_uint64),
        ("epilogue_launches", ctypes.c_uint64),
        ("other_launches", ctypes.c_uint64),
        ("contract_ms", ctypes.c_double),
        ("epilogue_ms", ctypes.c_double),
        ("contract_timed", ctypes.c_uint64),
        ("epilogue_timed", ctypes.c_uint64),
    ]


class MkTuning(ctypes.Structure):
    _fields_ = [
        ("tuned", ctypes.c_int32),
        ("umma_bn", ctypes.c_int32),
        ("epi_pairs", ctypes.c_int32),
        ("candidates", ctypes.c_int32),
        ("contract_ms", ctypes.c_float),
        ("epilogue_ms", ctypes.c_float),
    ]


_P = ctypes.c_void_p
_SIGS = {
    "mk_workspace_size": (ctypes.c_int, [ctypes.POINTER(MkDesc), ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "mk_plan": (ctypes.c_int, [ctypes.POINTER(MkDesc), ctypes.c_int32, _P, _P, ctypes.c_size_t,
                               ctypes.POINTER(_P)]),
    "mk_load_R": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "mk_set_Gd_window": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_double, ctypes.c_int32]),
    "mk_iterate": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "mk_fetch_fields": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, _P, ctypes.c_size_t, ctypes.c_int32]),
    "mk_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(MkStats), ctypes.c_int32]),
    "mk_set_fields": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint32, _P, ctypes.c_size_t, ctypes.c_int32,
                                     ctypes.c_int32]),
    "mk_destroy": (ctypes.c_int, [_P]),
    "mk_last_error": (ctypes.c_char_p, [_P]),
    "mk_image": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "mk_attach_R_host": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    "mk_load_R_time": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "mk_get_tuning": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(MkTuning)]),
    "mk_set_timing": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "mk_export_field_spectrum": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t, ctypes.c_int32]),
    "mk_import_field_spectrum": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_size_t, ctypes.c_int32]),
    "mk_run_noalloc": (ctypes.c_int, [ctypes.POINTER(MkDesc), _P, _P, _P, ctypes.c_double, ctypes.c_int32, _P, _P,
                                      _P]),
}
MK_NOALLOC_SCRATCH_BYTES = 64 << 20

_lib = None


def load() -> ctypes.CDLL:
    """Load libmarchenko.so (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                          f"g.build()\"` (needs nvcc); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
