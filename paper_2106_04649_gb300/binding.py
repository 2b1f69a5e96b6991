"""Thin Python binding of the C ABI: same names, argument marshalling only.

Every function takes plain integers for pointers (``tensor.data_ptr()``,
``array.ctypes.data``) and raises ``MarchenkoError`` on a non-zero status.
"""

from __future__ import annotations

import ctypes

from . import _native as N


class MarchenkoError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = N.STATUS_NAMES[status] if 0 <= status < len(N.STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


def _check(st: int, plan) -> None:
    if st != N.MK_OK:
        msg = N.load().mk_last_error(plan)
        raise MarchenkoError(st, msg.decode() if msg else "")


def _descs(descs) -> tuple:
    arr = (N.MkDesc * len(descs))()
    for i, d in enumerate(descs):
        for name, _ in N.MkDesc._fields_:
            setattr(arr[i], name, getattr(d, name))
    return arr, len(descs)


def mk_workspace_size(descs) -> int:
    arr, n = _descs(descs)
    out = ctypes.c_size_t(0)
    _check(N.load().mk_workspace_size(arr, n, ctypes.byref(out)), None)
    return int(out.value)


def mk_plan(descs, cuda_stream: int, workspace: int, workspace_bytes: int) -> int:
    arr, n = _descs(descs)
    out = ctypes.c_void_p(0)
    _check(N.load().mk_plan(arr, n, ctypes.c_void_p(cuda_stream), ctypes.c_void_p(workspace),
                            workspace_bytes, ctypes.byref(out)), None)
    return int(out.value)


def mk_load_R(plan: int, survey: int, Rw: int, w_begin: int, w_count: int, src_on_device: int) -> None:
    """src_on_device: MK_SRC_HOST (0), MK_SRC_DEVICE (1) or MK_SRC_HOST_ASYNC (2)."""
    _check(N.load().mk_load_R(plan, survey, Rw, w_begin, w_count, int(src_on_device)), plan)


def mk_set_timing(plan: int, stride: int, reserve_pairs: int) -> None:
    _check(N.load().mk_set_timing(plan, stride, reserve_pairs), plan)


def mk_get_tuning(plan: int, survey: int) -> dict:
    t = N.MkTuning()
    _check(N.load().mk_get_tuning(plan, survey, ctypes.byref(t)), plan)
    return {name: getattr(t, name) for name, _ in N.MkTuning._fields_}


def mk_load_R_time(plan: int, survey: int, Rt: int, src_on_device: bool) -> None:
    _check(N.load().mk_load_R_time(plan, survey, Rt, 1 if src_on_device else 0), plan)


def mk_attach_R_host(plan: int, survey: int, Rpad: int, nbytes: int) -> None:
    _check(N.load().mk_attach_R_host(plan, survey, Rpad, nbytes), plan)


def mk_set_Gd_window(plan: int, survey: int, Gd: int, td: int, eps_s: float, src_on_device: bool) -> None:
    _check(N.load().mk_set_Gd_window(plan, survey, Gd, td, eps_s, int(src_on_device)), plan)


def mk_iterate(plan: int, niter: int, energy: int | None) -> None:
    _check(N.load().mk_iterate(plan, niter, energy), plan)


def mk_fetch_fields(plan: int, survey: int, mask: int, out: int, out_bytes: int, dst_on_device: bool) -> None:
    _check(N.load().mk_fetch_fields(plan, survey, mask, out, out_bytes, int(dst_on_device)), plan)


def mk_set_fields(plan: int, survey: int, mask: int, data: int, nbytes: int, iteration: int,
                  src_on_device: bool) -> None:
    _check(N.load().mk_set_fields(plan, survey, mask, data, nbytes, iteration, int(src_on_device)), plan)


def mk_image(plan: int, survey: int, image: int, dst_on_device: bool) -> None:
    _check(N.load().mk_image(plan, survey, image, int(dst_on_device)), plan)


def mk_export_field_spectrum(plan: int, survey: int, dst: int, nbytes: int, dst_on_device: bool) -> None:
    _check(N.load().mk_export_field_spectrum(plan, survey, dst, nbytes, int(dst_on_device)), plan)


def mk_import_field_spectrum(plan: int, survey: int, src: int, row_begin: int, row_count: int, nbytes: int,
                             src_on_device: bool) -> None:
    _check(N.load().mk_import_field_spectrum(plan, survey, src, row_begin, row_count, nbytes, int(src_on_device)),
           plan)


def mk_get_stats(plan: int, reset: bool = False) -> dict:
    st = N.MkStats()
    _check(N.load().mk_get_stats(plan, ctypes.byref(st), int(reset)), plan)
    return {name: getattr(st, name) for name, _ in N.MkStats._fields_}


def mk_destroy(plan: int) -> None:
    _check(N.load().mk_destroy(plan), None)


def mk_last_error(plan: int | None) -> str:
    msg = N.load().mk_last_error(plan)
    return msg.decode() if msg else ""


def mk_run_noalloc(desc, R: int, Gd: int, td: int, eps_s: float, niter: int, fields: int, energy: int | None,
                   cuda_stream: int) -> None:
    """No-allocation run (device pointers only); errors via mk_last_error(None)."""
    arr, _ = _descs([desc])
    _check(N.load().mk_run_noalloc(arr, R, Gd, td, eps_s, niter, fields, energy, ctypes.c_void_p(cuda_stream)),
           None)
