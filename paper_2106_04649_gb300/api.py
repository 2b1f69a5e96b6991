"""PyTorch-facing wrapper of the C ABI.

PyTorch provides the device workspace (one uint8 tensor from its caching
allocator) and the CUDA stream; every computation runs in libmarchenko.so.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N
from . import binding as B


@dataclass
class Desc:
    """Mirror of the C ``mk_desc`` (one survey)."""

    nsrc: int
    nrec: int
    nt: int
    nfocal: int
    dt: float
    dx: float
    fmax_hz: float = 0.0
    rprec: int = N.MK_R_C64
    flags: int = 0
    row_begin: int = 0   # shot-row sharding: first output position held
    row_count: int = 0   # output positions held (0: all)

    @property
    def nw(self) -> int:
        if not self.fmax_hz > 0:
            return self.nt // 2 + 1
        return min(self.nt // 2, int(np.floor(self.fmax_hz * self.nt * self.dt))) + 1


def _ptr_host(a: np.ndarray, dtype) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


class Plan:
    """A plan over one or more surveys on one CUDA device.

    Inputs may be NumPy arrays (host) or CUDA tensors (device); outputs are
    NumPy arrays unless a CUDA tensor ``out`` is given.
    """

    def __init__(self, descs, device=None, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: libmarchenko has no CPU path")
        self.descs = list(descs)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = B.mk_workspace_size(self.descs)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
            self.handle = B.mk_plan(self.descs, self.stream.cuda_stream, self.workspace.data_ptr(), nbytes)
        self.workspace_bytes = nbytes

    # -- inputs ---------------------------------------------------------------
    def load_R(self, survey: int, Rw, w_begin: int = 0) -> None:
        """Band spectra R[m][k][r] (complex64) for bins w_begin .. w_begin + len - 1."""
        if isinstance(Rw, torch.Tensor):
            assert Rw.is_cuda and Rw.dtype == torch.complex64 and Rw.is_contiguous()
            B.mk_load_R(self.handle, survey, Rw.data_ptr(), w_begin, Rw.shape[0], True)
        else:
            a, p = _ptr_host(Rw, np.complex64)
            B.mk_load_R(self.handle, survey, p, w_begin, a.shape[0], False)

    def load_R_time(self, survey: int, Rt) -> None:
        """R as time traces float32 [nsrc][nrec][nt] (device tensor or host array)."""
        if isinstance(Rt, torch.Tensor) and Rt.is_cuda:
            assert Rt.dtype == torch.float32 and Rt.is_contiguous()
            B.mk_load_R_time(self.handle, survey, Rt.data_ptr(), True)
        elif isinstance(Rt, torch.Tensor):
            assert Rt.dtype == torch.float32 and Rt.is_contiguous()
            B.mk_load_R_time(self.handle, survey, Rt.data_ptr(), False)
        else:
            a, p = _ptr_host(Rt, np.float32)
            B.mk_load_R_time(self.handle, survey, p, False)

    def attach_R_host(self, survey: int, Rpad) -> None:
        """Out-of-core R (MK_FLAG_STREAM_R): a pinned torch CPU tensor, complex64
        [n_w][nsrc][r_pad] (padding zero), kept alive by this plan."""
        assert isinstance(Rpad, torch.Tensor) and Rpad.is_pinned() and Rpad.dtype == torch.complex64
        assert Rpad.is_contiguous()
        self._host_R = getattr(self, "_host_R", {})
        self._host_R[survey] = Rpad
        B.mk_attach_R_host(self.handle, survey, Rpad.data_ptr(), Rpad.numel() * 8)

    def set_Gd_window(self, survey: int, Gd, td, eps: float) -> None:
        """First arrivals G_d [F][n][nt] (float32) and t_d [F][n] (float64, s)."""
        if isinstance(Gd, torch.Tensor):
            assert Gd.is_cuda and isinstance(td, torch.Tensor) and td.is_cuda
            Gd = Gd.contiguous().to(torch.float32)
            td = td.contiguous().to(torch.float64)
            B.mk_set_Gd_window(self.handle, survey, Gd.data_ptr(), td.data_ptr(), float(eps), True)
        else:
            g, gp = _ptr_host(Gd, np.float32)
            t, tp = _ptr_host(td, np.float64)
            B.mk_set_Gd_window(self.handle, survey, gp, tp, float(eps), False)

    # -- iterations -----------------------------------------------------------
    def iterate(self, niter: int, energy: bool = True):
        """Run niter Neumann iterations; returns energies [niter][sum F] or None."""
        if not energy:
            B.mk_iterate(self.handle, niter, None)
            return None
        ftot = sum(d.nfocal for d in self.descs)
        e = np.zeros((niter, ftot), dtype=np.float64)
        B.mk_iterate(self.handle, niter, e.ctypes.data if niter else None)
        return e

    # -- outputs --------------------------------------------------------------
    def image(self, survey: int):
        """Double-focusing image [F] (zero lag of G^- * f1plus)."""
        out = np.zeros(self.descs[survey].nfocal, dtype=np.float64)
        B.mk_image(self.handle, survey, out.ctypes.data, False)
        return out

    def rows(self, survey: int) -> int:
        """Output positions the plan holds for a survey (a shard's rows, else nsrc)."""
        d = self.descs[survey]
        return d.row_count if 0 < d.row_count < d.nsrc else d.nsrc

    def fetch_fields(self, survey: int, mask: int = 0x3F, out=None):
        d = self.descs[survey]
        nf = bin(mask).count("1")
        shape = (nf, d.nfocal, self.rows(survey), d.nt)
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        if isinstance(out, torch.Tensor):
            assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
            B.mk_fetch_fields(self.handle, survey, mask, out.data_ptr(), out.numel() * 4, True)
        else:
            assert out.dtype == np.float32 and out.flags.c_contiguous
            B.mk_fetch_fields(self.handle, survey, mask, out.ctypes.data, out.nbytes, False)
        return out

    def set_fields(self, survey: int, fields, iteration: int, mask: int = 0x1F) -> None:
        """Resume from saved fields [popcount(mask)][F][n][nt] (N, f1plus, f1min, f2p, pmin order)."""
        if isinstance(fields, torch.Tensor):
            assert fields.is_cuda and fields.dtype == torch.float32 and fields.is_contiguous()
            B.mk_set_fields(self.handle, survey, mask, fields.data_ptr(), fields.numel() * 4, iteration, True)
        else:
            a, ptr = _ptr_host(fields, np.float32)
            B.mk_set_fields(self.handle, survey, mask, ptr, a.nbytes, iteration, False)

    # -- shot-row sharding ------------------------------------------------------
    def spectrum_bytes(self, survey: int, rows: int) -> int:
        """Bytes of `rows` packed rows of the survey's field spectrum."""
        d = self.descs[survey]
        parts = 1 if d.rprec in (N.MK_R_C64, N.MK_R_SPLIT_F16) else (3 if d.rprec == N.MK_R_SPLIT3_BF16 else 2)
        return parts * d.nw * d.nfocal * rows * 8

    def export_spectrum(self, survey: int, out: torch.Tensor | None = None) -> torch.Tensor:
        """The plan's own rows of the field spectrum, packed, into a uint8 CUDA tensor."""
        n = self.spectrum_bytes(survey, self.rows(survey))
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, device=self.device)
        assert out.is_cuda and out.is_contiguous() and out.numel() * out.element_size() >= n
        B.mk_export_field_spectrum(self.handle, survey, out.data_ptr(), n, True)
        return out

    def import_spectrum(self, survey: int, buf: torch.Tensor, row_begin: int, row_count: int) -> None:
        """Rows row_begin .. row_begin + row_count - 1 of the field spectrum from a packed CUDA buffer."""
        n = self.spectrum_bytes(survey, row_count)
        assert buf.is_cuda and buf.is_contiguous() and buf.numel() * buf.element_size() >= n
        B.mk_import_field_spectrum(self.handle, survey, buf.data_ptr(), row_begin, row_count, n, True)

    def tuning(self, survey: int) -> dict:
        """Kernel shapes of a survey (timed at its first set_Gd_window with MK_FLAG_AUTOTUNE)."""
        return B.mk_get_tuning(self.handle, survey)

    def stats(self, reset: bool = False) -> dict:
        return B.mk_get_stats(self.handle, reset)

    def close(self) -> None:
        if getattr(self, "handle", 0):
            B.mk_destroy(self.handle)
            self.handle = 0
            self.workspace = None  # return the device memory to torch's allocator

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
