"""Device-side assembly of the synthetic reflection response (input generation).

``reflection_band`` builds R on the host: R_m(k, r) = T_m(|k - r|) * scale(k, r)
with the offset spectra T (FP64, ``_offset_spectra``) and the reciprocal
jitter scale (1 + 0.01 u(k, r)) * kappa / dt.  For the large workloads the
host gather is slow, so this module does the same gather and product in FP64
on a torch device, chunk by chunk over frequencies, and hands each chunk to a
callback (typically the library's R load).  The arithmetic is the same FP64
product as on the host, element for element.
"""

from __future__ import annotations

import numpy as np

from .layered import Survey, _offset_spectra, amplitude_scale, jitter_matrix


def reflection_band_chunks(s: Survey, device, chunk: int = 8, dtype=None, w_begin: int = 0, w_count=None):
    """Yield (w0, R_chunk) with R_chunk a [c][n][n] tensor on ``device``
    (complex64 by default) covering bins w0 .. w0 + c - 1."""
    import torch
    dtype = torch.complex64 if dtype is None else dtype
    if w_count is None:
        w_count = s.nw - w_begin
    T = torch.from_numpy(_offset_spectra(s, w_begin, w_count)).to(device)                  # [w][n] complex128
    scale = (1.0 + 0.01 * jitter_matrix(s.seed, s.n)) * (amplitude_scale(s) / s.dt)      # [n][n] float64
    scale = torch.from_numpy(scale).to(device)
    idx = torch.arange(s.n, device=device)
    off = (idx[:, None] - idx[None, :]).abs()                                            # [n][n]
    for c in range(0, w_count, chunk):
        e = min(w_count, c + chunk)
        block = T[c:e][:, off] * scale[None]                                             # complex128
        yield w_begin + c, block.to(dtype)


def reflection_band_torch(s: Survey, device, dtype=None, chunk: int = 8):
    """The whole band [nw][n][n] on ``device`` (see ``reflection_band``)."""
    import torch
    dtype = torch.complex64 if dtype is None else dtype
    out = torch.empty((s.nw, s.n, s.n), dtype=dtype, device=device)
    for w0, blk in reflection_band_chunks(s, device, chunk, dtype):
        out[w0:w0 + blk.shape[0]] = blk
    return out
