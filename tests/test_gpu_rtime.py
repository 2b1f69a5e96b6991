"""R loaded from its time traces (mk_load_R_time) against the FP64 oracle.

The time traces are a synthetic real R(k, r, t) (the inverse transform of the
generator's band spectra, so the same reflection response as the spectral
tests).  The oracle takes the FP64 forward transform of the same traces as
its R_m, so the comparison covers the on-device transform, the layout
transposition (trace (k, r) to row k, column r of R_m) and the storage
conversion.
"""

import numpy as np
import pytest

from oracle import marchenko as M
from tests.conftest import rel_l2, small_survey
from tests.helpers import FIELD_NAMES, desc_for, survey_inputs

pytestmark = pytest.mark.gpu

C64, SPLIT3 = 0, 4


def _time_traces(R, nt):
    """float32 [k][r][t] whose band spectra are R [m][k][r] (bins above the band zero)."""
    nw = R.shape[0]
    full = np.zeros((R.shape[1], R.shape[2], nt // 2 + 1), dtype=np.complex128)
    full[:, :, :nw] = np.transpose(R, (1, 2, 0))
    return np.ascontiguousarray(np.fft.irfft(full, n=nt, axis=-1), dtype=np.float32)


def _fields(s, rprec, load, Gd, td, niter):
    from paper_2106_04649_gb300.api import Plan
    plan = Plan([desc_for(s, rprec=rprec)])
    load(plan)
    plan.set_Gd_window(0, Gd, td, s.eps)
    e = plan.iterate(niter)
    f = plan.fetch_fields(0)
    plan.close()
    return e, f


@pytest.mark.parametrize("rprec,tol", [(C64, 1e-5), (SPLIT3, 1e-5)])
def test_time_traces_match_oracle(rprec, tol):
    s = small_survey(n=257, dx=10.0, nt=1024, dt=0.004, nfocal=3, calibrate=0.9, fmax_hz=60.0, seed=11)
    R, td, Gd = survey_inputs(s)
    Rt = _time_traces(R, s.nt)
    Rw = np.ascontiguousarray(np.transpose(M.forward_band(Rt, s.nw), (2, 0, 1)))
    st = M.run(Rw, Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 6)
    ref = [st.N, st.f1plus, st.f1min, st.f2p, st.pmin, M.total_green(st.f2p, st.pmin)]
    e, f = _fields(s, rprec, lambda p: p.load_R_time(0, Rt), Gd, td, 6)
    for j, name in enumerate(FIELD_NAMES):
        err = rel_l2(f[j], ref[j])
        assert err <= tol, f"{name}: {err:.3e}"
    assert np.max(np.abs(e - np.array(st.energy)) / np.array(st.energy)) <= 2 * tol


def test_time_trace_sources_agree():
    """Device tensor, pinned host and pageable host (staged F rows at a time) give identical fields."""
    import torch
    s = small_survey(n=101, dx=10.0, nt=512, dt=0.004, nfocal=2, calibrate=0.9, fmax_hz=60.0, seed=5)
    R, td, Gd = survey_inputs(s)
    Rt = _time_traces(R, s.nt)
    dev = torch.from_numpy(Rt).cuda()
    pinned = torch.from_numpy(Rt).pin_memory()
    runs = [_fields(s, C64, lambda p, x=x: p.load_R_time(0, x), Gd, td, 4) for x in (dev, pinned, Rt)]
    for e, f in runs[1:]:
        assert np.array_equal(e, runs[0][0])
        for j in range(6):
            assert np.array_equal(f[j], runs[0][1][j])
    # and close to a load of the same spectra computed on the host
    Rw = np.transpose(np.fft.rfft(Rt.astype(np.float64), axis=-1)[..., :s.nw], (2, 0, 1)).astype(np.complex64)
    e1, f1 = _fields(s, C64, lambda p: p.load_R(0, Rw), Gd, td, 4)
    for j in range(6):
        assert rel_l2(runs[0][1][j], f1[j]) <= 2e-6
