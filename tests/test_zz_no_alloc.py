"""mk_run_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (a framework that owns all GPU memory through its own pool, a
process with a fixed memory budget) cannot hand mk_plan a workspace.
mk_run_noalloc runs the same series with its intermediate data in a static
device array; here its output is checked against the plan-based entry points
(mk_plan / mk_set_Gd_window / mk_iterate / mk_fetch_fields) on two calls in a
row, so that the contents the first call leaves in the shared array cannot
leak into the second.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import synthetic as S
from tests.conftest import rel_l2, small_survey
from tests.helpers import desc_for, survey_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2, the per-iteration gate of the parity tests


def _plan_fields(s, R, Gd, td, niter):
    from paper_2106_04649_gb300.api import Plan
    from paper_2106_04649_gb300 import _native as N
    p = Plan([desc_for(s)])
    p.load_R(0, R)
    p.set_Gd_window(0, Gd, td, s.eps)
    e = p.iterate(niter)
    mask = N.MK_F_N | N.MK_F_F1P | N.MK_F_F1M | N.MK_F_F2P | N.MK_F_PMIN
    f = p.fetch_fields(0, mask)
    p.close()
    return f, e


def _padded_R(R):
    import torch
    nw, n, _ = R.shape
    r_pad = (n + 31) // 32 * 32
    Rp = torch.zeros((nw, n, r_pad), dtype=torch.complex64, device="cuda")
    Rp[:, :, :n] = torch.from_numpy(R).cuda()
    return Rp


@pytest.mark.parametrize("niter,with_energy", [(5, True), (5, False), (0, True)])
@pytest.mark.parametrize("case", ["tiny", "small-F3"])
def test_noalloc_matches_plan_two_calls(case, niter, with_energy):
    # niter = 0 leaves the initial fields (no inverse transform, pmin zero);
    # energy = NULL sends the energies to the array's own slot
    import torch
    from paper_2106_04649_gb300 import binding as B
    if case == "tiny":
        s = S.tiny_survey()
    else:
        s = small_survey(n=25, nt=128, nfocal=3, fmax_hz=40.0)
    R, td, Gd = survey_inputs(s)
    ref_f, ref_e = _plan_fields(s, R, Gd, td, niter)

    Rp = _padded_R(R)
    Gdd = torch.from_numpy(Gd).cuda()
    tdd = torch.from_numpy(td).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        fields = torch.full((5, s.nfocal, s.n, s.nt), float("nan"), dtype=torch.float32, device="cuda")
        energy = torch.full((niter, s.nfocal), float("nan"), dtype=torch.float64, device="cuda")
        eptr = energy.data_ptr() if (with_energy and niter > 0) else None
        B.mk_run_noalloc(desc_for(s), Rp.data_ptr(), Gdd.data_ptr(), tdd.data_ptr(), s.eps, niter,
                         fields.data_ptr(), eptr, stream.cuda_stream)
        torch.cuda.synchronize()
        f = fields.cpu().numpy()
        assert np.all(np.isfinite(f)), f"call {call}: non-finite output (a device wait ran out?)"
        for i in range(5):
            if niter == 0 and not np.any(ref_f[i]):
                assert not np.any(f[i]), f"call {call} field {i} should be zero"
                continue
            err = rel_l2(f[i], ref_f[i])
            assert err <= TOL, f"call {call} field {i}: rel L2 {err:.3e}"
        if eptr is not None:
            e = energy.cpu().numpy()
            assert np.allclose(e, ref_e, rtol=TOL, atol=0), f"call {call} energies"


def test_noalloc_rejects_oversize_survey():
    from paper_2106_04649_gb300 import binding as B
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Desc
    import torch
    big = Desc(4001, 4001, 4096, 64, 0.004, 5.0, 60.0)
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")  # never read: the size check comes first
    p = buf.data_ptr()
    with pytest.raises(B.MarchenkoError) as ei:
        B.mk_run_noalloc(big, p, p, p, 0.012, 1, p, None, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == N.MK_ERR_ARG
    assert "MK_NOALLOC_SCRATCH_BYTES" in B.mk_last_error(None)
