"""Out-of-core R: frequency chunks streamed from pinned host memory.

A survey planned with MK_FLAG_STREAM_R keeps only two chunk buffers of R on
the device and copies the band from page-locked host memory during every
contraction (the paper's answer to R larger than device memory, Algorithm 2).
Each frequency is contracted by the same kernel on the same data as in the
resident plan, so every field is bit-identical to the resident run.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2, small_survey
from tests.helpers import FIELD_NAMES, desc_for, survey_inputs

pytestmark = pytest.mark.gpu

MK_FLAG_STREAM_R = 4


def _padded_host(R):
    import torch
    nw, ns, nr = R.shape
    r_pad = (nr + 31) // 32 * 32
    H = torch.zeros((nw, ns, r_pad), dtype=torch.complex64).pin_memory()
    H[:, :, :nr] = torch.from_numpy(np.ascontiguousarray(R, dtype=np.complex64))
    return H


def _run(survey, R, Gd, td, niter, stream):
    from paper_2106_04649_gb300.api import Plan
    plan = Plan([desc_for(survey, flags=MK_FLAG_STREAM_R if stream else 0)])
    if stream:
        plan.attach_R_host(0, _padded_host(R))
    else:
        plan.load_R(0, R)
    plan.set_Gd_window(0, Gd, td, survey.eps)
    e = plan.iterate(niter)
    f = plan.fetch_fields(0)
    plan.close()
    return e, f


@pytest.mark.parametrize("n,nt,nfocal", [(101, 512, 1), (257, 1024, 3), (333, 512, 1)])
def test_streamed_equals_resident(n, nt, nfocal):
    s = small_survey(n=n, dx=10.0, nt=nt, dt=0.004, nfocal=nfocal, calibrate=0.9, fmax_hz=60.0, seed=7)
    R, td, Gd = survey_inputs(s)
    e0, f0 = _run(s, R, Gd, td, 6, False)
    e1, f1 = _run(s, R, Gd, td, 6, True)
    assert np.array_equal(e0, e1)
    for j, name in enumerate(FIELD_NAMES):
        assert np.array_equal(f0[j], f1[j]), name
    # and against the oracle
    st = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 6)
    assert rel_l2(f1[1], st.f1plus) <= 1e-5
    assert rel_l2(f1[5], M.total_green(st.f2p, st.pmin)) <= 1e-5


def test_stream_call_order_and_arguments():
    import torch
    from paper_2106_04649_gb300 import binding as B
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Plan
    s = small_survey(n=101, dx=10.0, nt=512, dt=0.004, nfocal=1, calibrate=0.9, fmax_hz=60.0, seed=3)
    R, td, Gd = survey_inputs(s)
    plan = Plan([desc_for(s, flags=MK_FLAG_STREAM_R), desc_for(s)])
    # resident upload refused on a streamed survey, attach refused on a resident one
    with pytest.raises(B.MarchenkoError) as ei:
        plan.load_R(0, R)
    assert ei.value.status == N.MK_ERR_STATE
    H = _padded_host(R)
    with pytest.raises(B.MarchenkoError) as ei:
        plan.attach_R_host(1, H)
    assert ei.value.status == N.MK_ERR_STATE
    # pageable memory and a wrong size are rejected
    pageable = torch.zeros_like(H, device="cpu")
    with pytest.raises(B.MarchenkoError) as ei:
        B.mk_attach_R_host(plan.handle, 0, pageable.data_ptr(), pageable.numel() * 8)
    assert ei.value.status == N.MK_ERR_ARG
    with pytest.raises(B.MarchenkoError) as ei:
        B.mk_attach_R_host(plan.handle, 0, H.data_ptr(), H.numel() * 8 - 8)
    assert ei.value.status == N.MK_ERR_ARG
    plan.attach_R_host(0, H)
    plan.load_R(1, R)
    for i in range(2):
        plan.set_Gd_window(i, Gd, td, s.eps)
    e = plan.iterate(4)
    f0 = plan.fetch_fields(0)
    f1 = plan.fetch_fields(1)
    for j in range(6):
        assert np.array_equal(f0[j], f1[j])
    assert np.array_equal(e[:, 0], e[:, 1])
    plan.close()
