"""Tensor-core contraction (tcgen05) with 16-bit R storage vs the FP64 oracle.

The oracle runs on the dequantised R (the exact values the GPU stores, from a
round-to-nearest-even emulation written here), so the gate measures the
kernel, not the storage format; split BF16 is also compared with the exact R.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2, small_survey
from tests.helpers import FIELD_NAMES, desc_for, survey_inputs

pytestmark = pytest.mark.gpu

C64, CBF16, CF16, SPLIT, SPLIT3, SPLITF16 = 0, 1, 2, 3, 4, 5


def bf16_rne(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32 (finite inputs)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def dequantised(R, rprec):
    """The complex values the library stores for complex64 R in precision rprec."""
    re = np.ascontiguousarray(R.real, dtype=np.float32)
    im = np.ascontiguousarray(R.imag, dtype=np.float32)
    if rprec == CBF16:
        q = [bf16_rne(re), bf16_rne(im)]
    elif rprec == CF16:
        q = [re.astype(np.float16).astype(np.float32), im.astype(np.float16).astype(np.float32)]
    elif rprec == SPLIT:
        hr, hi = bf16_rne(re), bf16_rne(im)
        lr, li = bf16_rne(re - hr), bf16_rne(im - hi)
        q = [hr.astype(np.float64) + lr, hi.astype(np.float64) + li]
    else:
        hr, hi = bf16_rne(re), bf16_rne(im)
        mr, mi = bf16_rne(re - hr), bf16_rne(im - hi)
        lr, li = bf16_rne(re - hr - mr), bf16_rne(im - hi - mi)
        q = [hr.astype(np.float64) + mr + lr, hi.astype(np.float64) + mi + li]
    return q[0].astype(np.float64) + 1j * q[1].astype(np.float64)


def _run(s, R, Gd, td, rprec, niter, per_iter=False):
    from paper_2106_04649_gb300.api import Plan
    p = Plan([desc_for(s, rprec=rprec)])
    p.load_R(0, R)
    p.set_Gd_window(0, Gd, td, s.eps)
    out = []
    if per_iter:
        for _ in range(niter):
            e = p.iterate(1)
            out.append((e, p.fetch_fields(0)))
    else:
        e = p.iterate(niter)
        out.append((e, p.fetch_fields(0)))
    p.close()
    return out


def _ref(st):
    return [st.N, st.f1plus, st.f1min, st.f2p, st.pmin, M.total_green(st.f2p, st.pmin)]


@pytest.mark.parametrize("rprec", [CBF16, SPLIT, SPLIT3])
@pytest.mark.parametrize("n,nt,nfocal,fmax", [(25, 128, 3, None), (40, 128, 8, 40.0), (7, 64, 1, None)])
def test_bf16_forms_per_iteration(rprec, n, nt, nfocal, fmax):
    s = small_survey(n=n, nt=nt, nfocal=min(nfocal, 3), fmax_hz=fmax)
    if nfocal > 3:
        xs = np.linspace(0.2, 0.8, nfocal) * (n - 1) * s.dx
        s.focal = np.stack([xs, np.full(nfocal, 650.0)], axis=1)
    R, td, Gd = survey_inputs(s)
    Rq = dequantised(R, rprec)
    _, hist = M.run(Rq, Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 6, history=True)
    got = _run(s, R, Gd, td, rprec, 6, per_iter=True)
    for i, (e, f) in enumerate(got):
        ref = _ref(hist[i])
        for j, name in enumerate(FIELD_NAMES):
            err = rel_l2(f[j], ref[j])
            tol = 1e-4 if name == "N" else 1e-5
            assert err <= tol, f"rprec {rprec} n={n} F={nfocal} iter {i} {name}: {err:.3e}"


def test_split_bf16_vs_exact_oracle_tiny(tiny_inputs):
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    st = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 16)
    (e, f), = _run(s, R, Gd, td, SPLIT, 16)
    ref = _ref(st)
    for j, name in enumerate(FIELD_NAMES):
        assert rel_l2(f[j], ref[j]) <= 1e-4, name
    for j in (1, 2, 3, 4, 5):
        assert rel_l2(f[j], ref[j]) <= 1e-5, FIELD_NAMES[j]


def test_fp16_form_accumulated_fields(tiny_inputs):
    # FP16 keeps 11 significant bits but little range: the shrinking late N_i
    # lose relative precision, the accumulated fields stay within 1e-5
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    Rq = dequantised(R, CF16)
    st = M.run(Rq, Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 8)
    (e, f), = _run(s, R, Gd, td, CF16, 8)
    ref = _ref(st)
    for j in (1, 2, 3, 4, 5):
        assert rel_l2(f[j], ref[j]) <= 1e-5, FIELD_NAMES[j]


def test_paper_small_F64_split_bf16_sampled():
    # split BF16 keeps ~16 significant bits per operand: on this survey the
    # first synthesis already carries 1.5e-5 relative error vs the exact R
    # (cancellation in the contraction), so its gate here is 3e-5 / 1e-4
    s = S.paper_small_survey(64)
    R, td, Gd = survey_inputs(s)
    (e, f), = _run(s, R, Gd, td, SPLIT, 16)
    sel = [0, 31, 63]
    st = M.run(R.astype(np.complex128), Gd[sel].astype(np.float64), td[sel], s.eps, s.dt, s.dx, 16)
    ref = _ref(st)
    for j, name in enumerate(FIELD_NAMES):
        err = rel_l2(f[j][sel], ref[j])
        assert err <= (1e-4 if name == "N" else 3e-5), f"{name}: {err:.3e}"


@pytest.mark.parametrize("rprec,exact", [(CBF16, False), (SPLIT, False), (SPLIT3, False), (SPLIT3, True),
                                         (SPLITF16, True)])
def test_paper_small_per_iteration_identical_inputs(rprec, exact):
    # one tensor-core synthesis + epilogue from the oracle's state, vs the oracle on
    # the dequantised R (exact=False) or on the exact complex64 R (split form, exact=True)
    from paper_2106_04649_gb300.api import Plan
    s = S.paper_small_survey(64)
    sel = [0, 21, 42, 63]
    s.focal = s.focal[sel]
    R, td, Gd = survey_inputs(s)
    Rref = R.astype(np.complex128) if exact else dequantised(R, rprec)
    _, hist = M.run(Rref, Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 4, history=True)
    p = Plan([desc_for(s, rprec=rprec)])
    p.load_R(0, R)
    p.set_Gd_window(0, Gd, td, s.eps)
    prev = M.initialise(Gd.astype(np.float64))
    for i in range(4):
        p.set_fields(0, np.stack([prev.N, prev.f1plus, prev.f1min, prev.f2p, prev.pmin]).astype(np.float32), i)
        p.iterate(1)
        f = p.fetch_fields(0)
        ref = _ref(hist[i])
        e = [rel_l2(f[j], ref[j]) for j in range(6)]
        # the 3-product split keeps ~16 significant bits of each operand: ~1.4e-5 here
        tol = 2e-5 if rprec == SPLIT else 1e-5
        assert max(e) <= tol, f"rprec {rprec} exact={exact} iter {i}: {e}"
        prev = hist[i]
    p.close()


def test_paper_small_F64_split3_bf16_vs_exact():
    # the 6-product 3-way split: <= 1e-5 relative L2 against the exact FP64 oracle after 16 iterations
    s = S.paper_small_survey(64)
    R, td, Gd = survey_inputs(s)
    (e, f), = _run(s, R, Gd, td, SPLIT3, 16)
    sel = [0, 31, 63]
    st = M.run(R.astype(np.complex128), Gd[sel].astype(np.float64), td[sel], s.eps, s.dt, s.dx, 16)
    ref = _ref(st)
    for j, name in enumerate(FIELD_NAMES):
        err = rel_l2(f[j][sel], ref[j])
        assert err <= (1e-4 if name == "N" else 1e-5), f"{name}: {err:.3e}"


@pytest.mark.parametrize("n,nt,nfocal,fmax", [(25, 128, 3, None), (40, 128, 8, 40.0), (7, 64, 1, None),
                                              (75, 256, 5, 60.0)])
def test_scaled_fp16_split_vs_exact_oracle_per_iteration(n, nt, nfocal, fmax):
    # the 3-product form with both operands split into FP16 hi + lo and scaled by
    # powers of two (R per frequency, the field per frequency and focal point):
    # <= 1e-5 against the exact FP64 oracle at every iteration, like the 6-product form
    s = small_survey(n=n, nt=nt, nfocal=min(nfocal, 3), fmax_hz=fmax)
    if nfocal > 3:
        xs = np.linspace(0.2, 0.8, nfocal) * (n - 1) * s.dx
        s.focal = np.stack([xs, np.full(nfocal, 650.0)], axis=1)
    R, td, Gd = survey_inputs(s)
    _, hist = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 6, history=True)
    got = _run(s, R, Gd, td, SPLITF16, 6, per_iter=True)
    for i, (e, f) in enumerate(got):
        ref = _ref(hist[i])
        for j, name in enumerate(FIELD_NAMES):
            err = rel_l2(f[j], ref[j])
            assert err <= (1e-4 if name == "N" else 1e-5), f"n={n} F={nfocal} iter {i} {name}: {err:.3e}"


def test_paper_small_F64_scaled_fp16_split_vs_exact():
    # the 3-product scaled FP16 split on the paper-small survey: <= 1e-5 relative L2
    # against the exact FP64 oracle after 16 iterations (sampled focal points)
    s = S.paper_small_survey(64)
    R, td, Gd = survey_inputs(s)
    (e, f), = _run(s, R, Gd, td, SPLITF16, 16)
    sel = [0, 31, 63]
    st = M.run(R.astype(np.complex128), Gd[sel].astype(np.float64), td[sel], s.eps, s.dt, s.dx, 16)
    ref = _ref(st)
    for j, name in enumerate(FIELD_NAMES):
        err = rel_l2(f[j][sel], ref[j])
        assert err <= (1e-4 if name == "N" else 1e-5), f"{name}: {err:.3e}"
    eref = np.array(st.energy)
    assert np.max(np.abs(e[:, sel] - eref) / eref) <= 1e-4


def test_scaled_fp16_split_load_paths_agree():
    # host (pageable, staged), pinned and device sources give the same scales and parts
    import torch
    from paper_2106_04649_gb300.api import Plan
    s = small_survey(n=40, nt=128, nfocal=3, fmax_hz=40.0)
    R, td, Gd = survey_inputs(s)
    outs = []
    for mode in ("pageable", "pinned", "device"):
        p = Plan([desc_for(s, rprec=SPLITF16)])
        if mode == "pageable":
            p.load_R(0, R[:10])
            p.load_R(0, R[10:], w_begin=10)
        elif mode == "pinned":
            Rp = torch.from_numpy(R).pin_memory()
            from paper_2106_04649_gb300 import binding as B
            B.mk_load_R(p.handle, 0, Rp.data_ptr(), 0, R.shape[0], 0)
        else:
            p.load_R(0, torch.from_numpy(R).cuda())
        p.set_Gd_window(0, Gd, td, s.eps)
        e = p.iterate(3)
        outs.append((e, p.fetch_fields(0)))
        p.close()
    for e, f in outs[1:]:
        assert np.array_equal(e, outs[0][0]) and np.array_equal(f, outs[0][1])
