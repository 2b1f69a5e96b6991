"""Large survey: 4001 x 4001 positions, nt = 4096, 984 kept bins, one focal
batch of 32 points of the 4001-point line, R held as 3-way split BF16
(3 x 63 GB) or as the scaled FP16 split (2 x 63 GB).  FP64 R at this size is 252 GB, so the oracle follows sampled
focal points through the series with R rebuilt element by element from the
generator's factors (``synthesis_factored``, a plain C contraction):

* the first iteration at sampled output positions, from rows of R;
* four focal points of the batch through four Neumann iterations, every
  field in full;
* properties that hold at any size: exact linearity in G_d (doubling G_d
  doubles every field bit for bit over 8 iterations) and a contracting
  series."""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2
from tests.helpers import desc_for

pytestmark = pytest.mark.gpu

SPLIT3, SPLIT_F16 = 4, 5
TOL_ACC = 1e-5   # accumulated fields (rel L2)
TOL_N = 1e-4     # the current N_i


@pytest.mark.parametrize("rprec", [SPLIT3, SPLIT_F16], ids=["split3", "splitf16"])
def test_large_series_sampled_focal_points_and_linearity(rprec):
    import torch
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Plan
    from synthetic.torch_gen import reflection_band_chunks
    s = S.large_survey(nfocal=32)
    plan = Plan([desc_for(s, rprec=rprec)])
    for w0, blk in reflection_band_chunks(s, "cuda", chunk=4):
        plan.load_R(0, blk.contiguous(), w_begin=w0)
    torch.cuda.synchronize()
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float32)
    Gdd = torch.from_numpy(Gd).cuda()
    tdd = torch.from_numpy(td).cuda()
    plan.set_Gd_window(0, Gdd, tdd, s.eps)
    e1 = plan.iterate(1)
    Nf = torch.empty((1, s.nfocal, s.n, s.nt), dtype=torch.float32, device="cuda")
    plan.fetch_fields(0, N.MK_F_N, out=Nf)
    rows = [0, 777, 2000, 3333, 4000]
    sel2 = [0, 31]
    got = Nf[0][sel2][:, rows].cpu().numpy()
    # oracle: N_0 = -theta s_0(-t) at the sampled outputs, from rows of R regenerated on the host
    Rrows = S.reflection_band(s, rows=rows)                       # [nw][len(rows)][n]
    s0 = M.synthesis(Rrows, M.reverse_time(Gd[sel2].astype(np.float64)), s.dx * s.dt)
    theta = M.theta_mask(td[sel2][:, rows], s.eps, s.nt, s.dt)
    N0 = -theta * M.reverse_time(s0)
    assert rel_l2(got, N0) <= 1e-5
    assert abs(e1[0, 0] - np.sum(Nf[0, 0].double().cpu().numpy() ** 2)) <= 1e-6 * e1[0, 0]
    del Nf

    # four focal points through four iterations, against the oracle on the factored R
    e3 = plan.iterate(3)
    sel = [0, 10, 21, 31]
    f4 = torch.empty((4, s.nfocal, s.n, s.nt), dtype=torch.float32, device="cuda")
    plan.fetch_fields(0, N.MK_F_N | N.MK_F_F1P | N.MK_F_F1M | N.MK_F_F2P, out=f4)
    got4 = f4[:, sel].cpu().numpy()
    del f4
    Rf = S.reflection_factors(s)
    c = s.dx * s.dt
    thetas = M.theta_mask(td[sel], s.eps, s.nt, s.dt)
    st = M.initialise(Gd[sel].astype(np.float64))
    for _ in range(4):
        st = M.iterate_once(st, Rf, thetas, c, synth=M.synthesis_factored)
    for j, (name, ref) in enumerate(zip(("N", "f1plus", "f1min", "f2p"), (st.N, st.f1plus, st.f1min, st.f2p))):
        err = rel_l2(got4[j], ref)
        assert err <= (TOL_N if name == "N" else TOL_ACC), f"large, 4 iterations, {name}: rel L2 {err:.3e}"
    eref = np.array(st.energy)            # [4][len(sel)]
    egot = np.concatenate([e1, e3])[:, sel]
    assert np.max(np.abs(egot - eref) / eref) <= 1e-4

    # the series contracts at full size, and is exactly linear in G_d: 2 G_d
    # gives 2x every field, bit for bit (two series of 8 iterations; a fetch of
    # f2p, pmin or G mid-series would restore the contraction's operand through
    # another transform, which differs at the FP32 rounding level)
    plan.set_Gd_window(0, Gdd, tdd, s.eps)
    e = plan.iterate(8)
    assert np.all(np.isfinite(e)) and np.all(e[-1] < e[0])
    f_a = torch.empty((3, s.nfocal, s.n, s.nt), dtype=torch.float32, device="cuda")
    plan.fetch_fields(0, N.MK_F_N | N.MK_F_F1P | N.MK_F_F1M, out=f_a)
    plan.set_Gd_window(0, 2 * Gdd, tdd, s.eps)
    plan.iterate(8)
    f_b = torch.empty_like(f_a)
    plan.fetch_fields(0, N.MK_F_N | N.MK_F_F1P | N.MK_F_F1M, out=f_b)
    assert torch.equal(f_b, 2 * f_a)
    plan.close()
