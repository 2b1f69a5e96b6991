"""Relative L2 error against the FP64 oracle, iteration by iteration, for every R form.

The precision workload: the paper-small survey with 601 focal points along
z = 1200 m; the GPU runs all 601 and the oracle follows four of them (the
same complex64 R, FP64).  After each of
the 16 iterations the fields of those four are compared.  The table is
printed (pytest -s shows it); the gates are the contract's: complex FP32, the
3-way split BF16 (6 products) and the scaled FP16 split (3 products) within
1e-5 for f1+, f1- and G at every iteration and 1e-4 for N; the 16-bit forms
(R stored with 8 or 11 significant bits) and the 3-product BF16 split are
reported, with only a loose sanity bound.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2
from tests.helpers import desc_for

pytestmark = pytest.mark.gpu

FORMS = [("c64", 0), ("cbf16", 1), ("cf16", 2), ("split", 3), ("split3", 4), ("splitf16", 5)]
SEL = [0, 200, 400, 600]
NITER = 16


def test_per_iteration_error_table():
    import torch
    from paper_2106_04649_gb300.api import Plan
    from synthetic.torch_gen import reflection_band_torch
    s = S.precision_survey()
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float32)
    # the GPU gets complex64 R; the oracle takes the same values in FP64
    R = S.reflection_band(s, dtype=np.complex64).astype(np.complex128)
    _, hist = M.run(R, Gd[SEL].astype(np.float64), td[SEL], s.eps, s.dt, s.dx, NITER, history=True)
    R_dev = reflection_band_torch(s, "cuda")
    out = torch.empty((6, s.nfocal, s.n, s.nt), dtype=torch.float32, device="cuda")
    sel = torch.tensor(SEL, device="cuda")
    table = {}
    for name, rp in FORMS:
        p = Plan([desc_for(s, rprec=rp)])
        p.load_R(0, R_dev)
        p.set_Gd_window(0, Gd, td, s.eps)
        rows = []
        for i in range(NITER):
            p.iterate(1)
            p.fetch_fields(0, 0x3F, out=out)
            f = out.index_select(1, sel).cpu().numpy()
            st = hist[i]
            ref = [st.N, st.f1plus, st.f1min, M.total_green(st.f2p, st.pmin)]
            rows.append([rel_l2(f[j], r) for j, r in zip((0, 1, 2, 5), ref)])
        p.close()
        table[name] = np.array(rows)
    print("\nrelative L2 vs FP64 oracle, precision workload, focal points", SEL, "of 601")
    print("iter " + " ".join(f"{n + ' N':>12s} {n + ' G':>12s}" for n, _ in FORMS))
    for i in range(NITER):
        print(f"{i:4d} " + " ".join(f"{table[n][i, 0]:12.3e} {table[n][i, 3]:12.3e}" for n, _ in FORMS))
    for name in ("c64", "split3", "splitf16"):
        t = table[name]
        assert np.all(t[:, 1:] <= 1e-5), (name, t[:, 1:].max())
        assert np.all(t[:, 0] <= 1e-4), (name, t[:, 0].max())
    for name in ("cbf16", "cf16", "split"):
        assert np.all(np.isfinite(table[name])) and table[name][:, 1:].max() < 0.1, name
