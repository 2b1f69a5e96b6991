"""Batching: twelve independent surveys of uneven size in one plan.

Surveys s = 0..11 (n from 201 to 1201, nt 1024..4096, dt 2..4 ms, 5..15
layers, 1..256 focal points); even surveys keep R in complex FP32, odd ones
in the 3-way split BF16 form.  The GPU run covers all of them; the FP64
oracle checks sampled focal points of the surveys it can afford.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2
from tests.helpers import FIELD_NAMES, desc_for

pytestmark = pytest.mark.gpu

C64, SPLIT3 = 0, 4


def test_twelve_surveys_one_plan():
    import torch
    from paper_2106_04649_gb300.api import Plan
    from synthetic.torch_gen import reflection_band_chunks
    surveys = S.batching_surveys()
    descs = [desc_for(s, rprec=C64 if i % 2 == 0 else SPLIT3) for i, s in enumerate(surveys)]
    plan = Plan(descs)
    tds, gds = [], []
    for i, s in enumerate(surveys):
        for w0, blk in reflection_band_chunks(s, "cuda", chunk=16):
            plan.load_R(i, blk.contiguous(), w_begin=w0)
        td = S.survey_td(s)
        Gd = S.gd_traces(s, td, np.float32)
        plan.set_Gd_window(i, Gd, td, s.eps)
        tds.append(td)
        gds.append(Gd)
    torch.cuda.synchronize()
    e = plan.iterate(16)
    assert e.shape == (16, sum(s.nfocal for s in surveys))
    assert np.all(np.isfinite(e)) and np.all(e > 0)
    # every series contracts: the last energy is far below the first
    assert np.all(e[-1] < 1e-3 * e[0])
    # oracle parity on sampled focal points of the affordable surveys
    for i in (0, 1, 4, 8, 10):
        s = surveys[i]
        sel = [0, s.nfocal - 1] if s.nfocal > 1 else [0]
        R = S.reflection_band(s)
        st = M.run(R, gds[i][sel].astype(np.float64), tds[i][sel], s.eps, s.dt, s.dx, 16)
        f = plan.fetch_fields(i)
        ref = [st.N, st.f1plus, st.f1min, st.f2p, st.pmin, M.total_green(st.f2p, st.pmin)]
        for j, name in enumerate(FIELD_NAMES):
            err = rel_l2(f[j][sel], ref[j])
            assert err <= 1e-4, f"survey {i} {name}: {err:.3e}"
        foff = sum(x.nfocal for x in surveys[:i])
        eref = np.array(st.energy)
        assert np.max(np.abs(e[:, [foff + q for q in sel]] - eref) / eref) <= 1e-4
    plan.close()
