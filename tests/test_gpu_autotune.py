"""Autotuned kernel shapes (MK_FLAG_AUTOTUNE): the choice changes speed, never results.

The tuner times each N tile of the tensor-core contraction and each epilogue
block size on the survey's own buffers before its fields are initialised.
Every candidate computes each output element with the same operations in the
same order, so a tuned plan must reproduce the untuned plan bit for bit; a
second plan of the same shape must take its choice from the cache.
"""

import numpy as np
import pytest

import synthetic as S
from tests.conftest import small_survey
from tests.helpers import desc_for, survey_inputs

pytestmark = pytest.mark.gpu

MK_FLAG_AUTOTUNE = 8


def _run(surveys, rprecs, flags, niter=4):
    import torch
    from paper_2106_04649_gb300.api import Plan
    from synthetic.torch_gen import reflection_band_chunks
    plan = Plan([desc_for(s, rprec=rp, flags=flags) for s, rp in zip(surveys, rprecs)])
    for i, s in enumerate(surveys):
        for w0, blk in reflection_band_chunks(s, "cuda", chunk=32):
            plan.load_R(i, blk.contiguous(), w_begin=w0)
        td = S.survey_td(s)
        plan.set_Gd_window(i, S.gd_traces(s, td, np.float32), td, s.eps)
    torch.cuda.synchronize()
    e = plan.iterate(niter)
    f = [plan.fetch_fields(i) for i in range(len(surveys))]
    t = [plan.tuning(i) for i in range(len(surveys))]
    plan.close()
    return e, f, t


def test_tuned_plan_is_bit_identical_and_cached():
    surveys = [S.paper_small_survey(64), S.paper_small_survey(64),
               small_survey(n=257, dx=10.0, nt=1024, dt=0.004, nfocal=3, calibrate=0.9, fmax_hz=60.0, seed=2)]
    rprecs = [4, 0, 1]   # split3 (tensor path, N tiles 16..128), c64 (SIMT), cbf16 (N tiles 16)
    e0, f0, t0 = _run(surveys, rprecs, 0)
    e1, f1, t1 = _run(surveys, rprecs, MK_FLAG_AUTOTUNE)
    assert np.array_equal(e0, e1)
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)
    assert all(t["tuned"] == 0 for t in t0)
    assert t0[0]["umma_bn"] == 128 and t0[1]["umma_bn"] == 0
    assert all(t["tuned"] in (1, 2) for t in t1)
    assert t1[0]["umma_bn"] in (16, 32, 64, 128) and t1[0]["contract_ms"] > 0
    assert t1[1]["umma_bn"] == 0 and t1[1]["epi_pairs"] in (1, 2, 4) and t1[1]["epilogue_ms"] > 0
    # the same shapes again: every choice comes from the cache
    _, _, t2 = _run(surveys, rprecs, MK_FLAG_AUTOTUNE, niter=1)
    assert all(t["tuned"] == 2 for t in t2)
    assert [(t["umma_bn"], t["epi_pairs"]) for t in t2] == [(t["umma_bn"], t["epi_pairs"]) for t in t1]
