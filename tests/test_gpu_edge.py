"""Degenerate and extreme cases of the method on the GPU, against the FP64 oracle.

* R = 0: nothing is synthesised; N_i = 0, f1+ = f2p = G_d(-t), f1- = pmin = 0, energies 0.
* empty windows (t_d <= eps everywhere): theta = 0, so N_0 = 0 and the series stops after one
  synthesis (pmin = s_0).
* full windows (t_d far beyond the trace): theta = 1 on every sample.
* zero iterations: the fields stay at their initial values.
* the smallest trace length (nt = 32) with two positions, and an odd number of traces.
"""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2, small_survey
from tests.helpers import FIELD_NAMES, desc_for, survey_inputs

pytestmark = pytest.mark.gpu


def _run(s, R, Gd, td, niter):
    from paper_2106_04649_gb300.api import Plan
    p = Plan([desc_for(s)])
    p.load_R(0, R.astype(np.complex64))
    p.set_Gd_window(0, Gd.astype(np.float32), td, s.eps)
    e = p.iterate(niter)
    f = p.fetch_fields(0)
    p.close()
    return e, f


def _oracle(s, R, Gd, td, niter):
    st = M.run(R.astype(np.complex64).astype(np.complex128), Gd.astype(np.float32).astype(np.float64), td,
               s.eps, s.dt, s.dx, niter)
    return st, [st.N, st.f1plus, st.f1min, st.f2p, st.pmin, M.total_green(st.f2p, st.pmin)]


def _check(f, ref, tol=1e-5, tol_n=1e-4):
    for j, name in enumerate(FIELD_NAMES):
        if not np.any(ref[j]):
            assert not np.any(f[j]), f"{name} should be exactly zero"
        else:
            assert rel_l2(f[j], ref[j]) <= (tol_n if name == "N" else tol), name


@pytest.fixture(scope="module")
def small():
    s = small_survey(n=101, dx=10.0, nt=512, dt=0.004, nfocal=2, calibrate=0.9, fmax_hz=60.0, seed=9)
    R, td, Gd = survey_inputs(s, dtype=np.complex128)
    return s, R, td, Gd


def test_zero_reflection_response(small):
    s, R, td, Gd = small
    R0 = np.zeros_like(R)
    e, f = _run(s, R0, Gd, td, 3)
    st, ref = _oracle(s, R0, Gd, td, 3)
    assert np.all(e == 0.0)
    _check(f, ref)
    Gr = M.reverse_time(Gd.astype(np.float32).astype(np.float64))
    assert rel_l2(f[1], Gr) == 0.0 and rel_l2(f[3], Gr) == 0.0   # f1+ = f2p = G_d(-t), exactly


def test_empty_windows(small):
    s, R, td, Gd = small
    td0 = np.full_like(td, s.eps * 0.5)   # t_d - eps < 0: theta keeps nothing
    e, f = _run(s, R, Gd, td0, 4)
    st, ref = _oracle(s, R, Gd, td0, 4)
    assert np.all(e == 0.0)
    assert not np.any(f[0]) and not np.any(f[2])   # N and f1- vanish
    _check(f, ref)


def test_full_windows(small):
    s, R, td, Gd = small
    tdf = np.full_like(td, 1e6)           # theta keeps every sample
    e, f = _run(s, R, Gd, tdf, 5)
    st, ref = _oracle(s, R, Gd, tdf, 5)
    _check(f, ref)
    assert np.max(np.abs(e - np.array(st.energy)) / np.array(st.energy)) <= 1e-4


def test_zero_iterations(small):
    s, R, td, Gd = small
    e, f = _run(s, R, Gd, td, 0)
    assert e.shape[0] == 0
    Gr = M.reverse_time(Gd.astype(np.float32).astype(np.float64))
    assert rel_l2(f[0], Gr) == 0.0 and rel_l2(f[1], Gr) == 0.0 and rel_l2(f[3], Gr) == 0.0
    assert not np.any(f[2]) and not np.any(f[4])


@pytest.mark.parametrize("n,nt,nfocal", [(2, 32, 1), (3, 64, 1), (5, 128, 3)])
def test_smallest_surveys(n, nt, nfocal):
    s = small_survey(n=n, dx=20.0, nt=nt, dt=0.008, nfocal=nfocal, calibrate=0.7, fmax_hz=None, seed=4)
    R, td, Gd = survey_inputs(s, dtype=np.complex128)
    e, f = _run(s, R, Gd, td, 6)
    st, ref = _oracle(s, R, Gd, td, 6)
    _check(f, ref)
