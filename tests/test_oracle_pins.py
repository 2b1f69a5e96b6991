"""Pins of the FP64 oracle against things other than itself (no GPU).

* the DFT helpers against a naive O(nt^2) DFT written here, and Parseval;
* the synthesis against brute-force time-domain circular convolution;
* signs, reversals, mask and parity against exact rational spike algebra
  (n_r = 1, c = 1, dt = 1) and a hand-worked example;
* the converged Neumann sum against a dense direct solve of the Marchenko
  equation on the window unknowns;
* invariants: R = 0, linearity and superposition in G_d, theta idempotent and
  symmetric, reciprocity, the even/odd accumulation identities;
* a planted-mistake check: each plausible mistake, planted into the oracle on
  the CPU, must make at least one of these pins fail.
"""

import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2, small_survey


# --------------------------------------------------------------------------
# independent helpers (naive DFT, brute-force convolution, exact spikes)
# --------------------------------------------------------------------------

def naive_dft(x):
    nt = x.shape[-1]
    j = np.arange(nt)
    E = np.exp(-2j * np.pi * np.outer(j, j) / nt)
    return x @ E.T


def naive_real_idft(X_band, nt):
    """x_j = (1/nt) [Re X_0 + 2 sum_{0<m<nt/2} Re(X_m e^{2 pi i jm/nt}) + Re X_{nt/2} (-1)^j]."""
    nw = X_band.shape[-1]
    j = np.arange(nt)
    x = np.zeros(X_band.shape[:-1] + (nt,))
    for m in range(nw):
        ph = np.exp(2j * np.pi * j * m / nt)
        w = 1.0 if (m == 0 or 2 * m == nt) else 2.0
        x += w * np.real(X_band[..., m:m + 1] * ph)
    return x / nt


def brute_synthesis(Rbl, N, c):
    """s(k, f, j) = c sum_r sum_j' R_bl(k, r, (j - j') mod nt) N(f, r, j')."""
    n, _, nt = Rbl.shape
    F = N.shape[0]
    s = np.zeros((F, n, nt))
    jj = np.arange(nt)
    lag = (jj[:, None] - jj[None, :]) % nt
    for k in range(n):
        for r in range(n):
            C = Rbl[k, r][lag]  # [j][j']
            s[:, k, :] += N[:, r, :] @ C.T
    return c * s


def sp_conv(a, b, nt):
    out = {}
    for ta, va in a.items():
        for tb, vb in b.items():
            t = (ta + tb) % nt
            out[t] = out.get(t, 0) + va * vb
    return {t: v for t, v in out.items() if v != 0}


def sp_rev(a, nt):
    return {(-t) % nt: v for t, v in a.items()}


def sp_add(a, b, s=1):
    out = dict(a)
    for t, v in b.items():
        out[t] = out.get(t, 0) + s * v
    return {t: v for t, v in out.items() if v != 0}


def sp_mute(a, half, nt):
    return {t: v for t, v in a.items() if min(t, nt - t) < half}


def sp_dense(a, nt):
    x = np.zeros(nt)
    for t, v in a.items():
        x[t] = float(v)
    return x


def exact_spike_run(spikes, td, eps, nt, niter):
    """Algorithm 1 in exact rationals for one trace (n_r = 1, c = 1, dt = 1)."""
    R = dict(spikes)
    N = {(-td) % nt: Fr(1)}
    f1p, f2p, f1m, pmin = dict(N), dict(N), {}, {}
    hist = []
    for it in range(niter):
        s = sp_conv(R, N, nt)
        pmin = sp_add(pmin, s)
        Ni = sp_mute({t: -v for t, v in sp_rev(s, nt).items()}, td - eps, nt)
        f2p = sp_add(f2p, Ni)
        if it % 2 == 0:
            f1m = sp_add(f1m, sp_rev(Ni, nt), -1)
        else:
            f1p = sp_add(f1p, Ni)
        N = Ni
        hist.append(dict(N=N, f1plus=f1p, f1min=f1m, f2p=f2p, pmin=pmin))
    return hist


def spike_oracle_inputs(spikes, td, nt):
    m = np.arange(nt // 2 + 1)
    Rw = np.zeros((nt // 2 + 1, 1, 1), dtype=np.complex128)
    for t, v in spikes.items():
        Rw[:, 0, 0] += float(v) * np.exp(-2j * np.pi * m * t / nt)
    Gd = np.zeros((1, 1, nt))
    Gd[0, 0, td] = 1.0
    return Rw, Gd, np.array([[float(td)]])


# --------------------------------------------------------------------------
# pins, written as functions so the planted-mistake test can re-run them
# --------------------------------------------------------------------------

SPIKES = {20: Fr(1, 2), 7: Fr(-1, 3), 3: Fr(1, 5)}
TD, EPS, NT = 60, 3, 256


def pin_spike_algebra(niter=7):
    hist = exact_spike_run(SPIKES, TD, EPS, NT, niter)
    Rw, Gd, td = spike_oracle_inputs(SPIKES, TD, NT)
    _, ohist = M.run(Rw, Gd, td, float(EPS), 1.0, 1.0, niter, c=1.0, history=True)
    worst = 0.0
    for h, o in zip(hist, ohist):
        for name in ("N", "f1plus", "f1min", "f2p", "pmin"):
            worst = max(worst, np.max(np.abs(getattr(o, name)[0, 0] - sp_dense(h[name], NT))))
    return worst


def pin_worked_example():
    """R = 1/2 delta(t - 40), G_d = delta(t - 50), eps = 3 (dt = 1), worked by
    hand: N_{-1} = delta(t + 50); s_0 = R * N_{-1} = 1/2 delta(t + 10);
    N_0 = -theta s_0(-t) = -1/2 delta(t - 10) (inside |t| < 47);
    s_1 = R * N_0 = -1/4 delta(t - 50), whose reversal lies at t = -50,
    outside the window, so N_1 = 0; f1min = -N_0(-t) = 1/2 delta(t + 10);
    pmin = s_0 + s_1."""
    nt = 256
    Rw, Gd, td = spike_oracle_inputs({40: Fr(1, 2)}, 50, nt)
    _, h = M.run(Rw, Gd, td, 3.0, 1.0, 1.0, 2, c=1.0, history=True)
    N0 = np.zeros(nt); N0[10] = -0.5
    f1m = np.zeros(nt); f1m[nt - 10] = 0.5
    pmin = np.zeros(nt); pmin[nt - 10] = 0.5; pmin[50] = -0.25
    errs = [np.max(np.abs(h[0].N[0, 0] - N0)), np.max(np.abs(h[1].N[0, 0])),
            np.max(np.abs(h[1].f1min[0, 0] - f1m)), np.max(np.abs(h[1].pmin[0, 0] - pmin))]
    return max(errs)


def pin_brute_force(seed=5, n=6, nt=32, F=2, nw=None):
    """Random non-reciprocal R band: pins the index order of the contraction."""
    rng = np.random.default_rng(seed)
    nw = nt // 2 + 1 if nw is None else nw
    Rw = rng.standard_normal((nw, n, n)) + 1j * rng.standard_normal((nw, n, n))
    N = rng.standard_normal((F, n, nt))
    Rbl = naive_real_idft(Rw.transpose(1, 2, 0), nt)  # [k][r][t]
    c = 0.37
    return rel_l2(M.synthesis(Rw, N, c), brute_synthesis(Rbl, N, c))


def pin_direct_solve():
    s = small_survey()
    R = S.reflection_band(s)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float64)
    st = M.run(R, Gd, td, s.eps, s.dt, s.dx, 60)
    _, f2inf = M.direct_solution(R, Gd, td, s.eps, s.dt, s.dx)
    return rel_l2(st.f2p, f2inf)


def pin_accumulation_identities(tiny_inputs, niter):
    s, R, td, Gd = tiny_inputs
    c = s.dx * s.dt
    st, hist = M.run(R, Gd, td, s.eps, s.dt, s.dx, niter + 1, history=True)
    st = hist[niter - 1]
    theta = M.theta_mask(td, s.eps, s.nt, s.dt)
    Nm1 = M.reverse_time(Gd)
    errs = []
    # f2p = f1plus - f1min(-t)  (every N_i goes to f2p, odd ones to f1plus, even ones reversed to f1min)
    errs.append(rel_l2(st.f2p, st.f1plus - M.reverse_time(st.f1min)))
    # pmin = synthesis(f2p - N_last)  (linearity: pmin sums the syntheses of N_{-1} .. N_{niter-2})
    errs.append(rel_l2(st.pmin, M.synthesis(R, st.f2p - st.N, c)))
    if niter % 2 == 1:
        # f1min = theta * synthesis(f1plus)
        errs.append(rel_l2(st.f1min, theta * M.synthesis(R, st.f1plus, c)))
    else:
        # f1plus = N_{-1} + theta * [synthesis(f1min(-t))](-t)
        errs.append(rel_l2(st.f1plus, Nm1 + theta * M.reverse_time(M.synthesis(R, M.reverse_time(st.f1min), c))))
        # theta * synthesis(f1plus) = f1min - N_niter(-t)
        errs.append(rel_l2(theta * M.synthesis(R, st.f1plus, c), st.f1min - M.reverse_time(hist[niter].N)))
    return max(errs)


# --------------------------------------------------------------------------
# tests
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nt,dt,fmax,expect", [
    (512, 0.004, None, 257),      # tiny survey: full band 0 .. nt/2
    (2048, 0.004, 60.0, 492),     # paper-small: 60 Hz * 8.192 s = 491.52 -> bins 0 .. 491
    (4096, 0.004, 60.0, 984),     # large survey: 60 Hz * 16.384 s = 983.04 -> bins 0 .. 983
    (64, 0.004, 1000.0, 33),      # above Nyquist: capped at nt/2
    (1000 // 8 * 8, 0.002, 0.0, 501),  # fmax <= 0 keeps the full band
    (128, 0.008, 40.0, 41),       # 40 Hz * 1.024 s = 40.96 -> bins 0 .. 40
    (128, 0.0078125, 32.0, 33),   # exactly on a bin: 32 Hz * 1 s = 32 -> bins 0 .. 32 kept
])
def test_band_bins_closed_forms(nt, dt, fmax, expect):
    # the kept band ("padding" of the Implementation section): every bin m with
    # f_m = m / (nt dt) <= fmax up to Nyquist, counted here by brute force in
    # exact rationals
    from fractions import Fraction
    assert M.band_bins(nt, dt, fmax) == expect
    if fmax:
        T = Fraction(nt) * Fraction(dt)
        brute = sum(1 for m in range(nt // 2 + 1) if Fraction(m) / T <= Fraction(fmax))
        assert brute == expect


def test_band_bins_of_every_workload():
    # the oracle's band equals the inputs' band on every seeded workload
    import synthetic as S
    surveys = [S.tiny_survey(), S.paper_small_survey(1), S.large_survey(1)] + S.batching_surveys()
    for sv in surveys:
        assert M.band_bins(sv.nt, sv.dt, sv.fmax_hz) == S.band_count(sv.nt, sv.dt, sv.fmax_hz) == sv.nw


def test_forward_band_matches_naive_dft():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 64))
    X = M.forward_band(x, 20)
    assert np.max(np.abs(X - naive_dft(x)[:, :20])) < 1e-12


@pytest.mark.parametrize("nw", [33, 17, 1])
def test_inverse_band_matches_naive(nw):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, nw)) + 1j * rng.standard_normal((2, nw))
    assert np.max(np.abs(M.inverse_band(X, 64) - naive_real_idft(X, 64))) < 1e-13


def test_parseval():
    rng = np.random.default_rng(2)
    nt = 128
    x = rng.standard_normal(nt)
    X = M.forward_band(x, nt // 2 + 1)
    w = np.full(nt // 2 + 1, 2.0)
    w[0] = w[-1] = 1.0
    assert abs(np.sum(x * x) - np.sum(w * np.abs(X) ** 2) / nt) < 1e-10
    assert np.allclose(M.inverse_band(X, nt), x, atol=1e-13)


@pytest.mark.parametrize("nw", [None, 9])
def test_synthesis_matches_brute_force(nw):
    assert pin_brute_force(nw=nw) < 1e-12


def test_synthesis_brute_force_tiny_subset(tiny_inputs):
    # the tiny survey on a subset of positions (the operator restricted to them)
    s, R, td, Gd = tiny_inputs
    idx = np.arange(0, 101, 10)
    Rs = R[:, idx][:, :, idx]
    N = M.reverse_time(Gd[:, idx])
    Rbl = naive_real_idft(Rs.transpose(1, 2, 0), s.nt)
    assert rel_l2(M.synthesis(Rs, N, s.dx * s.dt), brute_synthesis(Rbl, N, s.dx * s.dt)) < 1e-12


def test_exact_spike_algebra():
    assert pin_spike_algebra() < 1e-13


def test_worked_example():
    assert pin_worked_example() < 1e-14


def test_theta_mask_properties():
    td = np.array([[0.1005, 0.2005, 0.0]])
    th = M.theta_mask(td, 0.012, 128, 0.004)
    assert np.array_equal(th * th, th)
    assert np.array_equal(th, M.reverse_time(th))
    # |t| < t_d - eps counted by hand: 0.0885/0.004 = 22.1 -> |j| <= 22 kept
    assert int(th[0, 0].sum()) == 2 * 22 + 1
    assert th[0, 2].sum() == 0
    # strict inequality at an exact boundary (binary-exact numbers): t_d - eps = 25 dt is not kept
    th2 = M.theta_mask(np.array([[6.25]]), 0.0, 128, 0.25)
    assert th2[0, 0, 25] == 0 and th2[0, 0, 24] == 1 and th2[0, 0, 128 - 24] == 1 and th2[0, 0, 128 - 25] == 0


def test_zero_reflectivity(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    st = M.run(np.zeros_like(R), Gd, td, s.eps, s.dt, s.dx, 3)
    assert np.all(st.N == 0) and np.all(st.f1min == 0) and np.all(st.pmin == 0)
    assert np.array_equal(st.f1plus, M.reverse_time(Gd)) and np.array_equal(st.f2p, M.reverse_time(Gd))


def test_linearity_and_superposition(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    rng = np.random.default_rng(3)
    G2 = rng.standard_normal(Gd.shape)
    a = M.run(R, Gd, td, s.eps, s.dt, s.dx, 4)
    b = M.run(R, G2, td, s.eps, s.dt, s.dx, 4)
    ab = M.run(R, 2.5 * Gd - G2, td, s.eps, s.dt, s.dx, 4)
    for name in ("N", "f1plus", "f1min", "f2p", "pmin"):
        assert rel_l2(getattr(ab, name), 2.5 * getattr(a, name) - getattr(b, name)) < 1e-12


def test_reciprocity_transposed_contraction(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    N = M.reverse_time(Gd)
    c = s.dx * s.dt
    assert rel_l2(M.synthesis(R.transpose(0, 2, 1), N, c), M.synthesis(R, N, c)) < 1e-14


@pytest.mark.parametrize("niter", [5, 6])
def test_accumulation_identities(tiny_inputs, niter):
    assert pin_accumulation_identities(tiny_inputs, niter) < 1e-12


def test_energy_is_sum_of_squares(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    _, h = M.run(R, Gd, td, s.eps, s.dt, s.dx, 3, history=True)
    for i, st in enumerate(h):
        assert abs(st.energy[i][0] - np.sum(st.N[0] ** 2)) <= 1e-12 * st.energy[i][0]


def test_total_green_definition(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    st = M.run(R, Gd, td, s.eps, s.dt, s.dx, 2)
    G = M.total_green(st.f2p, st.pmin)
    j = 7
    assert G[0, 3, j] == st.f2p[0, 3, s.nt - j] + st.pmin[0, 3, j]


def test_direct_solve_matches_converged_series():
    assert pin_direct_solve() < 1e-12


def test_sixteen_iterations_within_neumann_tail():
    s = small_survey()
    R = S.reflection_band(s)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float64)
    _, h = M.run(R, Gd, td, s.eps, s.dt, s.dx, 16, history=True)
    _, f2inf = M.direct_solution(R, Gd, td, s.eps, s.dt, s.dx)
    e = np.array([np.sqrt(x.energy[-1]) for x in h])  # [iter][F]
    rho = np.max(e[-1] / e[-2])
    assert rho < 0.6
    tail = np.linalg.norm(e[-1]) * rho / (1 - rho)
    err = np.linalg.norm(h[-1].f2p - f2inf)
    assert err <= 1.5 * tail
    assert err >= 0.2 * tail  # the tail estimate is the actual size of the error


def test_tiny_series_converges(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    st = M.run(R, Gd, td, s.eps, s.dt, s.dx, 16)
    e = np.sqrt(np.array(st.energy)[:, 0] / np.sum(Gd ** 2))
    assert e[0] < 0.5 and e[-1] < 1e-5
    assert np.all(np.diff(e) < 0)


# --------------------------------------------------------------------------
# planted mistakes: every one must break a pin
# --------------------------------------------------------------------------

def _mutant_iterate(kind):
    def it(st, Rw, theta, c):
        iRN = M.synthesis(Rw.transpose(0, 2, 1) if kind == "transpose" else Rw, st.N,
                          c / 0.004 if kind == "scale" else c)
        st.pmin = st.pmin + (M.reverse_time(iRN) if kind == "pmin_rev" else iRN)
        Ni = -M.reverse_time(iRN)
        if kind == "sign":
            Ni = -Ni
        if kind == "no_reverse":
            Ni = -iRN
        if kind != "no_mask":
            Ni = Ni * theta
        st.f2p = st.f2p + (M.reverse_time(Ni) if kind == "f2p_rev" else Ni)
        even = st.iteration % 2 == 0
        if kind == "parity":
            even = not even
        if even:
            st.f1min = st.f1min - (Ni if kind == "f1min_norev" else M.reverse_time(Ni))
        else:
            st.f1plus = st.f1plus + Ni
        st.N = Ni
        st.energy.append(np.sum(Ni * Ni, axis=(1, 2)))
        st.iteration += 1
        return st
    return it


@pytest.mark.parametrize("kind", ["sign", "no_reverse", "no_mask", "parity", "scale",
                                  "transpose", "pmin_rev", "f2p_rev", "f1min_norev"])
def test_planted_mistake_is_caught(monkeypatch, tiny_inputs, kind):
    monkeypatch.setattr(M, "iterate_once", _mutant_iterate(kind))
    if kind == "transpose":
        # reciprocal surveys cannot see it; a general R can
        rng = np.random.default_rng(9)
        n, nt = 5, 32
        Rw = rng.standard_normal((17, n, n)) + 1j * rng.standard_normal((17, n, n))
        Gd = rng.standard_normal((1, n, nt))
        Rbl = naive_real_idft(Rw.transpose(1, 2, 0), nt)
        st = M.run(Rw, Gd, np.full((1, n), 1e9), 0.0, 1.0, 1.0, 1, c=1.0)
        expect = -M.reverse_time(brute_synthesis(Rbl, M.reverse_time(Gd), 1.0))
        assert rel_l2(st.N, expect) > 1e-3
        return
    caught = [pin_spike_algebra() > 1e-9, pin_worked_example() > 1e-9]
    assert any(caught), kind


def test_tiny_energy_regression(tiny_inputs):
    # stored by tests/golden/make_golden.py from this oracle; guards its arithmetic
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_energy.txt")
    ref = np.loadtxt(path)
    s, R, td, Gd = tiny_inputs
    st = M.run(R, Gd, td, s.eps, s.dt, s.dx, 16)
    assert np.allclose(np.array(st.energy)[:, 0], ref[:, 1], rtol=1e-10, atol=0)


def test_green_up_down_sum_identity(tiny_inputs):
    # G - G^+ - G^- = -synthesis(N_last): pins the signs and reversals of G^+ against G's reading
    s, R, td, Gd = tiny_inputs
    c = s.dx * s.dt
    for niter in (3, 8):
        st = M.run(R, Gd, td, s.eps, s.dt, s.dx, niter)
        G = M.total_green(st.f2p, st.pmin)
        Gm = M.green_minus(R, st.f1plus, st.f1min, c)
        Gp = M.green_plus(R, st.f1plus, st.f1min, c)
        assert rel_l2(G - Gp - Gm, -M.synthesis(R, st.N, c)) < 1e-12


def test_green_minus_definition_spikes():
    # 1D spikes: G^- = R * f1plus - f1min exactly (exact rational algebra)
    niter = 5
    hist = exact_spike_run(SPIKES, TD, EPS, NT, niter)
    h = hist[-1]
    gm_exact = sp_add(sp_conv(SPIKES, h["f1plus"], NT), h["f1min"], -1)
    Rw, Gd, td = spike_oracle_inputs(SPIKES, TD, NT)
    st = M.run(Rw, Gd, td, float(EPS), 1.0, 1.0, niter, c=1.0)
    gm = M.green_minus(Rw, st.f1plus, st.f1min, 1.0)
    assert np.max(np.abs(gm[0, 0] - sp_dense(gm_exact, NT))) < 1e-13
    # image = zero lag of G^- * f1plus, by the exact spike product
    img_exact = sum(v * h["f1plus"].get((-t) % NT, 0) for t, v in gm_exact.items())
    assert abs(M.image(gm, st.f1plus, 1.0, 1.0)[0] - float(img_exact)) < 1e-13


def test_image_brute_force(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    st = M.run(R, Gd, td, s.eps, s.dt, s.dx, 4)
    Gm = M.green_minus(R, st.f1plus, st.f1min, s.dx * s.dt)
    nt = s.nt
    acc = 0.0
    for k in range(0, s.n, 25):
        for j in range(nt):
            acc += Gm[0, k, j] * st.f1plus[0, k, (nt - j) % nt]
    sub = Gm[:, ::25], st.f1plus[:, ::25]
    assert abs(M.image(*sub, s.dx, s.dt)[0] - s.dx * s.dt * acc) < 1e-12 * abs(acc) * s.dx * s.dt + 1e-300


# --------------------------------------------------------------------------
# the factored-R synthesis (plain C contraction) of the large-survey checks
# --------------------------------------------------------------------------

def _factored_case(n=7, nt=32, nw=13, F=3, seed=5):
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((nw, n)) + 1j * rng.standard_normal((nw, n))
    g = 1.0 + 0.3 * rng.standard_normal((n, n))          # not symmetric: pins which index is which
    N = rng.standard_normal((F, n, nt))
    off = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    R = T[:, off] * g[None]                               # R_m(k, r) = T[m][|k - r|] g[k][r]
    return T, g, N, R


def test_factored_synthesis_matches_brute_force():
    # Eq. (1) as a time-domain circular convolution with the band-limited R
    T, g, N, R = _factored_case()
    nt = N.shape[-1]
    Rbl = naive_real_idft(R.transpose(1, 2, 0), nt)
    got = M.synthesis_factored((T, g), N, 0.37)
    assert rel_l2(got, brute_synthesis(Rbl, N, 0.37)) < 1e-12


def test_factored_synthesis_matches_dense_on_a_survey():
    # the generator's dense R (the product of its factors) through the NumPy
    # oracle vs the factors through the C contraction
    s = small_survey(n=25, nt=128, nfocal=3, fmax_hz=40.0)
    T, g = S.reflection_factors(s)
    R = S.reflection_band(s)
    td = S.survey_td(s)
    N = M.reverse_time(S.gd_traces(s, td, np.float64))
    c = s.dx * s.dt
    assert rel_l2(M.synthesis_factored((T, g), N, c), M.synthesis(R, N, c)) < 1e-13


def test_factored_synthesis_catches_transposed_scale():
    # a transposed jitter scale (g[r][k] for g[k][r]) must change the result
    T, g, N, R = _factored_case()
    ref = M.synthesis(R, N, 1.0)
    assert rel_l2(M.synthesis_factored((T, g.T.copy()), N, 1.0), ref) > 1e-3
    assert rel_l2(M.synthesis_factored((T, g), N, 1.0), ref) < 1e-13


def test_factored_iteration_follows_algorithm_1(tiny_inputs):
    # the iteration with the factored synthesis equals the dense one
    s, R, td, Gd = tiny_inputs
    T, g = S.reflection_factors(s)
    theta = M.theta_mask(td, s.eps, s.nt, s.dt)
    c = s.dx * s.dt
    a = M.initialise(Gd)
    b = M.initialise(Gd)
    for _ in range(3):
        a = M.iterate_once(a, R, theta, c)
        b = M.iterate_once(b, (T, g), theta, c, synth=M.synthesis_factored)
    for x, y in ((a.N, b.N), (a.f1plus, b.f1plus), (a.f1min, b.f1min), (a.pmin, b.pmin)):
        assert rel_l2(y, x) < 1e-12
