"""FP64 CPU oracle of iterative Marchenko synthesis (test infrastructure only).

This module is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import
it.  It shares no code with the CUDA path and imports nothing from the product
package; its inputs come from the ``synthetic`` generators.

It is the paper's algorithm written out plainly in NumPy float64/complex128
(plus one plain-C loop, ``csynth.c``, for the contraction of surveys whose
dense FP64 R does not fit in memory),
step by step in the order of Algorithm 1, with the synthesis of Eq. (1) done
in the frequency domain as the paper's Theory section states (forward DFT of
the field, per-frequency product with R and integral over the surface
positions, inverse DFT of the result).  ``numpy.fft`` and ``numpy.matmul``
serve as library steps; nothing is blocked, fused or reordered.

Conventions (readings of the paper, see the design notes):

* circular time grid of nt samples; sample j has signed time j*dt for
  j < nt/2 and (j - nt)*dt otherwise; X(-t)[j] = X[(nt - j) mod nt];
* forward DFT unnormalised, inverse DFT normalised by 1/nt; only bins
  0 .. n_w-1 are kept, the others are zero ("padding" before the inverse
  transform, Implementation section);
* the space integral is the Riemann sum over positions, the time integral the
  sum over samples: the synthesis scale is c = dx * dt;
* theta keeps |t| < t_d(x_k) - eps of the output trace x_k and zeroes the rest
  (symmetric in +-t, a hard 0/1 mask);
* N_i = -theta * s_i(-t): the sign and reversal of Algorithm 1 ("multiplied
  by -1"), which Eq. (1) omits;
* niter iterations are iter = 0 .. niter-1, N_{-1} being the initialiser.

Every public function below cites the passage it follows.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------------------
# Time/frequency helpers (Theory section: convolutions in the frequency domain)
# ---------------------------------------------------------------------------

def band_bins(nt: int, dt: float, fmax_hz) -> int:
    """Kept bins 0 .. floor(fmax * nt * dt), at most nt/2 (Nyquist); full band
    when fmax is None or <= 0.  (The band limit is the "padding" of the
    Implementation section: bins outside it are zero.)"""
    if fmax_hz is None or fmax_hz <= 0:
        return nt // 2 + 1
    return min(nt // 2, int(np.floor(fmax_hz * nt * dt))) + 1


def forward_band(x: np.ndarray, nw: int) -> np.ndarray:
    """Forward (unnormalised) DFT of real traces along the last axis, bins
    0 .. nw-1 (Theory: "a direct ... Fourier transform of field N_i")."""
    return np.fft.rfft(np.asarray(x, dtype=np.float64), axis=-1)[..., :nw]


def inverse_band(X: np.ndarray, nt: int) -> np.ndarray:
    """Inverse DFT (1/nt) of a band spectrum zero-padded to nt/2+1 bins; the
    imaginary parts of the DC and Nyquist bins do not enter a real trace
    (Theory: "reverse Fourier transform"; Implementation: "padding")."""
    full = np.zeros(X.shape[:-1] + (nt // 2 + 1,), dtype=np.complex128)
    full[..., : X.shape[-1]] = X
    return np.fft.irfft(full, n=nt, axis=-1)


def reverse_time(x: np.ndarray) -> np.ndarray:
    """X(-t): sample j <- sample (nt - j) mod nt (Algorithm 1, iRN(-t)), i.e.
    sample 0 stays and samples 1 .. nt-1 are reversed."""
    return np.concatenate([x[..., :1], x[..., :0:-1]], axis=-1)


def signed_time(nt: int, dt: float) -> np.ndarray:
    """Signed time of each sample of the circular grid."""
    j = np.arange(nt)
    return np.where(j < nt // 2, j, j - nt).astype(np.float64) * dt


def theta_mask(td: np.ndarray, eps: float, nt: int, dt: float) -> np.ndarray:
    """theta[f][k][j] = 1 where |t_j| < t_d(f, x_k) - eps, else 0 (Theory:
    the window theta_t and the first-arrival time t_d; applyMute of
    Algorithm 1).  td is [F][n] in seconds."""
    tau = np.abs(signed_time(nt, dt))
    return (tau[None, None, :] < (np.asarray(td, np.float64)[:, :, None] - eps)).astype(np.float64)


# ---------------------------------------------------------------------------
# Synthesis, Eq. (1)
# ---------------------------------------------------------------------------

def synthesis(Rw: np.ndarray, N: np.ndarray, c: float) -> np.ndarray:
    """s(x_k, t) = c * sum_r sum_t' R(x_k, x_r, t - t') N(x_r, t') (Eq. 1 before
    the mute), done per frequency: S_m(k, f) = c * sum_r R_m(k, r) N_m(r, f).

    Rw: [n_w][n][n] band spectra R[m][k][r] (R(x_R = x_k, x = x_r)).
    N:  [F][n][nt] real time-domain field N(x_r, x_F, t).
    Returns s: [F][n][nt]."""
    return inverse_band(synthesis_spectrum(Rw, N, c), N.shape[-1])


def synthesis_factored(Rf, N: np.ndarray, c: float) -> np.ndarray:
    """``synthesis`` for a reflection response given by its two factors,
    Rf = (T [n_w][n] complex, g [n][n] real) with R_m(k, r) = T[m][|k-r|] g[k][r]:
    the same steps (forward DFT of N, the per-frequency sum over r of Eq. 1,
    inverse DFT), with R rebuilt element by element inside a plain C loop
    instead of held as a dense array (surveys whose FP64 R does not fit in
    memory)."""
    from . import _clib
    T, g = Rf
    nw = T.shape[0]
    Nw = np.ascontiguousarray(np.transpose(forward_band(N, nw), (2, 1, 0)))  # [m][r][F]
    S = _clib.contract_factored(T, g, Nw, c)                                  # [m][k][F]
    return inverse_band(np.transpose(S, (2, 1, 0)), N.shape[-1])


def synthesis_spectrum(Rw: np.ndarray, N: np.ndarray, c: float) -> np.ndarray:
    """The band spectrum S[F][k][m] of ``synthesis`` (same steps, before the
    inverse transform)."""
    nw = Rw.shape[0]
    Nw = np.ascontiguousarray(np.transpose(forward_band(N, nw), (2, 1, 0)))  # [m][r][F]
    S = np.matmul(Rw, Nw)                                                    # [m][k][F]
    return c * np.transpose(S, (2, 1, 0))                                    # [F][k][m]


# ---------------------------------------------------------------------------
# Algorithm 1: Neumann iterations and accumulation
# ---------------------------------------------------------------------------

@dataclass
class State:
    """Fields of Algorithm 1 after ``iteration`` iterations, each [F][n][nt]:
    N (the last N_i), f1plus, f1min, f2p, pmin; ``energy`` holds
    sum_{k,t} N_i^2 per focal point for each completed iteration."""

    N: np.ndarray
    f1plus: np.ndarray
    f1min: np.ndarray
    f2p: np.ndarray
    pmin: np.ndarray
    iteration: int = 0
    energy: list = field(default_factory=list)

    def copy(self) -> "State":
        return State(self.N.copy(), self.f1plus.copy(), self.f1min.copy(), self.f2p.copy(),
                     self.pmin.copy(), self.iteration, [e.copy() for e in self.energy])


def initialise(Gd: np.ndarray) -> State:
    """N_{-1} = f1plus = f2p = G_d(x_R, x_F, -t); f1min = pmin = 0 (Theory:
    initialisation; Algorithm 1, the two lines before the second loop)."""
    N = reverse_time(np.asarray(Gd, dtype=np.float64))
    z = np.zeros_like(N)
    return State(N=N.copy(), f1plus=N.copy(), f1min=z.copy(), f2p=N.copy(), pmin=z.copy())


def iterate_once(st: State, Rw, theta: np.ndarray, c: float, synth=None) -> State:
    """One Neumann iteration, in the order of Algorithm 1:
    iRN = synthesis(N_{i-1}); pmin += iRN; N_i = -iRN(-t); mute N_i;
    f2p += N_i; iteration even: f1min -= N_i(-t); odd: f1plus += N_i.
    ``synth`` is the synthesis of Eq. (1) to use (default ``synthesis`` on a
    dense Rw; ``synthesis_factored`` for R given by its factors)."""
    iRN = (synthesis if synth is None else synth)(Rw, st.N, c)
    st.pmin = st.pmin + iRN
    Ni = -reverse_time(iRN)
    Ni = Ni * theta
    st.f2p = st.f2p + Ni
    if st.iteration % 2 == 0:
        st.f1min = st.f1min - reverse_time(Ni)
    else:
        st.f1plus = st.f1plus + Ni
    st.N = Ni
    st.energy.append(np.sum(Ni * Ni, axis=(1, 2)))
    st.iteration += 1
    return st


def run(Rw: np.ndarray, Gd: np.ndarray, td: np.ndarray, eps: float, dt: float, dx: float,
        niter: int, c: float | None = None, history: bool = False):
    """Algorithm 1 from G_d to ``niter`` iterations.  Returns the final State,
    or (final, [State after each iteration]) when ``history``."""
    nt = Gd.shape[-1]
    c = dx * dt if c is None else c
    theta = theta_mask(td, eps, nt, dt)
    st = initialise(Gd)
    hist = []
    for _ in range(niter):
        st = iterate_once(st, Rw, theta, c)
        if history:
            hist.append(st.copy())
    return (st, hist) if history else st


def total_green(f2p: np.ndarray, pmin: np.ndarray) -> np.ndarray:
    """G(t) = f2p(-t) + pmin(t): the total Green's function from f_2 and p^-
    (Theory: "the latter two fields can be used to determine G").  The paper
    gives no formula; this convention is a reading."""
    return reverse_time(f2p) + pmin


# ---------------------------------------------------------------------------
# Limit of the series: plain definition (direct solve)
# ---------------------------------------------------------------------------

def direct_solution(Rw: np.ndarray, Gd: np.ndarray, td: np.ndarray, eps: float, dt: float,
                    dx: float, c: float | None = None):
    """Converged sum y = sum_{i>=0} N_i as the solution of (I - A) y = N_0 on
    the window unknowns, with the time-domain operator
    A[(k,j),(r,j')] = -theta_k(j) c R_bl(x_k, x_r, (-j - j') mod nt)
    (Theory: the Marchenko equation is an inverse problem that can be solved
    directly; the iterative scheme is its Neumann series).  R_bl is the inverse
    DFT of the band spectra.  Dense, for small surveys only.  Returns
    (y [F][n][nt], f2p_inf = N_{-1} + y)."""
    nw, n, _ = Rw.shape
    F, _, nt = Gd.shape
    c = dx * dt if c is None else c
    Rbl = inverse_band(Rw.transpose(1, 2, 0), nt)          # [k][r][t]
    theta = theta_mask(td, eps, nt, dt)
    jj = np.arange(nt)
    lag = (-jj[:, None] - jj[None, :]) % nt                  # [j][j']
    # Full operator rows (k, j), columns (r, j'):  -theta c R_bl(k, r, lag)
    Afull = -c * Rbl[:, :, lag].transpose(0, 2, 1, 3).reshape(n * nt, n * nt)
    Nm1 = reverse_time(np.asarray(Gd, np.float64))
    y = np.zeros((F, n, nt))
    for f in range(F):
        th = theta[f].reshape(-1)
        A = th[:, None] * Afull
        N0 = A @ Nm1[f].reshape(-1)
        win = np.nonzero(th)[0]
        Aw = A[np.ix_(win, win)]
        yw = np.linalg.solve(np.eye(win.size) - Aw, N0[win])
        yf = np.zeros(n * nt)
        yf[win] = yw
        y[f] = yf.reshape(n, nt)
    return y, Nm1 + y


# ---------------------------------------------------------------------------
# After the iterations: up/down-going Green's functions and the image
# ---------------------------------------------------------------------------

def green_minus(Rw: np.ndarray, f1plus: np.ndarray, f1min: np.ndarray, c: float) -> np.ndarray:
    """G^-(t) = synthesis(f1plus)(t) - f1min(t): the extra synthesis after the
    loop in Algorithm 1 ("cuda_synthesis(Refl, f1plus, iRN); Gmin = iRN - f1min")."""
    return synthesis(Rw, f1plus, c) - f1min


def green_plus(Rw: np.ndarray, f1plus: np.ndarray, f1min: np.ndarray, c: float) -> np.ndarray:
    """G^+(t) = f1plus(-t) - synthesis(f1min(-t))(t): the down-going part with
    its own extra synthesis (Theory section, citing the coupled Marchenko
    representations; the formula is a reading: G^+(-t) = f1plus(t) minus the
    correlation of R with f1min).  With the readings used here
    G - G^+ - G^- = -synthesis(N_last) exactly."""
    return reverse_time(f1plus) - synthesis(Rw, reverse_time(f1min), c)


def image(Gmin: np.ndarray, f1plus: np.ndarray, dx: float, dt: float) -> np.ndarray:
    """Double-focusing image per focal point: the zero-time sample of the
    time convolution of G^- with f1plus, integrated over the surface
    positions (Theory section): dx dt sum_k sum_j G^-(k, j) f1plus(k, -j)."""
    return dx * dt * np.sum(Gmin * reverse_time(f1plus), axis=(1, 2))
