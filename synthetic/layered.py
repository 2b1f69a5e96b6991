"""Analytic flat-layered surveys (primaries only) in FP64.

Everything here is input modelling, not the Marchenko method:

* a flat layered velocity model, fixed or drawn from a seeded SplitMix64 stream;
* the band spectra of the reflection response R(x_R, x, omega): Ricker
  primaries at hyperbolic traveltimes with a small reciprocal amplitude jitter;
* the direct-arrival traveltime t_d from a focal point to every surface
  position (the paper's Theory section says G_d may come from an eikonal
  solver; for a flat layered medium the exact transmitted-ray time is used);
* the first arrival G_d, a zero-phase Ricker centred on t_d;
* focal-point lines at a fixed depth.

Conventions used by every array produced here:

* surface positions x_i = i * dx, i = 0 .. n-1 (sources and receivers coincide);
* the time grid is circular with nt samples; the signed time of sample j is
  j*dt for j < nt/2 and (j - nt)*dt otherwise;
* frequency bin m has f_m = m / (nt * dt); the kept band is m = 0 .. n_w-1;
* R is returned frequency-major, ``R[m][k][r]`` = R(x_R = x_k, x = x_r, f_m),
  the last axis contiguous (receivers fastest within a row).  The model is
  exactly reciprocal, so ``R[m][k][r] == R[m][r][k]``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15  # SplitMix64 increment (Steele, Lea & Flood 2014)
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def splitmix64_mix(z):
    """SplitMix64 output function on uint64 values (scalar int or ndarray)."""
    if isinstance(z, (int, np.integer)):
        z = int(z) & _MASK
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        return z ^ (z >> 31)
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Scalar SplitMix64 stream: state += GAMMA; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + GAMMA) & _MASK
        return splitmix64_mix(self.state)

    def uniform(self, lo: float, hi: float) -> float:
        """Uniform double in [lo, hi) from the top 53 bits of one draw."""
        u = (self.next_u64() >> 11) * 2.0**-53
        return lo + (hi - lo) * u


def jitter_matrix(seed: int, n: int, rows=None) -> np.ndarray:
    """Reciprocal counter-hash jitter u(k, r) in [-1, 1), shape [len(rows)][n].

    u(k, r) = 2 * (z >> 11) * 2^-53 - 1 with
    z = mix(key + (a * 2^32 + b) * GAMMA mod 2^64), a = min(k, r), b = max(k, r),
    key = first output of SplitMix64(seed).  Any row can be regenerated alone.
    """
    key = SplitMix64(seed).next_u64()
    k = np.arange(n, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64)
    r = np.arange(n, dtype=np.uint64)
    a = np.minimum(k[:, None], r[None, :])
    b = np.maximum(k[:, None], r[None, :])
    with np.errstate(over="ignore"):
        ctr = (a << np.uint64(32)) | b
        z = splitmix64_mix(np.uint64(key) + ctr * np.uint64(GAMMA))
    return 2.0 * (z >> np.uint64(11)).astype(np.float64) * 2.0**-53 - 1.0


@dataclass
class LayeredModel:
    """Flat layers: interfaces at depths ``z`` (m, increasing) and velocities
    ``v`` (m/s); v[0] is the top layer, v[i] lies between z[i-1] and z[i],
    v[-1] is the half-space below the last interface.  Constant density."""

    z: np.ndarray
    v: np.ndarray

    def __post_init__(self):
        self.z = np.asarray(self.z, dtype=np.float64)
        self.v = np.asarray(self.v, dtype=np.float64)
        assert self.v.shape == (self.z.size + 1,)
        assert np.all(np.diff(self.z) > 0) and self.z[0] > 0

    def reflection_coefficients(self) -> np.ndarray:
        """Normal-incidence r_i = (v_below - v_above)/(v_below + v_above)."""
        return (self.v[1:] - self.v[:-1]) / (self.v[1:] + self.v[:-1])

    def primaries(self):
        """(t0, vrms, r) per interface: two-way vertical time, Dix RMS velocity
        and reflection coefficient."""
        dz = np.diff(np.concatenate([[0.0], self.z]))
        tau = dz / self.v[:-1]  # one-way vertical time per layer
        ctau = np.cumsum(tau)
        t0 = 2.0 * ctau
        vrms = np.sqrt(np.cumsum(self.v[:-1] ** 2 * tau) / ctau)
        return t0, vrms, self.reflection_coefficients()


def fixed_model(depths, velocities, halfspace_v) -> LayeredModel:
    return LayeredModel(np.asarray(depths, float), np.concatenate([np.asarray(velocities, float), [halfspace_v]]))


def random_model(seed: int, n_interfaces: int, zmin=100.0, zmax=3000.0, min_gap=40.0,
                 vmin=1500.0, vmax=3500.0) -> LayeredModel:
    """Seeded random flat model.  Draw order from one SplitMix64(seed) stream:
    n_interfaces depths U(zmin, zmax), sorted; the whole set is redrawn while
    any gap (including the one to the surface) is below min_gap; then
    n_interfaces + 1 velocities U(vmin, vmax), top to bottom."""
    g = SplitMix64(seed)
    while True:
        z = np.sort([g.uniform(zmin, zmax) for _ in range(n_interfaces)])
        if np.all(np.diff(np.concatenate([[0.0], z])) >= min_gap):
            break
    v = np.array([g.uniform(vmin, vmax) for _ in range(n_interfaces + 1)])
    return LayeredModel(z, v)


def band_count(nt: int, dt: float, fmax_hz) -> int:
    """Number of kept bins n_w = min(nt/2, floor(fmax_hz * nt * dt)) + 1
    (left-to-right FP64 product); fmax_hz None or <= 0 keeps the full band."""
    if fmax_hz is None or fmax_hz <= 0:
        return nt // 2 + 1
    return min(nt // 2, int(math.floor(fmax_hz * nt * dt))) + 1


def signed_times(nt: int, dt: float) -> np.ndarray:
    """Signed time of each sample of the circular grid."""
    j = np.arange(nt)
    return np.where(j < nt // 2, j, j - nt) * dt


def ricker_wavelet(t, f0: float) -> np.ndarray:
    """Zero-phase Ricker w(t) = (1 - 2 pi^2 f0^2 t^2) exp(-pi^2 f0^2 t^2)."""
    a = (math.pi * f0 * np.asarray(t, dtype=np.float64)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def ricker_spectrum(f, f0: float) -> np.ndarray:
    """Fourier transform (kernel exp(-2 pi i f t)) of ``ricker_wavelet``:
    W(f) = (2/sqrt(pi)) f^2 / f0^3 exp(-f^2/f0^2)."""
    f = np.asarray(f, dtype=np.float64)
    return (2.0 / math.sqrt(math.pi)) * f**2 / f0**3 * np.exp(-(f**2) / f0**2)


@dataclass
class Survey:
    """One seeded line survey: n sources = n receivers at spacing dx."""

    name: str
    n: int
    dx: float
    nt: int
    dt: float
    f0: float
    fmax_hz: float | None
    model: LayeredModel
    seed: int
    eps: float
    focal: np.ndarray  # [F][2] focal points (x, z) in metres
    calibrate: float | None = None  # target Toeplitz-symbol bound of max_m ||c R_m||_2
    meta: dict = field(default_factory=dict)

    @property
    def nfocal(self) -> int:
        return int(self.focal.shape[0])

    @property
    def nw(self) -> int:
        return band_count(self.nt, self.dt, self.fmax_hz)

    @property
    def x(self) -> np.ndarray:
        return np.arange(self.n) * self.dx


def _offset_spectra(s: Survey, w_begin: int, w_count: int) -> np.ndarray:
    """T[m][o] = sum_i A_i(h) W(f_m) exp(-2 pi i f_m t_i(h)) at h = o*dx."""
    t0, vrms, rc = s.model.primaries()
    h = np.arange(s.n) * s.dx
    t = np.sqrt(t0[None, :] ** 2 + (h[:, None] / vrms[None, :]) ** 2)  # [o][i]
    amp = rc[None, :] * np.sqrt(t0[None, :] / t)
    f = (w_begin + np.arange(w_count)) / (s.nt * s.dt)
    out = np.zeros((w_count, s.n), dtype=np.complex128)
    for i in range(rc.size):
        out += amp[None, :, i] * np.exp(-2j * math.pi * f[:, None] * t[None, :, i])
    out *= ricker_spectrum(f, s.f0)[:, None]
    return out


def amplitude_scale(s: Survey) -> float:
    """Calibration factor kappa applied to R (1 when ``s.calibrate`` is None).

    Without the transmission losses and scaling of recorded data, the analytic
    primaries of a many-layer model make the Neumann series diverge.  R is
    therefore calibrated so that an upper bound of max_m ||c R_m||_2, with
    c = dx*dt, equals ``s.calibrate`` (< 1 makes the series converge).  The
    bound uses the jitter-free R, a symmetric Toeplitz matrix per frequency,
    whose spectral norm is at most the maximum modulus of its symbol
    sum_o T_m(|o|) e^{i kappa o}; that maximum is taken over a 4n-point (or
    finer) FFT grid and multiplied by 1.01 for the +-1% jitter.
    """
    if s.calibrate is None:
        return 1.0
    if "kappa" not in s.meta:
        T = _offset_spectra(s, 0, s.nw) / s.dt
        n = s.n
        L = 1 << int(math.ceil(math.log2(4 * n)))
        emb = np.zeros((T.shape[0], L), dtype=np.complex128)
        emb[:, :n] = T
        emb[:, L - n + 1:] = T[:, 1:][:, ::-1]
        bound = s.dx * s.dt * 1.01 * np.abs(np.fft.fft(emb, axis=1)).max()
        s.meta["kappa"] = float(s.calibrate / bound)
    return s.meta["kappa"]


def reflection_factors(s: Survey, w_begin: int = 0, w_count: int | None = None, rows=None):
    """The two factors of R: (T [w_count][n] complex128, g [len(rows)][n] float64)
    with R_m(k, r) = T[m][|k - r|] * g[k][r] -- the offset spectra of the
    flat-layered primaries and the reciprocal jitter scale
    g(k, r) = (1 + 0.01 u(k, r)) kappa / dt.  ``reflection_band`` is their
    product; a consumer that cannot hold R whole rebuilds any element from them."""
    if w_count is None:
        w_count = s.nw - w_begin
    T = _offset_spectra(s, w_begin, w_count)
    g = (1.0 + 0.01 * jitter_matrix(s.seed, s.n, rows)) * (amplitude_scale(s) / s.dt)
    return T, g


def reflection_band(s: Survey, w_begin: int = 0, w_count: int | None = None,
                    dtype=np.complex128, rows=None, chunk: int = 16) -> np.ndarray:
    """Band spectra of R, shape [w_count][len(rows)][n], frequency-major.

    R_m(k, r) = (kappa/dt) (1 + 0.01 u(k, r)) sum_i A_i(h) W(f_m) exp(-2 pi i f_m t_i(h)),
    h = |x_k - x_r|, with u the reciprocal jitter of ``jitter_matrix`` and
    kappa the calibration of ``amplitude_scale`` (the product of the factors
    of ``reflection_factors``).
    """
    if w_count is None:
        w_count = s.nw - w_begin
    rows = np.arange(s.n) if rows is None else np.asarray(rows)
    T, scale = reflection_factors(s, w_begin, w_count, rows)
    off = np.abs(rows[:, None] - np.arange(s.n)[None, :])
    out = np.empty((w_count, rows.size, s.n), dtype=dtype)
    for c in range(0, w_count, chunk):
        e = min(w_count, c + chunk)
        out[c:e] = T[c:e][:, off] * scale[None]
    return out


def first_arrival_times(model: LayeredModel, xf: float, zf: float, x: np.ndarray,
                        iters: int = 160) -> np.ndarray:
    """Transmitted first-arrival time from (xf, zf) to surface points x.

    t_d(X) = max over p in [0, p_max] of p*X + sum_l dz_l sqrt(1/v_l^2 - p^2),
    summed over the layer pieces between the surface and zf, p_max = 1/max v_l.
    The bracketed function is concave in p; golden-section search in FP64.
    """
    bounds = np.concatenate([[0.0], model.z])
    dz, vl = [], []
    for l in range(model.v.size):
        top = bounds[l]
        bot = model.z[l] if l < model.z.size else np.inf
        if top >= zf:
            break
        dz.append(min(bot, zf) - top)
        vl.append(model.v[l])
    dz, vl = np.array(dz), np.array(vl)
    pmax = 1.0 / vl.max()
    X = np.abs(np.asarray(x, dtype=np.float64) - xf)

    def T(p):
        q = np.maximum(1.0 / vl[None, :] ** 2 - p[:, None] ** 2, 0.0)
        return p * X + np.sum(dz[None, :] * np.sqrt(q), axis=1)

    a = np.zeros_like(X)
    b = np.full_like(X, pmax)
    g = (math.sqrt(5.0) - 1.0) / 2.0
    c = b - g * (b - a)
    d = a + g * (b - a)
    fc, fd = T(c), T(d)
    for _ in range(iters):
        left = fc > fd  # maximum lies in [a, d]
        b = np.where(left, d, b)
        a = np.where(left, a, c)
        c_new = b - g * (b - a)
        d_new = a + g * (b - a)
        c, d = c_new, d_new
        fc, fd = T(c), T(d)
    p = 0.5 * (a + b)
    return np.maximum(np.maximum(T(p), T(np.zeros_like(p))), T(np.full_like(p, pmax)))


def gd_traces(s: Survey, td: np.ndarray, dtype=np.float32) -> np.ndarray:
    """First arrivals G_d(x_r, t) = w(t - t_d(x_r)) sampled on the signed
    circular grid; ``td`` is [F][n], the result [F][n][nt]."""
    tau = signed_times(s.nt, s.dt)
    return ricker_wavelet(tau[None, None, :] - td[:, :, None], s.f0).astype(dtype)


def focal_line(s_n: int, dx: float, count: int, z: float, mode: str = "central80") -> np.ndarray:
    """Focal points at depth z.  ``central80``: mid-points of ``count`` equal
    bins spanning the central 80% of the aperture [0, (n-1) dx];
    ``every``: one per surface position."""
    A = (s_n - 1) * dx
    if mode == "every":
        xs = np.arange(s_n) * dx
    else:
        lo, hi = 0.1 * A, 0.9 * A
        w = (hi - lo) / count
        xs = lo + w * (np.arange(count) + 0.5)
    return np.stack([xs, np.full_like(xs, z)], axis=1)


def focal_shard(focal: np.ndarray, world: int, rank: int) -> np.ndarray:
    """Focal points of one rank when a focal line is split over ``world``
    ranks: rank r takes points r, r + world, r + 2 world, ..."""
    return np.asarray(focal)[rank::world]


def survey_td(s: Survey) -> np.ndarray:
    """t_d[F][n] for every focal point of the survey."""
    return np.stack([first_arrival_times(s.model, xf, zf, s.x) for xf, zf in s.focal])
