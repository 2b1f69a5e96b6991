"""Pins of the seeded input generators (no GPU)."""

import math

import numpy as np
import pytest

import synthetic as S
from synthetic.layered import LayeredModel, first_arrival_times, signed_times


def test_splitmix64_published_vectors():
    # Reference outputs of SplitMix64 (Steele, Lea & Flood 2014) for seeds 0 and 1234567.
    g = S.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    g = S.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(5)] == [6457827717110365317, 3203168211198807973,
                                                9817491932198370423, 4593380528125082431,
                                                16408922859458223821]


def test_vectorised_mix_matches_scalar():
    z = np.array([0, 1, 2**63, 12345678901234567], dtype=np.uint64)
    v = S.splitmix64_mix(z)
    assert [int(x) for x in v] == [S.splitmix64_mix(int(x)) for x in z]


def test_jitter_symmetric_bounded_and_row_regenerable():
    u = S.jitter_matrix(7, 40)
    assert np.array_equal(u, u.T)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.1
    assert np.array_equal(S.jitter_matrix(7, 40, rows=[3, 17]), u[[3, 17]])
    assert not np.array_equal(S.jitter_matrix(8, 40), u)


def test_ricker_dft_matches_closed_form_spectrum():
    # The DFT of a Ricker sampled on the circular grid equals the Poisson sum
    # (1/dt) sum_q W(f_m - q/dt) e^{-2 pi i (f_m - q/dt) t_s}; the images |q| >= 2
    # and the wrap-around in time are far below 1e-12 here.
    nt, dt, f0, ts = 512, 0.004, 30.0, 0.3
    w = S.ricker_wavelet(signed_times(nt, dt) - ts, f0)
    X = np.fft.rfft(w)
    f = np.arange(nt // 2 + 1) / (nt * dt)
    Y = sum(S.ricker_spectrum(f - q / dt, f0) * np.exp(-2j * math.pi * (f - q / dt) * ts)
            for q in (-1, 0, 1)) / dt
    assert np.max(np.abs(X - Y)) < 1e-12 * np.max(np.abs(Y))
    # in the 0-60 Hz band of the workloads the q = 0 term alone suffices
    b = f <= 60.0
    Y0 = S.ricker_spectrum(f, f0) * np.exp(-2j * math.pi * f * ts) / dt
    assert np.max(np.abs(X[b] - Y0[b])) < 1e-12 * np.max(np.abs(Y0))


def test_band_counts():
    assert S.band_count(512, 0.004, None) == 257
    assert S.band_count(2048, 0.004, 60.0) == 492
    assert S.band_count(4096, 0.004, 60.0) == 984
    assert S.band_count(2048, 0.004, 1e9) == 1025


def test_reflection_band_reciprocal_and_structure(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    assert R.shape == (257, 101, 101)
    assert np.array_equal(R, R.transpose(0, 2, 1))
    assert np.all(R[0] == 0)  # the Ricker spectrum vanishes at DC
    # rows regenerate alone (used for sampled checks of big surveys)
    sub = S.reflection_band(s, 10, 5, rows=[4, 50])
    assert np.array_equal(sub, R[10:15][:, [4, 50]])


def test_first_arrival_closed_forms():
    # one homogeneous layer above the focal point: straight ray sqrt(X^2 + z^2)/v
    m = LayeredModel([2000.0], [2000.0, 2500.0])
    x = np.linspace(0, 3000, 31)
    td = first_arrival_times(m, 1000.0, 800.0, x)
    assert np.max(np.abs(td - np.hypot(x - 1000.0, 800.0) / 2000.0)) < 1e-9
    # layered: vertical time at zero offset, monotone in offset
    s = S.tiny_survey()
    td = S.survey_td(s)[0]
    vert = 300 / 1800 + 200 / 2200 + 150 / 2600
    assert abs(td[50] - vert) < 1e-12
    assert np.all(np.diff(td[50:]) > 0) and np.all(np.diff(td[:51]) < 0)


def test_first_arrival_snell_consistency():
    # a transmitted ray with slowness p reaches offset X(p) = sum dz p v / sqrt(1 - p^2 v^2)
    # at time T(p) = sum dz / (v sqrt(1 - p^2 v^2)); t_d(X(p)) must equal T(p)
    m = LayeredModel([300.0, 500.0, 800.0], [1800.0, 2200.0, 2600.0, 3000.0])
    dz = np.array([300.0, 200.0, 150.0])
    v = np.array([1800.0, 2200.0, 2600.0])
    for p in [1e-5, 1e-4, 2e-4, 3e-4]:
        q = np.sqrt(1 - (p * v) ** 2)
        X = np.sum(dz * p * v / q)
        T = np.sum(dz / (v * q))
        assert abs(first_arrival_times(m, 0.0, 650.0, np.array([X]))[0] - T) < 1e-9


def test_gd_traces_peak_at_td(tiny_inputs):
    s, R, td, Gd = tiny_inputs
    assert Gd.shape == (1, 101, 512)
    j = np.argmax(Gd[0], axis=1)
    assert np.all(np.abs(j * s.dt - td[0]) <= s.dt / 2 + 1e-12)


@pytest.mark.slow
def test_calibration_bounds_operator_norm():
    # the calibrated R must satisfy max_m ||c R_m||_2 <= calibrate (checked on a subset)
    s = S.batching_surveys()[0]
    R = S.reflection_band(s, 0, None)
    c = s.dx * s.dt
    worst = max(np.linalg.norm(c * R[m], 2) for m in range(0, R.shape[0], 7))
    assert worst <= s.calibrate
    assert worst > 0.5 * s.calibrate  # and the bound is not vacuous


def test_torch_assembly_matches_host_generator():
    torch = pytest.importorskip("torch")
    from synthetic.torch_gen import reflection_band_torch
    for s in (S.tiny_survey(), S.batching_surveys()[0]):
        ref = S.reflection_band(s, dtype=np.complex128)
        got = reflection_band_torch(s, "cpu", dtype=torch.complex128).numpy()
        assert np.array_equal(got, ref)
