"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2, small_survey
from tests.helpers import FIELD_NAMES, desc_for, survey_inputs

pytestmark = pytest.mark.gpu

# relative L2 gates (float32 path vs FP64 oracle)
TOL_ITER = 1e-5     # accumulated fields, every iteration
TOL_N = 1e-4        # the current N_i (a small, shrinking term) and after 16 iterations
TOL_E = 1e-4        # energies


def _plan(survey, R, Gd, td, nfocal=None):
    from paper_2106_04649_gb300.api import Plan
    p = Plan([desc_for(survey, nfocal=nfocal)])
    p.load_R(0, R)
    p.set_Gd_window(0, Gd, td, survey.eps)
    return p


def _oracle_fields(st):
    return [st.N, st.f1plus, st.f1min, st.f2p, st.pmin, M.total_green(st.f2p, st.pmin)]


def _compare(fields, st, tol_acc, tol_n, label=""):
    ref = _oracle_fields(st)
    errs = {name: rel_l2(fields[i], ref[i]) for i, name in enumerate(FIELD_NAMES)}
    for name, e in errs.items():
        tol = tol_n if name == "N" else tol_acc
        assert e <= tol, f"{label} {name}: rel L2 {e:.3e} > {tol:.0e} ({errs})"
    return errs


def test_tiny_trajectory_16_iterations(tiny_inputs):
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    _, hist = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 16, history=True)
    p = _plan(s, R, Gd, td)
    f0 = p.fetch_fields(0)
    st0 = M.initialise(Gd.astype(np.float64))
    _compare(f0, st0, 1e-7, 1e-7, "init")
    for i in range(16):
        e = p.iterate(1)
        f = p.fetch_fields(0)
        _compare(f, hist[i], TOL_ITER, TOL_N, f"iter {i}")
        assert abs(e[0, 0] - hist[i].energy[i][0]) <= TOL_E * hist[i].energy[i][0]
    p.close()


def test_tiny_energies_match_oracle(tiny_inputs):
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    st = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 16)
    p = _plan(s, R, Gd, td)
    e = p.iterate(16)
    assert e.shape == (16, 1)
    assert np.max(np.abs(e[:, 0] - np.array(st.energy)[:, 0]) / np.array(st.energy)[:, 0]) <= TOL_E
    _compare(p.fetch_fields(0), st, TOL_N, TOL_N, "after 16")
    p.close()


@pytest.mark.parametrize("n,nt,nfocal,fmax", [(25, 128, 2, None), (25, 128, 3, 40.0), (7, 32, 1, None),
                                              (1, 64, 1, None), (3, 64, 2, 30.0), (33, 256, 1, 50.0)])
def test_small_ragged_surveys(n, nt, nfocal, fmax):
    s = small_survey(n=n, nt=nt, nfocal=min(nfocal, 3), fmax_hz=fmax)
    R, td, Gd = survey_inputs(s)
    st, hist = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 6, history=True)
    p = _plan(s, R, Gd, td)
    for i in range(6):
        p.iterate(1)
        _compare(p.fetch_fields(0), hist[i], TOL_ITER, TOL_N, f"n={n} nt={nt} F={nfocal} iter {i}")
    p.close()


def test_deterministic_repeat(tiny_inputs):
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    out = []
    for _ in range(2):
        p = _plan(s, R, Gd, td)
        e = p.iterate(5)
        out.append((e, p.fetch_fields(0)))
        p.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_restart_resets_series(tiny_inputs):
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    p = _plan(s, R, Gd, td)
    e1 = p.iterate(3)
    p.set_Gd_window(0, Gd, td, s.eps)
    e2 = p.iterate(3)
    assert np.array_equal(e1, e2)
    p.close()


def test_paper_small_F1_full_size():
    s = S.paper_small_survey(1)
    R, td, Gd = survey_inputs(s)
    st = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 16)
    p = _plan(s, R, Gd, td)
    e = p.iterate(16)
    _compare(p.fetch_fields(0), st, TOL_N, TOL_N, "paper-small F=1 after 16")
    ref = np.array(st.energy)[:, 0]
    assert np.max(np.abs(e[:, 0] - ref) / ref) <= TOL_E
    p.close()


def test_device_inputs_and_outputs(tiny_inputs):
    import torch
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    from paper_2106_04649_gb300.api import Plan
    p = Plan([desc_for(s)])
    p.load_R(0, torch.from_numpy(R).cuda())
    p.set_Gd_window(0, torch.from_numpy(Gd).cuda(), torch.from_numpy(td).cuda(), s.eps)
    p.iterate(4)
    dev = torch.empty((6, 1, s.n, s.nt), dtype=torch.float32, device="cuda")
    p.fetch_fields(0, out=dev)
    host = p.fetch_fields(0)
    assert np.array_equal(dev.cpu().numpy(), host)
    p.close()


def test_call_order_errors(tiny_inputs):
    from paper_2106_04649_gb300.api import Plan
    from paper_2106_04649_gb300.binding import MarchenkoError
    from paper_2106_04649_gb300 import _native as N
    s, R64, td, Gd64 = tiny_inputs
    p = Plan([desc_for(s)])
    with pytest.raises(MarchenkoError) as ei:
        p.iterate(1)
    assert ei.value.status == N.MK_ERR_STATE
    p.load_R(0, R64[:10].astype(np.complex64))
    with pytest.raises(MarchenkoError) as ei:
        p.set_Gd_window(0, Gd64, td, s.eps)
    assert ei.value.status == N.MK_ERR_STATE
    with pytest.raises(MarchenkoError) as ei:
        p.load_R(0, R64[:10].astype(np.complex64), w_begin=250)
    assert ei.value.status == N.MK_ERR_ARG
    from paper_2106_04649_gb300 import binding as B
    out = np.empty(8, dtype=np.float32)
    with pytest.raises(MarchenkoError) as ei:
        B.mk_fetch_fields(p.handle, 5, N.MK_F_N, out.ctypes.data, out.nbytes, False)
    assert ei.value.status == N.MK_ERR_ARG
    p.close()


@pytest.mark.parametrize("n", [200, 353, 500, 700, 1000, 1201, 1400])
def test_contraction_row_lengths(n):
    # every register/ring variant of the F = 1 contraction (row lengths 256 .. 1408 complex)
    s = small_survey(n=n, nt=64, dt=0.008, nfocal=1, fmax_hz=8.0)
    R, td, Gd = survey_inputs(s)
    _, hist = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 2, history=True)
    p = _plan(s, R, Gd, td)
    for i in range(2):
        p.iterate(1)
        _compare(p.fetch_fields(0), hist[i], TOL_ITER, TOL_N, f"n={n} iter {i}")
    p.close()


def test_load_paths_agree(tiny_inputs):
    # pageable host, pinned host in out-of-order chunks (synchronous and
    # asynchronous in stream order), and device sources must give bit-identical runs
    import torch
    from paper_2106_04649_gb300 import binding as B
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Plan
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    outs = []
    for mode in ("pageable", "pinned", "pinned-async", "device"):
        p = Plan([desc_for(s)])
        if mode == "pageable":
            p.load_R(0, R)
        elif mode.startswith("pinned"):
            Rp = torch.from_numpy(R).pin_memory()
            nw, n = R.shape[0], R.shape[1]
            how = N.MK_SRC_HOST_ASYNC if mode == "pinned-async" else N.MK_SRC_HOST
            for a, b in [(200, nw), (0, 77), (77, 200)]:
                B.mk_load_R(p.handle, 0, Rp.data_ptr() + a * n * n * 8, a, b - a, how)
            if how == N.MK_SRC_HOST_ASYNC:
                # pageable memory cannot be read asynchronously
                with pytest.raises(B.MarchenkoError) as ei:
                    B.mk_load_R(p.handle, 0, R.ctypes.data, 0, 1, how)
                assert ei.value.status == N.MK_ERR_ARG
        else:
            p.load_R(0, torch.from_numpy(R).cuda())
        p.set_Gd_window(0, Gd, td, s.eps)
        e = p.iterate(3)
        outs.append((e, p.fetch_fields(0)))
        p.close()
    for e, f in outs[1:]:
        assert np.array_equal(e, outs[0][0])
        assert np.array_equal(f, outs[0][1])


def test_paper_small_F64_sampled_focal_points():
    # the 64-point line at full size; the oracle computes sampled focal points one by one
    s = S.paper_small_survey(64)
    R, td, Gd = survey_inputs(s)
    p = _plan(s, R, Gd, td)
    e = p.iterate(16)
    f = p.fetch_fields(0)
    p.close()
    sel = [0, 17, 40, 63]
    st = M.run(R.astype(np.complex128), Gd[sel].astype(np.float64), td[sel], s.eps, s.dt, s.dx, 16)
    ref = _oracle_fields(st)
    for i, name in enumerate(FIELD_NAMES):
        err = rel_l2(f[i][sel], ref[i])
        assert err <= TOL_N, f"F=64 {name}: rel L2 {err:.3e}"
    eref = np.array(st.energy)
    assert np.max(np.abs(e[:, sel] - eref) / eref) <= TOL_E


def _state_array(st):
    return np.stack([st.N, st.f1plus, st.f1min, st.f2p, st.pmin]).astype(np.float32)


@pytest.mark.parametrize("case", ["tiny", "paper-small-F4"])
def test_per_iteration_from_identical_inputs(case, tiny_inputs):
    # one synthesis + epilogue from the oracle's own (FP32-rounded) state: <= 1e-5 per iteration
    if case == "tiny":
        s, R64, td, Gd64 = tiny_inputs
        R = R64.astype(np.complex64)
        Gd = Gd64.astype(np.float32)
        niter = 16
    else:
        s = S.paper_small_survey(64)
        sel = [0, 21, 42, 63]
        s.focal = s.focal[sel]
        R, td, Gd = survey_inputs(s)
        niter = 6
    st0 = M.initialise(Gd.astype(np.float64))
    _, hist = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, niter, history=True)
    p = _plan(s, R, Gd, td)
    prev = st0
    for i in range(niter):
        p.set_fields(0, _state_array(prev), i)
        p.iterate(1)
        f = p.fetch_fields(0)
        ref = _oracle_fields(hist[i])
        for j, name in enumerate(FIELD_NAMES):
            err = rel_l2(f[j], ref[j])
            assert err <= TOL_ITER, f"{case} iter {i} {name}: {err:.3e}"
        prev = hist[i]
    p.close()


@pytest.mark.parametrize("rprec", [0, 4])
def test_green_up_down_and_image(tiny_inputs, rprec):
    # G^- (Algorithm 1 after the loop), G^+ and the double-focusing image vs the oracle
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Plan
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    c = s.dx * s.dt
    st = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 8)
    gm = M.green_minus(R.astype(np.complex128), st.f1plus, st.f1min, c)
    gp = M.green_plus(R.astype(np.complex128), st.f1plus, st.f1min, c)
    img = M.image(gm, st.f1plus, s.dx, s.dt)
    p = Plan([desc_for(s, rprec=rprec)])
    p.load_R(0, R)
    p.set_Gd_window(0, Gd, td, s.eps)
    p.iterate(8)
    # output in bit order: f1plus, G, G^-, G^+
    f = p.fetch_fields(0, N.MK_F_GMINUS | N.MK_F_GPLUS | N.MK_F_G | N.MK_F_F1P)
    assert rel_l2(f[0], st.f1plus) <= 1e-5
    assert rel_l2(f[1], M.total_green(st.f2p, st.pmin)) <= 1e-5
    assert rel_l2(f[2], gm) <= 1e-5
    assert rel_l2(f[3], gp) <= 1e-5
    # forming G^+ / G^- must not disturb the series: continue and compare again
    im = p.image(0)
    assert abs(im[0] - img[0]) <= 1e-5 * abs(img[0])
    p.iterate(2)
    st2 = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 10)
    f2 = p.fetch_fields(0)
    _compare(f2, st2, TOL_ITER, TOL_N, "after G+/G- and 2 more iterations")
    p.close()


def test_graph_replay_matches_stream_launches(tiny_inputs):
    # MK_FLAG_GRAPH: iterations replayed as one captured graph (two surveys on
    # parallel branches) give bit-identical fields and energies
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Plan
    s, R64, td, Gd64 = tiny_inputs
    R = R64.astype(np.complex64)
    Gd = Gd64.astype(np.float32)
    s2 = small_survey(n=25, nt=128, nfocal=3)
    R2, td2, Gd2 = survey_inputs(s2)
    outs = []
    for flags in (0, N.MK_FLAG_GRAPH):
        p = Plan([desc_for(s, flags=flags), desc_for(s2, rprec=4, flags=flags)])
        p.load_R(0, R)
        p.load_R(1, R2)
        p.set_Gd_window(0, Gd, td, s.eps)
        p.set_Gd_window(1, Gd2, td2, s2.eps)
        e = np.concatenate([p.iterate(3), p.iterate(5)])
        outs.append((e, p.fetch_fields(0), p.fetch_fields(1)))
        p.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("nfocal", [1, 3])
def test_new_R_between_iterations(nfocal):
    # mk_load_R of a second R (from device memory, so a load kernel precedes the
    # next contraction on the stream) between iterations, without a new
    # mk_set_Gd_window: the series continues from its state with the new R, and
    # the first contraction after the load must read the new R
    import torch
    s = small_survey(n=33, nt=128, nfocal=nfocal)
    R1, td, Gd = survey_inputs(s)
    s2 = small_survey(n=33, nt=128, nfocal=nfocal, seed=11, calibrate=0.6)
    R2 = S.reflection_band(s2, dtype=np.complex64)
    c = s.dx * s.dt
    theta = M.theta_mask(td, s.eps, s.nt, s.dt)
    st = M.initialise(Gd.astype(np.float64))
    for _ in range(2):
        st = M.iterate_once(st, R1.astype(np.complex128), theta, c)
    for _ in range(3):
        st = M.iterate_once(st, R2.astype(np.complex128), theta, c)
    p = _plan(s, R1, Gd, td)
    p.iterate(2)
    p.load_R(0, torch.from_numpy(R2).cuda())
    e = p.iterate(3)
    f = p.fetch_fields(0)
    p.close()
    ref = [st.N, st.f1plus, st.f1min, st.f2p]
    for j, name in enumerate(FIELD_NAMES[:4]):
        err = rel_l2(f[j], ref[j])
        assert err <= (TOL_N if name == "N" else TOL_ITER), f"F={nfocal} {name}: {err:.3e}"
    # pmin after a change of R is formed with the current R: synthesis of f2p - N_last
    pmin = M.synthesis(R2.astype(np.complex128), st.f2p - st.N, c)
    assert rel_l2(f[4], pmin) <= TOL_ITER
    assert rel_l2(f[5], M.total_green(st.f2p, pmin)) <= TOL_ITER
    assert np.max(np.abs(e[-1] - st.energy[-1]) / st.energy[-1]) <= TOL_E


@pytest.mark.parametrize("fmax", [None, 60.0])
def test_longest_traces_nt8192(fmax):
    # nt = 8192, the longest trace the library accepts (its own epilogue shape:
    # 512 threads, one CTA per SM, in-place transforms), per iteration
    s = small_survey(n=9, dx=20.0, nt=8192, dt=0.0005, nfocal=2, fmax_hz=fmax)
    R, td, Gd = survey_inputs(s)
    _, hist = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 4, history=True)
    p = _plan(s, R, Gd, td)
    for i in range(4):
        e = p.iterate(1)
        _compare(p.fetch_fields(0), hist[i], TOL_ITER, TOL_N, f"nt=8192 fmax={fmax} iter {i}")
        assert np.max(np.abs(e[0] - hist[i].energy[i]) / hist[i].energy[i]) <= TOL_E
    p.close()


def _many_focal(n, nt, dt, F, fmax):
    s = small_survey(n=n, nt=nt, dt=dt, nfocal=3, fmax_hz=fmax)
    xs = np.linspace(0.15, 0.85, F) * (n - 1) * s.dx
    zs = 600.0 + 100.0 * np.linspace(0.0, 1.0, F)
    s.focal = np.stack([xs, zs], axis=1)
    return s


@pytest.mark.parametrize("nt,dt,fmax,rprec", [(64, 0.016, None, 0), (128, 0.008, 40.0, 0), (256, 0.008, None, 0),
                                              (512, 0.004, 60.0, 0), (1024, 0.002, 90.0, 0), (2048, 0.001, 150.0, 0),
                                              (2048, 0.001, 150.0, 4), (512, 0.004, 60.0, 4), (1024, 0.002, 90.0, 1),
                                              (256, 0.008, None, 2), (4096, 0.0005, 200.0, 0),
                                              (4096, 0.0005, 480.0, 4), (4096, 0.0005, 480.0, 5),
                                              (4096, 0.0005, None, 0)])
def test_register_epilogue_shapes(nt, dt, fmax, rprec):
    # enough traces (33 positions x 80 focal points) for the register epilogue
    # where the shape fits its shared memory (nt = 64, 512 with a narrow band,
    # 1024, 2048, and 4096 with two warps per trace up to 984 bins for the
    # complex FP32 spectrum; the others run the shared-memory epilogue):
    # ragged blocks (33 is no multiple of the block size), full and limited
    # bands, and each output form (complex FP32 field spectrum, also quantised
    # by the scaled FP16 split; the 2- and 3-part 16-bit embeddings, BF16 and
    # FP16), per iteration
    from tests.test_gpu_tensor import dequantised
    from paper_2106_04649_gb300.api import Plan
    s = _many_focal(33, nt, dt, 80, fmax)
    R, td, Gd = survey_inputs(s)
    Rref = R.astype(np.complex128) if rprec in (0, 4, 5) else dequantised(R, rprec)
    _, hist = M.run(Rref, Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 3, history=True)
    p = Plan([desc_for(s, rprec=rprec)])
    p.load_R(0, R)
    p.set_Gd_window(0, Gd, td, s.eps)
    for i in range(3):
        e = p.iterate(1)
        _compare(p.fetch_fields(0), hist[i], TOL_ITER, TOL_N, f"nt={nt} rprec={rprec} iter {i}")
        assert np.max(np.abs(e[0] - hist[i].energy[i]) / hist[i].energy[i]) <= TOL_E
    p.close()


@pytest.mark.parametrize("n,F", [(25, 5), (75, 8), (300, 5), (500, 2), (500, 5), (75, 9)])
def test_few_focal_points_complex_fp32(n, F):
    # complex FP32 R with 2 .. 8 focal points: the GEMV takes 4 of them per pass
    # over R where their field slices fit in registers (rows of at most 384
    # positions), else 2, with a ragged last pass (F = 5); F = 9 is the first
    # count that runs the SIMT GEMM.  Per iteration against the oracle.
    from paper_2106_04649_gb300.api import Plan
    s = _many_focal(n, 128, 0.008, F, 40.0)
    R, td, Gd = survey_inputs(s)
    _, hist = M.run(R.astype(np.complex128), Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 4, history=True)
    p = Plan([desc_for(s)])
    p.load_R(0, R)
    p.set_Gd_window(0, Gd, td, s.eps)
    for i in range(4):
        e = p.iterate(1)
        _compare(p.fetch_fields(0), hist[i], TOL_ITER, TOL_N, f"n={n} F={F} iter {i}")
        assert np.max(np.abs(e[0] - hist[i].energy[i]) / hist[i].energy[i]) <= TOL_E
    p.close()


@pytest.mark.parametrize("nt,dt,fmax,F,rprec", [(2048, 0.001, 150.0, 80, 4), (4096, 0.004, 60.0, 80, 0),
                                                (4096, 0.0005, 480.0, 80, 5), (128, 0.008, 40.0, 3, 0)])
def test_fetch_mid_series(nt, dt, fmax, F, rprec):
    # Reading N, f1plus and f1min mid-series leaves the series untouched, bit
    # for bit.  Fields that need a synthesis (f2p with pmin, G, G^- and G^+)
    # overwrite the contraction's operand, which is then restored from N_last
    # through the shared-memory transform, and a plan resumed from fetched N,
    # f1plus and f1min starts from that transform too: both continue the
    # series to FP32 rounding (register epilogue at nt = 2048 and 4096, whose
    # own transform rounds differently, and the shared-memory epilogue).
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.api import Plan
    s = _many_focal(33, nt, dt, F, fmax)
    R, td, Gd = survey_inputs(s)
    state = N.MK_F_N | N.MK_F_F1P | N.MK_F_F1M

    def plan():
        p = Plan([desc_for(s, rprec=rprec)])
        p.load_R(0, R)
        p.set_Gd_window(0, Gd, td, s.eps)
        return p

    def series(fetch_at=(), mask=N.MK_F_ALL):
        p = plan()
        for i in range(6):
            p.iterate(1)
            if i in fetch_at:
                p.fetch_fields(0, mask)
        out = p.fetch_fields(0)
        p.close()
        return out

    plain = series()
    assert np.array_equal(series(fetch_at=(1, 3), mask=state), plain)
    assert rel_l2(series(fetch_at=(1, 3)), plain) <= 1e-6
    p = plan()
    p.iterate(3)
    fields = p.fetch_fields(0, state)
    p.close()
    q = plan()
    q.set_fields(0, np.ascontiguousarray(fields), 3, state)
    q.iterate(3)
    resumed = q.fetch_fields(0)
    q.close()
    assert rel_l2(resumed, plain) <= 1e-6
