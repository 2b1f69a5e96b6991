"""Shot-row sharding on one GPU: the paper splits the synthesis over GPUs by
shots (Implementation section); here two or three plans each hold a block of
output positions of one survey (mk_desc.row_begin / row_count), and between
iterations every shard exports its rows of the field spectrum and imports the
others' (mk_export_field_spectrum / mk_import_field_spectrum), as the ranks
of a multi-GPU run would around an all-gather.  The shards run one after the
other on one device (no kernel waits on another); the gathered fields must
match the FP64 oracle of the whole survey per iteration, and the shards'
energies must add up to the whole survey's."""

import numpy as np
import pytest

import synthetic as S
from oracle import marchenko as M
from tests.conftest import rel_l2, small_survey
from tests.helpers import FIELD_NAMES, desc_for, survey_inputs

pytestmark = pytest.mark.gpu

TOL_ITER, TOL_N, TOL_E = 1e-5, 1e-4, 1e-4


def _survey(n, nt, F, fmax):
    s = small_survey(n=n, nt=nt, nfocal=min(F, 3), fmax_hz=fmax)
    if F > 3:
        xs = np.linspace(0.15, 0.85, F) * (n - 1) * s.dx
        s.focal = np.stack([xs, np.full(F, 650.0)], axis=1)
    return s


def _shards(s, R, Gd, td, rprec, bounds):
    from paper_2106_04649_gb300.api import Plan
    plans = []
    for a, b in bounds:
        d = desc_for(s, rprec=rprec)
        d.row_begin, d.row_count = a, b - a
        p = Plan([d])
        p.load_R(0, np.ascontiguousarray(R[:, a:b, :]))
        p.set_Gd_window(0, np.ascontiguousarray(Gd[:, a:b]), np.ascontiguousarray(td[:, a:b]), s.eps)
        plans.append(p)
    return plans


def _exchange(plans, bounds):
    bufs = [p.export_spectrum(0) for p in plans]
    for i, p in enumerate(plans):
        for j, (a, b) in enumerate(bounds):
            if j != i:
                p.import_spectrum(0, bufs[j], a, b - a)


@pytest.mark.parametrize("n,nt,F,fmax,rprec,bounds", [
    (40, 128, 1, None, 0, [(0, 32), (32, 40)]),                 # F = 1: GEMV, pmin spectrum
    (75, 128, 3, 40.0, 0, [(0, 32), (32, 64), (64, 75)]),       # GEMV, 3 focal points per pass, three shards
    (75, 256, 3, None, 4, [(0, 64), (64, 75)]),                 # tcgen05, 3-way split embedding
    (70, 128, 2, 40.0, 1, [(0, 32), (32, 70)]),                 # tcgen05, BF16 R
    (75, 1024, 80, 30.0, 0, [(0, 32), (32, 64), (64, 75)]),     # register epilogue on the full shards
])
def test_sharded_series_matches_oracle(n, nt, F, fmax, rprec, bounds):
    from tests.test_gpu_tensor import dequantised
    s = _survey(n, nt, F, fmax)
    R, td, Gd = survey_inputs(s)
    Rref = R.astype(np.complex128) if rprec in (0, 4) else dequantised(R, rprec)
    _, hist = M.run(Rref, Gd.astype(np.float64), td, s.eps, s.dt, s.dx, 4, history=True)
    plans = _shards(s, R, Gd, td, rprec, bounds)
    _exchange(plans, bounds)
    for i in range(4):
        e = sum(p.iterate(1) for p in plans)
        _exchange(plans, bounds)
        f = np.concatenate([p.fetch_fields(0) for p in plans], axis=2)  # positions of all shards
        ref = [hist[i].N, hist[i].f1plus, hist[i].f1min, hist[i].f2p, hist[i].pmin,
               M.total_green(hist[i].f2p, hist[i].pmin)]
        for j, name in enumerate(FIELD_NAMES):
            err = rel_l2(f[j], ref[j])
            assert err <= (TOL_N if name == "N" else TOL_ITER), f"iter {i} {name}: rel L2 {err:.3e}"
        assert np.max(np.abs(e[0] - hist[i].energy[i]) / hist[i].energy[i]) <= TOL_E
    for p in plans:
        p.close()


def test_shard_export_import_round_trip():
    # a shard's exported rows imported into an unsharded plan and exported back
    # are the same bytes; sizes and ranges are checked
    from paper_2106_04649_gb300 import _native as N
    from paper_2106_04649_gb300.binding import MarchenkoError
    s = _survey(40, 128, 3, 40.0)
    R, td, Gd = survey_inputs(s)
    (sh,) = _shards(s, R, Gd, td, 4, [(32, 40)])
    (full,) = _shards(s, R, Gd, td, 4, [(0, 40)])
    buf = sh.export_spectrum(0)
    full.import_spectrum(0, buf, 32, 8)
    whole = full.export_spectrum(0)                      # rows 0 .. 39, packed per part
    parts, nw, rows = 3, s.nw, 40
    w = whole.cpu().numpy().reshape(parts, nw * 2 * s.nfocal, 2 * rows * 2)
    b = buf.cpu().numpy().reshape(parts, nw * 2 * s.nfocal, 2 * 8 * 2)
    assert np.array_equal(w[:, :, 2 * 32 * 2:], b)
    with pytest.raises(MarchenkoError) as ei:
        full.import_spectrum(0, buf, 36, 8)              # rows beyond nrec
    assert ei.value.status == N.MK_ERR_ARG
    with pytest.raises(MarchenkoError) as ei:
        sh.fetch_fields(0, N.MK_F_GMINUS)                # needs every shard's fields
    assert ei.value.status == N.MK_ERR_UNSUPPORTED
    sh.close()
    full.close()
