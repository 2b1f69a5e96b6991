"""Multi-rank host logic on CPU (gloo, world size 2): focal-point sharding
and shot-row sharding.

Focal points are independent Neumann series over the same R, so the N > 1
path gives each rank its own focal points (no collective on the data path).
Here two gloo ranks each run the FP64 oracle on their shard; the gathered
fields must equal the unsharded run, and the max-over-ranks timing reduction
used by the benchmark must return the slowest rank.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synthetic as S
    from oracle import marchenko as M
    from tests.conftest import small_survey
    s = small_survey(n=21, nt=64, nfocal=3)
    focal = S.focal_shard(s.focal, world, rank)
    R = S.reflection_band(s)
    tds = np.stack([S.first_arrival_times(s.model, xf, zf, s.x) for xf, zf in focal])
    Gd = S.gd_traces(s, tds, np.float64)
    st = M.run(R, Gd, tds, s.eps, s.dt, s.dx, 4)
    mine = torch.from_numpy(np.ascontiguousarray(st.f2p))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.shape[0]]))
    maxf = int(max(x.item() for x in sizes))
    pad = torch.zeros((maxf,) + tuple(mine.shape[1:]), dtype=mine.dtype)
    pad[: mine.shape[0]] = mine
    got = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(got, pad)
    t = torch.tensor([10.0 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        parts = [got[r][: int(sizes[r].item())].numpy() for r in range(world)]
        np.savez(out_path, t=t.numpy(), **{f"p{r}": p for r, p in enumerate(parts)})
    dist.barrier()
    dist.destroy_process_group()


def test_focal_sharding_equals_unsharded(tmp_path):
    import synthetic as S
    from oracle import marchenko as M
    from tests.conftest import small_survey
    world = 2
    out = str(tmp_path / "gathered.npz")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    d = np.load(out)
    assert float(d["t"][0]) == 20.0  # max over ranks
    s = small_survey(n=21, nt=64, nfocal=3)
    R = S.reflection_band(s)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float64)
    full = M.run(R, Gd, td, s.eps, s.dt, s.dx, 4).f2p
    # shard r holds focal points r, r + world, ...
    for r in range(world):
        idx = list(range(r, s.nfocal, world))
        assert np.allclose(d[f"p{r}"], full[idx], rtol=0, atol=1e-12)


def test_focal_shard_partition():
    import synthetic as S
    focal = np.arange(10 * 2, dtype=float).reshape(10, 2)
    parts = [S.focal_shard(focal, 4, r) for r in range(4)]
    assert sum(p.shape[0] for p in parts) == 10
    assert sorted(np.concatenate(parts)[:, 0].tolist()) == sorted(focal[:, 0].tolist())


# --------------------------------------------------------------------------
# shot-row sharding: each rank holds a block of output positions (rows of R)
# and all-gathers the new field between iterations (the paper's multi-GPU
# split by shots, Implementation section)
# --------------------------------------------------------------------------

def _rows_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synthetic as S
    from oracle import marchenko as M
    from tests.conftest import small_survey
    s = small_survey(n=21, nt=64, nfocal=2)
    bounds = [(0, 11), (11, 21)]
    a, b = bounds[rank]
    R = S.reflection_band(s)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float64)
    c = s.dx * s.dt
    theta = M.theta_mask(td[:, a:b], s.eps, s.nt, s.dt)
    # the rank's rows of every field; the whole current N after each gather
    N_full = M.reverse_time(Gd)
    f1plus = N_full[:, a:b].copy()
    f2p = N_full[:, a:b].copy()
    f1min = np.zeros_like(f1plus)
    pmin = np.zeros_like(f1plus)
    energy = []
    for i in range(5):
        s_rows = M.synthesis(R[:, a:b, :], N_full, c)      # Eq. (1) with this rank's rows of R
        pmin = pmin + s_rows
        Ni = -M.reverse_time(s_rows) * theta
        f2p = f2p + Ni
        if i % 2 == 0:
            f1min = f1min - M.reverse_time(Ni)
        else:
            f1plus = f1plus + Ni
        e = torch.from_numpy(np.sum(Ni * Ni, axis=(1, 2)))
        dist.all_reduce(e)                                 # energies add up over the ranks
        energy.append(e.numpy())
        # all-gather of the new field (gloo wants equal sizes: pad to the
        # largest shard, trim after)
        rmax = max(hi - lo for lo, hi in bounds)
        mine = torch.zeros((Ni.shape[0], rmax, Ni.shape[2]), dtype=torch.float64)
        mine[:, : b - a] = torch.from_numpy(Ni)
        parts = [torch.zeros_like(mine) for _ in bounds]
        dist.all_gather(parts, mine)
        N_full = np.concatenate([p.numpy()[:, : hi - lo] for p, (lo, hi) in zip(parts, bounds)], axis=1)
    rmax = max(hi - lo for lo, hi in bounds)
    mine = torch.zeros((4, 2, rmax, s.nt), dtype=torch.float64)
    mine[:, :, : b - a] = torch.from_numpy(np.stack([f1plus, f1min, f2p, pmin]))
    gathered = [torch.zeros_like(mine) for _ in bounds]
    dist.all_gather(gathered, mine)
    if rank == 0:
        np.savez(out_path, N=N_full, E=np.array(energy),
                 **{f"p{r}": g.numpy()[:, :, : hi - lo] for r, (g, (lo, hi)) in enumerate(zip(gathered, bounds))})
    dist.barrier()
    dist.destroy_process_group()


def test_shot_row_sharding_equals_unsharded(tmp_path):
    import synthetic as S
    from oracle import marchenko as M
    from tests.conftest import small_survey
    out = str(tmp_path / "rows.npz")
    mp.start_processes(_rows_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    d = np.load(out)
    s = small_survey(n=21, nt=64, nfocal=2)
    R = S.reflection_band(s)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float64)
    st = M.run(R, Gd, td, s.eps, s.dt, s.dx, 5)
    fields = np.concatenate([d["p0"], d["p1"]], axis=2)   # [4][F][n][nt]
    for got, ref in zip(fields, (st.f1plus, st.f1min, st.f2p, st.pmin)):
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    assert np.allclose(d["N"], st.N, rtol=0, atol=1e-12 * np.max(np.abs(st.N)))
    assert np.allclose(d["E"], np.array(st.energy), rtol=1e-12, atol=0)
