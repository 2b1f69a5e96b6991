"""Benchmark of iterative Marchenko synthesis on GB300.

One step = one full pass of the hot path for one set of focal points: the
initialisation (first arrivals, windows, spectrum of N_{-1}) and 16 Neumann
iterations (contraction, inverse transform, reversal, mute, accumulation,
forward transform), all in libmarchenko.so kernels.  The default workload is
the paper-small survey: 601 x 601 positions at dx = 10 m, nt = 2048,
dt = 4 ms, R band-limited to 0-60 Hz (492 bins, complex FP32, 1.42 GB
resident in HBM), one focal point (--nfocal 64 for the 64-point line).

Metric: focal points per second to convergence (16 iterations), with the
contraction's HBM bandwidth and FLOP rate against the measured roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--nfocal F] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (the slow
baseline) on the same workload, on a bounded sample of focal points.
Multi-GPU (torchrun, one rank per GPU): each rank runs its own focal-point set
on its own copy of R (weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NITER = 16
L2_NOTE = "inputs larger than L2: R (1.42 GB) is streamed from HBM every iteration"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--nfocal", type=int, default=1, choices=[1, 64])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def survey(nfocal):
    import synthetic as S
    return S.paper_small_survey(nfocal)


def workload_config(s, nfocal):
    return {
        "workload": f"paper-small: {s.n}x{s.n} sources/receivers, dx={s.dx:g} m, nt={s.nt}, dt={s.dt * 1e3:g} ms, "
                    f"R band 0-60 Hz ({s.nw} bins) complex FP32 resident, {nfocal} focal point(s) at z=1200 m, "
                    f"{NITER} Neumann iterations",
        "nsrc": s.n, "nrec": s.n, "nt": s.nt, "nw": s.nw, "nfocal": nfocal, "niter": NITER, "rprec": "c64",
        "l2": L2_NOTE,
    }


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- roofline
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(src: str) -> str:
    with open(os.path.join(ROOT, "paper_2106_04649_gb300", "csrc", src), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic(workload_key: str):
    """DRAM bytes per contraction launch from the committed ncu summary, or None
    when the kernel's source file changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(workload_key)
    if not e or e.get("source_sha256_16") != kernel_source_hash(e.get("source", "")):
        return None
    return e.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- CPU oracle
def cpu_worker(spec: str):
    """Runs in a child process: time the FP64 oracle on a sample of the workload."""
    import synthetic as S
    from oracle import marchenko as M
    d = json.loads(spec)
    s = S.paper_small_survey(d["nfocal"])
    sel = np.array(d["focal_sample"])
    R = S.reflection_band(s, dtype=np.complex128)
    td = S.survey_td(s)[sel]
    Gd = S.gd_traces(s, td, np.float64)
    times = []
    for _ in range(d["reps"]):
        t = time.perf_counter()
        M.run(R, Gd, td, s.eps, s.dt, s.dx, NITER)
        times.append(time.perf_counter() - t)
    print(json.dumps({"times": times, "focal_per_rep": int(sel.size)}))


def run_cpu_oracle(nfocal: int, reps: int):
    cores = os.cpu_count() or 1
    sample = [0] if nfocal == 1 else [0, 21, 42, 63][: max(1, min(4, nfocal))]
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    spec = json.dumps({"nfocal": nfocal, "focal_sample": sample, "reps": reps})
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", spec], env=env,
                         capture_output=True, text=True, cwd=ROOT)
    if res.returncode != 0:
        raise RuntimeError(f"CPU oracle worker failed:\n{res.stderr[-2000:]}")
    out = json.loads(res.stdout.strip().splitlines()[-1])
    return out, cores, sample


# --------------------------------------------------------------------------- reference arm
def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    s = survey(args.nfocal)
    reps = args.warmup + args.steps
    out, cores, sample = run_cpu_oracle(args.nfocal, reps)
    times = out["times"][args.warmup:]
    total = float(sum(times))
    value = out["focal_per_rep"] * len(times) / total
    line = {
        "impl": "reference",
        "metric": "focal points/sec to convergence (16 Neumann iterations)",
        "value": value, "unit": "focal points/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(s, args.nfocal),
        "cpu_baseline": {"value": value, "unit": "focal points/s", "cores": cores, "kind": "oracle",
                         "sample": f"focal points {sample} of {args.nfocal}, {NITER} iterations per step, "
                                   f"FP64 NumPy oracle, {cores} BLAS threads"},
        "e2e": {"value": value, "unit": "focal points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def main_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    import synthetic as S
    from paper_2106_04649_gb300.api import Desc, Plan
    from paper_2106_04649_gb300 import _native as N

    s = survey(args.nfocal)
    F = s.nfocal
    R = S.reflection_band(s, dtype=np.complex64)
    td = S.survey_td(s)
    Gd = S.gd_traces(s, td, np.float32)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    desc = Desc(s.n, s.n, s.nt, F, s.dt, s.dx, s.fmax_hz, N.MK_R_C64, N.MK_FLAG_TIMING)
    plan = Plan([desc], device=local, stream=stream)
    Rd = torch.from_numpy(R).to(dev)
    Gdd = torch.from_numpy(Gd).to(dev)
    tdd = torch.from_numpy(td).to(dev)
    plan.load_R(0, Rd)
    torch.cuda.synchronize()
    del Rd
    torch.cuda.empty_cache()

    def step():
        plan.set_Gd_window(0, Gdd, tdd, s.eps)
        plan.iterate(NITER, energy=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.stats(reset=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    st = plan.stats(reset=True)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    ms_per_step = ms / args.steps
    value = world * F * args.steps / (ms / 1e3)

    # roofline of the dominant kernel (the contraction)
    n_w, n = s.nw, s.n
    bytes_launch = n_w * n * n * 8 + n_w * n * F * 8 + n_w * n * F * 8
    flops_launch = 8 * n_w * n * n * F
    c_ms = st["contract_ms"] / max(1, st["contract_timed"])
    e_ms = st["epilogue_ms"] / max(1, st["epilogue_timed"])
    peak, peak_kind = measured_peaks()
    achieved = bytes_launch / (c_ms * 1e-3) / 1e9
    key = f"paper-small-F{F}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(key), "kernel": "contraction (complex GEMV, F=1)" if F == 1 else
                "contraction (complex GEMM)", "peak_source": f"{peak_kind} hbm_gbs (copy)",
                "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": c_ms}
    synthesis = {"hbm_gbs": achieved, "tflops": flops_launch / (c_ms * 1e-3) / 1e12,
                 "contract_ms": c_ms, "epilogue_ms": e_ms,
                 "share_contract": st["contract_ms"] / max(1e-9, ms)}

    # end to end through the C ABI with host buffers (R, G_d, t_d in; energies and G out)
    e2e = None
    if not args.no_e2e:
        Rh = torch.from_numpy(R).pin_memory()
        Gh = torch.from_numpy(Gd).pin_memory()
        th = torch.from_numpy(td).pin_memory()
        from paper_2106_04649_gb300 import binding as B
        Gout = torch.empty((1, F, n, s.nt), dtype=torch.float32).pin_memory()
        energy = torch.empty((NITER, F), dtype=torch.float64).pin_memory()
        h2d = R.nbytes + Gd.nbytes + td.nbytes
        d2h = Gout.numel() * 4 + energy.numel() * 8

        def e2e_step():
            B.mk_load_R(plan.handle, 0, Rh.data_ptr(), 0, s.nw, False)
            B.mk_set_Gd_window(plan.handle, 0, Gh.data_ptr(), th.data_ptr(), s.eps, False)
            B.mk_iterate(plan.handle, NITER, energy.data_ptr())
            B.mk_fetch_fields(plan.handle, 0, N.MK_F_G, Gout.data_ptr(), Gout.numel() * 4, False)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * F * args.steps / el, "unit": "focal points/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * el / args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        out, cores, sample = run_cpu_oracle(args.nfocal, reps=2)
        tcpu = min(out["times"])
        cpu = {"value": out["focal_per_rep"] / tcpu, "unit": "focal points/s", "cores": cores, "kind": "oracle",
               "sample": f"focal points {sample} of {F}, {NITER} iterations, FP64 NumPy oracle, best of 2, "
                         f"{cores} BLAS threads"}

    plan.close()
    if rank == 0:
        line = {
            "metric": "focal points/sec to convergence (16 Neumann iterations)",
            "value": value, "unit": "focal points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(s, F) | {"parallelism": f"focal-point replicas x{world}"},
            "roofline": roofline, "synthesis": synthesis, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(st["launches"]), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.cpu_worker is not None:
        cpu_worker(args.cpu_worker)
        return
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
