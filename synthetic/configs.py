"""The five seeded workloads of the benchmark, as ``Survey`` objects.

Readings where the workload statement is silent (each is listed with its
reason in the design notes):

* tiny: half-space below 800 m at 3000 m/s; full band (0 .. nt/2); eps = 12 ms.
* paper-small: 10 interfaces (11 velocities) from ``random_model(1, 10)``;
  jitter seed 1; f0 = 25 Hz; band to 60 Hz; eps = 12 ms; one focal point at
  (3000 m, 1200 m) or 64 on the central-80% line at z = 1200 m.
* precision: the paper-small survey with one focal point per surface position
  at z = 1200 m.
* batching: survey s (0..11) draws its size from SplitMix64(10 + s) in the
  order n, nt, dt, interface count, F; its model is ``random_model(1010 + s)``.
* large: 4001 positions at dx = 5 m, nt = 4096, the paper-small model.
* every random-model survey calibrates R (``calibrate=0.9``, see
  ``amplitude_scale``) so that its Neumann series converges; the tiny fixed
  model is left as stated, its series converges as it is.
"""

from __future__ import annotations

import math

import numpy as np

from .layered import SplitMix64, Survey, fixed_model, focal_line, random_model


def tiny_survey() -> Survey:
    model = fixed_model([300.0, 500.0, 800.0], [1800.0, 2200.0, 2600.0], 3000.0)
    return Survey("tiny", n=101, dx=10.0, nt=512, dt=0.004, f0=30.0, fmax_hz=None,
                  model=model, seed=0, eps=0.012, focal=np.array([[500.0, 650.0]]))


def paper_small_survey(nfocal: int = 1) -> Survey:
    model = random_model(1, 10)
    if nfocal == 1:
        focal = np.array([[3000.0, 1200.0]])
    elif nfocal == 601:
        focal = focal_line(601, 10.0, 601, 1200.0, mode="every")
    else:
        focal = focal_line(601, 10.0, nfocal, 1200.0)
    return Survey(f"paper-small-F{nfocal}", n=601, dx=10.0, nt=2048, dt=0.004, f0=25.0,
                  fmax_hz=60.0, model=model, seed=1, eps=0.012, focal=focal, calibrate=0.9)


def precision_survey() -> Survey:
    s = paper_small_survey(601)
    s.name = "precision-F601"
    return s


def batching_surveys() -> list[Survey]:
    out = []
    for s in range(12):
        g = SplitMix64(10 + s)
        n = 201 + int(math.floor(g.uniform(0.0, 1.0) * 1001))
        nt = (1024, 2048, 4096)[int(g.uniform(0.0, 3.0))]
        dt = (0.002, 0.003, 0.004)[int(g.uniform(0.0, 3.0))]
        nif = 5 + int(math.floor(g.uniform(0.0, 11.0)))
        F = int(round(math.exp(g.uniform(0.0, math.log(256.0)))))
        if s == 0:
            n, F = 201, 1
        if s == 11:
            n, F = 1201, 256
        F = max(1, min(256, F))
        model = random_model(1010 + s, nif)
        focal = np.array([[(n - 1) * 10.0 / 2, 1200.0]]) if F == 1 else focal_line(n, 10.0, F, 1200.0)
        out.append(Survey(f"batch-{s}", n=n, dx=10.0, nt=nt, dt=dt, f0=25.0, fmax_hz=60.0,
                          model=model, seed=10 + s, eps=0.012, focal=focal, calibrate=0.9,
                          meta={"rprec": "c64" if s % 2 == 0 else "split_bf16"}))
    return out


def large_survey(nfocal: int = 4001) -> Survey:
    model = random_model(1, 10)
    focal = focal_line(4001, 5.0, 4001, 1200.0, mode="every") if nfocal == 4001 else \
        focal_line(4001, 5.0, nfocal, 1200.0)
    return Survey(f"large-F{nfocal}", n=4001, dx=5.0, nt=4096, dt=0.004, f0=25.0,
                  fmax_hz=60.0, model=model, seed=1, eps=0.012, focal=focal, calibrate=0.9)
