"""Host logic of bench.py (no GPU): roofline arithmetic, peaks, traffic lookup, workloads."""

import hashlib
import importlib.util
import json
import os

import pytest

import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_headline_roofline_is_hbm_with_algorithmic_bytes(bench):
    s = S.paper_small_survey(1)
    r = bench.roofline_for(s, 1, "c64", 0.2)
    b = s.nw * s.n * s.n * 8 + 2 * s.nw * s.n * 8   # R read once, Nw in, S out
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["algorithmic_bytes_per_launch"] == b
    assert r["achieved"] == pytest.approx(b / 0.2e-3 / 1e9)
    peaks, _ = bench.measured_peaks()
    assert r["frac"] == pytest.approx(r["achieved"] / peaks["hbm_gbs"])


def test_binding_bound_per_form(bench):
    # F = 64: the 16-bit forms move more bytes per flop than the tensor pipe needs (HBM-bound);
    # F = 601: the 3-way split is tensor-bound; complex FP32 with F > 1 is ALU-bound
    small, prec = S.paper_small_survey(64), S.precision_survey()
    assert bench.lower_bound_ms(small, 64, "split3")[0] == "hbm"
    assert bench.lower_bound_ms(small, 64, "cbf16")[0] == "hbm"
    assert bench.lower_bound_ms(prec, 601, "split3")[0] == "tensor"
    assert bench.lower_bound_ms(small, 64, "c64")[0] == "alu"
    # the reported roof equals the larger lower bound
    r = bench.roofline_for(prec, 601, "split3", 3.5)
    lb = r["lower_bounds_ms"]
    assert r["bound"] == max(lb, key=lb.get)
    assert r["frac"] == pytest.approx(max(lb.values()) / 3.5)


def test_lower_bound_scales_with_work(bench):
    # flops scale with F, R bytes do not: doubling F at most doubles the bound
    s64, s128 = S.large_survey(nfocal=64), S.large_survey(nfocal=128)
    a = bench.lower_bound_ms(s64, 64, "split3")[1]
    b = bench.lower_bound_ms(s128, 128, "split3")[1]
    assert a < b <= 2 * a + 1e-9


def test_measured_peaks_file(bench):
    peaks, kind = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured"
        assert peaks["hbm_gbs"] == json.load(open(path))["hbm_gbs"]
    else:
        assert kind == "fallback"
    for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
        assert peaks[k] > 0


def test_traffic_only_for_the_profiled_source(bench):
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, e in d.items():
        src = os.path.join(ROOT, "paper_2106_04649_gb300", "csrc", e["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        got = bench.profiled_traffic(key)
        assert got == (e["dram_bytes_per_launch"] if h == e["source_sha256_16"] else None)
        if got is not None:  # the DRAM bytes of a profiled launch cover at least R once
            s = S.paper_small_survey(1)
            assert got >= s.nw * s.n * s.n * 8
    assert bench.profiled_traffic("no-such-workload") is None


def test_workload_config_names_the_workload(bench):
    s = S.paper_small_survey(1)
    c = bench.workload_config(s, 1, "c64")
    assert "paper-small" in c["workload"] and c["nfocal"] == 1 and c["nw"] == s.nw
    assert "model" not in c
