"""The committed benchmark record (profiles/bench_sweep.json, one line of `python bench.py`
on one GPU) checked on the CPU: it carries every key of the output contract, and its
derived figures follow from its own measured ones and from the workload's shapes, so a
hand edit or a stale record fails here."""
import json
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads  # noqa: E402

REJECTED_CLOCK_REASONS = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}


@pytest.fixture(scope="module")
def rec():
    with open(os.path.join(ROOT, "profiles", "bench_sweep.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def wl():
    return workloads.workload(bench.WORKLOAD)


def test_contract_keys(rec):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in rec, k
    assert rec["metric"] == "whitened injections/sec" and rec["unit"] == "injections/s"
    assert rec["higher_is_better"] is True and rec["scaling"] == "weak"
    assert rec["warmup"] >= 3 and rec["steps"] >= 1 and rec["gpu_launches"] > 0
    assert rec["data"].startswith("synthetic") and rec["dtype"] == "f32"
    assert set(rec["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert set(rec["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert set(rec["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert set(rec["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}


def test_clocks_were_not_throttled(rec):
    assert not REJECTED_CLOCK_REASONS & set(rec["clocks"]["reasons"])
    assert rec["clocks"]["sm_mhz"] >= 0.9 * rec["clocks"]["sm_max_mhz"]


def test_value_follows_from_the_step_time(rec, wl):
    assert rec["config"]["global_batch"] == wl["B"] and rec["config"]["seq_len"] == wl["N"]
    assert rec["config"]["workload"].startswith(bench.WORKLOAD + ":")
    expect = rec["n_gpus"] * wl["B"] / (rec["ms_per_step"] * 1e-3)
    assert math.isclose(rec["value"], expect, rel_tol=1e-9)


def test_roofline_arithmetic(rec, wl):
    r = rec["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["flops_per_injection"] == bench.flops_per_injection(wl)
    assert r["injections_per_launch"] == wl["B"]
    achieved = r["flops_per_injection"] * r["injections_per_launch"] / (r["avg_launch_ms"] * 1e-3) / 1e12
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-9)
    # the derived FP32 peak: SMs x 128 lanes x 2 flop x the maximum SM clock
    peak = r["sm_count"] * bench.FP32_LANES_PER_SM * 2 * rec["clocks"]["sm_max_mhz"] * 1e6 / 1e12
    assert math.isclose(r["peak"], peak, rel_tol=1e-9)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-9)
    # the fused call is part of the step
    assert r["avg_launch_ms"] <= rec["ms_per_step"]
    assert r["algorithmic_bytes_per_launch"] == wl["B"] * len(wl["dets"]) * wl["N"] * 4


def test_traffic_is_the_tables_for_the_recorded_kernel(rec, wl):
    t = rec["roofline"]["traffic"]
    if t is not None:
        entry = bench.TRAFFIC[wl["name"]]
        assert t == entry["bytes_per_launch"] and entry["B"] == wl["B"]
        # no re-reads: within a few percent of the output bytes
        assert 0.95 <= t / rec["roofline"]["algorithmic_bytes_per_launch"] <= 1.05


def test_end_to_end_bytes(rec, wl):
    e = rec["e2e"]
    B, D, N, L = wl["B"], len(wl["dets"]), wl["N"], wl["L"]
    assert e["h2d_bytes_per_step"] == D * L * 4                       # the background strain
    assert e["d2h_bytes_per_step"] == B * D * N * 4 + 11 * B * 8 + B * 8   # strain, parameters, offsets
    assert e["value"] < rec["value"]
    if "d2h_link_gbs" in e:
        # bytes per step x steps per second (value / B)
        assert math.isclose(e["d2h_gbs"], e["d2h_bytes_per_step"] * e["value"] / wl["B"] / 1e9, rel_tol=1e-6)
        assert math.isclose(e["d2h_frac_of_link"], e["d2h_gbs"] / e["d2h_link_gbs"], rel_tol=1e-9)


def test_marginal_likelihood_leg_arithmetic(rec):
    """u inverse transforms of n = N/2 points per sample at 5 n log2 n flops each (the
    two-detector workload: N = 2048, u = 16), and the achieved rate from the call time."""
    t = rec["log_likelihood_tmarg"]
    r = t["roofline"]
    n, u = 1024, t["grid"]["oversample"]
    assert r["flops_per_sample"] == u * 5 * n * int(math.log2(n))
    assert math.isclose(t["samples_per_s"], t["samples"] / (t["ms_per_call"] * 1e-3), rel_tol=1e-9)
    assert math.isclose(r["achieved"], r["flops_per_sample"] * t["samples_per_s"] / 1e12, rel_tol=1e-9)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-9)
    assert math.isclose(r["peak"], rec["roofline"]["peak"], rel_tol=1e-9)


def test_gemm_leg_arithmetic(rec):
    """The 8192^3 bf16 product: 2 M N K flops over the measured time, for both arms, and
    the fraction of the measured bf16 peak."""
    g = rec["gemm_bf16"]
    flops = 2.0 * 8192 ** 3
    assert math.isclose(g["tflops"], flops / (g["ms"] * 1e-3) / 1e12, rel_tol=1e-9)
    assert math.isclose(g["cublas_tflops"], flops / (g["cublas_ms"] * 1e-3) / 1e12, rel_tol=1e-9)
    r = g["roofline"]
    assert r["bound"] == "tensor" and math.isclose(r["achieved"], g["tflops"], rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-9)


def test_four_second_window_leg_arithmetic(rec):
    """The 4 s-window workload (three detectors, N = 8192, 2048 draws per step): rate from
    the step time, the flop model of its shapes and the roofline fraction."""
    h = rec["hl3"]
    wl = workloads.workload("hl3")
    r = h["roofline"]
    assert math.isclose(h["injections_per_s"], wl["B"] / (h["ms_per_step"] * 1e-3), rel_tol=1e-9)
    assert r["flops_per_injection"] == bench.flops_per_injection(wl) and r["injections_per_launch"] == wl["B"]
    achieved = r["flops_per_injection"] * wl["B"] / (r["avg_launch_ms"] * 1e-3) / 1e12
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-9)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"], rel_tol=1e-9)
    assert r["algorithmic_bytes_per_launch"] == wl["B"] * len(wl["dets"]) * wl["N"] * 4
