"""Host logic of bench.py that needs no GPU: the clock record, the per-step
statistics, the reference arm's JSON line, and the projected oracle baseline
of the batched workload."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sampler_with(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_under_load_and_reasons():
    # clocks.sm, clocks.max.sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["345, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # idle sample
             "2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line"]
    s = sampler_with(lines).summary()
    assert s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["sm_mhz"] == 2055.0  # median of the samples under load (the idle 345 MHz one left out)
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown():
    lines = ["1500, 2070, 1300.0, 0x48, Active, Not Active, Active, Not Active"]
    assert sampler_with(lines).summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert sampler_with([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_reference_arm_json_line():
    """`bench.py --impl reference` on the 64^3 workload: one JSON line with the
    contract's keys, the oracle as the CPU baseline, no host copies."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "sweep64", "--steps", "1",
                        "--warmup", "0", "--cpu-sweeps", "2"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"]


def test_batched_baseline_projection():
    """The projected oracle rate is count / (sum of points x sweeps / measured
    sweep rate): twice the sweeps halve it."""
    sizes, seeds = bench.batch_problems(16)
    pts = np.array([a * b * c for a, b, c in sizes], dtype=float)
    iters = np.full(len(sizes), 100.0)
    one = bench.cpu_sample_batched(sizes, seeds, pts, iters, n_sample=2, sweeps=3)
    assert one["unit"] == "solves/s" and one["kind"] == "oracle" and one["value"] > 0
    rate = float(one["sample"].split("sweep rate ")[1].split(" GLUP/s")[0]) * 1e9
    assert abs(one["value"] - len(sizes) / ((pts * iters).sum() / rate)) <= 0.01 * one["value"]


def test_step_stats():
    class Ev:
        def __init__(self, t):
            self.t = t

        def elapsed_time(self, other):
            return other.t - self.t

    st = bench.step_stats([Ev(0.0), Ev(2.0), Ev(5.0), Ev(6.0)])
    assert st["n"] == 3 and st["min"] == 1.0 and st["median"] == 2.0 and abs(st["mean"] - 2.0) < 1e-12


def test_all_cores_baseline_is_the_oracles_sample_bitwise():
    """The bench's all-cores figure runs the oracle baseline's own sample
    (same seeded grid, sweeps and norm) through the multi-core host library:
    the result must be the oracle's bits, and float workloads get none."""
    wl = {"nx": 40, "ny": 33, "nz": 27, "r": 1, "dtype": "f64", "seed": 2}
    base, ref_out, ref_norm = bench.cpu_baseline(wl, 5, keep=True)
    assert base["kind"] == "oracle" and base["cores"] == 1 and base["value"] > 0
    d = bench.cpu_all_cores(wl, 5, ref_out, ref_norm)
    assert d["bitwise_oracle"] is True and d["norm_rel_diff_oracle"] <= 40 * 33 * 27 * 2.0 ** -53
    assert d["cores"] >= 1 and d["value"] > 0 and d["unit"] == "GLUP/s"
    assert bench.cpu_all_cores(dict(wl, dtype="f32"), 5) is None
    # both go into the bench's JSON line as they are
    line = json.loads(json.dumps({"cpu_baseline": base, "cpu_all_cores": d}))
    assert line["cpu_all_cores"]["bitwise_oracle"] is True


import pytest  # noqa: E402


@pytest.mark.parametrize("workload,extra", [("jacobi2d", ["--cpu-sweeps2d", "20"]), ("advect", [])])
def test_other_reference_arms(workload, extra):
    """The 2-D jacobi and advection reference arms: the oracle on a bounded
    sample, one JSON line with the contract's keys."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "1",
                        "--warmup", "0", *extra], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["workload"]


@pytest.mark.parametrize("workload", ["batch", "serve", "varcoef"])
def test_reference_arms_that_cannot_run_say_why(workload):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert d["impl"] == "reference" and "oracle" in d["unavailable"]


def test_lindley_single_server_fifo():
    """The plain per-request path serves one request at a time in arrival
    order: start = max(arrival, previous finish)."""
    import bench
    assert bench.lindley([0.0, 0.0, 0.0], [1.0, 2.0, 3.0]) == [1.0, 3.0, 6.0]   # all at once: queue
    assert bench.lindley([0.0, 10.0, 11.0], [1.0, 1.0, 1.0]) == [1.0, 1.0, 1.0]  # idle between arrivals
    assert bench.lindley([0.0, 0.5, 4.0], [1.0, 1.0, 1.0]) == [1.0, 1.5, 1.0]
    assert bench.lindley([], []) == []


def test_roofline_helpers():
    """The variable-coefficient line's HBM roofline (16 compulsory bytes per
    update; traffic scaled from the 512 x 512 x 256 ncu capture) and the
    FP64-pipe fraction used by the FP64 lines: achieved / peak, with the
    peak derived from 2 double ops per clock per SM on 152 SMs."""
    import bench
    fs = {"f32_sweep_hbm_gbs": 4800.0, "f32_sweep_ms": 0.75}
    r = bench.varcoef_roofline(fs)
    peaks, _ = bench.load_peaks()
    assert r["bound"] == "hbm" and r["achieved"] == 4800.0 and r["peak"] == float(peaks["hbm_gbs"])
    assert abs(r["frac"] - 4800.0 / float(peaks["hbm_gbs"])) < 1e-12
    assert abs(r["traffic"] / (768 * 768 * 384) - (837.3e6 + 250.5e6) / (512 * 512 * 256)) < 1e-9
    p = bench.fp64_pipe(6.0 * 1e9, 10.0, {"sm_max_mhz": 2070.0}, "x")
    assert abs(p["fp64_pipe_peak_tops"] - 2 * 152 * 2070e6 / 1e12) < 1e-12
    assert abs(p["fp64_pipe_achieved_tops"] - 6e9 / 10e-3 / 1e12) < 1e-12
    assert abs(p["fp64_pipe_frac"] - p["fp64_pipe_achieved_tops"] / p["fp64_pipe_peak_tops"]) < 1e-15
