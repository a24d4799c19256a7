#!/usr/bin/env python3
"""Benchmark of the 3D Jacobi stencil path on GB300 (one JSON line on stdout).

Workload (default, `--workload sweep512`): the 7-point FP64 Jacobi sweep on a
512x512x512 interior (Fortran layout, 1-cell zero Dirichlet halo, interior
U[0,1) from PCG64 seed 2, coefficients {0, 1/6}); one STEP is the whole job of
that configuration: 1000 sweeps (stencil_sweep_f64) followed by the fused
residual-norm reduction of the result (residual_norm_f64).  GLUP/s counts the
1000 sweeps only.  Each array is 1 GiB (> 129 MB of L2), so no flush is needed
between steps.  The paper's own jacobi benchmark (arXiv 2409.18824 Sec. 4) is
a 2D 1024^2 CPU run; its data are not published and this seeded grid stands in
for it.

Arms:
  default            the CUDA library through its C ABI, device-resident grids;
                     `e2e` repeats the step with pinned HOST grids (the library
                     stages them: H2D + D2H inside the timed region).
  --impl reference   the CPU oracle as it stands, on the host cores, each step
                     a bounded sample of the same workload (see `sample`).

Multi-GPU: the path does not shard (one grid per GPU, no exchange), so with
torchrun each rank runs an independent replica; value = all ranks' updates /
the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import stencil_inputs as si  # noqa: E402

WORKLOADS = {
    # name: (nx, ny, nz, r, sweeps, dtype, seed)
    "sweep512": dict(nx=512, ny=512, nz=512, r=1, sweeps=1000, dtype="f64", seed=2,
                     desc="7-point Jacobi, 512^3 FP64, zero halo, interior U[0,1) seed 2, "
                          "1000 sweeps + residual L2 norm"),
    "sweep64": dict(nx=64, ny=64, nz=64, r=1, sweeps=100, dtype="f64", seed=1,
                    desc="7-point Jacobi, 64^3 FP64, zero halo, interior U[0,1) seed 1, "
                         "100 sweeps + residual L2 norm"),
    "sweep320": dict(nx=320, ny=320, nz=320, r=1, sweeps=100, dtype="f64", seed=2,
                     desc="7-point Jacobi, 320^3 FP64 (268 MB per grid, profiling size), 100 sweeps"),
    "sweep320f32": dict(nx=320, ny=320, nz=320, r=1, sweeps=100, dtype="f32", seed=2,
                        desc="7-point Jacobi, 320^3 FP32 (134 MB per grid, profiling size), 100 sweeps"),
    "sweep512f32": dict(nx=512, ny=512, nz=512, r=1, sweeps=1000, dtype="f32", seed=2,
                        desc="7-point Jacobi, 512^3 FP32, zero halo, interior U[0,1) seed 2, "
                             "1000 sweeps + residual L2 norm"),
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes per lattice update of the default kernels, from one ncu capture
# each (dram__bytes_read.sum + dram__bytes_write.sum of a 320^3 launch divided
# by its 32.8 M updates; summaries under profiles/).  Set to None whenever the
# kernel changes until it is captured again.
TRAFFIC_BYTES_PER_LUP = {
    ("f64", 0): (271.3e6 + 220.2e6) / 320 ** 3,  # plane kernel (star_kernel<double,1>, 16-plane chunks)
    ("f32", 1): (143.0e6 + 82.2e6) / 320 ** 3,  # column kernel (star_col_kernel<float,1>, 2 planes prefetched)
    ("f32", 3): (151.5e6 + 81.4e6) / 320 ** 3,  # staged kernel (star_staged_kernel<float,1>, 152 blocks)
    ("f32", -1): (151.5e6 + 81.4e6) / 320 ** 3,  # automatic: the staged kernel for these large float grids
}

# DRAM bytes (read + write) of the other timed kernels, from their ncu
# captures, per unit the launch processes: the 2-D resident launch (1024^2,
# bulk-copy build), the dot product per element pair and the sum per element
# (2^27 elements), the self-advection per cell (512 x 512 x 256), and the
# variable-coefficient float sweep per update (512 x 512 x 256)
TRAFFIC_J2D_LAUNCH = 8.44e6 + 6.7e3
TRAFFIC_DOT_PER_PAIR = (2.1476e9 + 2.9e6) / 2 ** 27
TRAFFIC_SUM_PER_ELEMENT = (1.0738e9 + 3.1e6) / 2 ** 27
TRAFFIC_ADVECT_PER_CELL = (1.733e9 + 1.575e9) / (512 * 512 * 256)
TRAFFIC_VARCOEF_F32_PER_LUP = (837.3e6 + 250.5e6) / (512 * 512 * 256)  # var_tma_kernel

# FP64 issue rate of this GPU measured with a throughput probe: 2 double
# fused-multiply-add instructions per clock per SM (every double add and
# multiply of the sweep is issued as one), 152 SMs.
FP64_OPS_PER_CLK_SM = 2.0
N_SM = 152


def fp64_pipe(ops, kern_ms, peaks, what):
    """The FP64-pipe fraction of a kernel whose roofline is HBM but whose double
    operations cap it first: ops / kernel time against 2 FP64 instructions per
    clock per SM (measured with a throughput probe) x 152 SMs x the maximum SM
    clock."""
    sm_clock = float(peaks.get("sm_max_mhz", 2070.0))
    peak = FP64_OPS_PER_CLK_SM * N_SM * sm_clock * 1e6 / 1e12  # Tops/s
    achieved = ops / (kern_ms * 1e-3) / 1e12
    return {"fp64_pipe_achieved_tops": achieved, "fp64_pipe_peak_tops": peak,
            "fp64_pipe_frac": achieved / peak,
            "fp64_pipe_peak_kind": f"derived: {FP64_OPS_PER_CLK_SM:g} FP64 ops/clk/SM (measured probe) x "
                                   f"{N_SM} SMs x {sm_clock:g} MHz; {what}"}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [v for v in sm if v > 0.5 * (mx or max(sm))] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_info():
    """CPU model and core count of the machine running the benchmark."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
                if k == "cpu part" and model is None:
                    model = "arm cpu part " + ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return {"cpu": model or platform.machine(), "cores": os.cpu_count()}


def step_stats(events):
    """Per-step times (ms) from consecutive CUDA events: median, mean, min."""
    ts = [a.elapsed_time(b) for a, b in zip(events[:-1], events[1:])]
    return {"median": statistics.median(ts), "mean": statistics.fmean(ts), "min": min(ts), "n": len(ts)}


def max_over_ranks(ms, device):
    """The job's time: the slowest rank's (an all-reduce MAX over the process
    group; the local value when there is no group or only one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- CUDA arm --
def run_cuda(args, wl):
    import torch
    import paper_2409_18824_gb300 as stn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    nx, ny, nz, r, sweeps = wl["nx"], wl["ny"], wl["nz"], wl["r"], wl["sweeps"]
    f64 = wl["dtype"] == "f64"
    npdt = np.float64 if f64 else np.float32
    esize = 8 if f64 else 4
    coeffs = si.LAPLACE7
    u0 = si.uniform_interior(nx, ny, nz, r, seed=wl["seed"] + rank, dtype=npdt)
    d_in = torch.from_numpy(u0).to(dev)
    d_out = d_in.clone()
    sweep = stn.stencil_sweep_f64 if f64 else stn.stencil_sweep_f32
    resid = stn.residual_norm_f64 if f64 else stn.residual_norm_f32
    apply_ = stn.stencil_apply_f64 if f64 else stn.stencil_apply_f32
    stream = torch.cuda.current_stream(dev)
    stn.stencil_tune_set("star_variant", args.variant)
    stn.stencil_tune_set("temporal_depth", args.temporal)
    stn.stencil_tune_set("star_chunks", args.chunks)
    tuned = None
    if args.autotune:
        # before any timing: the autotuner times the candidate plans for these
        # extents and caches the fastest, which the sweeps below then use
        e = stn.stencil_autotune_sweep(nx, ny, nz, esize, r, coeffs, 24, stream=stream)
        tuned = {k: e[k] for k in ("variant", "chunks", "depth", "glups", "default_glups")}
        d_in.copy_(torch.from_numpy(u0).to(dev))

    if args.kernel_only:
        # a few launches of the dominant kernel alone (for profilers)
        for i in range(args.kernel_only):
            if i % 2 == 0:
                apply_(d_in, d_out, coeffs, r)
            else:
                apply_(d_out, d_in, coeffs, r)
        torch.cuda.synchronize(dev)
        return

    def step():
        sweep(d_in, d_out, coeffs, r, sweeps)
        return resid(d_out, coeffs, r)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    norms = []
    with ClockSampler(local) as clk:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        t_wall0 = time.perf_counter()
        evs[0].record(stream)
        for i in range(args.steps):
            norms.append(step())
            evs[i + 1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    e0, e1 = evs[0], evs[-1]
    ms = e0.elapsed_time(e1)
    per_step = step_stats(evs)
    ms = max_over_ranks(ms, dev)
    lups_rank = float(nx) * ny * nz * sweeps * args.steps
    value = lups_rank * ws / (ms * 1e-3) / 1e9

    # Dominant kernel alone: back-to-back single-sweep launches (stencil_apply,
    # one kernel each) between two events on the launching stream.
    n_apply = 20 if f64 else 60
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        apply_(d_in, d_out, coeffs, r)
    torch.cuda.synchronize(dev)
    a0.record(stream)
    for i in range(n_apply):
        if i % 2 == 0:
            apply_(d_in, d_out, coeffs, r)
        else:
            apply_(d_out, d_in, coeffs, r)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    kern_ms = a0.elapsed_time(a1) / n_apply

    # the same kernel's share inside the timed region
    step_ms = ms / args.steps
    launch_ms_in_step = step_ms / (sweeps + 1)

    # e2e through the C ABI with pinned host grids
    h_in = torch.from_numpy(u0).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    hin_np, hout_np = h_in.numpy(), h_out.numpy()
    sweep(hin_np, hout_np, coeffs, r, sweeps)  # warm the staging path
    resid(hout_np, coeffs, r)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sweep(hin_np, hout_np, coeffs, r, sweeps)
        resid(hout_np, coeffs, r)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    grid_bytes = u0.nbytes
    h2d = grid_bytes * 2        # in for the sweeps, out for the norm
    d2h = grid_bytes * 2 + 8    # out, clobbered in, and the norm
    e2e_val = float(nx) * ny * nz * sweeps / e2e_s / 1e9

    peaks, peak_kind = load_peaks()
    clocks = clk.summary()
    lups_kernel = float(nx) * ny * nz
    bytes_alg = 2.0 * esize * lups_kernel           # read u, write out: compulsory traffic
    tkey = (wl["dtype"], 0 if (f64 and args.variant in (-1, 0)) else (-1 if args.variant == -1 else args.variant))
    tpl = TRAFFIC_BYTES_PER_LUP.get(tkey)
    plan_is_default = tuned is None or tuned["glups"] == tuned["default_glups"]
    traffic = (tpl * lups_kernel if (tpl is not None and args.temporal in (0, 1) and args.chunks == 0
                                     and plan_is_default) else None)
    hbm_gbs = bytes_alg / (kern_ms * 1e-3) / 1e9
    hbm_peak = float(peaks["hbm_gbs"])
    if f64:
        # The roofline of this workload is HBM (16 B per update, compulsory);
        # the FP64 pipe caps the double sweep first (6 double ops per update
        # at 2 per clock per SM), so its fraction is given beside it.
        roofline = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_gbs / hbm_peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                    "peak_kind": peak_kind, "kernel_ms": kern_ms, "kernel_ms_in_step": launch_ms_in_step}
        roofline.update(fp64_pipe(6.0 * lups_kernel, kern_ms, peaks, "6 double ops per update"))
    else:
        roofline = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_gbs / hbm_peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                    "peak_kind": peak_kind,
                    "kernel_ms": kern_ms, "kernel_ms_in_step": launch_ms_in_step}

    out = {
        "metric": "GLUP/s (512^3 7-point Jacobi, FP64)" if wl is WORKLOADS["sweep512"] else f"GLUP/s ({args.workload})",
        "value": value,
        "unit": "GLUP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": wl["dtype"],
        "data": "synthetic",
        "config": {"workload": wl["desc"], "nx": nx, "ny": ny, "nz": nz, "radius": r,
                   "sweeps_per_step": sweeps, "kernel_variant": args.variant,
                   "temporal_depth": args.temporal, "k_chunks": args.chunks, "autotuned": tuned,
                   "l2": (f"inputs larger than L2 ({u0.nbytes / 2**30:.2f} GiB per grid), no flush"
                          if u0.nbytes > 129e6 else
                          f"grid of {u0.nbytes / 1e6:.1f} MB stays in L2 across sweeps (as in the solve), no flush"),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "e2e": {"value": e2e_val, "unit": "GLUP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * (1 + sweeps + 2),
        "roofline": roofline,
        "clocks": clocks,
        "wall_s_timed": t_wall,
        "step_ms": per_step,
        "host": host_info(),
        "residual_norm": norms[-1],
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            base, ref_out, ref_norm = cpu_baseline(wl, args.cpu_sweeps, keep=True)
            out["cpu_baseline"] = base
            try:
                allc = cpu_all_cores(wl, args.cpu_sweeps, ref_out, ref_norm)
            except Exception as e:  # context only: never costs the line
                allc = {"error": f"{type(e).__name__}: {e}"}
            if allc is not None:
                out["cpu_all_cores"] = allc
            del ref_out
        if ws == 1 and wl is WORKLOADS["sweep512"] and not args.no_extras:
            try:
                out["fp64_double_word"] = double_word_variant(stn, dev, u0, d_in, d_out, peaks)
            except Exception as e:  # recorded, never costs the headline line
                out["fp64_double_word"] = {"error": f"{type(e).__name__}: {e}"}
            del d_in, d_out
            torch.cuda.empty_cache()
            out.update(run_extras(args, dev))
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------- the paper's 2-D jacobi run ----
JACOBI2D = dict(nx=1024, ny=1024, r=1, sweeps=100000, seed=7,
                desc="the paper's jacobi benchmark: 2-D 5-point Laplace Jacobi, 1024 x 1024 FP64, "
                     "c = {0, 1/4}, zero halo, interior U[0,1) seed 7, 100000 iterations + residual L2 norm")
# The paper's runtime for exactly this run with its MLIR flow (Table 2: 249.08 s, one
# core of an AMD EPYC 7742; the precision is not stated), as GLUP/s.
PAPER_JACOBI2D_GLUPS = 1024 * 1024 * 100000 / 249.08 / 1e9


def cpu_sample2d(sweeps):
    import oracle
    w = JACOBI2D
    u0 = si.uniform_interior2d(w["nx"], w["ny"], w["r"], seed=w["seed"])
    oracle.build()
    t0 = time.perf_counter()
    out = oracle.stencil_sweep2d(u0, si.LAPLACE5, w["r"], sweeps)
    oracle.residual_norm2d(out, si.LAPLACE5, w["r"])
    t = time.perf_counter() - t0
    return float(w["nx"]) * w["ny"] * sweeps / t / 1e9, t


def run_jacobi2d(args):
    """The paper's jacobi run (Sec. 4, Tables 1-2): 100000 sweeps of a 1024^2
    grid held in the SMs' shared memory, then its residual norm."""
    import torch
    import paper_2409_18824_gb300 as stn

    w = JACOBI2D
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nx, ny, r = w["nx"], w["ny"], w["r"]
    sweeps = args.sweeps2d or w["sweeps"]
    c = si.LAPLACE5
    u0 = si.uniform_interior2d(nx, ny, r, seed=w["seed"] + rank)
    d_in = torch.from_numpy(u0).to(dev)
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream(dev)
    chunk = stn.stencil_tune_get("sweep2d_chunk")

    def step():
        stn.stencil_sweep2d_f64(d_in, d_out, c, r, sweeps)
        return stn.residual_norm2d_f64(d_out, c, r)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    norms = []
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            norms.append(step())
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dev)
    lups = float(nx) * ny * sweeps
    value = lups * args.steps * ws / (ms * 1e-3) / 1e9

    # the resident kernel alone: one launch of min(sweeps, chunk) sweeps
    k_sweeps = min(sweeps, chunk)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    stn.stencil_sweep2d_f64(d_in, d_out, c, r, k_sweeps)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    kern_ms = a0.elapsed_time(a1)
    launches_per_step = -(-sweeps // chunk) + 2  # resident launches + residual + finalize

    # e2e through the C ABI with pinned host grids
    h_in = torch.from_numpy(u0).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    hin_np, hout_np = h_in.numpy(), h_out.numpy()
    e2e_steps = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        stn.stencil_sweep2d_f64(hin_np, hout_np, c, r, sweeps)
        stn.residual_norm2d_f64(hout_np, c, r)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    ops = 4.0 * float(nx) * ny * k_sweeps  # 3 adds + 1 multiply per update
    sm_clock = float(load_peaks()[0].get("sm_max_mhz", 2070.0))
    fp64_peak = FP64_OPS_PER_CLK_SM * N_SM * sm_clock * 1e6 / 1e12
    achieved = ops / (kern_ms * 1e-3) / 1e12
    out = {
        "metric": "GLUP/s (the paper's 2-D jacobi: 1024^2, 100000 iterations, FP64)",
        "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_JACOBI2D_GLUPS if sweeps == w["sweeps"] else None,
        "vs_baseline_note": "against the paper's own runtime for this run (Table 2, MLIR flow: 249.08 s on "
                            "one EPYC 7742 core); other hardware, context only",
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "nx": nx, "ny": ny, "radius": r, "sweeps_per_step": sweeps,
                   "resident_launch_sweeps": chunk, "l2": "8 MB grid held in shared memory; HBM touched "
                   "once per launch", "parallelism": "replicas" if ws > 1 else "single"},
        "seconds_per_run": ms / args.steps / 1e3,
        "paper_seconds": {"mlir_flow_1core": 249.08, "flang_v20_1core": 277.67, "cray_1core": 109.89,
                          "gnu_1core": 232.62},
        "e2e": {"value": lups / e2e_s / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": 2 * u0.nbytes,
                "d2h_bytes_per_step": u0.nbytes + 8},
        "gpu_launches": args.steps * launches_per_step,
        # DRAM bytes of one resident launch (ncu on this grid, the bulk-copy build):
        # the grid read once (8.44 MB) and 6.7 KB written before the kernel ends
        # (the rest leaves L2 later)
        # The grid stays in shared memory for the whole launch, so HBM is touched
        # once per launch (16 B per point) and bounds nothing: the bound is the
        # FP64 pipe (4 double ops per update)
        "roofline": {"bound": "alu", "alu": "FP64 pipe (grid resident in shared memory; no HBM traffic per sweep)",
                     "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": TRAFFIC_J2D_LAUNCH, "traffic_unit": "bytes per launch",
                     "peak_kind": "derived: 2 FP64 FMA-pipe ops/clk/SM (measured probe) x 152 SMs x max SM clock",
                     "kernel": "j2d_resident_kernel<double,1>", "kernel_ms": kern_ms,
                     "kernel_sweeps": k_sweeps},
        "clocks": clk.summary(),
        "host": host_info(),
        "residual_norm": norms[-1],
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            k = args.cpu_sweeps2d
            val, t = cpu_sample2d(k)
            out["cpu_baseline"] = {"value": val, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                                   "sample": f"{k} sweeps + 1 residual norm of the same 1024x1024 grid, "
                                             f"plain C oracle, single thread ({t:.1f} s)"}
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_reference2d(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    k = args.cpu_sweeps2d
    for _ in range(args.warmup):
        cpu_sample2d(1)
    times = [cpu_sample2d(k)[1] for _ in range(args.steps)]
    total = sum(times)
    value = float(JACOBI2D["nx"]) * JACOBI2D["ny"] * k * args.steps / total / 1e9
    print(json.dumps({
        "impl": "reference",
        "metric": "GLUP/s (the paper's 2-D jacobi: 1024^2, 100000 iterations, FP64)",
        "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_JACOBI2D_GLUPS, "dtype": "f64", "data": "synthetic",
        "config": {"workload": JACOBI2D["desc"], "nx": JACOBI2D["nx"], "ny": JACOBI2D["ny"], "radius": 1,
                   "sweeps_per_step": k, "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: {k} sweeps + 1 residual norm (plain C oracle, one thread) "
                                   f"instead of 100000"},
        "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host": host_info(),
    }), flush=True)


# ----------------------- the paper's threaded jacobi on the host cores ----
# Table 4 of the paper: speed-up over serial of its OpenMP jacobi (its MLIR
# flow) on 2..64 cores of its CPU.  Context for the host path's scaling.
PAPER_OPENMP_JACOBI_SPEEDUP = {2: 1.95, 4: 4.01, 8: 5.77, 16: 13.14, 32: 26.14, 64: 72.62}


def run_jacobi2d_host(args):
    """The multi-core host path (libstencil_host.so) on the paper's jacobi
    grid: K timed steps of `--host-sweeps` sweeps on every hardware thread,
    then the scaling curve over 1, 2, 4, ... threads (one timed run each)."""
    import paper_2409_18824_gb300.host as hp

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    nx, ny, sweeps = JACOBI2D["nx"], JACOBI2D["ny"], args.host_sweeps
    u0 = si.uniform_interior2d(nx, ny, 1, seed=JACOBI2D["seed"])
    a, out = u0.copy(), np.zeros_like(u0)
    tmax = hp.threads()

    def run(T, k):
        a[...] = u0
        t0 = time.perf_counter()
        hp.stencil_host_sweep2d_f64(a, out, si.LAPLACE5, 1, k, nthreads=T)
        norm = hp.stencil_host_residual_norm2d_f64(out, si.LAPLACE5, 1, nthreads=T)
        return time.perf_counter() - t0, norm

    for _ in range(args.warmup):
        run(tmax, max(1, sweeps // 10))
    times = [run(tmax, sweeps)[0] for _ in range(args.steps)]
    total = sum(times)
    value = float(nx) * ny * sweeps * args.steps / total / 1e9
    curve = {}
    for T in sorted({t for t in (1, 2, 4, 8, 16, 32, 64) if t <= tmax} | {tmax}):
        dt, _ = run(T, sweeps)
        curve[T] = float(nx) * ny * sweeps / dt / 1e9
    speedup = {T: curve[T] / curve[1] for T in curve}
    full_s = {T: float(nx) * ny * JACOBI2D["sweeps"] / (curve[T] * 1e9) for T in curve}
    print(json.dumps({
        "metric": "GLUP/s (the paper's 2-D jacobi, 1024^2 FP64, multi-core host path)",
        "value": value, "unit": "GLUP/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": JACOBI2D["desc"] + "; host threads, each step " + f"{sweeps} sweeps + 1 residual "
                               "norm instead of 100000", "nx": nx, "ny": ny, "radius": 1, "sweeps_per_step": sweeps,
                   "threads": tmax, "parallelism": "host threads (libstencil_host.so)"},
        "scaling_curve": {"glups": curve, "speedup": speedup,
                          "paper_table4_speedup": PAPER_OPENMP_JACOBI_SPEEDUP,
                          "projected_full_run_s": full_s,
                          "paper_serial_s": {"mlir_flow": 249.08, "cray": 109.89}},
        "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
        "host": host_info(),
    }), flush=True)


# Table 4 of the paper: its threaded pw-advection (MLIR flow), speed-up over serial.
PAPER_OPENMP_PW_SPEEDUP = {2: 1.81, 4: 3.34, 8: 5.52, 16: 8.04, 32: 9.77, 64: 10.80}


def run_advect_host(args):
    """The advection stand-in on the host cores (libstencil_host.so): u, v, w
    advecting themselves on a 512 x 256 x 256 block of the pw-advection fields;
    K timed steps of one pass on every hardware thread, then the scaling curve."""
    import paper_2409_18824_gb300.host as hp

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    nx, ny, nz = 512, 256, 256
    NX, NY, NZ = nx + 2, ny + 2, nz + 2
    vel = [si.hash_field(NX, NY, 0, NZ, m) for m in range(3)]
    outs = [np.zeros_like(vel[0]) for _ in range(3)]
    c = (0.25, 0.25, 0.25)
    tmax = hp.threads()

    def run(T):
        t0 = time.perf_counter()
        hp.stencil_host_advect_f64(vel[0], vel[1], vel[2], outs, c, nthreads=T)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        run(tmax)
    times = [run(tmax) for _ in range(args.steps)]
    cells = float(nx) * ny * nz
    value = cells * args.steps / sum(times) / 1e9
    curve = {}
    for T in sorted({t for t in (1, 2, 4, 8, 16, 32, 64) if t <= tmax} | {tmax}):
        curve[T] = cells / min(run(T) for _ in range(2)) / 1e9
    print(json.dumps({
        "metric": "Gcells/s (advection stand-in, u, v, w advecting themselves, FP64, multi-core host path)",
        "value": value, "unit": "Gcells/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512 x 256 x 256 block of the pw-advection fields (hash_field), one pass per step",
                   "grid": [nx, ny, nz], "threads": tmax, "parallelism": "host threads (libstencil_host.so)"},
        "scaling_curve": {"gcells": curve, "speedup": {T: curve[T] / curve[1] for T in curve},
                          "paper_table4_speedup": PAPER_OPENMP_PW_SPEEDUP},
        "e2e": {"value": value, "unit": "Gcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
        "host": host_info(),
    }), flush=True)


# ------------------------------------ the paper's sum / dotproduct runs ----
INTRINSICS = {
    "sum": dict(n=32768 * 32768, seed=8, paper_s=1.63, flang_s=1.65,
                desc="the paper's sum intrinsic: sum of a 32768 x 32768 FP64 array (8.6 GB), U[0,1) seed 8"),
    "dot": dict(n=1 << 27, seed=9, paper_s=0.81, flang_s=2.70,
                desc="the paper's dotproduct intrinsic: two 2^27-element (134 M) FP64 vectors, N(0,1) seeds 9, 10"),
}


def intrinsic_inputs(kind, n=None):
    w = INTRINSICS[kind]
    n = n or w["n"]
    x = si.rng(w["seed"]).random(n) if kind == "sum" else si.rng(w["seed"]).standard_normal(n)
    y = None if kind == "sum" else si.rng(w["seed"] + 1).standard_normal(n)
    return x, y


def run_intrinsic(args, kind):
    """One step = one sum (or dot product) over the whole array, read from HBM."""
    import torch
    import paper_2409_18824_gb300 as stn

    w = INTRINSICS[kind]
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.elements or w["n"]  # a smaller case only for profiling
    x, y = intrinsic_inputs(kind, n)
    dx = torch.from_numpy(x).to(dev)
    dy = None if y is None else torch.from_numpy(y).to(dev)
    stream = torch.cuda.current_stream(dev)
    nbytes = 8.0 * n * (1 if kind == "sum" else 2)

    def step():
        return stn.reduce_sum_f64(dx) if kind == "sum" else stn.dot_f64(dx, dy)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    vals = []
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            vals.append(step())
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dev)
    sec = ms / args.steps / 1e3
    value = nbytes * ws / sec / 1e9
    # e2e: the arrays from pinned host memory through the C ABI every step
    hx = torch.from_numpy(x).pin_memory()
    hy = None if y is None else torch.from_numpy(y).pin_memory()
    hxn, hyn = hx.numpy(), (None if hy is None else hy.numpy())
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        stn.reduce_sum_f64(hxn) if kind == "sum" else stn.dot_f64(hxn, hyn)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    peaks, peak_kind = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    note = "timed through the synchronous call: kernel + fixed-order finalize + 8-byte read"
    if kind == "sum":
        # HBM roofline (8 B per element); one double add per element makes the
        # FP64 pipe the first cap, given beside it.  DRAM bytes of one launch:
        # ncu on a 2^27-element case read 8.02 B per element (no re-reads),
        # scaled by the elements
        roofline = {"bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": nbytes / sec / 1e9 / hbm_peak, "traffic": TRAFFIC_SUM_PER_ELEMENT * n,
                    "traffic_unit": "bytes per launch", "peak_kind": peak_kind,
                    "kernel": "sum_kernel", "kernel_ms": ms / args.steps, "note": note}
        roofline.update(fp64_pipe(float(n), ms / args.steps, peaks, "one double add per element"))
    else:
        # ncu on the full 2^27-element dot: 2.1476 GB read, 2.9 MB written
        roofline = {"bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": nbytes / sec / 1e9 / hbm_peak, "traffic": TRAFFIC_DOT_PER_PAIR * n,
                    "traffic_unit": "bytes per launch",
                    "peak_kind": peak_kind, "kernel": "vec_reduce_kernel<true>", "kernel_ms": ms / args.steps,
                    "note": note}
    out = {
        "metric": f"GB/s ({w['desc']})", "value": value, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "elements": n, "bytes_per_step": nbytes,
                   "l2": "inputs larger than L2, no flush", "parallelism": "replicas" if ws > 1 else "single"},
        "seconds_per_run": sec,
        "paper_seconds": {"mlir_flow_1core": w["paper_s"], "flang_v20_1core": w["flang_s"]},
        "e2e": {"value": nbytes / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": 8},
        "gpu_launches": args.steps * 2,
        "roofline": roofline,
        "clocks": clk.summary(),
        "host": host_info(),
        "result": vals[-1],
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            val, t = cpu_sample_intrinsic(kind, x, y)
            out["cpu_baseline"] = {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                   "sample": f"the whole workload {INTRINSIC_CPU_PASSES[kind]} times, plain C "
                                             f"oracle, one thread ({t:.1f} s)"}
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


INTRINSIC_CPU_PASSES = {"sum": 10, "dot": 100}  # ~10 s of one core each


def cpu_sample_intrinsic(kind, x, y, passes=None):
    import oracle
    oracle.build()
    passes = passes or INTRINSIC_CPU_PASSES[kind]
    t0 = time.perf_counter()
    for _ in range(passes):
        oracle.sum_(x) if kind == "sum" else oracle.dot(x, y)
    t = time.perf_counter() - t0
    return 8.0 * x.size * (1 if kind == "sum" else 2) * passes / t / 1e9, t


def run_reference_intrinsic(args, kind):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = INTRINSICS[kind]
    x, y = intrinsic_inputs(kind)
    for _ in range(args.warmup):
        cpu_sample_intrinsic(kind, x, y, 1)
    times = [cpu_sample_intrinsic(kind, x, y, 1)[1] for _ in range(args.steps)]
    total = sum(times)
    nbytes = 8.0 * w["n"] * (1 if kind == "sum" else 2)
    value = nbytes * args.steps / total / 1e9
    print(json.dumps({
        "impl": "reference", "metric": f"GB/s ({w['desc']})", "value": value, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "elements": w["n"], "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "each step: the whole workload, plain C oracle, one thread"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host": host_info(),
    }), flush=True)


# ------------------------------------------- the advection stand-in (pw-like) ----
ADVECT = dict(nx=2048, ny=1024, nz=1024, c=(0.25, 0.25, 0.25),
              desc="multi-field advection stand-in for the paper's pw-advection (its formulas are not "
                   "in the paper): u, v, w on 2048 x 1024 x 1024 FP64 advect themselves (second-order "
                   "centred flux form), fields from the integer hash of stencil_inputs.hash_field")
ADVECT_FP64_OPS = 48.0   # double ops per cell: one flux per face and field (3 each), 3 (diff, scale) pairs, 2 adds
ADVECT_BYTES = 48.0      # read u, v, w; write three tendencies


def hash_field_device(NX, NY, NZ, comp, dtype, device):
    """stencil_inputs.hash_field on the device, plane by plane (bitwise the same values)."""
    import torch
    a, b, c, d = si.HASH_MULS
    out = torch.empty((NZ, NY, NX), dtype=dtype, device=device)
    i = torch.arange(NX, device=device, dtype=torch.int64)
    j = torch.arange(NY, device=device, dtype=torch.int64)
    base = a * i[None, :] + b * j[:, None] + d * comp
    for k in range(NZ):
        h = (base + c * k) % 65536
        out[k] = (h.to(torch.float64) / 32768.0 - 1.0).to(dtype)
    return out


def run_advect(args):
    import torch
    import paper_2409_18824_gb300 as stn

    w = ADVECT
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    if args.kernel_only:
        nx, ny, nz = 512, 512, 256  # profiling size: 6 x 545 MB, above L2
    NX, NY, NZ = nx + 2, ny + 2, nz + 2
    vel = [hash_field_device(NX, NY, NZ, m, torch.float64, dev) for m in range(3)]
    if args.kernel_only:
        outs = [torch.empty_like(vel[0]) for _ in range(3)]
        for _ in range(args.kernel_only):
            stn.advect_f64(vel[0], vel[1], vel[2], outs, w["c"])
        torch.cuda.synchronize(dev)
        return
    outs = [torch.empty_like(vel[0]) for _ in range(3)]
    stream = torch.cuda.current_stream(dev)

    def step():
        stn.advect_f64(vel[0], vel[1], vel[2], outs, w["c"])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        for k in range(args.steps):
            step()
            evs[k + 1].record(stream)
        torch.cuda.synchronize(dev)
    ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), dev)
    cells = float(nx) * ny * nz
    sec = ms / args.steps / 1e3
    value = cells * ws / sec / 1e9
    checksum = float(outs[0][1:-1, 1:-1, 1:-1].double().abs().sum().item())
    del vel, outs
    torch.cuda.empty_cache()
    # e2e at the tra-adv grid size (1024 x 512 x 512, 1/4 of the cells): the
    # three fields from pinned host memory in, the three tendencies out
    ex, ey, ez = 1024, 512, 512
    hv = [torch.from_numpy(si.hash_field(ex + 2, ey + 2, 0, ez + 2, m)).pin_memory() for m in range(3)]
    ho = [torch.empty_like(hv[0]).pin_memory() for _ in range(3)]
    dv = [torch.empty(hv[0].shape, dtype=torch.float64, device=dev) for _ in range(3)]
    do = [torch.empty_like(dv[0]) for _ in range(3)]
    for dd, hh in zip(dv, hv):
        dd.copy_(hh, non_blocking=True)
    stn.advect_f64(dv[0], dv[1], dv[2], do, w["c"])
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(2):
        for dd, hh in zip(dv, hv):
            dd.copy_(hh, non_blocking=True)
        stn.advect_f64(dv[0], dv[1], dv[2], do, w["c"])
        for hh, dd in zip(ho, do):
            hh.copy_(dd, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / 2
    peaks, peak_kind = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    hbm_gbs = cells * ADVECT_BYTES / sec / 1e9
    # HBM roofline (3 fields in, 3 tendencies out); the FP64 pipe caps it
    # first and its fraction is given beside it.  ncu on a 512 x 512 x 256
    # case: 3.308 GB for 67.1 M cells = 49.3 B per cell (5 % halo re-reads),
    # scaled by the cells of this launch
    roofline = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
                "traffic": TRAFFIC_ADVECT_PER_CELL * cells, "traffic_unit": "bytes per launch",
                "peak_kind": peak_kind, "bytes_per_cell": ADVECT_BYTES, "kernel": "advect_kernel<double,3,self>",
                "kernel_ms": ms / args.steps}
    roofline.update(fp64_pipe(cells * ADVECT_FP64_OPS, ms / args.steps, peaks,
                              f"{ADVECT_FP64_OPS} double ops per cell"))
    out = {
        "metric": "Gcells/s (advection stand-in, pw-like, 2048 x 1024 x 1024 FP64)",
        "value": value, "unit": "Gcells/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "nx": nx, "ny": ny, "nz": nz, "fields": 3,
                   "l2": "inputs larger than L2 (17 GB per field), no flush",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "paper_context": "pw-advection: one EPYC core 86.47 s (MLIR flow, Table 2), V100 OpenACC 22.78 s at "
                         "1.1 billion cells (Table 5); iteration counts not stated, so not comparable",
        "e2e": {"value": float(ex) * ey * ez / e2e_s / 1e9, "unit": "Gcells/s",
                "h2d_bytes_per_step": 3 * hv[0].numel() * 8, "d2h_bytes_per_step": 3 * hv[0].numel() * 8,
                "grid": [ex, ey, ez]},
        "gpu_launches": args.steps,
        "roofline": roofline,
        "step_ms": step_stats(evs),
        "clocks": clk.summary(),
        "host": host_info(),
        "checksum_abs_su": checksum,
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            val, t = cpu_sample_advect()
            out["cpu_baseline"] = {"value": val, "unit": "Gcells/s", "cores": 1, "kind": "oracle",
                                   "sample": f"{ADVECT_CPU_PASSES} passes over a 256 x 128 x 128 corner of the "
                                             f"same fields, plain C oracle, one thread ({t:.1f} s)"}
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


ADVECT_CPU_PASSES = 100  # passes over the CPU sample (~10 s of one core)


def cpu_sample_advect(passes=ADVECT_CPU_PASSES):
    import oracle
    nx, ny, nz = 256, 128, 128
    f = [si.hash_field(nx + 2, ny + 2, 0, nz + 2, m) for m in range(3)]
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(passes):
        for m in range(3):
            oracle.advect(f[0], f[1], f[2], f[m], ADVECT["c"])
    t = time.perf_counter() - t0
    return float(nx) * ny * nz * passes / t / 1e9, t


def run_reference_advect(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_sample_advect(1)
    passes = 20
    times = [cpu_sample_advect(passes)[1] for _ in range(args.steps)]
    value = 256.0 * 128 * 128 * passes * args.steps / sum(times) / 1e9
    print(json.dumps({
        "impl": "reference", "metric": "Gcells/s (advection stand-in, pw-like, 2048 x 1024 x 1024 FP64)",
        "value": value, "unit": "Gcells/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": ADVECT["desc"], "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "Gcells/s", "cores": 1, "kind": "oracle",
                         "sample": "each step: 20 passes over a 256 x 128 x 128 corner of the fields, plain C "
                                   "oracle, one thread"},
        "e2e": {"value": value, "unit": "Gcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host": host_info(),
    }), flush=True)


# ------------------------------------------------------- batched solves ----
def batch_problems(count, seed_sizes=4, seed_rhs=5):
    """Per-axis sizes log-uniform in [16, 128] (PCG64 seed 4); right-hand sides
    N(0,1), problem i drawn from PCG64 seed 5 * 1000003 + i; zero halo."""
    sizes = si.log_uniform_sizes(count, 16, 128, seed_sizes)
    return [tuple(int(v) for v in s) for s in sizes], [seed_rhs * 1000003 + i for i in range(count)]


def run_batched(args):
    import torch
    import paper_2409_18824_gb300 as stn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sizes, seeds = batch_problems(args.batch)
    tol = 1e-8
    # one allocation per array kind; problems are views into it
    counts = [(nx + 2) * (ny + 2) * (nz + 2) for nx, ny, nz in sizes]
    offs = np.concatenate([[0], np.cumsum(counts)])
    total = int(offs[-1])
    h_rhs = torch.empty(total, dtype=torch.float64).pin_memory()
    hr = h_rhs.numpy()
    for i, (nx, ny, nz) in enumerate(sizes):
        hr[offs[i]:offs[i + 1]] = si.normal_interior(nx, ny, nz, 1, seed=seeds[i]).ravel()
    d_rhs = h_rhs.to(dev)
    d_u = torch.zeros(total, dtype=torch.float64, device=dev)
    us = [d_u[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]
    bs = [d_rhs[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]
    refined = args.refined

    def step():
        d_u.zero_()
        if refined:
            rc, infos = stn.jacobi_solve_batched_refined(us, bs, si.LAPLACE7, 1, tol, args.inner_max,
                                                         args.inner_tol, 50, 40)
        else:
            rc, infos = stn.jacobi_solve_batched_f64(us, bs, si.LAPLACE7, 1, tol, 10 ** 7, 100)
        return rc, infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    times, lups, all_infos = [], 0.0, None
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, infos = step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
            all_infos = infos
    ms = sum(times)
    ms = max_over_ranks(ms, dev)
    pts = np.array([nx * ny * nz for nx, ny, nz in sizes], dtype=np.float64)
    iters = np.array([i["iters"] for i in all_infos], dtype=np.float64)
    lups = float((pts * iters).sum())
    conv = sum(1 for i in all_infos if i["status"] == 0)
    value = args.batch * ws * args.steps / (ms * 1e-3)
    # e2e: right-hand sides from pinned host memory in, solutions out, inside the timed region
    h_u = torch.empty(total, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    d_rhs.copy_(h_rhs, non_blocking=True)
    step()
    h_u.copy_(d_u, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    out = {
        "metric": "batched solves/s (2048 Jacobi/Poisson solves, sizes log-U[16,128], tol 1e-8)",
        "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 refined" if refined else "f64", "data": "synthetic",
        "config": {"workload": f"{args.batch} independent 7-point Poisson solves u = S u + b, per-axis sizes "
                               f"log-uniform in [16,128] (seed 4), b ~ N(0,1), tol 1e-8, one persistent "
                               f"{'cluster' if stn.stencil_tune_get('batch_engine') == 1 else 'work-unit scheduler'} launch"
                               + (", FP32 sweeps with FP64 refinement" if refined else ", FP64"),
                   "batch": args.batch, "points": int(pts.sum()), "l2": "no flush (each solve re-reads its grid)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "e2e": {"value": args.batch / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": total * 8,
                "d2h_bytes_per_step": total * 8},
        "gpu_launches": args.steps * 1,
        "aggregate_glups": lups / (ms / args.steps * 1e-3) / 1e9,
        "scheduler_counters": stn.stencil_sched_stats(),
        "converged": conv,
        "sweeps_max": int(iters.max()), "sweeps_median": float(np.median(iters)),
        "clocks": clk.summary(),
        "host": host_info(),
    }
    if rank == 0:
        if not args.no_cpu_baseline and not refined:
            out["cpu_baseline"] = cpu_sample_batched(sizes, seeds, pts, iters)
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------- variable coefficient (r=2) --
def cpu_sample_batched(sizes, seeds, pts, iters, n_sample=8, sweeps=1000):
    """The oracle's Jacobi sweep rate (one thread) on every 256th problem of the
    mix, `sweeps` sweeps each, projected onto the whole batch with the sweep
    counts this run took: solves/s = count / sum(points x sweeps / rate)."""
    import oracle
    idx = list(range(0, len(sizes), max(1, len(sizes) // n_sample)))[:n_sample]
    lup, sec = 0.0, 0.0
    for i in idx:
        nx, ny, nz = sizes[i]
        b = si.normal_interior(nx, ny, nz, 1, seed=seeds[i])
        t0 = time.perf_counter()
        oracle.stencil_sweep(b, si.LAPLACE7, 1, sweeps)  # the problem's own values as the grid
        sec += time.perf_counter() - t0
        lup += float(nx) * ny * nz * sweeps
    rate = lup / sec
    total_s = float((pts * iters).sum()) / rate
    return {"value": len(sizes) / total_s, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"projected: the oracle's sweep rate {rate / 1e9:.3f} GLUP/s (one thread, {sweeps} sweeps "
                      f"on each of problems {idx}, {sec:.1f} s) times the sweep counts of this run's "
                      f"{len(sizes)} solves ({total_s:.0f} s of oracle work)"}


def varcoef_problem(stn, dev, nx, ny, nz):
    """The variable-coefficient workload's problem: a ~ U[0.5,1.5] (seed 3),
    the (1,1,1) sine mode as the solution u*, f = A u* (device grids)."""
    import torch
    W, R = si.VARCOEF_W, 2
    a = torch.from_numpy(si.uniform_full(nx, ny, nz, R, seed=3)).to(dev)
    ustar = torch.from_numpy(si.sine_mode(nx, ny, nz, R)).to(dev)
    f = torch.zeros_like(ustar)
    stn.varcoef_apply_f64(ustar, a, f, W, R)  # manufactured right-hand side f = A u*
    return a, f, ustar


def varcoef_rates(stn, dev):
    """Full-size (768 x 768 x 384) sweep rates, float and double, and the
    complete refined and plain FP64 solves to 1e-10 on 96 x 96 x 48.  Returns
    (measurements, the two solves, clocks, the 96 x 96 x 48 grids)."""
    import torch
    W, R = si.VARCOEF_W, 2

    def problem(nx, ny, nz):
        return varcoef_problem(stn, dev, nx, ny, nz)

    out = {"workload": "varcoef"}
    with ClockSampler(0) as clk:
        # full size: rates
        nx, ny, nz = 768, 768, 384
        a, f, ustar = problem(nx, ny, nz)
        a32, f32 = a.float(), f.float()
        e0 = torch.zeros_like(f32)
        e1 = torch.zeros_like(f32)
        sweeps = 20
        stn.varcoef_sweep_f32(e0, e1, a32, f32, W, R, 2)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        stn.varcoef_sweep_f32(e0, e1, a32, f32, W, R, sweeps)
        ev1.record()
        torch.cuda.synchronize()
        ms32 = ev0.elapsed_time(ev1) / sweeps
        u = torch.zeros_like(f)
        stn.varcoef_residual_norm_f64(u, a, f, W, R)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(3):
            stn.varcoef_residual_norm_f64(u, a, f, W, R)
        ev1.record()
        torch.cuda.synchronize()
        ms_res = ev0.elapsed_time(ev1) / 3
        u64a, u64b = torch.zeros_like(f), torch.zeros_like(f)
        ev0.record()
        stn.varcoef_sweep_f64(u64a, u64b, a, f, W, R, 3)
        ev1.record()
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1) / 3
        pts = float(nx) * ny * nz
        out["full_size"] = {"grid": [nx, ny, nz], "f32_sweep_ms": ms32, "f32_sweep_glups": pts / ms32 / 1e6,
                            "f32_sweep_hbm_gbs": 16.0 * pts / ms32 / 1e6, "f64_residual_ms": ms_res,
                            "f64_sweep_ms": ms64, "f64_sweep_glups": pts / ms64 / 1e6}
        del a, f, ustar, a32, f32, e0, e1, u, u64a, u64b
        torch.cuda.empty_cache()
        # reduced grid: complete solves
        nx, ny, nz = 96, 96, 48
        a, f, ustar = problem(nx, ny, nz)
        res = {}
        for name in ("refined", "plain_f64"):
            u = torch.zeros_like(f)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "refined":
                rc, info = stn.jacobi_solve_varcoef_refined(a, f, u, W, R, 1e-10, 4000, 40)
            else:
                rc, info = stn.jacobi_solve_varcoef_f64(a, f, u, W, R, 1e-10, 10 ** 6, 200)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            err = float((u - ustar).abs().max() / ustar.abs().max())
            res[name] = {"seconds": dt, "rc": rc, "rel_res": info["rel_res"], "sweeps": info["iters"],
                         "outer": info["outer"], "err_vs_manufactured": err}
        out["reduced_96x96x48"] = res
        clocks = clk.summary()
    return out, res, clocks, (a, f, ustar)


def varcoef_roofline(fs):
    """HBM roofline of the full-size float sweep (16 compulsory bytes per update)."""
    peaks, peak_kind = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    # ncu on a 512 x 512 x 256 float sweep of the TMA-staged kernel: 837.3 MB
    # read + 250.5 MB written for 67.1 M updates = 16.2 B per update, scaled to
    # the full grid
    return {"bound": "hbm", "achieved": fs["f32_sweep_hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": fs["f32_sweep_hbm_gbs"] / hbm_peak, "traffic": TRAFFIC_VARCOEF_F32_PER_LUP * 768 * 768 * 384,
            "traffic_unit": "bytes per launch", "peak_kind": peak_kind,
            "kernel": "var_tma_kernel (TMA-staged float sweep, radius 2, one sweep at 768 x 768 x 384)",
            "kernel_ms": fs["f32_sweep_ms"]}


def run_varcoef(args):
    """768x768x384 radius-2 variable-coefficient Poisson problem: per-sweep rates at
    full size (float Jacobi sweep, double residual), and complete solves to a
    1e-10 relative residual on a 96x96x48 grid of the same construction (FP32
    sweeps with FP64 refinement vs plain FP64 Jacobi)."""
    import torch
    import paper_2409_18824_gb300 as stn

    dev = torch.device("cuda", 0)
    W = si.VARCOEF_W
    R = 2

    if args.kernel_only:
        # the float variable-coefficient sweep alone at 512 x 512 x 256 (for profilers)
        nx, ny, nz = 512, 512, 256
        a32 = torch.from_numpy(si.uniform_full(nx, ny, nz, R, seed=3, dtype=np.float32)).to(dev)
        f32 = torch.from_numpy(si.normal_interior(nx, ny, nz, R, seed=4, dtype=np.float32)).to(dev)
        e0 = torch.zeros_like(f32)
        e1 = torch.zeros_like(f32)
        stn.varcoef_sweep_f32(e0, e1, a32, f32, W, R, args.kernel_only)
        torch.cuda.synchronize()
        return

    def problem(nx, ny, nz):
        return varcoef_problem(stn, dev, nx, ny, nz)

    full_solve = None
    if not args.varcoef_reduced:
        full_solve = varcoef_full_solve(stn, dev, problem, with_cpu=not args.no_cpu_baseline)
        torch.cuda.empty_cache()
    out, res, clocks, (a, f, ustar) = varcoef_rates(stn, dev)
    ratio = res["plain_f64"]["seconds"] / res["refined"]["seconds"]
    # e2e: the refined solve through the C ABI with host (numpy) grids, copies included
    a_h, f_h, us_h = (t.cpu().numpy() for t in (a, f, ustar))
    u_h = np.zeros_like(f_h)
    t0 = time.perf_counter()
    stn.jacobi_solve_varcoef_refined(a_h, f_h, u_h, W, R, 1e-10, 4000, 40)
    e2e_s = time.perf_counter() - t0
    roofline = varcoef_roofline(out["full_size"])
    if full_solve is not None:
        fs_solve = full_solve
        line_metric = ("time to a 1e-10 relative residual, 768x768x384 variable-coefficient r=2 Poisson, "
                       "FP32 sweeps + FP64 refinement")
        value, unit, hib = fs_solve["seconds"], "s", False
        ms_step = fs_solve["seconds"] * 1e3
        launches = int(fs_solve["sweeps"] + 4 * fs_solve["outer"])
        wl_desc = ("768x768x384 variable-coefficient 13-point Poisson, a ~ U[0.5,1.5] (seed 3), manufactured (1,1,1) "
                   "sine solution, solved once at full size to 1e-10 (refined); full-size sweep rates and complete "
                   "refined and FP64 solves on 96x96x48 beside it")
    else:
        line_metric = "time to 1e-10 relative residual, variable-coefficient r=2 Poisson (refined vs FP64)"
        value, unit, hib = ratio, "speedup (x)", True
        ms_step = res["refined"]["seconds"] * 1e3
        launches = int(res["refined"]["sweeps"] + 4 * res["refined"]["outer"])
        wl_desc = ("768x768x384 variable-coefficient 13-point Poisson, a ~ U[0.5,1.5] (seed 3), manufactured (1,1,1) "
                   "sine solution; full-size sweep rates + complete solves on 96x96x48")
    line = {"metric": line_metric,
            "value": value, "unit": unit, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": ms_step, "higher_is_better": hib, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 refined", "data": "synthetic",
            "config": {"workload": wl_desc},
            "e2e": {"value": res["plain_f64"]["seconds"] / e2e_s, "unit": "speedup (x)",
                    "h2d_bytes_per_step": 3 * f_h.nbytes, "d2h_bytes_per_step": f_h.nbytes},
            # kernels of the timed refined solve: one float sweep each, and per outer
            # step the residual, its maximum, the scaling and the update
            "gpu_launches": launches,
            "roofline": roofline,
            "clocks": clocks,
            "host": host_info(),
            "detail": out}
    if full_solve is not None:
        line["full_solve"] = full_solve
        line["reduced_96x96x48_speedup_refined_vs_f64"] = ratio
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample_varcoef()
        if full_solve is not None and "oracle_check" in full_solve:
            line["cpu_baseline"]["oracle_check"] = full_solve.pop("oracle_check")
    print(json.dumps(line), flush=True)


def varcoef_full_solve(stn, dev, problem, with_cpu, inner=40000, max_outer=80):
    """The variable-coefficient configuration solved once at full size: FP32
    sweeps with FP64 refinement to a 1e-10 relative residual (inner sweeps per
    outer step fixed at `inner`), timed with CUDA events; the error against
    the manufactured solution; the FP64 plain solve's time projected from its
    measured full-size sweep time; and, in the CPU leg, the oracle's own FP64
    residual ||f - A u|| / ||f|| of the returned u at full size."""
    import torch
    W, R = si.VARCOEF_W, 2
    nx, ny, nz = 768, 768, 384
    a, f, ustar = problem(nx, ny, nz)
    u = torch.zeros_like(f)
    # the double sweep's time at this size, for the plain projection
    u64a, u64b = torch.zeros_like(f), torch.zeros_like(f)
    stn.varcoef_sweep_f64(u64a, u64b, a, f, W, R, 1)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    stn.varcoef_sweep_f64(u64a, u64b, a, f, W, R, 4)
    ev[1].record()
    torch.cuda.synchronize()
    ms64 = ev[0].elapsed_time(ev[1]) / 4
    del u64a, u64b
    torch.cuda.empty_cache()
    with ClockSampler(dev.index or 0) as clk:
        t0 = time.perf_counter()
        ev[2].record()
        rc, info = stn.jacobi_solve_varcoef_refined(a, f, u, W, R, 1e-10, inner, max_outer)
        ev[3].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    sec = ev[2].elapsed_time(ev[3]) / 1e3
    err = float((u - ustar).abs().max() / ustar.abs().max())
    out = {"grid": [nx, ny, nz], "seconds": sec, "wall_s": wall, "rc": rc, "rel_res": info["rel_res"],
           "sweeps": info["iters"], "outer": info["outer"], "inner_sweeps_per_outer": inner,
           "err_vs_manufactured_max_rel": err, "clocks": clk.summary(),
           "f32_sweep_ms_mean": sec * 1e3 / max(1, info["iters"]),
           "plain_f64_projected": {"seconds": info["iters"] * ms64 * 1e-3, "f64_sweep_ms": ms64,
                                   "sweeps": info["iters"],
                                   "how": "projected: the measured full-size FP64 sweep time x the refined solve's "
                                          "total sweep count (the same Jacobi iteration matrix; a plain solve needs "
                                          "at most that many, give or take one group of inner sweeps)"}}
    out["speedup_vs_plain_projected"] = out["plain_f64_projected"]["seconds"] / sec
    if with_cpu:
        import oracle
        uh, ah, fh = u.cpu().numpy(), a.cpu().numpy(), f.cpu().numpy()
        t0 = time.perf_counter()
        rr = oracle.varcoef_residual_norm(uh, ah, fh, W, R) / oracle.interior_norm(fh, R)
        out["oracle_check"] = {"rel_res_oracle": rr, "tol": 1e-10, "within_tol": bool(rr <= 1e-10),
                               "seconds": time.perf_counter() - t0,
                               "what": "the oracle's own FP64 ||f - A u|| / ||f|| of the returned u, full size"}
    del a, f, ustar, u
    return out


def cpu_sample_varcoef():
    """The oracle's own refined vs plain FP64 solves to 1e-10 on a 24 x 24 x 12
    grid of the workload's construction (one thread; the speedup, the metric's
    unit), and its float sweep rate on a 192 x 192 x 96 block."""
    import oracle
    W, R = si.VARCOEF_W, 2
    nx, ny, nz = 24, 24, 12
    a = si.uniform_full(nx, ny, nz, R, seed=3)
    f = oracle.varcoef_apply(si.sine_mode(nx, ny, nz, R), a, W, R)
    t0 = time.perf_counter()
    oracle.varcoef_refined_solve(a, f, np.zeros_like(f), W, R, 1e-10, 4000, 40)
    t_ref = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.varcoef_jacobi_solve(a, f, np.zeros_like(f), W, R, 1e-10, 10 ** 6, 200)
    t_plain = time.perf_counter() - t0
    bx, by, bz = 192, 192, 96
    a32 = si.uniform_full(bx, by, bz, R, seed=3, dtype=np.float32)
    f32 = si.normal_interior(bx, by, bz, R, seed=4, dtype=np.float32)
    e = np.zeros_like(f32)
    t0 = time.perf_counter()
    for _ in range(2):
        e = oracle.varcoef_sweep(e, a32, f32, W, R)
    t_sw = time.perf_counter() - t0
    return {"value": t_plain / t_ref, "unit": "speedup (x)", "cores": 1, "kind": "oracle",
            "sample": f"refined ({t_ref:.2f} s) vs plain FP64 ({t_plain:.2f} s) oracle solves to 1e-10 on a "
                      f"24 x 24 x 12 grid of the same construction; float sweep {bx * by * bz * 2 / t_sw / 1e9:.3f} "
                      f"GLUP/s on {bx} x {by} x {bz}"}


# ------------------------------------------------------------- serving -----
def serve_requests(count, seed_sizes=6, seed_rhs=7):
    """Per-axis sizes log-uniform in [32, 256] (PCG64 seed 6); right-hand sides
    N(0,1), request i from PCG64 seed 7 * 1000003 + i; zero halo and guess."""
    sizes = si.log_uniform_sizes(count, 32, 256, seed_sizes)
    return [tuple(int(v) for v in s) for s in sizes], [seed_rhs * 1000003 + i for i in range(count)]


def run_serving(args):
    import torch
    import paper_2409_18824_gb300 as stn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    sizes, seeds = serve_requests(args.requests)
    rhss = [si.normal_interior(nx, ny, nz, 1, seed=sd) for (nx, ny, nz), sd in zip(sizes, seeds)]
    budget = 40 << 30
    refined = not args.plain

    def run_trace(arrivals):
        """Submits request i at arrivals[i] seconds; returns (makespan, latencies)."""
        with stn.Server(hbm_budget=budget, tol=args.tol, refined=refined, inner_sweeps=200000, inner_tol=1e-2,
                        check_every=50, max_outer=40, max_inflight=64) as srv:
            t0 = time.perf_counter()
            tickets = []
            for i, at in enumerate(arrivals):
                d = at - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                tickets.append(srv.submit(rhss[i]))
            lat, status = [], []
            for t in tickets:
                r = srv.wait(t, 3600.0)
                lat.append(r["latency_s"])
                status.append(r["status"])
                srv.release(t)
            return time.perf_counter() - t0, lat, status

    def run_trace_per_request(arrivals):
        """The plain comparison: one double Jacobi solve per request, in arrival
        order, each through jacobi_solve_f64 (its own CUDA-graph solve)."""
        import queue
        q = queue.Queue()
        done = [None] * len(arrivals)
        status = [None] * len(arrivals)

        def worker():
            while True:
                item = q.get()
                if item is None:
                    return
                i, t_sub = item
                d_b = torch.from_numpy(rhss[i]).cuda()
                d_u = torch.zeros_like(d_b)
                rc, info = stn.jacobi_solve_f64(d_b, d_u, si.LAPLACE7, 1, args.tol, 10 ** 7, 50)
                d_u.cpu()
                done[i] = time.perf_counter() - t_sub
                status[i] = info["status"]

        th = threading.Thread(target=worker)
        th.start()
        t0 = time.perf_counter()
        for i, at in enumerate(arrivals):
            d = at - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            q.put((i, time.perf_counter()))
        q.put(None)
        th.join()
        return time.perf_counter() - t0, done, status

    trace = run_trace_per_request if args.per_request else run_trace
    n = len(rhss)
    # capacity: every request at t = 0
    with ClockSampler(local) as clk:
        span, lat, status = trace([0.0] * n)
        capacity = n / span
        loads = []
        rates = args.rates or [frac * capacity for frac in args.loads]
        for k, rate in enumerate(rates):
            frac = rate / capacity
            arr = si.poisson_arrival_times(n, rate, seed=8).tolist()
            span_l, lat_l, st_l = trace(arr)
            loads.append({"offered_frac": frac, "offered_per_s": rate, "solves_per_s": n / span_l,
                          "p50_s": float(np.percentile(lat_l, 50)), "p99_s": float(np.percentile(lat_l, 99)),
                          "converged": int(sum(1 for x in st_l if x == 0))})
    out = {
        "metric": f"serving solves/s and p50/p99 latency (Poisson arrivals, sizes log-U[32,256], tol {args.tol:g})",
        "value": capacity, "unit": "solves/s", "n_gpus": ws, "steps": 1, "warmup": 0,
        "ms_per_step": span * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if (args.per_request or not refined) else "f32+f64 refined", "data": "synthetic",
        "config": {"workload": f"{n} Poisson solve requests, per-axis sizes log-uniform in [32,256] (seed 6), "
                               f"rhs N(0,1), tol {args.tol:g}, " + (
                                   "one double jacobi_solve_f64 per request in arrival order (the plain path)"
                                   if args.per_request else
                                   "40 GiB admission budget, continuous batching"
                                   + ("" if refined else ", double Jacobi")),
                   "requests": n},
        "saturation": {"solves_per_s": capacity, "p50_s": float(np.percentile(lat, 50)),
                       "p99_s": float(np.percentile(lat, 99)), "converged": int(sum(1 for x in status if x == 0))},
        "loads": loads,
        "e2e": {"value": capacity, "unit": "solves/s",
                "h2d_bytes_per_step": int(sum(b.nbytes for b in rhss)) * 2,
                "d2h_bytes_per_step": int(sum(b.nbytes for b in rhss))},
        "clocks": clk.summary(),
        "host": host_info(),
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def double_word_variant(stn, dev, u0, d_in, d_out, peaks):
    """The opt-in double sweep in double-word float arithmetic (knob
    fp64_double_word) on the headline grid: its sweep rate (20 sweeps, CUDA
    events) and, from the workload's own grid, its largest difference from the
    exact path after the workload's 1000 sweeps.  Not the headline: it is not
    bitwise the canonical order (error bound about 40 * 2^-48 of the grid's
    largest value per sweep)."""
    import torch
    sweeps = 1000
    n = float(u0.shape[0] - 2) * (u0.shape[1] - 2) * (u0.shape[2] - 2)
    d_in.copy_(torch.from_numpy(u0))
    stn.stencil_sweep_f64(d_in, d_out, si.LAPLACE7, 1, sweeps)
    exact = d_out.clone()
    stn.stencil_tune_set("fp64_double_word", 1)
    try:
        d_in.copy_(torch.from_numpy(u0))
        stn.stencil_sweep_f64(d_in, d_out, si.LAPLACE7, 1, sweeps)
        torch.cuda.synchronize(dev)
        exact_max = float(exact.abs().max())
        err = float((d_out - exact).abs().max()) / exact_max
        stn.stencil_sweep_f64(d_in, d_out, si.LAPLACE7, 1, 2)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        stn.stencil_sweep_f64(d_in, d_out, si.LAPLACE7, 1, 20)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 20
    finally:
        stn.stencil_tune_set("fp64_double_word", 0)
    del exact
    hbm = 16.0 * n / (ms * 1e-3) / 1e9
    out = {"opt_in": "knob fp64_double_word = 1; not the canonical order, not bitwise",
           "glups": n / (ms * 1e-3) / 1e9, "kernel_ms": ms, "hbm_gbs": hbm,
           "hbm_frac": hbm / float(peaks["hbm_gbs"]),
           "max_rel_diff_vs_exact_after_1000_sweeps": err,
           "bound_after_1000_sweeps": 1000 * 40.0 * 2.0 ** -48 * float(np.max(np.abs(u0))) / exact_max,
           "bound_note": "per sweep at most 40 * 2^-48 of the largest |u| (split, five double-word additions, "
                         "the product with c1, the final rounding); the Jacobi update is non-expansive in the "
                         "max norm, so n sweeps stay within n times that"}
    out.update(fp64_pipe(1.0 * n, ms, peaks, "one double add per update (the final rejoin)"))
    return out


# ------------------------------------------ the metric's other configurations --
# The default run adds, after the 512^3 headline, the other parts of the
# benchmark metric under their own keys of the same JSON line: the 64^3
# configuration ("c1"), the variable-coefficient configuration's sweep rates
# and reduced solves ("c3"), the 2048-solve batch ("batched") and the serving
# loop ("serving").  They run in this order within a wall-clock budget
# (--extras-budget); a part that would not fit is recorded as skipped.

SERVE_REQUESTS = 200
SERVE_LOADS = (0.5, 0.8, 1.1)
SERVE_WORKERS = 4


def lindley(arrivals, service):
    """Latencies of a single first-come-first-served server: request i starts
    when it has arrived and request i-1 has finished, and runs for service[i]."""
    lat, free = [], 0.0
    for a, sv in zip(arrivals, service):
        start = max(a, free)
        free = start + sv
        lat.append(free - a)
    return lat


def pct(x, q):
    return float(np.percentile(np.asarray(x, dtype=np.float64), q))


def extra_c1(stn, dev, with_cpu):
    """64^3 FP64, U[0,1) seed 1, zero halo, c = {0, 1/6}: 100 sweeps, then the
    residual L2 norm.  The grid (2.3 MB) stays in L2, so the bound is the
    kernel latency and the FP64 pipe, not HBM."""
    import torch
    n, sweeps, steps = 64, 100, 20
    u0 = si.uniform_interior(n, n, n, 1, seed=1)
    d_in = torch.from_numpy(u0).to(dev)
    d_out = torch.zeros_like(d_in)
    stream = torch.cuda.current_stream(dev)

    def step():
        stn.stencil_sweep_f64(d_in, d_out, si.LAPLACE7, 1, sweeps)
        return stn.residual_norm_f64(d_out, si.LAPLACE7, 1)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index or 0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            norm = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    lups = float(n) ** 3 * sweeps
    out = {"workload": "7-point Jacobi, 64^3 FP64, zero halo, interior U[0,1) seed 1, 100 sweeps + residual L2 norm",
           "value": lups / (ms * 1e-3) / 1e9, "unit": "GLUP/s", "ms_per_step": ms, "steps": steps, "warmup": 3,
           "us_per_sweep": ms * 1e3 / (sweeps + 1), "residual_norm": norm, "clocks": clk.summary(),
           "roofline": {"bound": "latency", "note": "the grid (2.3 MB per array) stays in L2: a sweep is bound by "
                        "kernel latency and the FP64 pipe, not HBM"}}
    out["roofline"].update(fp64_pipe(6.0 * lups, ms, load_peaks()[0], "6 double ops per update"))
    h_in, h_out = u0.copy(), np.zeros_like(u0)
    t0 = time.perf_counter()
    for _ in range(3):
        stn.stencil_sweep_f64(h_in, h_out, si.LAPLACE7, 1, sweeps)
        stn.residual_norm_f64(h_out, si.LAPLACE7, 1)
    e2e_s = (time.perf_counter() - t0) / 3
    out["e2e"] = {"value": lups / e2e_s / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": 2 * u0.nbytes,
                  "d2h_bytes_per_step": 2 * u0.nbytes + 8}
    if with_cpu:
        import oracle
        # the timed steps reuse `in` as the ping-pong buffer; one more step from
        # the configuration's own grid gives the result the oracle checks
        d_in.copy_(torch.from_numpy(u0))
        norm = step()
        t0 = time.perf_counter()
        ref = oracle.stencil_sweep(u0, si.LAPLACE7, 1, sweeps)
        rnorm = oracle.residual_norm(ref, si.LAPLACE7, 1)
        t = time.perf_counter() - t0
        got = d_out.cpu().numpy()
        out["cpu_baseline"] = {"value": lups / t / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                               "sample": f"the whole configuration, plain C oracle, one thread ({t:.2f} s)",
                               "bitwise_oracle": bool(np.array_equal(got.view(np.uint64), ref.view(np.uint64))),
                               "norm_rel_diff_oracle": abs(norm - rnorm) / rnorm}
    return out


def extra_batched(stn, dev, refined, with_cpu):
    """The 2048-solve batch (per-axis sizes log-U[16,128] seed 4, b ~ N(0,1),
    tol 1e-8) in one persistent scheduler launch: device time of the solve
    (CUDA events) and, in the same run, the end-to-end time including the
    right-hand sides' copy in from pinned host memory and the solutions' copy
    out."""
    import torch
    sizes, seeds = batch_problems(2048)
    tol = 1e-8
    counts = [(nx + 2) * (ny + 2) * (nz + 2) for nx, ny, nz in sizes]
    offs = np.concatenate([[0], np.cumsum(counts)])
    total = int(offs[-1])
    h_rhs = torch.empty(total, dtype=torch.float64).pin_memory()
    hr = h_rhs.numpy()
    for i, (nx, ny, nz) in enumerate(sizes):
        hr[offs[i]:offs[i + 1]] = si.normal_interior(nx, ny, nz, 1, seed=seeds[i]).ravel()
    h_u = torch.empty(total, dtype=torch.float64).pin_memory()
    d_rhs = torch.empty(total, dtype=torch.float64, device=dev)
    d_u = torch.zeros(total, dtype=torch.float64, device=dev)
    us = [d_u[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]
    bs = [d_rhs[offs[i]:offs[i + 1]].view(nz + 2, ny + 2, nx + 2) for i, (nx, ny, nz) in enumerate(sizes)]

    def solve(u_list, b_list):
        if refined:
            return stn.jacobi_solve_batched_refined(u_list, b_list, si.LAPLACE7, 1, tol, 200000, 1e-2, 50, 40)
        return stn.jacobi_solve_batched_f64(u_list, b_list, si.LAPLACE7, 1, tol, 10 ** 7, 100)

    d_rhs.copy_(h_rhs)
    solve(us[:64], bs[:64])  # warm-up: the first 64 problems
    d_u.zero_()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index or 0) as clk:
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        t0 = time.perf_counter()
        d_rhs.copy_(h_rhs, non_blocking=True)
        e[0].record(stream)
        rc, infos = solve(us, bs)
        e[1].record(stream)
        h_u.copy_(d_u, non_blocking=True)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    ms = e[0].elapsed_time(e[1])
    pts = np.array([nx * ny * nz for nx, ny, nz in sizes], dtype=np.float64)
    iters = np.array([i["iters"] for i in infos], dtype=np.float64)
    out = {"workload": "2048 independent 7-point Poisson solves u = S u + b, per-axis sizes log-uniform in [16,128] "
                       "(seed 4), b ~ N(0,1), tol 1e-8, one persistent work-unit scheduler launch, "
                       + ("FP32 sweeps with FP64 refinement" if refined else "FP64"),
           "value": 2048 / (ms * 1e-3), "unit": "solves/s", "seconds": ms * 1e-3,
           "aggregate_glups": float((pts * iters).sum()) / (ms * 1e-3) / 1e9,
           "converged": int(sum(1 for i in infos if i["status"] == 0)),
           "sweeps_median": float(np.median(iters)), "sweeps_max": int(iters.max()),
           "e2e": {"value": 2048 / wall, "unit": "solves/s", "h2d_bytes_per_step": total * 8,
                   "d2h_bytes_per_step": total * 8},
           "gpu_launches": 1, "scheduler_counters": stn.stencil_sched_stats(), "clocks": clk.summary(),
           "roofline": {"bound": "latency", "note": "most grids stay in L2 (<= 17.6 MB per array); the scheduler's "
                        "unit sweeps are bound by latency and, in double, the FP64 pipe"}}
    if not refined:
        # every update of the FP64 batch is a canonical double sweep update
        out["roofline"].update(fp64_pipe(6.0 * float((pts * iters).sum()), ms, load_peaks()[0],
                                         "6 double ops per update over all sweeps of the batch"))
    if with_cpu:
        import oracle
        idx = list(range(0, 2048, 256)) + [int(np.argmax(pts))]
        hu = h_u.numpy()
        rels = []
        for i in idx:
            nx, ny, nz = sizes[i]
            u = hu[offs[i]:offs[i + 1]].reshape(nz + 2, ny + 2, nx + 2)
            b = hr[offs[i]:offs[i + 1]].reshape(nz + 2, ny + 2, nx + 2)
            rels.append(oracle.residual_norm(u, si.LAPLACE7, 1, b) / oracle.interior_norm(b, 1))
        out["cpu_baseline"] = cpu_sample_batched(sizes, seeds, pts, iters)
        out["cpu_baseline"]["oracle_check"] = {
            "problems": idx, "max_rel_res": max(rels), "tol": tol, "all_within_tol": bool(max(rels) <= tol),
            "what": "the oracle's own FP64 residual ||S u + b - u|| / ||b|| of the returned u"}
    return out


def extra_c3(stn, dev, with_cpu):
    """The variable-coefficient configuration (768 x 768 x 384, radius 2,
    a ~ U[0.5,1.5], manufactured sine solution): the full-size float sweep's
    rate and HBM roofline, the double sweep and residual rates, and complete
    refined and plain FP64 solves to 1e-10 on 96 x 96 x 48.  The full-size
    solve to 1e-10 (about ten minutes) runs under --workload varcoef."""
    import torch
    out, res, clocks, _ = varcoef_rates(stn, dev)
    torch.cuda.empty_cache()
    fs = out["full_size"]
    d = {"workload": "768x768x384 variable-coefficient 13-point Poisson, a ~ U[0.5,1.5] (seed 3), manufactured "
                     "(1,1,1) sine solution: full-size float sweep rate; complete solves to 1e-10 on 96x96x48",
         "value": fs["f32_sweep_glups"], "unit": "GLUP/s (float sweep, 768x768x384)",
         "full_size": fs, "reduced_96x96x48": res,
         "speedup_refined_vs_f64_96x96x48": res["plain_f64"]["seconds"] / res["refined"]["seconds"],
         "roofline": varcoef_roofline(fs), "clocks": clocks}
    if with_cpu:
        d["cpu_baseline"] = cpu_sample_varcoef()
    return d


def serve_pool(stn, rhss, arrivals, tol, keep=()):
    """One trace through the refined pool server (engine 1): request i is
    submitted at arrivals[i] s.  Returns (span_s, latencies, statuses, kept
    solutions by index)."""
    kept = {}
    with stn.Server(hbm_budget=40 << 30, tol=tol, refined=True, inner_sweeps=200000, inner_tol=1e-2,
                    check_every=50, max_outer=40, max_inflight=SERVE_WORKERS, engine=1) as srv:
        t0 = time.perf_counter()
        tickets = []
        for i, at in enumerate(arrivals):
            d = at - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit(rhss[i]))
        lat, status = [], []
        for i, t in enumerate(tickets):
            r = srv.wait(t, 3600.0)
            lat.append(r["latency_s"])
            status.append(r["status"])
            if i in keep:
                kept[i] = srv.result(t, rhss[i].shape)
            srv.release(t)
        span = time.perf_counter() - t0
    return span, lat, status, kept


def plain_service_times(stn, rhss, tols, deadline):
    """The plain comparison: one FP64 jacobi_solve_f64 per request, one at a
    time on the whole GPU, in arrival order.  Each request is copied in,
    solved to tols[0], copied out (its service time at tols[0]) and then, from
    that iterate, solved on to tols[1] and copied out again (the continuation
    is the same sequence of sweeps as a direct solve to tols[1]: groups of 50
    from the start).  Returns per-tol service times and statuses, or None past
    the deadline."""
    import torch
    svc = {t: [] for t in tols}
    st = {t: [] for t in tols}
    for i, b in enumerate(rhss):
        if time.perf_counter() > deadline:
            return None, None
        t0 = time.perf_counter()
        d_b = torch.from_numpy(b).cuda()
        d_u = torch.zeros_like(d_b)
        rc, info = stn.jacobi_solve_f64(d_b, d_u, si.LAPLACE7, 1, tols[0], 10 ** 7, 50)
        ta = time.perf_counter()
        d_u.cpu()
        tb = time.perf_counter()
        rc2, info2 = stn.jacobi_solve_f64(d_b, d_u, si.LAPLACE7, 1, tols[1], 10 ** 7, 50)
        d_u.cpu()
        t2 = time.perf_counter()
        svc[tols[0]].append(tb - t0)                 # in, solve to tols[0], out
        st[tols[0]].append(info["status"])
        svc[tols[1]].append((ta - t0) + (t2 - tb))   # in, solve to tols[1], out
        st[tols[1]].append(info2["status"])
    return svc, st


def extra_serving(stn, dev, deadline, with_cpu):
    """Serving (sizes log-U[32,256] seed 6, b ~ N(0,1), Poisson arrivals seed 8,
    40 GiB budget): the FP32-refined pool server at saturation and at three
    offered loads of SERVE_REQUESTS requests each, against the plain FP64
    per-request path on the same requests at the same offered rates, to 1e-10
    and to 1e-8."""
    sizes, seeds = serve_requests(SERVE_REQUESTS)
    rhss = [si.normal_interior(nx, ny, nz, 1, seed=sd) for (nx, ny, nz), sd in zip(sizes, seeds)]
    n = len(rhss)
    pts = np.array([nx * ny * nz for nx, ny, nz in sizes], dtype=np.float64)
    keep = set(range(0, n, 40)) | {int(np.argmax(pts))}
    out = {"workload": f"{n} Poisson solve requests per trace, per-axis sizes log-uniform in [32,256] (seed 6), "
                       "rhs N(0,1), Poisson arrivals (seed 8), 40 GiB admission budget",
           "requests_per_load": n, "engine": f"pool of {SERVE_WORKERS} worker streams on the full-grid kernels",
           "plain": "one jacobi_solve_f64 per request, in arrival order, on the whole GPU; latencies at each "
                    "offered rate from its measured per-request service times through the single-server "
                    "first-come-first-served recursion"}
    solutions = {}

    def refined_block(tol):
        res = {}
        with ClockSampler(dev.index or 0) as clk:
            span, lat, status, kept = serve_pool(stn, rhss, [0.0] * n, tol, keep)
        cap = n / span
        solutions[tol] = kept
        res["saturation"] = {"solves_per_s": cap, "p50_s": pct(lat, 50), "p99_s": pct(lat, 99),
                             "converged": int(sum(1 for x in status if x == 0)), "clocks": clk.summary()}
        res["loads"] = []
        for frac in SERVE_LOADS:
            rate = frac * cap
            est = n / rate * 1.1 + 5
            if time.perf_counter() + est > deadline:
                res["loads"].append({"offered_frac": frac, "skipped": f"time budget (about {est:.0f} s)"})
                continue
            arr = si.poisson_arrival_times(n, rate, seed=8).tolist()
            with ClockSampler(dev.index or 0) as clk:
                span_l, lat_l, st_l, _ = serve_pool(stn, rhss, arr, tol)
            res["loads"].append({"offered_frac": frac, "offered_per_s": rate, "solves_per_s": n / span_l,
                                 "p50_s": pct(lat_l, 50), "p99_s": pct(lat_l, 99),
                                 "converged": int(sum(1 for x in st_l if x == 0)), "clocks": clk.summary()})
        out[f"tol_{tol:g}"] = {"refined": res}

    # the spec comparison first: refined to 1e-10, then the plain path
    # (both tolerances in one pass), then refined to 1e-8
    refined_block(1e-10)
    svc = st = None
    plain_clocks = None
    if time.perf_counter() + 60 > deadline:
        out["plain_skipped"] = "time budget"
    else:
        with ClockSampler(dev.index or 0) as clk:
            svc, st = plain_service_times(stn, rhss, (1e-8, 1e-10), deadline)
        plain_clocks = clk.summary()
        if svc is None:
            out["plain_skipped"] = "time budget (stopped part way)"
    if time.perf_counter() + 30 < deadline:
        refined_block(1e-8)
    else:
        out["tol_1e-08"] = {"skipped": "time budget"}
    if svc is not None:
        for tol in (1e-10, 1e-8):
            key = f"tol_{tol:g}"
            if "refined" not in out.get(key, {}):
                continue
            s_t = svc[tol]
            sat_lat = lindley([0.0] * n, s_t)
            plain = {"saturation": {"solves_per_s": n / sum(s_t), "p50_s": pct(sat_lat, 50), "p99_s": pct(sat_lat, 99),
                                    "converged": int(sum(1 for x in st[tol] if x == 0))},
                     "service_s": {"median": pct(s_t, 50), "max": max(s_t), "sum": sum(s_t)},
                     "clocks": plain_clocks, "loads": []}
            for ld in out[key]["refined"]["loads"]:
                if "offered_per_s" not in ld:
                    continue
                arr = si.poisson_arrival_times(n, ld["offered_per_s"], seed=8).tolist()
                lat_p = lindley(arr, s_t)
                plain["loads"].append({"offered_per_s": ld["offered_per_s"], "p50_s": pct(lat_p, 50),
                                       "p99_s": pct(lat_p, 99),
                                       "solves_per_s": n / max(a + l for a, l in zip(arr, lat_p))})
            out[key]["plain"] = plain
            ref = out[key]["refined"]
            cmp = {"solves_per_s_ratio": ref["saturation"]["solves_per_s"] / plain["saturation"]["solves_per_s"],
                   "p99_ratio_at_saturation": plain["saturation"]["p99_s"] / ref["saturation"]["p99_s"]}
            for lr, lp in zip([x for x in ref["loads"] if "offered_per_s" in x], plain["loads"]):
                cmp[f"p99_ratio_at_{lr['offered_frac']:g}"] = lp["p99_s"] / lr["p99_s"]
            cmp["refined_wins"] = bool(cmp["solves_per_s_ratio"] > 1 and all(
                v > 1 for k, v in cmp.items() if k.startswith("p99_ratio")))
            out[key]["refined_vs_plain"] = cmp
    if with_cpu:
        import oracle
        checks = {}
        t0 = time.perf_counter()
        for tol, kept in solutions.items():
            rels = [oracle.residual_norm(u, si.LAPLACE7, 1, rhss[i]) / oracle.interior_norm(rhss[i], 1)
                    for i, u in kept.items()]
            checks[f"tol_{tol:g}"] = {"requests": sorted(kept), "max_rel_res": max(rels),
                                      "all_within_tol": bool(max(rels) <= tol)}
        t_chk = time.perf_counter() - t0
        # oracle timing sample: the plain C oracle's sweep rate on the median-size request
        i_med = int(np.argsort(pts)[n // 2])
        nx, ny, nz = sizes[i_med]
        t0 = time.perf_counter()
        oracle.stencil_sweep(rhss[i_med], si.LAPLACE7, 1, 200)
        t = time.perf_counter() - t0
        rate = float(nx) * ny * nz * 200 / t
        out["cpu_baseline"] = {"value": rate / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                               "sample": f"200 sweeps of request {i_med} ({nx}x{ny}x{nz}, the median size), plain C "
                                         f"oracle, one thread ({t:.2f} s); the solves themselves would take hours",
                               "oracle_check": checks, "oracle_check_s": t_chk,
                               "what": "the oracle's own FP64 residual ||S u + b - u|| / ||b|| of served solutions "
                                       "(every 40th request and the largest, from the saturation runs)"}
    return out


def run_extras(args, dev):
    import paper_2409_18824_gb300 as stn
    deadline = time.perf_counter() + args.extras_budget
    with_cpu = not args.no_cpu_baseline
    out = {}
    for key, fn in (("c1", lambda: extra_c1(stn, dev, with_cpu)),
                    ("c3", lambda: extra_c3(stn, dev, with_cpu)),
                    ("batched_refined", lambda: extra_batched(stn, dev, True, with_cpu)),
                    ("batched_f64", lambda: extra_batched(stn, dev, False, with_cpu)),
                    ("serving", lambda: extra_serving(stn, dev, deadline, with_cpu))):
        if time.perf_counter() > deadline:
            out[key] = {"skipped": "time budget"}
            continue
        t0 = time.perf_counter()
        try:
            out[key] = fn()
        except Exception as e:  # recorded, never costs the headline line
            out[key] = {"error": f"{type(e).__name__}: {e}"}
        out[key]["wall_s"] = time.perf_counter() - t0
    return out


# ------------------------------------------------------------ oracle (CPU) --
def cpu_sample(wl, sweeps, keep=False):
    import oracle
    nx, ny, nz, r = wl["nx"], wl["ny"], wl["nz"], wl["r"]
    npdt = np.float64 if wl["dtype"] == "f64" else np.float32
    u0 = si.uniform_interior(nx, ny, nz, r, seed=wl["seed"], dtype=npdt)
    oracle.build()
    t0 = time.perf_counter()
    out = oracle.stencil_sweep(u0, si.LAPLACE7, r, sweeps)
    norm = oracle.residual_norm(out, si.LAPLACE7, r)
    t = time.perf_counter() - t0
    val = float(nx) * ny * nz * sweeps / t / 1e9
    return (val, t, out, norm) if keep else (val, t)


def cpu_baseline(wl, sweeps, keep=False):
    val, t, *rest = cpu_sample(wl, sweeps, keep=True)
    d = {"value": val, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
         "sample": f"{sweeps} sweeps + 1 residual norm of the same {wl['nx']}x{wl['ny']}x{wl['nz']} "
                   f"grid, plain C oracle, single thread ({t:.1f} s)"}
    return (d, *rest) if keep else d


def cpu_all_cores(wl, sweeps, ref_out=None, ref_norm=None):
    """The single-thread oracle's sample on every host core, through the
    multi-core host library (libstencil_host.so), whose sweeps are bitwise the
    oracle's for any thread count: checked here against the oracle's output
    when it is given.  Context beside the oracle baseline; FP64 workloads
    only (None otherwise)."""
    if wl["dtype"] != "f64":
        return None
    import paper_2409_18824_gb300.host as host
    nx, ny, nz, r = wl["nx"], wl["ny"], wl["nz"], wl["r"]
    u0 = si.uniform_interior(nx, ny, nz, r, seed=wl["seed"])
    out = np.zeros_like(u0)
    threads = host.threads()
    t0 = time.perf_counter()
    host.stencil_host_sweep_f64(u0, out, si.LAPLACE7, r, sweeps, nthreads=threads)
    norm = host.stencil_host_residual_norm_f64(out, si.LAPLACE7, r, nthreads=threads)
    t = time.perf_counter() - t0
    d = {"value": float(nx) * ny * nz * sweeps / t / 1e9, "unit": "GLUP/s", "cores": threads,
         "kind": "host library (the oracle's arithmetic, multi-threaded)",
         "sample": f"{sweeps} sweeps + 1 residual norm of the same {nx}x{ny}x{nz} grid on {threads} threads "
                   f"({t:.2f} s)"}
    if ref_out is not None:
        d["bitwise_oracle"] = bool(np.array_equal(out.view(np.uint64), ref_out.view(np.uint64)))
    if ref_norm is not None:
        d["norm_rel_diff_oracle"] = abs(norm - ref_norm) / ref_norm if ref_norm else 0.0
    return d


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    times = []
    sweeps = args.cpu_sweeps
    for _ in range(args.warmup):
        cpu_sample(wl, 1)
    for _ in range(args.steps):
        _, t = cpu_sample(wl, sweeps)
        times.append(t)
    total = sum(times)
    value = float(wl["nx"]) * wl["ny"] * wl["nz"] * sweeps * args.steps / total / 1e9
    out = {
        "impl": "reference",
        "metric": "GLUP/s (512^3 7-point Jacobi, FP64)" if wl is WORKLOADS["sweep512"] else f"GLUP/s ({args.workload})",
        "value": value, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
        "config": {"workload": wl["desc"], "nx": wl["nx"], "ny": wl["ny"], "nz": wl["nz"], "radius": wl["r"],
                   "sweeps_per_step": sweeps, "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: {sweeps} sweeps + 1 residual norm of the workload's grid "
                                   f"(plain C oracle, one thread) instead of the full sweep count"},
        "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host": host_info(),
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep512",
                    choices=sorted(WORKLOADS) + ["batch", "serve", "varcoef", "jacobi2d", "jacobi2d_host", "sum",
                                                 "dot", "advect", "advect_host"])
    ap.add_argument("--elements", type=int, default=0,
                    help="sum/dot: elements instead of the paper's size (for profiling a smaller case)")
    ap.add_argument("--host-sweeps", type=int, default=2000,
                    help="jacobi2d_host: sweeps per timed step of the multi-core host path")
    ap.add_argument("--requests", type=int, default=48, help="serving workload: requests per trace")
    ap.add_argument("--loads", type=float, nargs="*", default=[0.5, 0.8, 1.1],
                    help="serving workload: offered loads as fractions of the measured capacity")
    ap.add_argument("--plain", action="store_true", help="serving workload: double Jacobi instead of refinement")
    ap.add_argument("--per-request", action="store_true",
                    help="serving workload: one double solve per request in arrival order (the plain comparison)")
    ap.add_argument("--rates", type=float, nargs="*", default=None,
                    help="serving workload: absolute offered rates (solves/s) instead of --loads fractions")
    ap.add_argument("--batch", type=int, default=2048, help="problems in the batched workload")
    ap.add_argument("--tol", type=float, default=1e-8,
                    help="serving workload: relative residual each request is solved to")
    ap.add_argument("--refined", action="store_true", help="batched workload: FP32 sweeps + FP64 refinement")
    ap.add_argument("--inner-tol", type=float, default=1e-2)
    ap.add_argument("--inner-max", type=int, default=200000)
    ap.add_argument("--cpu-sweeps", type=int, default=20, help="oracle sweeps per CPU sample (~10 s at 512^3)")
    ap.add_argument("--cpu-sweeps2d", type=int, default=4000, help="jacobi2d: oracle sweeps per CPU sample")
    ap.add_argument("--sweeps2d", type=int, default=0, help="jacobi2d: sweeps per step (0: the paper's 100000)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=-1,
                    help="star-kernel variant (-1 automatic, 0 one point/thread, 1/2 register-blocked)")
    ap.add_argument("--chunks", type=int, default=0,
                    help="k chunks per tile column of the star kernels (0 automatic)")
    ap.add_argument("--temporal", type=int, default=0,
                    help="sweeps fused per HBM pass (0 automatic, 1 off, 2..4)")
    ap.add_argument("--autotune", action="store_true",
                    help="sweep workloads: run the sweep autotuner on the workload's extents before timing")
    ap.add_argument("--varcoef-reduced", action="store_true",
                    help="varcoef workload: skip the full-size solve to 1e-10 (about 12 minutes)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the 64^3, batched and serving parts of the line")
    ap.add_argument("--extras-budget", type=float, default=1020.0,
                    help="wall-clock seconds for the 64^3, batched and serving parts of the default line")
    ap.add_argument("--kernel-only", type=int, default=0,
                    help="run only this many single-sweep launches (for profilers), print nothing")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("steps >= 1, warmup >= 0")
    if args.workload == "varcoef":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "variable-coefficient workload: the oracle's "
                              "solve of the 768x768x384 grid to 1e-10 takes days of one core; the tests check "
                              "the GPU against it at 96x96x48 and on sampled windows"}))
            return
        run_varcoef(args)
        return
    if args.workload == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "serving workload: the oracle's solves of "
                              "48 grids of up to 256^3 take about an hour of one core per step; the tests check served results "
                              "against the batched path and it against the oracle"}))
            return
        run_serving(args)
        return
    if args.workload == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "batched workload: the oracle's 2048 solves "
                              "take hours of one core per step; the tests check sampled solves bitwise and the "
                              "default line's cpu_baseline projects the rate"}))
            return
        run_batched(args)
        return
    if args.workload == "advect":
        if args.impl == "reference":
            run_reference_advect(args)
        else:
            run_advect(args)
        return
    if args.workload in INTRINSICS:
        if args.impl == "reference":
            run_reference_intrinsic(args, args.workload)
        else:
            run_intrinsic(args, args.workload)
        return
    if args.workload == "jacobi2d":
        if args.impl == "reference":
            run_reference2d(args)
        else:
            run_jacobi2d(args)
        return
    if args.workload == "advect_host":
        if args.impl == "reference":
            run_reference_advect(args)
        else:
            run_advect_host(args)
        return
    if args.workload == "jacobi2d_host":
        if args.impl == "reference":
            run_reference2d(args)
        else:
            run_jacobi2d_host(args)
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_cuda(args, wl)


if __name__ == "__main__":
    main()
