#!/usr/bin/env python
"""Benchmark of the explicit ARK step on GB300.

Workload (default): 3D Rayleigh-Benard layer, 512 x 512 x 256 cells, box
2 x 2 x 1, polytrope m = 0.1, chi = 1.1, Ra = 1e7, Pr = 1, no-slip
fixed-temperature walls in z, periodic in x and y, velocity perturbation
U(-1e-3, 1e-3) from numpy default_rng(4) -- synthetic data built by
``paper_1903_09043_gb300.inputs``.  A step is one launch of the fused step
kernel over all 64 Mi cells (acoustic faces, tilde states, transport,
viscous and heat fluxes, next CFL time step).

Paths timed: ``f32split`` (headline: FP32 state and stencil arithmetic, FP64
base state) and ``f64`` (FP64 throughout) on that workload; ``f32split_2d``
on the 2D Rayleigh-Benard layer (8192 x 4096); ``gresho_f32split``,
``gresho_f32`` (plain FP32 state) and ``gresho_f64`` on the inviscid Gresho
vortex (8192 x 8192, Sec. 4.2), where the step does the fewest operations per
byte; and the 256-run ensemble.
``--impl reference`` times the FP64 CPU oracle on slabs of the same workload
instead.

Output: one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per time step"
UNIT = "cell-updates/s"
WORKLOAD = {"workload": "rayleigh_benard_3d_512x512x256", "dim": 3, "n": [512, 512, 256], "box": [2.0, 2.0, 1.0],
            "polytrope_m": 0.1, "chi": 1.1, "Ra": 1e7, "Pr": 1.0, "perturbation": 1e-3, "seed": 4,
            "bc": "periodic x,y; no-slip fixed-T walls z", "low_mach": 1, "cfl": 0.8}
# algorithmic HBM bytes per cell-update: every conserved field read once and written once
ALG_BYTES = {("f64", 3): 80, ("f32", 3): 40, ("f32split", 3): 40, ("f64", 2): 64, ("f32", 2): 32, ("f32split", 2): 32}
STEP_KERNEL = "ark_step_kernel"
# algorithmic floating-point operations per cell-update of the scheme (each add,
# sub, mul, div, sqrt, abs, min, max counted once; every face computed once and
# shared by its two cells): primitives, acoustic faces, tilde state, upwind
# transport, viscous and heat fluxes, CFL wave rate.  Per-row counts are
# tabulated with the kernel descriptions in the design notes.
ALG_FLOPS = {(3, True): 392, (3, False): 213, (2, True): 225, (2, False): 144}
# ALU peaks from unit counts and the maximum SM clock: 152 SMs x 128 FP32 lanes
# x 2 (FMA) x 2.07 GHz; FP64: 152 SMs x 2 FP64 FMA per clock x 2 x 2.07 GHz.
SMS, SM_GHZ = 152, 2.07
ALU_PEAK_TFLOPS = {"f32": SMS * 128 * 2 * SM_GHZ / 1e3, "f64": SMS * 2 * 2 * SM_GHZ / 1e3}
# instruction issue peak: 4 schedulers per SM, one warp instruction each per clock
ISSUE_PEAK_GWARP = SMS * 4 * SM_GHZ


# 2D roofline line: the Rayleigh-Benard layer of Sec. 4.5 (2D polytrope m = 1.3,
# chi = 1.1, box 2 x 1, Ra = 1.1 Ra_c, perturbation 1e-4 from default_rng(2)) on
# 8192 x 4096 cells (FP32 state 0.54 GB, larger than L2).
WORKLOAD_2D = {"workload": "rayleigh_benard_2d_8192x4096", "dim": 2, "n": [8192, 4096], "box": [2.0, 1.0],
               "polytrope_m": 1.3, "chi": 1.1, "Ra": 1.1 * 1707.76, "Pr": 1.0, "perturbation": 1e-4, "seed": 2,
               "bc": "periodic x; no-slip fixed-T walls y", "low_mach": 1, "cfl": 0.8}
# Roofline line where HBM can bind: the inviscid Gresho vortex of Sec. 4.2
# (periodic unit square, rho0 = 1, Ma = 1e-2, low-Mach correction on) on
# 8192 x 8192 cells (FP32 state 1.07 GB, FP64 2.1 GB), 144 flops per cell.
WORKLOAD_GRESHO = {"workload": "gresho_2d_8192x8192", "dim": 2, "n": [8192, 8192], "box": [1.0, 1.0],
                   "mach": 1e-2, "bc": "periodic x,y", "inviscid": True, "low_mach": 1, "cfl": 0.8}
# path name -> (precision, workload kind)
PATHS = {"f32split": ("f32split", "3d"), "f64": ("f64", "3d"), "f32": ("f32", "3d"),
         "f32split_2d": ("f32split", "2d"), "gresho_f32split": ("f32split", "gresho"),
         "gresho_f64": ("f64", "gresho"), "gresho_f32": ("f32", "gresho")}

# A smaller case of the same set-up (state 160 MB FP32 / 320 MB FP64, still larger
# than L2) used for ncu captures, which replay each launch many times.
SMALL = dict(WORKLOAD, workload="rayleigh_benard_3d_256x256x128", n=[256, 256, 128])
SMALL_2D = dict(WORKLOAD_2D, workload="rayleigh_benard_2d_4096x2048", n=[4096, 2048])   # FP32 state 134 MB
SMALL_GRESHO = dict(WORKLOAD_GRESHO, workload="gresho_2d_4096x4096", n=[4096, 4096])    # FP32 state 268 MB


def make_workload(w=WORKLOAD):
    from paper_1903_09043_gb300 import inputs as I
    if w["workload"].startswith("gresho"):
        return I.gresho(w["n"][0], mach=w["mach"], low_mach=w["low_mach"], cfl=w["cfl"])
    return I.rayleigh_benard(w["dim"], tuple(w["n"]), m=w["polytrope_m"], chi=w["chi"], Ra=w["Ra"], Pr=w["Pr"],
                             amp=w["perturbation"], seed=w["seed"], low_mach=w["low_mach"], cfl=w["cfl"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_traffic(path, key="bytes_per_launch_full"):
    """DRAM bytes per launch of the step kernel (or, with ``key``, another
    recorded figure) from the committed ncu figures
    (profiles/step_kernel_traffic.txt), valid only while the step kernel
    sources are unchanged (their hash is recorded with the figures)."""
    import hashlib
    try:
        rec = {}
        with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 2 and not line.startswith("#"):
                    rec[parts[0]] = parts[1]
        h = hashlib.sha256()
        for name in ("ark_common.cuh", "ark_step.cuh", "ark_step2.cuh"):
            with open(os.path.join(ROOT, "paper_1903_09043_gb300", "csrc", name), "rb") as g:
                h.update(g.read())
        if rec.get("source_sha256") != h.hexdigest():
            return None
        v = rec.get(f"{path}.{key}")
        return float(v) if v is not None else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(", ") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 7:
                continue
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except ValueError:
                continue
            for k, v in zip(names, r[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(k)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier_and_max(value, world):
    """Maximum of a per-rank value over all ranks (the slowest rank's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank, ms_per_step_local, world):
    """Whole-job cell-updates/s: every rank advances its own replica of the
    workload, so the job processes world x cells per step in the slowest rank's time."""
    ms_max = barrier_and_max(ms_per_step_local, world)
    return cells_per_rank * world / (ms_max * 1e-3), ms_max


def cpu_baseline(prob, U, seconds=10.0, single_seconds=4.0):
    """The FP64 oracle on one-step slabs of the workload (8 z planes each), on
    all host cores (the reported value) and on one core."""
    import oracle as O
    cores = os.cpu_count() or 1
    dt = O.dt(prob, U)
    nz = prob.n[2]

    def rate(threads, budget):
        O.set_threads(threads)
        cells, k = 0, 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget:
            z0 = (8 * k) % (nz - 8)
            O.step_window(prob, U, dt, [0, 0, z0], [prob.n[0], prob.n[1], z0 + 8])
            cells += prob.n[0] * prob.n[1] * 8
            k += 1
        return cells / (time.perf_counter() - t0), k

    value, k = rate(cores, seconds)
    single, k1 = rate(1, single_seconds)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} one-step slabs of 512x512x8 cells of the workload (FP64 oracle, OpenMP {cores} threads)",
            "single_thread": {"value": single, "unit": UNIT, "cores": 1,
                              "sample": f"{k1} one-step slabs of 512x512x8 cells, one thread"},
            "configs": cpu_configs(cores)}


def cpu_configs(cores, budget=1.0):
    """The FP64 oracle on the smaller stated configurations, whole-grid CFL
    steps for about ``budget`` seconds each, on all cores and on one core:
    the 128 x 128 isothermal atmosphere, the 256 x 128 Rayleigh-Benard layer
    and the 1024 x 1024 Gresho vortex (Ma = 1e-2)."""
    import oracle as O
    from paper_1903_09043_gb300 import inputs as I
    cases = {"atmosphere_2d_128x128": I.atmosphere((128, 128)),
             "rayleigh_benard_2d_256x128": I.rayleigh_benard(2, (256, 128)),
             "gresho_2d_1024x1024": I.gresho(1024, mach=1e-2)}
    out = {}
    for name, (prob, U) in cases.items():
        row = {}
        for threads in (cores, 1):
            O.set_threads(threads)
            V, k = U, 0
            t0 = time.perf_counter()
            while k == 0 or time.perf_counter() - t0 < budget:
                V = O.step(prob, V, O.dt(prob, V))
                k += 1
            el = time.perf_counter() - t0
            row["all_cores" if threads == cores else "one_core"] = {
                "value": prob.ncells * k / el, "ms_per_step": 1e3 * el / k, "steps": k, "cores": threads}
        out[name] = row
    O.set_threads(cores)
    return out


def run_config(workload, world):
    """The ``config`` object of the result line (the same in both arms)."""
    return dict(workload, l2="inputs (0.5-2.7 GB) exceed L2 (129 MB); no flush",
                parallelism="replicas" if world > 1 else "single GPU")


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle as O
    prob, U = make_workload()
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    dt = O.dt(prob, U)
    nz = prob.n[2]
    slab = 2
    cells = prob.n[0] * prob.n[1] * slab

    def one(k):
        z0 = (slab * k) % (nz - slab)
        O.step_window(prob, U, dt, [0, 0, z0], [prob.n[0], prob.n[1], z0 + slab])

    for k in range(args.warmup):
        one(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(k)
    el = time.perf_counter() - t0
    value = cells * args.steps / el
    sample = f"each step: one FP64 oracle step of a 512x512x{slab} slab of the workload ({cells} cells)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(WORKLOAD, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_path(prob, U, precision, args, world, stream, sampler=None, min_sampled_s=1.0, max_blocks=100):
    """Device time of K back-to-back steps (CUDA events on the launching stream).
    With a clock sampler the timed block of exactly K steps is repeated until
    the sampled region lasts ``min_sampled_s`` (a short block holds too few
    nvidia-smi samples), and the median block is reported."""
    import torch
    from paper_1903_09043_gb300 import ark
    s = ark.Solver(prob, precision, stream=stream.cuda_stream)
    s.set_state(U)
    s.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
    blocks = []
    t_start = time.perf_counter()
    while True:
        torch.cuda.synchronize()
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        blocks.append(ev0.elapsed_time(ev1) / args.steps)
        if not sampler or len(blocks) >= max_blocks or time.perf_counter() - t_start >= min_sampled_s:
            break
    clocks = sampler.stop() if sampler else None
    ms = statistics.median(blocks)
    ms_max = barrier_and_max(ms, world)
    d = s.diagnostics(check=False)
    shape = s.launch_shape()
    s.close()
    return ms, ms_max, d, shape, clocks, len(blocks)


E2E_BLOCKS = 5


def e2e_path(prob, U, path, args, stream):
    """Through the C ABI with host buffers: upload the FP64 state from pinned
    host memory, K steps each followed by a read of (t, dt), download the state."""
    import numpy as np
    import torch
    from paper_1903_09043_gb300 import ark
    pinned = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
    host = pinned.numpy()
    host[...] = U
    out = torch.empty(U.shape, dtype=torch.float64, pin_memory=True).numpy()
    s = ark.Solver(prob, path, stream=stream.cuda_stream)
    s.set_state(host)
    s.step(args.warmup)
    s.time()
    s.get_state(out)      # both host buffers have been through a copy before the timed blocks
    torch.cuda.synchronize()
    # E2E_BLOCKS timed blocks, the median reported: a host<->device copy of the
    # state takes from one to four times its usual time from call to call.
    els = []
    for _ in range(E2E_BLOCKS):
        t0 = time.perf_counter()
        s.set_state(host)
        for _ in range(args.steps):
            s.step(1)
            s.time()
        s.get_state(out)
        els.append(time.perf_counter() - t0)
    s.close()
    el = sorted(els)[len(els) // 2]
    nbytes = U.nbytes
    return {"value": prob.ncells * args.steps / el, "unit": UNIT,
            "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": 16 + nbytes / args.steps,
            "steps_per_upload": args.steps, "blocks": E2E_BLOCKS,
            "block_values": [prob.ncells * args.steps / e for e in els],
            "note": (f"one FP64 state upload, {args.steps} steps each followed by a 16-byte (t, dt) read, "
                     f"one FP64 state download; median of {E2E_BLOCKS} such blocks; the rate rises with the "
                     "steps per upload")}


def batch_path(args, stream, hbm):
    """Ensemble of 256 independent 2D Rayleigh-Benard runs (grids 64x32 to 512x256,
    Ra in [1e3, 1e6], seeded), FP32-split: one launch per step for all runs (CUDA
    graph replay, autotuned tiles), against the same runs advanced one at a time."""
    import torch
    from paper_1903_09043_gb300 import ark, inputs as I
    runs = I.ensemble(256, seed=5)
    probs = [p for p, _ in runs]
    cells = sum(p.ncells for p in probs)
    b = ark.Batch(probs, "f32split", stream=stream.cuda_stream)
    for i, (_, U) in enumerate(runs):
        b.set_state(i, U)
    tx, planes = b.tune(reps=3)
    b.step(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    shape = b.shape()
    bad = sum(1 for i in range(len(runs)) if b.diagnostics(i, check=False)["status"])
    b.close()
    # the same runs, one at a time (one grid, one launch per step, runs in sequence)
    solvers = []
    for p, U in runs:
        s = ark.Solver(p, "f32split", stream=stream.cuda_stream)
        s.set_state(U)
        s.step(args.warmup)
        solvers.append(s)
    torch.cuda.synchronize()
    ev0.record(stream)
    for s in solvers:
        s.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_one = ev0.elapsed_time(ev1) / args.steps
    for s in solvers:
        s.close()
    achieved = cells * ALG_BYTES[("f32split", 2)] / (ms * 1e-3) / 1e9
    flops = ALG_FLOPS[(2, all(p.mu > 0 or p.kappa > 0 for p in probs))]
    tflops = cells * flops / (ms * 1e-3) / 1e12
    wipc = kernel_traffic("batch", "warp_inst_per_cell")
    issue = None
    if wipc is not None:
        gw = wipc * cells / (ms * 1e-3) / 1e9
        issue = {"achieved": gw, "peak": ISSUE_PEAK_GWARP, "unit": "G warp-instructions/s",
                 "frac": gw / ISSUE_PEAK_GWARP, "warp_inst_per_cell": wipc,
                 "peak_kind": "4 issue slots per SM per clock at the maximum SM clock; instructions per cell from ncu"}
    return {"value": cells / (ms * 1e-3), "ms_per_step": ms, "runs": len(runs), "cells": cells, "dtype": "f32",
            "one_at_a_time_value": cells / (ms_one * 1e-3), "one_at_a_time_ms_per_step": ms_one,
            "speedup_vs_one_at_a_time": ms_one / ms, "tile": shape, "tuned": {"tx": tx, "planes": planes},
            "launches_per_step": 1, "runs_with_status": bad,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "alg_bytes_per_cell": ALG_BYTES[("f32split", 2)], "traffic": kernel_traffic("batch"),
                         "alu": {"achieved": tflops, "peak": ALU_PEAK_TFLOPS["f32"], "unit": "TFLOP/s",
                                 "frac": tflops / ALU_PEAK_TFLOPS["f32"], "alg_flops_per_cell": flops},
                         "issue": issue}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--paths", default="f32split,f64,f32split_2d,gresho_f32split,gresho_f32,gresho_f64",
                    help="comma list of " + ", ".join(PATHS) + "; the first is the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--workload", default="full", choices=["full", "small"],
                    help="small: 256x256x128 case of the same set-up, for profiler captures")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1903_09043_gb300 import ark  # noqa: F401  (fails loudly without libark.so)
    wl = SMALL if args.workload == "small" else WORKLOAD
    prob, U = make_workload(wl)
    stream = torch.cuda.Stream()
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    paths = [p for p in args.paths.split(",") if p]
    for p in paths:
        if p not in PATHS:
            raise SystemExit(f"unknown path {p}; choose from {', '.join(PATHS)}")
    small = args.workload == "small"
    wdefs = {"3d": wl, "2d": SMALL_2D if small else WORKLOAD_2D, "gresho": SMALL_GRESHO if small else WORKLOAD_GRESHO}
    works = {"3d": (prob, U)}
    results = {}
    head = paths[0]
    timed_blocks = 1
    for path in paths:
        precision, kind = PATHS[path]
        if kind not in works:
            works[kind] = make_workload(wdefs[kind])
        pprob, pU = works[kind]
        with torch.cuda.stream(stream):
            sampler = ClockSampler(local) if (rank == 0 and path == head) else None
            ms, ms_max, d, shape, clocks, nblocks = time_path(pprob, pU, precision, args, world, stream, sampler)
        if path == head:
            timed_blocks = nblocks
        cells = pprob.ncells
        B = ALG_BYTES[(precision, pprob.dim)]
        achieved = cells * B / (ms * 1e-3) / 1e9
        traffic = kernel_traffic(path)
        dt_kind = "f64" if precision == "f64" else "f32"
        flops = ALG_FLOPS[(pprob.dim, pprob.mu > 0 or pprob.kappa > 0)]
        tflops = cells * flops / (ms * 1e-3) / 1e12
        alu_peak = ALU_PEAK_TFLOPS[dt_kind]
        wipc = kernel_traffic(path, "warp_inst_per_cell")
        issue = None
        if wipc is not None:
            gw = wipc * cells / (ms * 1e-3) / 1e9
            issue = {"achieved": gw, "peak": ISSUE_PEAK_GWARP, "unit": "G warp-instructions/s",
                     "frac": gw / ISSUE_PEAK_GWARP, "warp_inst_per_cell": wipc,
                     "peak_kind": "4 issue slots per SM per clock at the maximum SM clock; instructions per cell from ncu"}
        results[path] = {
            "value": cells * world / (ms_max * 1e-3), "ms_per_step": ms_max, "dtype": dt_kind,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic, "alg_bytes_per_cell": B,
                         "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                         "alu": {"achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak,
                                 "alg_flops_per_cell": flops,
                                 "peak_kind": f"{dt_kind.upper()} peak from unit counts and the maximum SM clock"},
                         "issue": issue},
            "launch": shape, "final_t": d["t"], "final_dt": d["dt"], "status": d["status"], "clocks": clocks,
            "workload": wdefs[kind]["workload"],
        }
    h = results[head]
    line = {"metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": h["dtype"], "data": "synthetic",
            "config": run_config(wdefs[PATHS[head][1]], world),
            "path": head,
            "timed_blocks": (f"{timed_blocks} blocks of exactly {args.steps} steps, median reported "
                             "(repeated so that the clock sampler sees the timed region)"),
            "roofline": h["roofline"], "clocks": h["clocks"], "gpu_launches": args.steps,
            "paths": {p: {k: v for k, v in r.items() if k != "clocks"} for p, r in results.items()}}
    if not args.no_batch:
        with torch.cuda.stream(stream):
            line["paths"]["batch"] = batch_path(args, stream, hbm)
    # speed-ups at the accuracies the tests hold (FP64 within 1e-12 of the oracle,
    # the FP32 forms within their per-step budget)
    sp = {}
    if "f32split" in results and "f64" in results:
        sp["f32split_vs_f64"] = results["f64"]["ms_per_step"] / results["f32split"]["ms_per_step"]
    if "batch" in line["paths"]:
        sp["batch_vs_one_at_a_time"] = line["paths"]["batch"]["speedup_vs_one_at_a_time"]
    if sp:
        line["speedups"] = sp
    if rank == 0 and not args.no_e2e:
        with torch.cuda.stream(stream):
            hprec, hkind = PATHS[head]
            hprob, hU = works[hkind]
            line["e2e"] = e2e_path(hprob, hU, hprec, args, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "full":
        line["cpu_baseline"] = cpu_baseline(prob, U)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
