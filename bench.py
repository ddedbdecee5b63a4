#!/usr/bin/env python
"""Benchmark of the IBM step (3D heated sphere, 256^3 FP32).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload sphere|batched|cylinders|adjoint]

One step = the whole hot path: fluid stage 1 (L(U^n), dt), fluid stage 2
(SSP-RK2 predictor), interpolation + direct forcing at the markers,
spreading + forced update, force/heat sums.  The markers are at rest, so the
bins, the quadrature weights and the spreading operator are built once at
set-up, and the force/heat sums run inside the spreading launch (the kernel
split reports them under "spread_apply").

--workload cylinders times the small L2-resident 2D cases (the heated
cylinder, FP64, static; the transversely oscillating cylinder, FP32, with
its markers, bins and weights rebuilt every step) with direct launches and
with step graphs, and the kernel split of the direct launches.

With N > 1 (torchrun, one process per GPU) every rank runs its own
independent sphere case (Mach x wall-temperature variants): weak scaling,
no collective on the data path.  Rank 0 prints one JSON line.

At N = 1 the sphere line also carries two short passes of the other forms
on the same GPU (skip with --no-extras): "batched" (20 steps of the 64-case
batch against the plain per-case loop) and "adjoint" (50 recorded steps of
the 128^3 sphere, checkpoint every 10, reversed by ibm_backward).

--impl reference times the FP64 CPU oracle on this host's cores on a slab
sample of the same workload (rank 0 only).

--workload batched times 64 independent 2D heated-cylinder cases of uneven
size (128^2 to 512^2, 1 to 8 cylinders each) advanced as one batch: one
persistent launch per stage over (case, tile) work items, the step replayed
from a CUDA graph, tile shape and markers per block autotuned; the plain
per-case loop of single-grid steps is timed beside it on the same cases.
With N > 1 the cases are dealt out to the ranks (weak scaling).

--workload adjoint records K steps of the 128^3 FP32 sphere (Ma 0.5,
Re 100, 804 markers) with a checkpoint every --every steps, then times the
discrete adjoint (ibm_backward: gradient of C_d + Nu with respect to every
marker position and wall temperature) over all K steps.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2301_09349_gb300 import cases as C  # noqa: E402

METRIC = "cell-updates/s + marker-updates/s per IBM step at 1 GB300; % HBM roofline"
UNIT = "cell-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256, help="grid cells per axis")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target seconds of oracle work for the cpu_baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="sphere line without the short batched and adjoint passes")
    p.add_argument("--workload", default="sphere",
                   choices=["sphere", "batched", "adjoint", "cylinders"])
    p.add_argument("--every", type=int, default=50, help="adjoint checkpoint interval")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def case_for(rank: int, world: int, n: int) -> C.Case:
    from paper_2301_09349_gb300 import replicas
    return replicas.case_for_rank(rank, world, n)


def workload_name(c: C.Case, n_kept: int) -> str:
    return ("3D heated sphere %d^3 FP32, Ma %.1f, T_w %.1f, Re 300, %d Fibonacci markers "
            "(%d after one-per-cell dedup)" % (c.grid.n[0], c.grid.Mach, c.Tw[0], len(c.X), n_kept))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash(path: str) -> str:
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; otherwise None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        ent = t[kernel]
        src = os.path.join(ROOT, ent["source"])
        if source_hash(src) != ent["source_sha256_16"]:
            return None
        return float(ent["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, gpu_id: str):
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), "ibm_clocks_%d.csv" % os.getpid())
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--id=" + gpu_id, "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_slab(c: C.Case, nz: int):
    """A z-slab of the workload: same spacing, x-y extent, BCs and physics;
    nz planes centred on the body; markers kept where their support fits."""
    import dataclasses
    g = c.grid
    nz = max(8, min(nz, g.n[2]))
    z0 = -0.5 * nz * g.h
    gs = dataclasses.replace(g, n=(g.n[0], g.n[1], nz), lo=(g.lo[0], g.lo[1], z0))
    cz = np.floor((c.X[:, 2] - z0) / g.h)
    sel = (cz >= 2) & (cz <= nz - 3)
    return gs, c.X[sel], c.Tw[sel]


def oracle_rate(c: C.Case, target_s: float, steps: int, warmup: int, threads: int):
    """Time `steps` oracle steps (after `warmup`) on a slab sized so that the
    whole run takes about target_s seconds.  Returns (cells/s, details)."""
    from oracle import oracle as O
    O.build()
    O.set_threads(threads)
    g = c.grid
    # calibrate the per-cell cost on a 16-plane slab
    gs, X, Tw = oracle_slab(c, 16)
    U = C.initial_state(gs, c.seed).astype(np.float32).astype(np.float64)
    run = O.Run(gs, X, Tw)
    t = time.perf_counter()
    run.step(U)
    per_cell = (time.perf_counter() - t) / gs.ncells
    nz = int(target_s / max(steps + warmup, 1) / (per_cell * g.n[0] * g.n[1]))
    gs, X, Tw = oracle_slab(c, nz)
    U = C.initial_state(gs, c.seed).astype(np.float32).astype(np.float64)
    run = O.Run(gs, X, Tw)
    for _ in range(warmup):
        U = run.step(U)
    t = time.perf_counter()
    for _ in range(steps):
        U = run.step(U)
    el = time.perf_counter() - t
    rate = gs.ncells * steps / el
    sample = ("z-slab %dx%dx%d of the %s case (%d markers), %d timed step(s)"
              % (gs.n[0], gs.n[1], gs.n[2], "x".join(map(str, g.n[: g.dim])), len(run.X), steps))
    return rate, {"seconds": el, "sample": sample, "cells": gs.ncells,
                  "markers": len(run.X), "ms_per_step": 1e3 * el / steps}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    c = case_for(0, 1, args.n)
    threads = os.cpu_count() or 1
    target = max(60.0, min(150.0, 1.2 * (args.steps + args.warmup)))
    rate, det = oracle_rate(c, target, args.steps, args.warmup, threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": det["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(c, det["markers"]) + "; " + det["sample"]},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": det["sample"]},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import torch
    from paper_2301_09349_gb300 import build, ibm
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    c = case_for(rank, world, args.n)
    g = c.grid
    stream = torch.cuda.Stream()
    grid = ibm.Grid(g, max_markers=len(c.X), stream=stream)
    n_kept = grid.set_markers(c.X, c.Tw)
    grid.set_state(C.initial_state(g, c.seed).astype(np.float32))
    N = g.ncells

    grid.step(args.warmup)
    grid.sync()

    uuid = str(torch.cuda.get_device_properties(local).uuid)
    gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    clocks = ClockSampler(gpu_id)
    time.sleep(0.3)
    ibm.ibm_profile(grid.h, True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    grid.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ibm.ibm_profile_read(grid.h)
    ibm.ibm_profile(grid.h, False)
    clk = clocks.stop()
    grid.sync()

    # end to end through the C ABI with host buffers: per step the wall
    # temperatures go up from page-locked memory, the step runs, and the
    # force/heat result comes back (a synchronizing read)
    Tw_pin = torch.empty(n_kept, dtype=torch.float64, pin_memory=True).numpy()
    _, _, idx = grid.markers()
    Tw_pin[:] = c.Tw[idx]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ibm.ibm_set_wall_temperature(grid.h, Tw_pin)
        ibm.ibm_step(grid.h, 1)
        res = ibm.ibm_forces_and_nusselt(grid.h)
    e2e_s = time.perf_counter() - t0
    barrier()

    from paper_2301_09349_gb300 import replicas
    ms_max, e2e_ms_max, cells_all, markers_all = replicas.reduce_timings(
        dist, torch.device("cuda", local), ms, e2e_s * 1e3, float(N), float(n_kept))

    if rank == 0:
        steps = args.steps
        value = cells_all * steps / (ms_max * 1e-3)
        marker_rate = markers_all * steps / (ms_max * 1e-3)
        nc = g.ncomp
        bpe = g.fp_bytes
        alg = {"stage1": 2 * nc * bpe * N, "stage2": 3 * nc * bpe * N}
        peak, peak_kind = measured_peaks()
        kernels = {}
        total_ms = sum(v[0] for v in prof.values())
        for name, (kms, nl) in prof.items():
            if nl == 0:
                continue
            ent = {"launches": nl, "ms_per_launch": kms / nl, "share": kms / total_ms}
            if name in alg:
                ent["GB_per_s"] = alg[name] / (kms / nl * 1e-3) / 1e9
            kernels[name] = ent
        dom = max(("stage1", "stage2"), key=lambda k: prof[k][0])
        dms = prof[dom][0] / prof[dom][1]
        achieved = alg[dom] / (dms * 1e-3) / 1e9
        traffic = traffic_for(dom)
        # the whole step against the same roofline (100 B per cell-step)
        step_bytes = (alg["stage1"] + alg["stage2"]) * steps
        step_frac = step_bytes / (ms / 1e3 if world == 1 else ms_max / 1e3) / 1e9 / peak
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded free stream + 1e-3 density noise; Fibonacci markers)",
            "config": {"workload": workload_name(c, n_kept),
                       "grid": list(g.n), "markers_in": len(c.X), "markers_kept": n_kept,
                       "cases_per_rank": "one independent sphere case per GPU",
                       "l2": "inputs larger than L2 (each state array %.0f MB > 129 MB)"
                             % (nc * bpe * N / 1e6)},
            "marker_updates_per_s": marker_rate,
            "hbm_roofline_frac_step": step_frac,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                                        if peak_kind == "measured" else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": alg[dom]},
            "kernels": kernels,
            "gpu_launches": int(sum(v[1] for v in prof.values())) * world,
            "e2e": {"value": cells_all * steps / (e2e_ms_max * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": 8 * n_kept, "d2h_bytes_per_step": 64,
                    "path": "ibm_set_wall_temperature(pinned host) + ibm_step + "
                            "ibm_forces_and_nusselt per step"},
            "clocks": clk,
            "result": {"Cd": res["Cd"], "Cl": res["Cl"], "Nu": res["Nu"]},
        }
        if world == 1 and not args.no_extras:
            # the batched and adjoint forms, timed briefly on the same GPU so
            # that every run of the default line carries them
            grid.close()
            line["batched"] = extra_batched(20, 3, gpu_id)
            line["adjoint"] = extra_adjoint(50, 10, gpu_id)
        if world == 1 and not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            rate, det = oracle_rate(c, args.cpu_seconds, 1, 0, threads)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads,
                                    "kind": "oracle", "sample": det["sample"]}
            rate1, det1 = oracle_rate(c, max(2.0, args.cpu_seconds / 5.0), 1, 0, 1)
            line["cpu_baseline_single_thread"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                                  "kind": "oracle", "sample": det1["sample"]}
        print(json.dumps(line), flush=True)
    grid.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# batched 2D cylinders
# ---------------------------------------------------------------------------

BATCH_METRIC = ("cell-updates/s of a batch of 64 uneven 2D heated-cylinder cases at 1 GB300 "
                "(one launch per stage over all cases); speed-up over the per-case loop")


def batch_cases(rank: int, world: int):
    """the 64-case batch, cases dealt round-robin to the ranks"""
    cs = C.batched_cylinders()
    return [c for i, c in enumerate(cs) if i % world == rank]


def batch_workload_name(cs) -> str:
    sizes = sorted({c.grid.n[0] for c in cs})
    return ("batch of %d 2D heated-cylinder cases FP32, n^2 cells with n in %s over "
            "[-4,12]x[-8,8], 1-8 cylinders (D = 1) per case, %d markers, T_w~U[0.5,2], "
            "Ma~U[0.1,0.5], Re~U[40,200]"
            % (len(cs), sizes, sum(len(c.X) for c in cs)))


def oracle_batch_rate(cs, target_s: float, threads: int):
    """The oracle over the cases of the batch, one step each (set-up untimed),
    until about target_s seconds of stepping have been spent."""
    from oracle import oracle as O
    O.build()
    O.set_threads(threads)
    cells, el, used = 0, 0.0, 0
    for c in cs:
        run = O.Run(c.grid, c.X, c.Tw)
        U = C.initial_state(c.grid, c.seed).astype(np.float32).astype(np.float64)
        t = time.perf_counter()
        run.step(U)
        el += time.perf_counter() - t
        cells += c.grid.ncells
        used += 1
        if el >= target_s:
            break
    sample = "one step of each of the first %d of the %d cases (%d cells)" % (used, len(cs), cells)
    return cells / el, {"seconds": el, "sample": sample, "ms_per_step": 1e3 * el}


def run_reference_batched(args, rank, world):
    if rank != 0:
        return 0
    cs = batch_cases(0, 1)
    threads = os.cpu_count() or 1
    target = max(30.0, min(150.0, 1.0 * (args.steps + args.warmup)))
    rate, det = oracle_batch_rate(cs, target, threads)
    line = {
        "impl": "reference", "metric": BATCH_METRIC, "value": rate, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": det["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": batch_workload_name(cs) + "; " + det["sample"]},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": det["sample"]},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_and_loop(cs, stream, steps, warmup, barrier, tune_reps, gpu_id=None, profile=False):
    """Set up the cases as one batch (autotuned), time `steps` batched steps,
    then the plain per-case loop of single-grid steps on the same cases.
    Returns the batch (still open), both times in ms, the kept marker counts,
    the tuning, the kernel split (profile=True) and the clock samples taken
    during the batched steps (gpu_id given)."""
    import torch
    from paper_2301_09349_gb300 import ibm
    b = ibm.Batch([c.grid for c in cs], [len(c.X) for c in cs], stream=stream)
    kept = []
    for cg, c in zip(b.cases, cs):
        kept.append(cg.set_markers(c.X, c.Tw))
        cg.set_state(C.initial_state(c.grid, c.seed).astype(np.float32))
    tune_ms = b.autotune(reps=tune_reps)
    tuning = b.tuning()

    def timed(fn, k):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(k)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1)

    b.step(warmup)
    b.sync()
    clocks = ClockSampler(gpu_id) if gpu_id else None
    if clocks is not None:
        time.sleep(0.3)
    ms = timed(b.step, steps)
    clk = clocks.stop() if clocks is not None else None
    b.sync()

    prof = None
    if profile:
        # the same steps launched kernel by kernel with event pairs: the split
        ibm.ibm_batch_profile(b.h, True)
        b.step(steps)
        prof = ibm.ibm_batch_profile_read(b.h)
        ibm.ibm_batch_profile(b.h, False)
        b.sync()

    # the plain per-case loop: one single-grid step per case per step
    loop = []
    for c in cs:
        gr = ibm.Grid(c.grid, max_markers=len(c.X), stream=stream)
        gr.set_markers(c.X, c.Tw)
        gr.set_state(C.initial_state(c.grid, c.seed).astype(np.float32))
        loop.append(gr)

    def loop_steps(k):
        for _ in range(k):
            for gr in loop:
                gr.step(1)

    loop_steps(warmup)
    ms_loop = timed(loop_steps, steps)
    for gr in loop:
        gr.sync()
    for gr in loop:
        gr.close()
    return {"batch": b, "ms": ms, "ms_loop": ms_loop, "kept": kept, "tune_ms": tune_ms,
            "tuning": tuning, "prof": prof, "clocks": clk}


def extra_batched(steps: int, warmup: int, gpu_id: str):
    """Short pass of the 64-case batch beside the sphere line: batched step
    against the plain per-case loop, same GPU, same cases."""
    import torch
    cs = C.batched_cylinders()
    stream = torch.cuda.Stream()
    bm = batch_and_loop(cs, stream, steps, warmup, lambda: None, tune_reps=3, gpu_id=gpu_id)
    bm["batch"].close()
    N = float(sum(c.grid.ncells for c in cs))
    return {"workload": batch_workload_name(cs), "steps": steps, "warmup": warmup,
            "tuning": bm["tuning"],
            "batched_ms_per_step": bm["ms"] / steps,
            "per_case_loop_ms_per_step": bm["ms_loop"] / steps,
            "speedup_of_batch": bm["ms_loop"] / bm["ms"],
            "batched_cell_updates_per_s": N * steps / (bm["ms"] * 1e-3),
            "per_case_loop_cell_updates_per_s": N * steps / (bm["ms_loop"] * 1e-3),
            "timing": "CUDA events on the batch's stream around each loop of steps",
            "clocks": bm["clocks"]}


def run_batched(args, rank, world, local):
    import torch
    from paper_2301_09349_gb300 import build, ibm
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    cs = batch_cases(rank, world)
    stream = torch.cuda.Stream()
    uuid = str(torch.cuda.get_device_properties(local).uuid)
    gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    bm = batch_and_loop(cs, stream, args.steps, args.warmup, barrier, tune_reps=10,
                        gpu_id=gpu_id, profile=True)
    b, ms, ms_loop, kept, tune_ms, tuning, prof, clk = (
        bm["batch"], bm["ms"], bm["ms_loop"], bm["kept"], bm["tune_ms"], bm["tuning"],
        bm["prof"], bm["clocks"])
    N = float(sum(c.grid.ncells for c in cs))

    # end to end through the C ABI with host buffers: per step the wall
    # temperatures of every case go up from page-locked memory in one copy,
    # the batch steps, and the forces of all cases come back in one read
    tws = []
    for cg, c in zip(b.cases, cs):
        _, _, idx = cg.markers()
        tws.append(c.Tw[idx])
    tw_all = np.concatenate(tws)
    Tw_pin = torch.empty(len(tw_all), dtype=torch.float64, pin_memory=True).numpy()
    Tw_pin[:] = tw_all
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ibm.ibm_batch_set_wall_temperature(b.h, Tw_pin)
        ibm.ibm_batch_step(b.h, 1)
        res = ibm.ibm_batch_forces(b.h, len(cs))
    e2e_s = time.perf_counter() - t0
    barrier()

    from paper_2301_09349_gb300 import replicas
    ms_max, e2e_ms_max, cells_all, markers_all = replicas.reduce_timings(
        dist, torch.device("cuda", local), ms, e2e_s * 1e3, N, float(sum(kept)))
    loop_max, _, _, _ = replicas.reduce_timings(
        dist, torch.device("cuda", local), ms_loop, 0.0, N, 0.0)

    if rank == 0:
        steps = args.steps
        value = cells_all * steps / (ms_max * 1e-3)
        nc, bpe = 4, 4
        alg = {"stage1": 2 * nc * bpe * N, "stage2": 3 * nc * bpe * N}
        peak, peak_kind = measured_peaks()
        kernels = {}
        total_ms = sum(v[0] for v in prof.values())
        for name, (kms, nl) in prof.items():
            if nl == 0:
                continue
            ent = {"launches": nl, "ms_per_launch": kms / nl, "share": kms / total_ms}
            if name in alg:
                ent["GB_per_s"] = alg[name] / (kms / nl * 1e-3) / 1e9
            kernels[name] = ent
        dom = max(("stage1", "stage2"), key=lambda k: prof[k][0])
        dms = prof[dom][0] / prof[dom][1]
        achieved = alg[dom] / (dms * 1e-3) / 1e9
        line = {
            "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms_max / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded free stream + 1e-3 density noise; circle markers)",
            "config": {"workload": batch_workload_name(cs), "cases": len(cs),
                       "cells": int(N), "markers_kept": int(sum(kept)),
                       "tuning": tuning,
                       "l2": "inputs larger than L2 (state %.0f MB + stage-1 buffer %.0f MB "
                             "> 129 MB)" % (nc * bpe * N / 1e6, nc * bpe * N / 1e6)},
            "per_case_loop": {"ms_per_step": loop_max / steps,
                              "value": cells_all * steps / (loop_max * 1e-3),
                              "launches_per_step": 5 * len(cs),
                              "speedup_of_batch": loop_max / ms_max},
            "autotune_ms": {"stage_ms_per_shape": list(map(float, tune_ms["stage_ms"])),
                            "interp_ms_per_warps": list(map(float, tune_ms["interp_ms"]))},
            "roofline": {"bound": "hbm", "kernel": "batch_" + dom, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic_for("batch_" + dom),
                         "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                                        if peak_kind == "measured" else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": alg[dom]},
            "kernels": kernels,
            "gpu_launches": 5 * steps * world,
            "e2e": {"value": cells_all * steps / (e2e_ms_max * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": 8 * int(sum(kept)),
                    "d2h_bytes_per_step": 64 * len(cs),
                    "path": "ibm_batch_set_wall_temperature (pinned host) + ibm_batch_step + "
                            "ibm_batch_forces per step"},
            "clocks": clk,
            "result": {"Cd_case0": float(res[0, 3]), "Nu_case0": float(res[0, 5])},
        }
        if world == 1 and not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            rate, det = oracle_batch_rate(cs, args.cpu_seconds, threads)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads,
                                    "kind": "oracle", "sample": det["sample"]}
        print(json.dumps(line), flush=True)
    b.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# discrete adjoint
# ---------------------------------------------------------------------------

ADJ_METRIC = ("reversed cell-steps/s of the discrete adjoint (gradient of C_d + Nu w.r.t. "
              "marker positions and wall temperatures) at 1 GB300")


def run_adjoint(args, rank, world, local):
    import torch
    from paper_2301_09349_gb300 import build, ibm
    build.build()
    torch.cuda.set_device(local)
    if rank != 0:
        return 0
    uuid = str(torch.cuda.get_device_properties(local).uuid)
    am = adjoint_measure(args.steps, args.every, "GPU-" + uuid if not uuid.startswith("GPU-")
                         else uuid)
    c, n_kept, S, fwd_ms, bwd_s, f, gX, gT, clk = (
        am["case"], am["n_kept"], am["steps"], am["fwd_ms"], am["bwd_s"], am["forces"],
        am["gX"], am["gT"], am["clocks"])
    N = c.grid.ncells
    line = {
        "metric": ADJ_METRIC, "value": N * S / bwd_s, "unit": UNIT, "n_gpus": 1,
        "steps": S, "warmup": 0, "ms_per_step": 1e3 * bwd_s / S, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded free stream + 1e-3 density noise; Fibonacci markers)",
        "config": {"workload": "3D sphere 128^3 FP32, Ma 0.5, Re 100, T_w 1.5, %d markers "
                               "(%d kept), %d recorded steps, checkpoint every %d"
                               % (len(c.X), n_kept, S, args.every)},
        "forward_ms_per_step_recording": fwd_ms / S,
        "backward_over_forward": (1e3 * bwd_s) / fwd_ms,
        "J": {"Cd": f["Cd"], "Nu": f["Nu"]},
        "gradient_norms": {"dJ_dX": float(np.linalg.norm(gX)), "dJ_dTw": float(np.linalg.norm(gT))},
        "clocks": clk,
        "timing": "host wall clock around the synchronizing ibm_backward call",
    }
    print(json.dumps(line), flush=True)
    return 0


def adjoint_measure(S: int, every: int, gpu_id=None):
    """Record S steps of the 128^3 adjoint sphere (checkpoint every `every`),
    then time ibm_backward over all of them (host wall clock around the
    synchronizing call)."""
    import torch
    from paper_2301_09349_gb300 import ibm
    c = C.adjoint_sphere()
    g = c.grid
    stream = torch.cuda.Stream()
    grid = ibm.Grid(g, max_markers=len(c.X), stream=stream)
    n_kept = grid.set_markers(c.X, c.Tw)
    grid.set_state(C.initial_state(g, c.seed).astype(np.float32))
    grid.record(S, every)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    grid.step(S)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    f = grid.forces()
    clocks = ClockSampler(gpu_id) if gpu_id else None
    if clocks is not None:
        time.sleep(0.3)
    t0 = time.perf_counter()
    gX, gT = grid.backward(1.0, 1.0)        # synchronizing
    bwd_s = time.perf_counter() - t0
    clk = clocks.stop() if clocks is not None else None
    grid.close()
    return {"case": c, "n_kept": n_kept, "steps": S, "every": every, "fwd_ms": fwd_ms,
            "bwd_s": bwd_s, "forces": f, "gX": gX, "gT": gT, "clocks": clk}


def extra_adjoint(S: int, every: int, gpu_id: str):
    """Short adjoint pass beside the sphere line."""
    am = adjoint_measure(S, every, gpu_id)
    c = am["case"]
    N = c.grid.ncells
    return {"workload": "3D sphere 128^3 FP32, Ma 0.5, Re 100, T_w 1.5, %d markers (%d kept), "
                        "%d recorded steps, checkpoint every %d"
                        % (len(c.X), am["n_kept"], S, every),
            "reversed_ms_per_step": 1e3 * am["bwd_s"] / S,
            "forward_ms_per_step_recording": am["fwd_ms"] / S,
            "backward_over_forward": 1e3 * am["bwd_s"] / am["fwd_ms"],
            "reversed_cell_steps_per_s": N * S / am["bwd_s"],
            "timing": "host wall clock around the synchronizing ibm_backward call",
            "clocks": am["clocks"]}


# ---------------------------------------------------------------------------
# small 2D cylinders: time per step, direct launches vs CUDA graphs
# ---------------------------------------------------------------------------

CYL_METRIC = "us per IBM step of the small 2D cylinder cases (L2-resident), direct vs CUDA graphs"


def run_cylinders(args, rank, world, local):
    import torch
    from paper_2301_09349_gb300 import build, ibm
    build.build()
    torch.cuda.set_device(local)
    if rank != 0:
        return 0
    stream = torch.cuda.Stream()
    out = {}
    for c in (C.heated_cylinder(), C.oscillating_cylinder()):
        g = c.grid
        res = {}
        for k in (0, 10):
            grid = ibm.Grid(g, max_markers=len(c.X), stream=stream)
            grid.set_markers(c.X, c.Tw, motion=c.motion)
            grid.set_state(C.initial_state(g, c.seed).astype(
                np.float32 if g.fp_bytes == 4 else np.float64))
            grid.use_graphs(k)
            grid.step(max(args.warmup, 10))
            grid.sync()
            if k == 0:       # the kernel split of direct launches
                ibm.ibm_profile(grid.h, True)
                grid.step(args.steps)
                prof = ibm.ibm_profile_read(grid.h)
                ibm.ibm_profile(grid.h, False)
                res["split_us_per_step"] = {n: 1e3 * ms / args.steps
                                            for n, (ms, nl) in prof.items() if nl}
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            grid.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            grid.sync()
            res["graphs" if k else "direct"] = 1e3 * e0.elapsed_time(e1) / args.steps
            grid.close()
        out[c.name] = {"cells": g.ncells, "fp": "f%d" % (8 * g.fp_bytes),
                       "moving_markers": c.motion is not None,
                       "us_per_step_direct": res["direct"], "us_per_step_graphs": res["graphs"],
                       "split_us_per_step": res["split_us_per_step"],
                       "launch_overhead_us_per_step": res["direct"] - res["graphs"]}
    osc = out[C.oscillating_cylinder().name]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle on the host cores, whole grids: the heated cylinder for
        # its 200 configured steps, the oscillating cylinder for 50 steps
        from oracle import oracle as O
        O.build()
        threads = os.cpu_count() or 1
        O.set_threads(threads)
        for c, nsteps in ((C.heated_cylinder(), 200), (C.oscillating_cylinder(), 50)):
            U = C.initial_state(c.grid, c.seed).astype(
                np.float32 if c.grid.fp_bytes == 4 else np.float64).astype(np.float64)
            run = O.Run(c.grid, c.X, c.Tw, motion=c.motion)
            t0 = time.perf_counter()
            for _ in range(nsteps):
                U = run.step(U)
            el = time.perf_counter() - t0
            out[c.name]["oracle"] = {"cell_updates_per_s": c.grid.ncells * nsteps / el,
                                     "us_per_step": 1e6 * el / nsteps, "steps": nsteps,
                                     "cores": threads}
        o = out[C.oscillating_cylinder().name]["oracle"]
        cpu = {"value": o["cell_updates_per_s"], "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "whole 1024x512 oscillating-cylinder grid, 50 steps (markers moved, "
                         "quadrature re-solved every step); the heated cylinder's 200 steps "
                         "are in cases"}
    line = {
        "metric": CYL_METRIC, "value": osc["cells"] * 1e6 / osc["us_per_step_graphs"],
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": osc["us_per_step_graphs"] / 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "2D heated cylinder 128x64 FP64 (static) and 2D oscillating "
                               "cylinder 1024x512 FP32 (moving markers, bins and quadrature "
                               "rebuilt every step); value = the latter with graphs",
                   "l2": "L2-resident by design (states of 0.26 and 8.4 MB)"},
        "cases": out,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload == "adjoint":
        return run_adjoint(args, rank, world, local)
    if args.workload == "cylinders":
        return run_cylinders(args, rank, world, local)
    if args.workload == "batched":
        if args.impl == "reference":
            return run_reference_batched(args, rank, world)
        return run_batched(args, rank, world, local)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
