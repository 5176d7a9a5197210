#!/usr/bin/env python
"""Throughput of the occupancy-grid sampling + compositing hot path on GB300.

One step = one pass of the path over one batch of synthetic rays (Algorithm 1
of NerfAcc, arXiv 2305.04966): occupancy-grid march with early termination
into packed samples, the analytic field at the samples (harness stand-in for
the radiance field), render_fwd, an L2 loss against a seeded target image
(harness), render_bwd.  Workload (default): the full 800x800 pinhole image
(640,000 rays) of the 8-blob scene with a 4-level 128^3 cascaded occupancy
grid and up to 1024 lattice steps per ray.

Prints ONE JSON line (rank 0).  ``value`` = rays/s over all ranks with
inputs resident in HBM, timed with CUDA events on the launching stream;
``e2e`` = the same metric through the public API with the step's inputs
copied from pinned host memory and the rendered image + loss copied back
inside the timed region.  ``--impl reference`` times the CPU oracle instead
(the reference arm of this comparison).

Multi-GPU (torchrun): every rank renders its own view (weak scaling, no
collective on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "rays/s & samples/s, march+composite fwd+bwd, % of HBM roofline, vs CPU oracle"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
L2_FLUSH_BYTES = 512 << 20  # > 129 MB of L2

# Algorithmic bytes (what the method must move), S = samples, R = rays.
#   march:      rays read once (24 R), packed samples written (12 S: ray id, t0, t1),
#               CSR offsets written (8 R)
#   render_fwd: t0, t1, sigma, rgb read (24 S), offsets (8 R), rgb/opacity/depth/T_N written (24 R)
#   render_bwd: t0, t1, sigma, rgb read (24 S), dsigma, drgb written (16 S), offsets (8 R),
#               per-ray upstream gradients (20 R)
BYTES = {
    "march": (12, 32),
    "render_fwd": (24, 32),
    "render_bwd": (40, 28),
}
# march with a field: two block summaries, run walk, early-stop pass, exact decisions of the rays it
# queued, scan, fill (and a 24-byte memset of the work counters)
KERNELS_PER_STEP = {"march": 7, "field": 1, "render_fwd": 1, "loss": 1, "render_bwd": 1}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--width", type=int, default=800)
    ap.add_argument("--height", type=int, default=800)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-aux", action="store_true", help="skip the grid-update / sample_pdf timings")
    ap.add_argument("--aux-legs", default="update,step,proposal,unbounded",
                    help="comma list of auxiliary legs: update (grid update / sample_pdf timings), step (the "
                         "training batch's whole step incl. the grid update as one CUDA graph), proposal "
                         "(learned and combined estimators), unbounded (grid vs proposal on unbounded scenes)")
    ap.add_argument("--unbounded-cams", type=int, default=16,
                    help="cameras of the unbounded-scene leg (16 = the 4,194,304-ray workload)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target oracle CPU time")
    ap.add_argument("--shard", choices=["view", "batch"], default="view",
                    help="N > 1: every rank renders its own camera view (weak scaling), or the ranks split the "
                         "rays of one view into contiguous ranges (strong scaling); no collective either way")
    ap.add_argument("--profile", choices=["image", "training", "unbounded"], default=None,
                    help="run only --warmup + --steps eager steps of one workload's training step (march, field, "
                         "render fwd, L2 loss, render bwd; the training batch adds the grid update; the unbounded "
                         "scene at K = 512) and print their mean time: the command the launch lists under "
                         "profiles/ are taken on")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed helpers (host logic, testable with gloo on CPU)
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def view_for_rank(rank: int) -> int:
    """Each rank renders its own camera view; rank 0 renders the reference view."""
    return rank


def ray_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous shard [lo, hi) of n rays that rank takes when one batch is
    split over the ranks (sizes differ by at most one; rays are independent, so
    the shards need no exchange)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_workload(args, rank: int, world: int):
    """The bench workload of one rank: its own camera view (--shard view, weak
    scaling) or its contiguous range of the rays of view 0 (--shard batch,
    strong scaling)."""
    if args.shard == "batch" and world > 1:
        w = workloads.c2_image(args.width, args.height, view=0)
        lo, hi = ray_range(w.n_rays, rank, world)
        return workloads.dataclasses.replace(
            w, name=f"{w.name}_rays{lo}-{hi}", rays_o=np.ascontiguousarray(w.rays_o[lo:hi]),
            rays_d=np.ascontiguousarray(w.rays_d[lo:hi]), target=np.ascontiguousarray(w.target[lo:hi]))
    return workloads.c2_image(args.width, args.height, view=view_for_rank(rank))


def reduce_max(value: float, dist=None) -> float:
    """Max of a float over ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        return self.summarise(rows)

    @classmethod
    def summarise(cls, rows):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows]
        util = [num(r[4]) for r in rows]
        load = [s for s, u in zip(sm, util) if s is not None and u is not None and u >= 50]
        if not load:
            load = [s for s in sm if s is not None]
        reasons = set()
        for r in rows:
            for name, v in zip(cls.REASONS, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load)}


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline / reference arm)
# ---------------------------------------------------------------------------

class OraclePipeline:
    """The oracle's march (FP32, early stop) + FP64 field + FP64 compositing +
    L2 gradient + FP64 adjoint on a subset of the workload's rays; per-stage
    wall times of the last run in ``stage_s``."""

    def __init__(self, w, threads=None, unbounded=False):
        import oracle
        self.orc = oracle
        self.w = w
        self.unbounded = unbounded
        if unbounded:
            self.bits, _ = oracle.density_grid_contracted(w.grid, w.blobs)
        else:
            self.bits, _ = oracle.density_grid(w.grid, w.blobs)
        self.threads = oracle.max_threads() if threads is None else int(threads)
        self.stage_s = {}

    def run(self, sel):
        orc, w, nt = self.orc, self.w, self.threads
        g, m = w.grid, w.march
        o, d = np.ascontiguousarray(w.rays_o[sel]), np.ascontiguousarray(w.rays_d[sel])
        t = [time.perf_counter()]
        if self.unbounded:
            ex = orc.march_unbounded(o, d, g.aabb_min, g.aabb_max, g.res, g.n_levels, self.bits, m.max_steps,
                                     m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps, n_threads=nt)
        else:
            ex = orc.march(o, d, g.aabb_min, g.aabb_max, g.res, g.n_levels, self.bits, m.step, m.max_steps,
                           m.t_min, m.t_max, blobs=w.blobs, eps=m.early_stop_eps, n_threads=nt)
        t.append(time.perf_counter())
        sig, rgb = orc.field_samples(o, d, ex["ray_indices"], ex["t_starts"], ex["t_ends"], w.blobs, n_threads=nt)
        t.append(time.perf_counter())
        out = orc.render_fwd(ex["offsets"], ex["t_starts"], ex["t_ends"], sig, rgb, bg=w.bg, n_threads=nt)
        t.append(time.perf_counter())
        n = len(sel)
        g_rgb = 2.0 * (out["rgb"] - w.target[sel]) / (3 * n)
        orc.render_bwd(ex["offsets"], ex["t_starts"], ex["t_ends"], sig, rgb, g_rgb, np.zeros(n),
                       np.zeros(n), bg=w.bg, n_threads=nt)
        t.append(time.perf_counter())
        self.stage_s = dict(zip(("march", "field", "render_fwd", "render_bwd"), np.diff(t).tolist()))
        return int(ex["offsets"][-1])


def _timed_sample(pipe, n, target_seconds):
    """Strided sample of the n rays sized for ~target_seconds of oracle work."""
    probe = np.arange(0, n, 256)
    t0 = time.perf_counter()
    pipe.run(probe)
    per_ray = max(time.perf_counter() - t0, 1e-3) / len(probe)
    k = int(min(n, max(len(probe), target_seconds / per_ray)))
    stride = max(1, n // k)
    sel = np.arange(0, n, stride)
    t0 = time.perf_counter()
    S = pipe.run(sel)
    return sel, stride, S, time.perf_counter() - t0


def cpu_baseline(w, target_seconds=10.0):
    """Oracle rays/s on a bounded, evenly strided sample of the workload's
    rays, on all host cores and (a smaller sample) on one core, with the
    per-stage split of the all-core run."""
    pipe = OraclePipeline(w)
    n = w.n_rays
    sel, stride, S, dt = _timed_sample(pipe, n, target_seconds)
    stages = {k: v for k, v in pipe.stage_s.items()}
    one = OraclePipeline(w, threads=1)
    sel1, stride1, S1, dt1 = _timed_sample(one, n, target_seconds / 4)
    return {"value": len(sel) / dt, "unit": "rays/s", "cores": pipe.threads, "kind": "oracle",
            "sample": f"every {stride}th ray of the {n}-ray image ({len(sel)} rays, {S} samples), "
                      f"march+field+fwd+loss+bwd, {dt:.1f} s",
            "samples_per_s": S / dt,
            "stage_s": stages,
            "single_core": {"value": len(sel1) / dt1, "unit": "rays/s", "cores": 1,
                            "sample": f"every {stride1}th ray ({len(sel1)} rays, {S1} samples), {dt1:.1f} s",
                            "stage_s": one.stage_s}}


def cpu_baseline_unbounded(n_cams=16, target_seconds=5.0, res=64):
    """The oracle on a strided ray subset of the unbounded-scene workload,
    reported per ray and labelled as a subset.  Its grid is built by the
    oracle itself at 4 x res^3 (the workload's 4 x 256^3 grid would take the
    host minutes to evaluate); the march's cost is the K lattice points per
    ray either way."""
    w = workloads.c5_unbounded(n_cams=n_cams, res=res)
    pipe = OraclePipeline(w, unbounded=True)
    sel, stride, S, dt = _timed_sample(pipe, w.n_rays, target_seconds)
    return {"value": len(sel) / dt, "unit": "rays/s", "cores": pipe.threads, "kind": "oracle",
            "sample": f"subset: every {stride}th ray of the {w.n_rays}-ray workload ({len(sel)} rays, {S} samples), "
                      f"grid 4x{res}^3, unbounded march (K = {w.march.max_steps}) + field + fwd + loss + bwd, "
                      f"{dt:.1f} s",
            "stage_s": pipe.stage_s}


def training_step_measure(torch, nacc, dev, flush, hbm, peak_src, steps=10):
    """The training batch's whole step -- march (early stop) -> field ->
    render_fwd -> L2 -> render_bwd -> grid points -> field at the points ->
    grid update (EMA, threshold, bits) -- captured as one CUDA graph and
    replayed; eager launches timed beside it, and once more with events at
    the stage boundaries for the path roofline.  262,144 rays, 64 blobs,
    4 x 128^3 grid."""
    w = workloads.c3_training()
    g, m = w.grid, w.march
    n = w.n_rays
    field = nacc.BlobField.from_numpy(w.blobs, dev)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels, dev)
    nacc.density_grid(grid, field, 0.01)
    o = torch.as_tensor(w.rays_o).to(dev)
    d = torch.as_tensor(w.rays_d).to(dev)
    tgt = torch.as_tensor(w.target).to(dev)
    cap = n * m.max_steps
    bufs = nacc.MarchBuffers(n, cap, dev)
    ubufs = nacc.UpdateBuffers(grid.n_cells, dev)
    sig = torch.empty(cap, device=dev)
    rgbs = torch.empty((cap, 3), device=dev)
    gsg = torch.empty(cap, device=dev)
    gcc = torch.empty((cap, 3), device=dev)
    pts = torch.empty((grid.n_cells, 3), device=dev)
    dens = torch.empty(grid.n_cells, device=dev)
    ck = nacc.render_ckpt_buffer(n, dev)

    def staged(mark, count):
        mark(0)
        count(True)
        pk = nacc.march_grid(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps, field=field,
                             buffers=bufs)
        count(False)
        mark(1)
        nacc.field_eval(field, o, d, pk, out=(sig, rgbs))
        mark(2)
        rgb, _, _, _, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, w.bg, 0.0, ckpt=ck)
        mark(3)
        loss, g_rgb = nacc.l2_loss(rgb, tgt)
        mark(4)
        nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, w.bg, 0.0, out=(gsg, gcc),
                        ckpt=ck)
        mark(5)
        nacc.grid_points(grid, seed=7, step=1, jitter=True, out=pts)
        nacc.field_points(field, pts, out=dens)
        nacc.update_grid(grid, dens, 0.95, 0.01, buffers=ubufs)
        mark(6)
        return loss

    def step():
        return staged(lambda i: None, lambda on: None)

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    eager_ms = timed(step)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream().wait_stream(s)
    gph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gph):
        step()
    graph_ms = timed(gph.replay)
    S = bufs.packed.n_samples()
    names = ["march", "field", "render_fwd", "loss", "render_bwd", "grid_update"]
    stage_ms, staged_ms, count_ms, _ = staged_timing(torch, nacc._abi.load(), flush, staged, names, steps=steps)
    out = {"workload": w.name, "n_rays": n, "samples": S, "cells": grid.n_cells,
           "kernels_per_step": KERNELS_PER_STEP["march"] + 4 + 5,
           "graph": {"ms": graph_ms, "rays/s": n / (graph_ms / 1e3), "samples/s": S / (graph_ms / 1e3)},
           "eager": {"ms": eager_ms, "rays/s": n / (eager_ms / 1e3)},
           "stage_ms": stage_ms, "staged_step_ms": staged_ms,
           "path_roofline": path_roofline(stage_ms, S, n, hbm, peak_src, count_ms, w.blobs.n,
                                          alu_peak_tflops(torch, dev))}
    del gph, bufs, sig, rgbs, gsg, gcc, pts, dens
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workloads.c2_image(args.width, args.height)
    pipe = OraclePipeline(w)
    n = w.n_rays
    stride = 16  # each step: a bounded 1/16 sample of the image
    times, samples = [], []
    for i in range(args.warmup + args.steps):
        sel = np.arange(i % stride, n, stride)
        t0 = time.perf_counter()
        S = pipe.run(sel)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            samples.append(S)
    nray = len(np.arange(0, n, stride))
    ms = 1000.0 * sum(times) / len(times)
    val = nray / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "rays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_rays": n, "step_sample": f"every {stride}th ray ({nray} rays)"},
        "samples_per_s": float(np.mean(samples)) / (ms / 1000.0),
        "cpu_baseline": {"value": val, "unit": "rays/s", "cores": pipe.threads, "kind": "oracle",
                         "sample": f"every {stride}th ray of the {n}-ray image per step"},
        "e2e": {"value": val, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def src_sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def recorded_traffic(stage, S, R):
    """DRAM bytes per launch of `stage` from the committed ncu summary, scaled to
    this launch, or None if absent or taken on an older version of the kernel."""
    try:
        rec = json.load(open(TRAFFIC_FILE)).get(stage)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2305_04966_gb300", "csrc", rec["source"])
    if not os.path.exists(src) or src_sha(src) != rec["source_sha"]:
        return None
    return rec["dram_bytes_per_sample"] * S + rec.get("dram_bytes_per_ray", 0.0) * R


def alu_peak_tflops(torch, dev) -> float:
    """FP32 (non-tensor) peak: SMs x 128 FP32 lanes x 2 FLOP per FMA x the
    2070 MHz maximum SM clock of the part."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * 2070e6 / 1e12


def count_pass_flop(S: int, n_blobs: int) -> float:
    """Algorithmic FP32 work of the march's count phase (the run walk and the
    early-stop pass, timed together through the library's event hook): the early-stop density
    at every emitted sample, 11 FLOP per blob (3 differences, |x-mu|^2 as a
    multiply and two FMAs, the exponent scale, the accumulating FMA; the
    exponent itself runs on the special-function unit) plus 14 per sample
    (t0, t1, midpoint, position as three FMAs, dt, tau and the depth sum).
    The lattice walk is not counted, so this is a lower bound on the work."""
    return float(S) * (11 * n_blobs + 14)


def staged_timing(torch, lib, flush, run, names, steps=5, warmup=2):
    """Mean time of each stage of `run` and of the whole call, with CUDA events
    on the current stream (L2 flushed before each call, outside the events).
    run(mark, count) executes one step: mark(i) records the event at stage
    boundary i (0 .. len(names)); count(True/False) turns the library's
    count-phase events of the marches on and off around a march call.
    Returns ({name: ms}, total ms, count-phase ms, run's last result)."""
    for _ in range(warmup):
        run(lambda i: None, lambda on: None)
    torch.cuda.synchronize()
    recs, out = [], None
    for _ in range(steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        cev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for e in cev:  # create the CUDA events behind the handles passed to the library
            e.record()
        flush.zero_()

        def count(on, cev=cev):
            if on:
                lib.nacc_set_march_count_events(cev[0].cuda_event, cev[1].cuda_event)
            else:
                lib.nacc_set_march_count_events(None, None)

        out = run(lambda i, ev=ev: ev[i].record(), count)
        recs.append((ev, cev))
    torch.cuda.synchronize()
    k = len(recs)
    stage = {nm: sum(ev[j].elapsed_time(ev[j + 1]) for ev, _ in recs) / k for j, nm in enumerate(names)}
    total = sum(ev[0].elapsed_time(ev[-1]) for ev, _ in recs) / k
    count_ms = sum(c[0].elapsed_time(c[1]) for _, c in recs) / k
    return stage, total, count_ms, out


def path_roofline(stage_ms, S, R, hbm, peak_src, count_ms=None, n_blobs=None, fp32_peak=None):
    """The method's path (march + render_fwd + render_bwd): its algorithmic
    bytes (BYTES per sample and per ray) over the sum of the three measured
    stage times, against the HBM peak; with each stage's own fraction, the
    DRAM traffic recorded by ncu for the three kernels (null when any record
    is missing or stale), and, given the count phase's time, its FP32 work
    (count_pass_flop) against the FP32 peak."""
    nbytes = sum(BYTES[s][0] * S + BYTES[s][1] * R for s in BYTES)
    ms = sum(stage_ms[s] for s in BYTES)
    ach = nbytes / (ms / 1000.0) / 1e9
    tr = [recorded_traffic(s, S, R) for s in BYTES]
    out = {"bound": "hbm", "kernel": "march + render_fwd + render_bwd", "achieved": ach, "peak": hbm,
           "unit": "GB/s", "frac": ach / hbm, "peak_source": peak_src, "ms": ms, "algorithmic_bytes": nbytes,
           "samples": S, "rays": R, "bytes_per_sample": {s: BYTES[s][0] for s in BYTES},
           "bytes_per_ray": {s: BYTES[s][1] for s in BYTES},
           "traffic": None if any(t is None for t in tr) else float(sum(tr)),
           "stages": {s: {"ms": stage_ms[s], "frac": (BYTES[s][0] * S + BYTES[s][1] * R) / (stage_ms[s] / 1e3) / 1e9
                          / hbm} for s in BYTES}}
    if count_ms is not None and count_ms > 0 and n_blobs is not None and fp32_peak:
        fl = count_pass_flop(S, n_blobs)
        out["count_phase"] = {"bound": "alu", "ms": count_ms, "algorithmic_flop": fl,
                              "achieved": fl / (count_ms / 1e3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                              "frac": fl / (count_ms / 1e3) / 1e12 / fp32_peak,
                              "peak_source": "derived: SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"}
    return out


def aux_measure(torch, nacc, dev, flush, hbm, steps=10):
    """The path's other boundary calls at the C3 / C4 sizes, each timed alone
    with CUDA events (L2 flushed before each call): the jittered cell points
    and the EMA grid update of a 4x128^3 grid (8,388,608 cells), and inverse-
    CDF resampling of 262,144 rays from 64 bins to 32 (stratified).  Inputs are
    seeded synthetic tensors; the algorithmic bytes are per cell / per ray."""
    g = torch.Generator(device=dev)
    g.manual_seed(0x5EED)
    grid = nacc.OccupancyGrid.empty((-1.5,) * 3, (1.5,) * 3, 128, 4, dev)
    nc = grid.n_cells
    dens = torch.rand(nc, generator=g, device=dev) * 10.0
    ubuf = nacc.UpdateBuffers(nc, dev)
    pts = torch.empty((nc, 3), dtype=torch.float32, device=dev)
    nr, nb, no = 262144, 64, 32
    edges = 2.0 + 4.0 * torch.sort(torch.rand((nr, nb + 1), generator=g, device=dev), dim=1).values
    weights = torch.rand((nr, nb), generator=g, device=dev)
    outp = torch.empty((nr, no + 1), dtype=torch.float32, device=dev)

    def comb_path():
        pk = combined.sample(o, d, m.t_min, m.t_max)
        nacc.field_eval(field, o, d, pk, out=(ps, pc))
        return nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, ps, pc, bg, 0.0)[3]

    def timed(fn):
        for _ in range(3):
            fn()
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / steps

    def entry(ms, nbytes, **kw):
        gbs = nbytes / (ms / 1000.0) / 1e9
        return dict(kw, ms=ms, algorithmic_bytes=nbytes, **{"GB/s": gbs}, frac=gbs / hbm)

    t_pts = timed(lambda: nacc.grid_points(grid, 7, 1, True, out=pts))
    t_upd = timed(lambda: nacc.update_grid(grid, dens, 0.95, 0.01, 0.0, buffers=ubuf))
    t_pdf = timed(lambda: nacc.sample_pdf(edges, weights, no, True, 5, out=outp))
    return {
        "grid_points": entry(t_pts, 12 * nc, cells=nc, bytes_per_cell=12),
        "update_grid": entry(t_upd, 16.125 * nc, cells=nc, bytes_per_cell=16.125),
        "sample_pdf": entry(t_pdf, (4 * (2 * nb + 1) + 4 * (no + 1)) * nr, rays=nr, bins=nb, n_out=no,
                            bytes_per_ray=4 * (2 * nb + 1) + 4 * (no + 1)),
    }


def weighted_points(torch, nacc, field, o, d, pk, bg, n_pts, gen):
    """n_pts points drawn along the rays with probability proportional to the
    rendering weights of a sample set (the grid path's): where the
    transmittance drops, each point uniform inside its sample's interval."""
    sig, rgbs = nacc.field_eval(field, o, d, pk)
    wts = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, bg, 0.0, want_weights=True)[4]
    S = pk.n_samples()
    cdf = torch.cumsum(wts[:S].double(), 0)
    del sig, rgbs, wts
    u = torch.rand(n_pts, generator=gen, device=o.device, dtype=torch.float64) * cdf[-1]
    idx = torch.searchsorted(cdf, u).clamp_(max=S - 1)
    del cdf, u
    a = torch.rand(n_pts, generator=gen, device=o.device)
    t = pk.t_starts[idx] + a * (pk.t_ends[idx] - pk.t_starts[idx])
    ri = pk.ray_indices[idx].long()
    return (o[ri] + d[ri] * t[:, None]).contiguous()


def train_proposal(torch, mlp, x, target, steps, batch, lr0, gen, windows=16):
    """Adam on (x, target) pairs, batches of a fresh permutation per epoch,
    learning rate cosine-annealed from lr0 to 1e-5.  Returns the time and the
    loss curve (mean batch MSE over `windows` equal stretches of the steps)."""
    import math as _m
    npairs = x.shape[0]
    perm = torch.randperm(npairs, generator=gen, device=x.device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    losses = []
    a.record()
    j = 0
    for it in range(steps):
        if j + batch > npairs:
            perm = torch.randperm(npairs, generator=gen, device=x.device)
            j = 0
        idx = perm[j:j + batch]
        j += batch
        lr = 1e-5 + 0.5 * (lr0 - 1e-5) * (1.0 + _m.cos(_m.pi * it / steps))
        losses.append(mlp.train_step(x[idx].contiguous(), target[idx].contiguous(), lr=lr))
    b.record()
    torch.cuda.synchronize()
    L = torch.stack(losses).cpu().numpy()
    win = max(1, steps // windows)
    return a.elapsed_time(b), [float(L[i:i + win].mean()) for i in range(0, steps, win)]


def proposal_measure(torch, nacc, dev, flush, steps=5, train_steps=4096, batch=65536, n_pairs=1 << 24,
                     sample_rays=2000):
    """The learned-proposal path and the combined path (grid range + proposal)
    beside the plain grid path on the 262,144-ray training batch (100
    cameras, 64-blob field).  The proposal network is
    first trained (timed, outside the step) on n_pairs (xyz, density) pairs
    drawn along the batch's rays -- uniform t in each ray's clip of the scene
    box for a quarter of them, in its occupied grid range for another
    quarter, by the grid path's rendering weights for the other half -- with
    the density of the analytic field; train_steps Adam steps of batch
    points, learning rate cosine-annealed.  Then each path runs the training step on the batch: sampling
    (grid = march with early stop; proposal = two rounds, 64 -> 32 -> 32
    bins; combined = the proposal rounds over the grid's occupied range),
    field, checkpointed render forward, L2 loss against the batch's target,
    checkpointed adjoint.  Returns rays/s of each, and their final
    transmittance on a fixed sample of rays (the exact values come from the
    CPU leg)."""
    w = workloads.c3_training()
    g, m = w.grid, w.march
    n = w.n_rays
    field = nacc.BlobField.from_numpy(w.blobs, dev)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels, dev)
    nacc.density_grid(grid, field, 0.01)
    box = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, 32, 1, dev)
    o = torch.as_tensor(w.rays_o).to(dev)
    d = torch.as_tensor(w.rays_d).to(dev)
    # training pairs
    gen = torch.Generator(device=dev)
    gen.manual_seed(0x5EED + 4)
    # a quarter of the pairs along each ray's scene-box range (where the
    # proposal path samples), a quarter along its occupied grid range (where
    # the combined path samples: the cascade reaches past the scene box), half
    # where the grid path's rendering weights are (where the transmittance
    # drops)
    e1 = nacc.uniform_edges(box, o, d, 1, m.t_min, m.t_max)
    lo, hi = nacc.occupied_range(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max)
    nu = n_pairs // 2
    ri = torch.randint(0, n, (nu,), generator=gen, device=dev)
    u = torch.rand(nu, generator=gen, device=dev)
    first = torch.arange(nu, device=dev) < nu // 2
    a0 = torch.where(first, e1[ri, 0], lo[ri])
    a1 = torch.where(first, e1[ri, 1], hi[ri])
    t = a0 + u * (a1 - a0)
    pk = nacc.march_grid(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps, field=field)
    xyz = torch.cat([(o[ri] + d[ri] * t[:, None]), weighted_points(torch, nacc, field, o, d, pk, w.bg,
                                                                   n_pairs - nu, gen)]).contiguous()
    del pk, ri, u, t, a0, a1, first
    torch.cuda.empty_cache()
    sig = nacc.field_points(field, xyz)
    mlp = nacc.ProposalMLP.init(seed=11, device=dev)
    train_ms, curve = train_proposal(torch, mlp, xyz, sig, train_steps, batch, 3e-3, gen)
    target_var = float(sig.var())
    del xyz, sig
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    bufs = nacc.MarchBuffers(n, n * m.max_steps, dev)
    fs = torch.empty(n * m.max_steps, device=dev)
    fc = torch.empty((n * m.max_steps, 3), device=dev)
    gfs, gfc = torch.empty_like(fs), torch.empty_like(fc)
    sampler = nacc.ProposalSampler(mlp, box, n, rounds=(64, 32), n_final=32, device=dev)
    combined = nacc.CombinedSampler(mlp, grid, n, m.step, m.max_steps, rounds=(64, 32), n_final=32, device=dev)
    ps = torch.empty(n * 32, device=dev)
    pc = torch.empty((n * 32, 3), device=dev)
    bg = w.bg
    tgt = torch.as_tensor(w.target).to(dev)
    ck = nacc.render_ckpt_buffer(n, dev)  # per-ray records from render_fwd for render_bwd

    def tail(pk, sig, rgbs, gs, gc):
        """field, checkpointed render forward, L2 loss, checkpointed adjoint;
        returns the final transmittance."""
        nacc.field_eval(field, o, d, pk, out=(sig, rgbs))
        rgb, _, _, tr, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, bg, 0.0, ckpt=ck)
        _, g_rgb = nacc.l2_loss(rgb, tgt)
        nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, bg, 0.0, out=(gs, gc),
                        ckpt=ck)
        return tr

    def grid_path():
        pk = nacc.march_grid(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps, field=field,
                             buffers=bufs)
        return tail(pk, fs, fc, gfs, gfc)

    def prop_path():
        return tail(sampler.sample(o, d, m.t_min, m.t_max), ps, pc, gfs, gfc)

    def comb_path():
        return tail(combined.sample(o, d, m.t_min, m.t_max), ps, pc, gfs, gfc)

    def timed(fn):
        for _ in range(2):
            fn()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps, out

    grid_ms, T_grid = timed(grid_path)
    grid_S = bufs.packed.n_samples()
    prop_ms, T_prop = timed(prop_path)
    comb_ms, T_comb = timed(comb_path)
    sel = np.linspace(0, n - 1, sample_rays).astype(np.int64)

    # equal-error sweep: the grid path on coarser lattices (step x mult over the
    # same distance), the proposal path with more bins
    sweep_T = {}
    grid_sweep, prop_sweep = [], []
    for mult in (1, 2, 4, 8, 16, 32):
        st, ks = m.step * mult, (m.max_steps + mult - 1) // mult

        def gp():
            pk = nacc.march_grid(grid, o, d, st, ks, m.t_min, m.t_max, m.early_stop_eps, field=field, buffers=bufs)
            return tail(pk, fs, fc, gfs, gfc)

        ms_, T_ = timed(gp)
        grid_sweep.append({"step": st, "max_steps": ks, "samples": bufs.packed.n_samples(), "ms": ms_,
                           "rays/s": n / (ms_ / 1e3)})
        sweep_T[f"grid step x{mult}"] = T_.cpu().numpy()[sel]
    for rounds, nf in (((64, 32), 32), ((128, 64), 64), ((256, 128), 128)):
        smp = nacc.ProposalSampler(mlp, box, n, rounds=rounds, n_final=nf, device=dev)
        ps2 = torch.empty(n * nf, device=dev)
        pc2 = torch.empty((n * nf, 3), device=dev)

        def pp():
            return tail(smp.sample(o, d, m.t_min, m.t_max), ps2, pc2, gfs, gfc)

        ms_, T_ = timed(pp)
        prop_sweep.append({"rounds": list(rounds), "final_samples_per_ray": nf, "ms": ms_, "rays/s": n / (ms_ / 1e3)})
        sweep_T[f"proposal {list(rounds)}->{nf}"] = T_.cpu().numpy()[sel]
        del smp, ps2, pc2
    return {
        "grid_sweep": grid_sweep, "proposal_sweep": prop_sweep,
        "workload": w.name, "n_rays": n,
        "grid_path": {"rays/s": n / (grid_ms / 1e3), "ms": grid_ms, "samples": grid_S,
                      "early_stop_eps": m.early_stop_eps},
        "proposal_path": {"rays/s": n / (prop_ms / 1e3), "ms": prop_ms, "samples": n * 32,
                          "rounds": [64, 32], "final_samples_per_ray": 32},
        "combined_path": {"rays/s": n / (comb_ms / 1e3), "ms": comb_ms, "samples": n * 32,
                          "rounds": [64, 32], "final_samples_per_ray": 32,
                          "initial_range": "first to last occupied lattice point of the grid"},
        "training": {"pairs": n_pairs, "steps": train_steps, "batch": batch, "ms": train_ms,
                     "schedule": "Adam, lr cosine 3e-3 -> 1e-5", "loss_curve": curve,
                     "mse_first": curve[0], "mse_last": curve[-1], "target_variance": target_var,
                     "points": "1/4 uniform in the scene-box range, 1/4 in the occupied grid range, 1/2 "
                               "by the grid path's rendering weights"},
        # the two paths integrate over different ranges (cascade vs scene box):
        # this difference includes the density outside the scene box
        "T_abs_diff_proposal_vs_grid": {"mean": float((T_prop - T_grid).abs().mean()),
                                        "p99": float((T_prop - T_grid).abs().quantile(0.99))},
        "_sample": {"rays": sel, "T_grid": T_grid.cpu().numpy()[sel], "T_prop": T_prop.cpu().numpy()[sel],
                    "T_comb": T_comb.cpu().numpy()[sel], "w": w, "sweep": sweep_T},
    }


def proposal_exact_error(prop):
    """CPU leg: the exact transmittance of the sampled rays (oracle closed
    form of the blob field's line integral) over each path's own range --
    the cascade's outermost box for the grid path, the scene box for the
    proposal's bins -- and each path's error against it."""
    import oracle
    from oracle import proposal as P
    s = prop.pop("_sample")
    w, sel = s["w"], s["rays"]
    o, d = w.rays_o[sel], w.rays_d[sel]
    out = {"rays": int(len(sel))}
    for name, levels, Tp in (("grid", w.grid.n_levels, s["T_grid"]), ("proposal", 1, s["T_prop"]),
                             ("combined", w.grid.n_levels, s["T_comb"])):
        tn, tf, hit = oracle.ray_clip(o, d, w.grid.aabb_min, w.grid.aabb_max, w.grid.res, levels, w.march.t_min,
                                      w.march.t_max)
        tau = P.exact_optical_depth(o, d, tn.astype(np.float64), np.where(hit, tf, tn).astype(np.float64),
                                    w.blobs.mu, w.blobs.std, w.blobs.peak)
        err = np.abs(Tp - np.exp(-tau))
        out[name + "_mean_abs"] = float(err.mean())
        out[name + "_p99"] = float(np.quantile(err, 0.99))
        out[name + "_range"] = "outermost cascade box" if levels > 1 else "scene box (level 0)"
    prop["T_error_vs_exact"] = out
    # the sweep, each path against the exact depth over its own range
    Tex = {}
    for levels in (1, w.grid.n_levels):
        tn, tf, hit = oracle.ray_clip(o, d, w.grid.aabb_min, w.grid.aabb_max, w.grid.res, levels, w.march.t_min,
                                      w.march.t_max)
        Tex[levels] = np.exp(-P.exact_optical_depth(o, d, tn.astype(np.float64),
                                                    np.where(hit, tf, tn).astype(np.float64), w.blobs.mu,
                                                    w.blobs.std, w.blobs.peak))
    mults = (1, 2, 4, 8, 16, 32)
    for row, mult in zip(prop["grid_sweep"], mults):
        e = np.abs(s["sweep"][f"grid step x{mult}"] - Tex[w.grid.n_levels])
        row["T_mean_abs_err"], row["T_p99_abs_err"] = float(e.mean()), float(np.quantile(e, 0.99))
    for row in prop["proposal_sweep"]:
        e = np.abs(s["sweep"][f"proposal {row['rounds']}->{row['final_samples_per_ray']}"] - Tex[1])
        row["T_mean_abs_err"], row["T_p99_abs_err"] = float(e.mean()), float(np.quantile(e, 0.99))
    # at each proposal configuration's error: the fastest grid configuration
    # that is at least as accurate
    eq = []
    for row in prop["proposal_sweep"]:
        ok = [g for g in prop["grid_sweep"] if g["T_mean_abs_err"] <= row["T_mean_abs_err"]]
        best = max(ok, key=lambda g: g["rays/s"]) if ok else None
        eq.append({"proposal": {"rounds": row["rounds"], "final": row["final_samples_per_ray"],
                                "rays/s": row["rays/s"], "T_mean_abs_err": row["T_mean_abs_err"]},
                   "grid": None if best is None else {"step": best["step"], "rays/s": best["rays/s"],
                                                      "T_mean_abs_err": best["T_mean_abs_err"]}})
    prop["equal_error"] = eq


def unbounded_measure(torch, nacc, dev, flush, hbm, peak_src, n_cams=16, steps=3,
                      grid_K=(128, 256, 512, 1024, 2048),
                      prop_cfg=(((64, 32), 32), ((128, 64), 64), ((256, 128), 128)), train_steps=32768,
                      batch=65536, n_pairs=1 << 24, sample_rays=1500):
    """Unbounded scenes: 4,194,304 rays from 16 inward-facing 1024x256 cameras
    over 256 blobs spread across radius 20, space contracted into [-2, 2]^3.
    Both estimators run the whole training step (sampling + field + the
    checkpointed render fwd + L2 loss + the checkpointed render bwd), timed
    whole and once more with events at the stage boundaries (grid
    configurations also report the path roofline of march + render fwd +
    bwd and the count phase's FP32 fraction):
      grid: the 4x256^3 grid over the contracted space (initialised from the
            field at the cell centres' scene points), the s-lattice march with
            early stop, at several lattice sizes K;
      proposal: the proposal network (trained first on (contracted point,
            density) pairs, half uniform in s along the rays and half where
            the grid path's rendering weights are, timed outside the step),
            rounds of inverse-CDF resampling from bins uniform in s, at
            several bin counts.
    Each configuration's final transmittance on a fixed sample of rays is
    compared (CPU leg) with the exact line integral over [t_near, t_far]; the
    proposal rounds driven by the exact density give the sampler's own bound."""
    w = workloads.c5_unbounded(n_cams=n_cams)
    m = w.march
    n = w.n_rays
    n_pairs = min(n_pairs, 4 * n)
    field = nacc.BlobField.from_numpy(w.blobs, dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    grid = nacc.OccupancyGrid.empty(w.grid.aabb_min, w.grid.aabb_max, w.grid.res, w.grid.n_levels, dev)
    a.record()
    nacc.density_grid_unbounded(grid, field, 0.01)
    b.record()
    torch.cuda.synchronize()
    init_ms = a.elapsed_time(b)
    occ = workloads.unpack_bits(grid.bits.cpu().numpy().view(np.uint32)).reshape(w.grid.n_levels, -1).mean(1)
    o = torch.as_tensor(w.rays_o).to(dev)
    d = torch.as_tensor(w.rays_d).to(dev)
    tgt = torch.as_tensor(w.target).to(dev)
    sel = np.linspace(0, n - 1, sample_rays).astype(np.int64)

    def timed(fn):
        for _ in range(2):
            fn()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps, out

    ck = nacc.render_ckpt_buffer(n, dev)  # per-ray records from render_fwd for render_bwd
    lib = nacc._abi.load()
    fp32_peak = alu_peak_tflops(torch, dev)
    names = ["sampling", "field", "render_fwd", "loss", "render_bwd"]

    def train_step(sample, sig, rgbs, gs, gc, mark=lambda i: None, count=lambda on: None):
        mark(0)
        count(True)
        pk = sample()
        count(False)
        mark(1)
        nacc.field_eval(field, o, d, pk, out=(sig, rgbs))
        mark(2)
        rgb, _, _, tr, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, w.bg, 0.0, ckpt=ck)
        mark(3)
        _, g_rgb = nacc.l2_loss(rgb, tgt)
        mark(4)
        nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, w.bg, 0.0, out=(gs, gc),
                        ckpt=ck)
        mark(5)
        return tr

    def stages(sample, sig, rgbs, gs, gc):
        st, tot, cnt, tr = staged_timing(torch, lib, flush, lambda mk, ct: train_step(sample, sig, rgbs, gs, gc, mk, ct),
                                         names, steps=steps)
        return st, tot, cnt, tr

    out = {"workload": w.name, "n_rays": n, "grid_spec": f"{w.grid.n_levels}x{w.grid.res}^3 over [-2,2]^3",
           "t_near": m.t_min, "t_far": m.t_max, "grid_init_ms": init_ms,
           "occupied_fraction_per_level": [float(v) for v in occ], "grid": [], "proposal": [], "_T": {}}
    for K in grid_K:
        pk = nacc.march_unbounded(grid, o, d, K, m.t_min, m.t_max, m.early_stop_eps, field=field)
        S = pk.n_samples()
        del pk
        bufs = nacc.MarchBuffers(n, S, dev)
        sig = torch.empty(S, device=dev)
        rgbs = torch.empty((S, 3), device=dev)
        gs, gc = torch.empty_like(sig), torch.empty_like(rgbs)

        def march():
            return nacc.march_unbounded(grid, o, d, K, m.t_min, m.t_max, m.early_stop_eps, field=field,
                                        buffers=bufs)

        ms, tr = timed(lambda: train_step(march, sig, rgbs, gs, gc))
        march_ms, _ = timed(march)
        st, _, cnt, _ = stages(march, sig, rgbs, gs, gc)
        st["march"] = st.pop("sampling")
        out["grid"].append({"K": K, "samples": S, "samples_per_ray": S / n, "step_ms": ms, "march_ms": march_ms,
                            "rays/s": n / (ms / 1e3), "stage_ms": st,
                            "path_roofline": path_roofline(st, S, n, hbm, peak_src, cnt, w.blobs.n, fp32_peak)})
        out["_T"][f"grid K={K}"] = tr.cpu().numpy()[sel]
        del bufs, sig, rgbs, gs, gc
        torch.cuda.empty_cache()

    # training pairs: half uniform in s along random rays, half by the
    # rendering weights of the grid path at K = 1024 (where the transmittance
    # drops); the density of the field there, the network at the contracted point
    gen = torch.Generator(device=dev)
    gen.manual_seed(0x5EED + 5)
    nu = n_pairs // 2
    ri = torch.randint(0, n, (nu,), generator=gen, device=dev)
    s = torch.rand(nu, generator=gen, device=dev)
    t = 1.0 / ((1.0 / m.t_min) * (1.0 - s) + (1.0 / m.t_max) * s)
    pk = nacc.march_unbounded(grid, o, d, 1024, m.t_min, m.t_max, m.early_stop_eps, field=field)
    x = torch.cat([o[ri] + d[ri] * t[:, None], weighted_points(torch, nacc, field, o, d, pk, w.bg, n_pairs - nu,
                                                                gen)]).contiguous()
    del pk, ri, s, t
    torch.cuda.empty_cache()
    target = nacc.field_points(field, x)
    c = nacc.contract_points(x)
    del x
    mlp = nacc.ProposalMLP.init(seed=12, device=dev)
    train_ms, curve = train_proposal(torch, mlp, c, target, train_steps, batch, 1e-2, gen)
    out["training"] = {"pairs": n_pairs, "steps": train_steps, "batch": batch, "ms": train_ms,
                       "schedule": "Adam, lr cosine 1e-2 -> 1e-5", "loss_curve": curve,
                       "mse_first": curve[0], "mse_last": curve[-1], "target_variance": float(target.var()),
                       "points": "1/2 uniform in s, 1/2 by the grid path's rendering weights (K = 1024)"}
    del c, target

    for rounds, nf in prop_cfg:
        sampler = nacc.UnboundedProposalSampler(mlp, n, m.t_min, m.t_max, rounds=rounds, n_final=nf, device=dev)
        S = n * nf
        sig = torch.empty(S, device=dev)
        rgbs = torch.empty((S, 3), device=dev)
        gs, gc = torch.empty_like(sig), torch.empty_like(rgbs)
        ms, tr = timed(lambda: train_step(lambda: sampler.sample(o, d), sig, rgbs, gs, gc))
        samp_ms, _ = timed(lambda: sampler.sample(o, d))
        st, _, _, _ = stages(lambda: sampler.sample(o, d), sig, rgbs, gs, gc)
        name = f"proposal {list(rounds)}->{nf}"
        out["proposal"].append({"rounds": list(rounds), "final_samples_per_ray": nf, "samples": S, "step_ms": ms,
                                "sampler_ms": samp_ms, "rays/s": n / (ms / 1e3), "stage_ms": st})
        out["_T"][name] = tr.cpu().numpy()[sel]
        # the same rounds driven by the exact density at the bin midpoints
        e = nacc.phi_edges(n, rounds[0], m.t_min, m.t_max, dev)
        for i, nb in enumerate(rounds):
            tm = 0.5 * (e[:, :-1] + e[:, 1:])
            sg = torch.empty((n, nb), device=dev)
            for c0 in range(0, n, 1 << 19):
                c1 = min(n, c0 + (1 << 19))
                xm = (o[c0:c1, None, :] + d[c0:c1, None, :] * tm[c0:c1, :, None]).reshape(-1, 3).contiguous()
                sg[c0:c1] = nacc.field_points(field, xm).reshape(c1 - c0, nb)
            wts = nacc.dense_weights(e, sg)
            e = nacc.sample_pdf(e, wts, rounds[i + 1] if i + 1 < len(rounds) else nf)
        pk = nacc.edges_to_packed(e)
        sig2, rgb2 = nacc.field_eval(field, o, d, pk)
        out["_T"][f"exact-density {list(rounds)}->{nf}"] = nacc.render_fwd(
            pk.offsets, pk.t_starts, pk.t_ends, sig2, rgb2, w.bg, 0.0)[3].cpu().numpy()[sel]
        del sampler, sig, rgbs, gs, gc, e, tm, sg, wts, pk, sig2, rgb2
        torch.cuda.empty_cache()
    out["_sample"] = {"rays": sel, "w": w}
    return out


def unbounded_exact_error(unb):
    """CPU leg: the exact transmittance of the sampled rays over [t_near,
    t_far] (oracle closed form), each configuration's error against it, and
    the fastest configuration of each estimator within the error of the grid
    at K = 1024, and within the best error the proposal reaches."""
    from oracle import proposal as P
    s = unb.pop("_sample")
    Ts = unb.pop("_T")
    w, sel = s["w"], s["rays"]
    k = len(sel)
    tau = P.exact_optical_depth(w.rays_o[sel], w.rays_d[sel], np.full(k, w.march.t_min), np.full(k, w.march.t_max),
                                w.blobs.mu, w.blobs.std, w.blobs.peak)
    Tex = np.exp(-tau)
    err = {name: {"mean_abs": float(np.abs(T - Tex).mean()), "p99": float(np.quantile(np.abs(T - Tex), 0.99))}
           for name, T in Ts.items()}
    unb["T_error_vs_exact"] = {"rays": k, "exact_T_mean": float(Tex.mean()), **err}
    for row in unb["grid"]:
        row["T_mean_abs_err"] = err[f"grid K={row['K']}"]["mean_abs"]
    for row in unb["proposal"]:
        row["T_mean_abs_err"] = err[f"proposal {row['rounds']}->{row['final_samples_per_ray']}"]["mean_abs"]
    def at_error(target):
        eq = {"target_T_mean_abs_err": target}
        for est in ("grid", "proposal"):
            ok = [r for r in unb[est] if target is not None and r["T_mean_abs_err"] <= target * 1.0001]
            best = max(ok, key=lambda r: r["rays/s"]) if ok else None
            eq[est] = None if best is None else {"rays/s": best["rays/s"], "T_mean_abs_err": best["T_mean_abs_err"],
                                                 "config": {kk: best[kk] for kk in best if kk in ("K", "rounds",
                                                            "final_samples_per_ray")}}
        return eq

    # at the error of the grid at K = 1024, and at the proposal's best error
    unb["equal_error"] = at_error(next((r["T_mean_abs_err"] for r in unb["grid"] if r["K"] == 1024), None))
    if unb["proposal"]:
        unb["equal_error_at_proposal_best"] = at_error(min(r["T_mean_abs_err"] for r in unb["proposal"]))


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2305_04966_gb300 as nacc
    nacc.load_library()

    w = rank_workload(args, rank, world)
    g, m = w.grid, w.march
    n = w.n_rays
    field = nacc.BlobField.from_numpy(w.blobs, dev)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels, dev)
    nacc.density_grid(grid, field, 0.01)
    o = torch.as_tensor(w.rays_o).to(dev)
    d = torch.as_tensor(w.rays_d).to(dev)
    tgt = torch.as_tensor(w.target).to(dev)
    cap = n * m.max_steps  # worst case: the march never synchronises
    bufs = nacc.MarchBuffers(n, cap, dev)
    sig = torch.empty(cap, dtype=torch.float32, device=dev)
    rgbs = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    gsg = torch.empty(cap, dtype=torch.float32, device=dev)
    gcc = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    ck = nacc.render_ckpt_buffer(n, dev)  # per-ray records from render_fwd for render_bwd
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stages = ["march", "field", "render_fwd", "loss", "render_bwd"]

    lib = nacc._abi.load()

    def step(o_, d_, tgt_, ev=None, before_loss=None, after_fwd=None):
        if ev is not None:
            ev[0].record()
            lib.nacc_set_march_count_events(ev[6].cuda_event, ev[7].cuda_event)
        pk = nacc.march_grid(grid, o_, d_, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps,
                             field=field, buffers=bufs)
        if ev is not None:
            lib.nacc_set_march_count_events(None, None)
            ev[1].record()
        nacc.field_eval(field, o_, d_, pk, out=(sig, rgbs))
        if ev is not None:
            ev[2].record()
        rgb, op, dep, tr, _ = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, w.bg, 0.0, ckpt=ck)
        if ev is not None:
            ev[3].record()
        if after_fwd is not None:
            after_fwd(rgb)
        if before_loss is not None:
            before_loss()
        loss, g_rgb = nacc.l2_loss(rgb, tgt_)
        if ev is not None:
            ev[4].record()
        nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, w.bg, 0.0,
                        out=(gsg, gcc), ckpt=ck)
        if ev is not None:
            ev[5].record()
        return rgb, loss

    for _ in range(max(args.warmup, 0)):
        step(o, d, tgt)
    torch.cuda.synchronize()
    S = bufs.packed.n_samples()

    clk = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    # 6 stage boundaries + the count kernel's two events (recorded by the library)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(args.steps)]
    for ev in evs:  # create the CUDA events behind the handles passed to the library
        ev[6].record()
        ev[7].record()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        step(o, d, tgt, evs[i])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    stage_ms = {s: 0.0 for s in stages}
    step_ms = []
    count_ms = 0.0
    for ev in evs:
        step_ms.append(ev[0].elapsed_time(ev[5]))
        for j, s in enumerate(stages):
            stage_ms[s] += ev[j].elapsed_time(ev[j + 1])
        count_ms += ev[6].elapsed_time(ev[7])
    stage_ms = {s: v / args.steps for s, v in stage_ms.items()}
    count_ms /= args.steps
    ms_local = sum(step_ms) / len(step_ms)
    ms = reduce_max(ms_local, dist)
    rays_total = reduce_sum(n, dist)
    samples_total = reduce_sum(S, dist)
    value = rays_total / (ms / 1000.0)

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    # the dominant kernel of the method's path: the march count phase (ALU-bound,
    # timed alone through the library's event hook) or an HBM-bound render kernel
    fp32_peak = alu_peak_tflops(torch, dev)
    count_flop = count_pass_flop(S, w.blobs.n)
    dom = max(["march_count", "render_fwd", "render_bwd"],
              key=lambda s: count_ms if s == "march_count" else stage_ms[s])
    if dom == "march_count":
        achieved = count_flop / (count_ms / 1000.0) / 1e12
        roofline = {"bound": "alu", "kernel": "k_march_runs+k_march_stop", "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak, "ms": count_ms,
                    "peak_source": "derived: SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz",
                    "traffic": recorded_traffic("march_count", S, n), "algorithmic_flop": count_flop}
    else:
        dom_bytes = BYTES[dom][0] * S + BYTES[dom][1] * n
        achieved = dom_bytes / (stage_ms[dom] / 1000.0) / 1e9
        roofline = {"bound": "hbm", "kernel": "k_" + dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "ms": stage_ms[dom], "peak_source": peak_src,
                    "traffic": recorded_traffic(dom, S, n), "algorithmic_bytes": dom_bytes}
    # the headline roofline is the whole path's (march + render_fwd + render_bwd), the quantity the
    # target is stated for; the dominant kernel's own figure is reported beside it
    path_roof = path_roofline(stage_ms, S, n, hbm, peak_src, count_ms, w.blobs.n, fp32_peak)
    kernel_roof = roofline
    stage_roof = {}
    for s in BYTES:
        b = BYTES[s][0] * S + BYTES[s][1] * n
        a = b / (stage_ms[s] / 1000.0) / 1e9
        stage_roof[s] = {"ms": stage_ms[s], "GB/s": a, "frac": a / hbm, "traffic": recorded_traffic(s, S, n)}

    e2e = None
    if not args.no_e2e:
        e2e = e2e_measure(args, torch, nacc, step, w, dev, n, flush, dist)
    aux = None
    if rank == 0 and not args.no_aux:
        legs = set(filter(None, args.aux_legs.split(",")))
        aux = aux_measure(torch, nacc, dev, flush, hbm) if "update" in legs else {}
        if "step" in legs:
            aux["training_step"] = training_step_measure(torch, nacc, dev, flush, hbm, peak_src)
        if "proposal" in legs:
            aux["proposal"] = proposal_measure(torch, nacc, dev, flush)
            if args.no_cpu_baseline:
                aux["proposal"].pop("_sample")
            else:
                proposal_exact_error(aux["proposal"])
        if "unbounded" in legs:
            aux["unbounded"] = unbounded_measure(torch, nacc, dev, flush, hbm, peak_src, n_cams=args.unbounded_cams)
            if args.no_cpu_baseline:
                aux["unbounded"].pop("_sample")
                aux["unbounded"].pop("_T")
            else:
                unbounded_exact_error(aux["unbounded"])
                aux["unbounded"]["cpu_baseline"] = cpu_baseline_unbounded(args.unbounded_cams)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if args.shard == "batch" and world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n_rays_per_gpu": n, "grid": f"{g.n_levels}x{g.res}^3",
                       "max_steps": m.max_steps, "blobs": w.blobs.n, "early_stop_eps": m.early_stop_eps,
                       "samples_per_gpu": S, "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"dp{world} ("
                                      + ("contiguous ray ranges of one view" if args.shard == "batch" and world > 1
                                         else "one view per GPU") + ")"},
            "samples_per_s": samples_total / (ms / 1000.0),
            "stage_ms": stage_ms,
            "roofline": path_roof,
            "kernel_roofline": kernel_roof,
            "stage_roofline": stage_roof,
            "aux": aux,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": sum(KERNELS_PER_STEP.values()) * args.steps,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def e2e_measure(args, torch, nacc, step, w, dev, n, flush, dist):
    """Same step with the inputs (rays, target) copied in from pinned host
    memory and the rendered image + loss copied back, all inside the events.
    The rays go in first on the step's stream (the march needs them); the
    target goes in on a copy stream while the march and field run (the loss
    waits for it), and the image comes back on the copy stream during the
    adjoint; the step's stream waits for every copy before its end event."""
    o_h = torch.as_tensor(w.rays_o).pin_memory()
    d_h = torch.as_tensor(w.rays_d).pin_memory()
    t_h = torch.as_tensor(w.target).pin_memory()
    rgb_h = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    loss_h = torch.empty(1, dtype=torch.float32).pin_memory()
    o_d = torch.empty_like(o_h, device=dev)
    d_d = torch.empty_like(d_h, device=dev)
    t_d = torch.empty_like(t_h, device=dev)
    cs = torch.cuda.Stream(device=dev)
    K = max(1, args.steps // 2)
    total = 0.0
    for i in range(2 + K):
        flush.zero_()
        main = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_in, f_done, rgb_out = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
        e0.record()
        cs.wait_event(e0)
        with torch.cuda.stream(cs):
            t_d.copy_(t_h, non_blocking=True)
            t_in.record(cs)
        o_d.copy_(o_h, non_blocking=True)
        d_d.copy_(d_h, non_blocking=True)

        def after_fwd(rgb):
            f_done.record(main)
            cs.wait_event(f_done)
            with torch.cuda.stream(cs):
                rgb_h.copy_(rgb, non_blocking=True)
                rgb_out.record(cs)

        rgb, loss = step(o_d, d_d, t_d, before_loss=lambda: main.wait_event(t_in), after_fwd=after_fwd)
        loss_h.copy_(loss, non_blocking=True)
        main.wait_event(rgb_out)
        e1.record()
        e1.synchronize()
        if i >= 2:
            total += e0.elapsed_time(e1)
    ms = reduce_max(total / K, dist)
    rays_total = reduce_sum(n, dist)
    h2d = o_h.numel() * 4 + d_h.numel() * 4 + t_h.numel() * 4
    d2h = rgb_h.numel() * 4 + 4
    return {"value": rays_total / (ms / 1000.0), "unit": "rays/s", "ms_per_step": ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": K,
            "overlap": "target in during the march and field, image out during the adjoint (copy stream)"}


def profile_run(args):
    """One workload's training step, eagerly, --warmup + --steps times (for an
    ncu launch list: every launch of a step is one of the library's kernels or
    the L2 loss's)."""
    import torch
    import paper_2305_04966_gb300 as nacc
    nacc.load_library()
    dev = torch.device("cuda", 0)
    if args.profile == "unbounded":
        w = workloads.c5_unbounded(n_cams=args.unbounded_cams)
    elif args.profile == "training":
        w = workloads.c3_training()
    else:
        w = workloads.c2_image(args.width, args.height)
    g, m = w.grid, w.march
    n = w.n_rays
    field = nacc.BlobField.from_numpy(w.blobs, dev)
    grid = nacc.OccupancyGrid.empty(g.aabb_min, g.aabb_max, g.res, g.n_levels, dev)
    o = torch.as_tensor(w.rays_o).to(dev)
    d = torch.as_tensor(w.rays_d).to(dev)
    tgt = torch.as_tensor(w.target).to(dev)
    if args.profile == "unbounded":
        nacc.density_grid_unbounded(grid, field, 0.01)
        K = 512
        S = nacc.march_unbounded(grid, o, d, K, m.t_min, m.t_max, m.early_stop_eps, field=field).n_samples()
        bufs = nacc.MarchBuffers(n, S, dev)

        def march():
            return nacc.march_unbounded(grid, o, d, K, m.t_min, m.t_max, m.early_stop_eps, field=field,
                                        buffers=bufs)
    else:
        nacc.density_grid(grid, field, 0.01)
        bufs = nacc.MarchBuffers(n, n * m.max_steps, dev)
        S = n * m.max_steps

        def march():
            return nacc.march_grid(grid, o, d, m.step, m.max_steps, m.t_min, m.t_max, m.early_stop_eps,
                                   field=field, buffers=bufs)
    sig, rgbs = torch.empty(S, device=dev), torch.empty((S, 3), device=dev)
    gs, gc = torch.empty_like(sig), torch.empty_like(rgbs)
    ck = nacc.render_ckpt_buffer(n, dev)
    if args.profile == "training":
        ubufs = nacc.UpdateBuffers(grid.n_cells, dev)
        pts = torch.empty((grid.n_cells, 3), device=dev)
        dens = torch.empty(grid.n_cells, device=dev)

    def step():
        pk = march()
        nacc.field_eval(field, o, d, pk, out=(sig, rgbs))
        rgb = nacc.render_fwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, w.bg, 0.0, ckpt=ck)[0]
        _, g_rgb = nacc.l2_loss(rgb, tgt)
        nacc.render_bwd(pk.offsets, pk.t_starts, pk.t_ends, sig, rgbs, g_rgb, None, None, w.bg, 0.0, out=(gs, gc),
                        ckpt=ck)
        if args.profile == "training":
            nacc.grid_points(grid, seed=7, step=1, jitter=True, out=pts)
            nacc.field_points(field, pts, out=dens)
            nacc.update_grid(grid, dens, 0.95, 0.01, buffers=ubufs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        step()
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "workload": w.name, "rays": n, "samples": bufs.packed.n_samples(),
                      "ms_per_step": a.elapsed_time(b) / max(args.steps, 1), "steps": args.steps,
                      "warmup": args.warmup}))
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return profile_run(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
