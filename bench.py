#!/usr/bin/env python
"""Benchmark of FGA registration on GB300 (one JSON line on stdout).

Default workload: large inhomogeneous clouds, N = M = 1M points sampled
independently from seeded piecewise-planar scenes (8-16 rectangles, 10x
density variation, 5 % uniform outliers, sigma = 0.01), uniform masses,
Barnes-Hut with theta = 0.5, 100 iterations of Algorithm 2, FP32 forces with
FP64 reductions and rigid fit. One step = one whole registration
(normalisation, masses, tree build, 100 iterations, de-normalisation) of one
pair whose inputs are already resident in device memory. The same line
carries the theta = 0.3 and 0.7 registrations and the tiled all-pairs sum on
the same pairs (a few steps each), as extra keys.

Metric: pair-interactions/s = force terms evaluated (accepted cells + leaf
particles, counted on the device) per second of registration time; the line
also carries registrations/s and p50/p99 latency. ``e2e`` repeats the
measurement through the same C call with pinned HOST inputs (host->device
copies and the result read-back inside the timed region).

Other workloads (``--workload``): the 120k LiDAR-like sweeps (Barnes-Hut,
16-NN masses), the 1k sphere and 262k planar all-pairs cases, the 256-pair
batch, the parameter grid and the served Poisson trace.

``--impl reference`` times the FP64 CPU oracle on the same workload (each step
a bounded sample of it) on the host cores.

Multi-GPU (torchrun): every rank registers its own pairs (no collective on the
data path); the timing is the max over ranks, the value the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

FLOPS_NOTE = "12 FP32 instructions + 1 MUFU rsqrt per interaction"
FP32_INSTR_PER_INTERACTION = 12
FP32_LANES_PER_SM = 128


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="planar-bh")
    ap.add_argument("--n", type=int, default=None, help="points per cloud (workload default)")
    ap.add_argument("--iters", type=int, default=None, help="iterations (workload default)")
    ap.add_argument("--theta", type=float, default=None, help="BH opening parameter")
    ap.add_argument("--pairs", type=int, default=2, help="distinct seeded pairs per rank")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--masses", choices=["default", "niv16", "knn16", "uniform"], default="default",
                    help="reference masses: the workload's default (16-NN for LiDAR, else uniform), the "
                         "NIV lattice, inverse density from the 16th nearest neighbour, or uniform")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=None,
                    help="oracle iterations in the CPU baseline's sample (workload default: about "
                         "10-30 s on 16 cores)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="planar-bh: skip the theta 0.3 / 0.7 and all-pairs runs")
    ap.add_argument("--sweep-steps", type=int, default=2,
                    help="timed registrations per extra theta (and all-pairs) run")
    ap.add_argument("--walk", type=int, default=0,
                    help="Barnes-Hut walk (fga_params.bh_walk; 0 = by template size)")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------- distributed helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_seeds(rank: int, world: int, pairs: int, base: int = 1000):
    """Seeds of the pairs a rank registers: disjoint across ranks (weak scaling)."""
    return [base * (rank + 1) + k for k in range(pairs)]


def reduce_max_sum(t_ms: float, units: float, world: int):
    """(max over ranks of t_ms, sum over ranks of units)."""
    if world == 1:
        return t_ms, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    a = torch.tensor([t_ms], dtype=torch.float64, device=dev)
    b = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- roofline

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


DEVICE_HEADER = "paper_2009_14005_gb300/csrc/fga_device.cuh"


def source_hash(paths):
    """Hash of the kernel's source: its own file and the shared device header."""
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_file: str, summary: str, extra=()):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on the
    current source of the kernel (line 'traffic_bytes_per_launch: <B> source_sha: <h>',
    h = source_hash of the kernel's file, the shared device header and `extra`)."""
    p = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(p):
        return None
    cur = source_hash([os.path.join(ROOT, kernel_file), os.path.join(ROOT, DEVICE_HEADER)] +
                      [os.path.join(ROOT, e) for e in extra])
    for ln in open(p):
        if ln.startswith("traffic_bytes_per_launch:"):
            parts = ln.split()
            if len(parts) >= 4 and parts[3] == cur:
                return float(parts[1])
    return None


# --------------------------------------------------------------------------- workload

WORKLOADS = {
    # the headline configuration: LiDAR-like sweeps, Barnes-Hut
    # (G = 1 from the paper's parameter range: with 66.7 the trajectory on this
    # cloud is chaotic, so no FP32 run can track the FP64 one)
    "lidar-bh": dict(gen="lidar", n=120_000, iters=200, method="bh", theta=0.5, niv=False,
                     masses="knn16", G=1.0, eps=0.2, eta=0.2, cpu_iters=24),
    # 1k x 1k points on the unit sphere, all-pairs sum
    "sphere-direct": dict(gen="sphere", n=1000, iters=100, method="direct", theta=0.5, niv=False,
                          G=66.7, eps=0.05, eta=0.1),
    # large piecewise-planar scenes, all-pairs sum (a few iterations per step)
    "planar-direct": dict(gen="planar", n=262_144, iters=5, method="direct", theta=0.5, niv=False,
                          G=66.7, eps=0.2, eta=0.2),
    # large piecewise-planar scenes, Barnes-Hut
    "planar-bh": dict(gen="planar", n=1_000_000, iters=100, method="bh", theta=0.5, niv=False,
                      G=66.7, eps=0.2, eta=0.2, cpu_iters=1, ref_template=262_144),
    # many independent pairs (N, M log-uniform in [500, 50k], sphere and planar
    # shapes, rotations <= 60 deg), all-pairs or Barnes-Hut per pair by size,
    # one graph-captured loop per step; n = number of pairs
    "batch": dict(gen="batch", n=256, iters=100, method="auto", theta=0.5, niv=False,
                  G=66.7, eps=0.2, eta=0.2),
    # served requests: Poisson arrivals at 200/s, N and M log-uniform in
    # [1k, 500k], overlap 30-100 %; one step = one request of the trace
    # a parameter grid as one batch: a 1k-point anisotropic box and its copy
    # under a 30 deg rotation, registered under 25 G x 20 eps x 20 eta = 10^4
    # parameter cells, all-pairs forces; n = number of cells
    "grid": dict(gen="grid", n=10_000, iters=100, method="direct", theta=0.5, niv=False,
                 G=66.7, eps=0.05, eta=0.1),
    "serve": dict(gen="serve", n=500_000, iters=100, method="auto", theta=0.5, niv=False,
                  G=66.7, eps=0.2, eta=0.2, rate=200.0, lo=1000),
}


def workload(a):
    w = dict(WORKLOADS[a.workload])
    for k in ("n", "iters", "theta"):
        v = getattr(a, k)
        if v is not None:
            w[k] = v
    masses = getattr(a, "masses", "default")
    if masses == "default":
        masses = w.get("masses", "niv16" if w["niv"] else "uniform")
    w["masses"] = masses
    w["niv"] = w["masses"] == "niv16"
    if getattr(a, "cpu_iters", None) is not None:
        w["cpu_iters"] = a.cpu_iters
    w.setdefault("cpu_iters", 24)
    return w


def workload_config(a):
    w = workload(a)
    if w["gen"] in ("batch", "serve", "grid"):
        return special_config(a, w)
    name = "%s-%dk-%s%s-%dit" % (
        {"lidar": "lidar-sweeps", "sphere": "unit-sphere", "planar": "planar-scene",
         "batch": "batch"}[w["gen"]],
        max(w["n"] // 1000, 1), "bh-theta%.1f" % w["theta"] if w["method"] == "bh" else "direct",
        "", w["iters"])
    return {"workload": name, "N": w["n"], "M": w["n"], "iterations": w["iters"],
            "method": "barnes-hut" if w["method"] == "bh" else "all-pairs",
            "theta": w["theta"] if w["method"] == "bh" else None,
            "masses": {"niv16": "NIV lattice 16 (reference), uniform (template)",
                       "knn16": "inverse density from the 16th nearest neighbour (reference), uniform "
                                "(template)",
                       "uniform": "uniform"}[w["masses"]],
            "eps": w["eps"], "eta": w["eta"], "dt": 0.1, "G": w["G"], "pairs_per_rank": a.pairs,
            "l2": "flushed between steps (256 MB device write outside the timed events)",
            "inputs": "resident in HBM at the start of each timed step"}


def grid_cells(n):
    """(G, eps, eta) of the grid workload: log-spaced G in [1, 300] and eps in
    [0.01, 0.5], linear eta in [0.02, 0.5]; the first n cells of the 25 x 20 x 20
    grid (G slowest)."""
    Gs = np.geomspace(1.0, 300.0, 25)
    es = np.geomspace(0.01, 0.5, 20)
    hs = np.linspace(0.02, 0.5, 20)
    cells = [(g, e, h) for g in Gs for e in es for h in hs]
    return cells[:n]


def special_config(a, w):
    if w["gen"] == "serve":
        return {"workload": "serve-poisson%d-%dk-%dk-%dit" % (w["rate"], w["lo"] // 1000, w["n"] // 1000,
                                                                w["iters"]),
                "requests": a.steps, "arrival_rate_per_s": w["rate"],
                "N_M": "log-uniform in [%d, %d], independently" % (w["lo"], w["n"]),
                "overlap": "uniform in [0.3, 1.0] (cropped piecewise-planar scenes)",
                "iterations": w["iters"],
                "method": "per pair: all-pairs if N <= the autotuned crossover, else barnes-hut "
                          "(theta %.1f)" % w["theta"],
                "masses": "uniform", "eps": w["eps"], "eta": w["eta"], "dt": 0.1, "G": w["G"],
                "timing": "host clock: first arrival to last result; latency = submit to result on host",
                "l2": "not flushed: the trace's inputs (hundreds of MB) exceed L2",
                "inputs": "device-resident at submit (value); pinned host (e2e)"}
    if w["gen"] == "grid":
        return {"workload": "grid-%d-cells-box-1k-%dit" % (w["n"], w["iters"]), "cells": w["n"],
                "pair": "1000 points uniform in a 2 x 1.2 x 0.6 box and the same points under a "
                        "30 deg rotation and t = (0.1, -0.05, 0.08) (seed 0)",
                "G": "25 values log-spaced in [1, 300]", "eps": "20 values log-spaced in [0.01, 0.5]",
                "eta": "20 values in [0.02, 0.5]", "iterations": w["iters"], "method": "all-pairs",
                "masses": "uniform", "dt": 0.1,
                "l2": "flushed between steps (256 MB device write outside the timed events)",
                "inputs": "resident in HBM at the start of each timed step; one preparation "
                          "shared by all cells"}
    if w["gen"] == "batch":
        return {"workload": "batch-%d-pairs-500-50k-%dit" % (w["n"], w["iters"]), "pairs": w["n"],
                "N_M": "log-uniform in [500, 50000], independently", "iterations": w["iters"],
                "method": "per pair: all-pairs if N <= the autotuned crossover, else barnes-hut "
                          "(theta %.1f)" % w["theta"],
                "masses": "uniform", "eps": w["eps"], "eta": w["eta"], "dt": 0.1, "G": w["G"],
                "pairs_per_rank": a.pairs,
                "l2": "flushed between steps (256 MB device write outside the timed events)",
                "inputs": "resident in HBM at the start of each timed step"}
    raise ValueError(w["gen"])


def make_pairs(seeds, a):
    w = workload(a)
    if w["gen"] == "batch":
        return [synth.batch_pairs(s, count=w["n"]) for s in seeds]
    if w["gen"] == "grid":
        return [[synth.box_pair(0, n=1000, deg=30.0)] for s in seeds]
    if w["gen"] == "serve":
        tr = synth.serve_trace(seeds[0], max(a.steps, 1), rate=w["rate"], lo=w["lo"], hi=w["n"])
        return [[(X, Y, R, t) for _, X, Y, R, t in tr]]
    gen = {"lidar": synth.lidar_pair, "sphere": synth.sphere_pair,
           "planar": synth.planar_scene_pair}[w["gen"]]
    return [gen(s, n=w["n"]) for s in seeds]


def lib_params(fga, a):
    w = workload(a)
    return fga.params(method={"bh": fga.FGA_BH, "direct": fga.FGA_DIRECT, "auto": fga.FGA_AUTO}[w["method"]],
                      theta=w["theta"], max_iter=w["iters"], G=w["G"], eps=w["eps"], eta=w["eta"],
                      mass_mode={"niv16": fga.FGA_MASS_NIV, "knn16": fga.FGA_MASS_KNN,
                                 "uniform": fga.FGA_MASS_UNIFORM}[w["masses"]], lattice=16, profile=1,
                      bh_walk=getattr(a, "walk", 0))


def cpu_single_thread(pair, a, iters: int = 20):
    """The oracle's rate on one core (the all-pairs sphere workload's second
    CPU figure), on `iters` iterations of the same pair."""
    import oracle
    oracle.build()
    before = oracle.max_threads()
    oracle.set_threads(1)
    try:
        i, t, _ = cpu_sample(pair, a, iters)
    finally:
        oracle.set_threads(before)
    return {"value": i / t, "unit": "interactions/s", "cores": 1,
            "sample": "%d of %d iterations on one core (%.2f s)" % (iters, workload(a)["iters"], t)}


def cpu_direct_sample(pair, a, m_sample: int = 4096):
    """The oracle's all-pairs force (Eq. 6, FP64) for the first `m_sample`
    template points against the whole normalised reference, one evaluation:
    the CPU rate of the all-pairs sum on a Barnes-Hut workload, labelled as a
    subsample."""
    import oracle
    oracle.build()
    X, Y, _, _ = pair
    Xn, Yn, _ = oracle.normalize(X, Y)
    Ys = Yn[:m_sample]
    w = workload(a)
    mX = np.full(len(Xn), 1.0 / len(Xn))
    t0 = time.perf_counter()
    oracle.direct_acc(Xn, mX, Ys, w["G"], w["eps"])
    t = time.perf_counter() - t0
    return {"value": len(Xn) * len(Ys) / t, "unit": "interactions/s", "cores": oracle.max_threads(),
            "sample": "all-pairs force of %d template points against all %d reference points, one "
                      "evaluation (%.2f s)" % (len(Ys), len(Xn), t)}


def direct_equivalent(pair_terms: float, t_ms: float):
    """All-pairs-equivalent rate of a Barnes-Hut run, labelled as such: N * M
    pairs per iteration, as if every pair were summed exactly, over the same
    time. The metric itself counts only the terms Barnes-Hut evaluates."""
    return {"value": pair_terms / (t_ms / 1e3) if t_ms > 0 else None, "unit": "pair-interactions/s",
            "note": "all-pairs equivalent (N * M per iteration); Barnes-Hut evaluates fewer terms"}


def cpu_sample(pair, a, iters, min_s: float = 3.0):
    """The FP64 oracle on one pair for `iters` iterations (bounded sample).

    For the all-pairs workloads whose sample would exceed ~2e10 terms, the
    template is cut to its first points (the time per term does not depend on
    which points)."""
    import oracle
    oracle.build()
    w = workload(a)
    if w["gen"] in ("batch", "serve", "grid"):
        pair = pair[0]
        w = dict(w, method="direct" if len(pair[0]) <= 32768 else "bh")
    X, Y, _, _ = pair
    if w["method"] == "direct":
        keep = int(max(1, min(len(Y), 2e10 / (len(X) * iters))))
        Y = Y[:keep]
    p = oracle.Params(method=oracle.FGA_BH if w["method"] == "bh" else oracle.FGA_DIRECT,
                      theta=w["theta"], max_iter=iters, niv_masses=w["niv"],
                      knn_masses=w["masses"] == "knn16", lattice=16, G=w["G"], eps=w["eps"], eta=w["eta"])
    # small samples are repeated until they have run for at least min_s seconds
    inter, dt, reps = 0, 0.0, 0
    while reps == 0 or (dt < min_s and reps < 1000):
        t0 = time.perf_counter()
        o = oracle.register_full(X, Y, p)
        dt += time.perf_counter() - t0
        inter += o["interactions"]
        reps += 1
    return inter, dt, oracle.max_threads()


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload(a)
    pair = make_pairs(shard_seeds(0, 1, 1), a)[0]
    m_ref = w.get("ref_template")
    if m_ref and w["gen"] not in ("batch", "serve", "grid"):
        X, Y, R, t = pair
        pair = (X, Y[:m_ref], R, t)
    for _ in range(a.warmup):
        cpu_sample(pair, a, 1, min_s=0.0)
    total_i, total_t, cores = 0, 0.0, 1
    for _ in range(a.steps):
        i, t, cores = cpu_sample(pair, a, 1, min_s=0.0)
        total_i += i
        total_t += t
    value = total_i / total_t
    if w["gen"] in ("batch", "serve", "grid"):
        what = "the workload's first pair"
    else:
        what = "the %d x %d pair" % (len(pair[0]), len(pair[1])) + (
            " (the first %d template points of the %d)" % (m_ref, w["n"]) if m_ref else "")
    sample = ("FP64 C oracle, Algorithm 2 (%s): normalisation, %s masses, %sand ONE iteration of the "
              "loop on %s per step" % ("BHForce" if w["method"] == "bh" else "all-pairs sum / BHForce by size",
                                       w["masses"], "tree " if w["method"] != "direct" else "", what))
    line = {"impl": "reference", "metric": "pair-interactions/s", "value": value,
            "unit": "interactions/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total_t / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(a),
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_registrations(fga, dev, p, steps, flush, stream, offset=0, gts=None):
    """`steps` whole registrations on device-resident pairs, each bracketed by
    CUDA events on the launch stream, the L2 flushed before each (outside the
    events). Returns per-step ms, the summed counters and, with `gts` (ground
    truth (R, t, bbox diagonal) per pair), each result's error against it."""
    import torch
    import oracle
    out = dict(step_ms=[], inter=0, force_ms=0.0, force_launches=0, pair_terms=0, gt_rot=[], gt_t=[])
    for k in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        Xd, Yd = dev[(k + offset) % len(dev)]
        e0.record(stream)
        R, t, st = fga.fga_register(Xd, Yd, p, stream=stream)
        e1.record(stream)
        e1.synchronize()
        out["step_ms"].append(e0.elapsed_time(e1))
        out["inter"] += st["interactions"]
        out["force_ms"] += st["force_ms"]
        out["force_launches"] += st["force_launches"]
        out["pair_terms"] += int(Xd.shape[0]) * int(Yd.shape[0]) * st["iterations"]
        if gts is not None:
            Rg, tg, diag = gts[(k + offset) % len(dev)]
            out["gt_rot"].append(oracle.rotation_error_deg(R, Rg))
            out["gt_t"].append(float(np.linalg.norm(np.asarray(t) - tg)) / diag)
    return out


def gt_summary(m):
    """Ground-truth error of the timed registrations (the synthetic pairs carry
    the motion that generated them)."""
    if not m["gt_rot"]:
        return None
    return {"rot_deg_median": float(np.median(m["gt_rot"])), "rot_deg_max": float(np.max(m["gt_rot"])),
            "t_rel_median": float(np.median(m["gt_t"])), "t_rel_max": float(np.max(m["gt_t"])),
            "note": "rotation (deg) and translation (/ bbox diagonal) of each timed result against the "
                    "motion that generated the synthetic pair"}


def roofline_of(kname, inter, force_ms, force_launches, t_local, peaks, peak_src, sms, summary):
    """FP32-issue roofline of the dominant force kernel from its CUDA-event launch times."""
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_rate = sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / FP32_INSTR_PER_INTERACTION
    launch_inter = inter / max(force_launches, 1)
    launch_s = force_ms / 1e3 / max(force_launches, 1)
    achieved = launch_inter / launch_s if launch_s > 0 else 0.0
    return {"bound": "alu", "kernel": kname, "achieved": achieved / 1e9, "peak": peak_rate / 1e9,
            "unit": "Ginteractions/s", "frac": achieved / peak_rate,
            "traffic": recorded_traffic("paper_2009_14005_gb300/csrc/fga_force.cu", summary),
            "peak_source": "%d SMs x %d FP32 lanes x %.0f MHz (sm_max_mhz, %s) / %d FP32 "
                           "instructions per interaction" % (sms, FP32_LANES_PER_SM, sm_mhz, peak_src,
                                                             FP32_INSTR_PER_INTERACTION),
            "launches": force_launches, "interactions_per_launch": launch_inter,
            "mean_launch_ms": 1e3 * launch_s, "share_of_step": force_ms / max(t_local, 1e-9)}


def small_loop_roofline(fga, pair, p, iters, stream, peaks, peak_src, sms, summary):
    """Roofline of the one-launch loop of a small all-pairs pair: CUDA events
    around fga_step(iters) of a state on the normalised pair, which is one
    launch of k_small_loop when the pair is small enough (else None)."""
    import torch
    Xn, Yn, _ = fga.fga_normalize(pair[0], pair[1], stream=stream)
    q = fga.params(**{k: getattr(p, k) for k, _ in p._fields_})
    q.profile = 0
    best = None
    for _ in range(3):
        s = fga.fga_state_create(Xn, None, Yn, None, q, stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n0 = fga.fga_launch_count()
        e0.record(stream)
        s.step(iters, stream=stream)
        e1.record(stream)
        e1.synchronize()
        launched = fga.fga_launch_count() - n0
        _, _, st = s.get(stream=stream)
        s.close()
        if launched != 1:
            return None
        ms = e0.elapsed_time(e1)
        if best is None or ms < best[0]:
            best = (ms, st["interactions"])
    ms, inter = best
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_rate = sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / FP32_INSTR_PER_INTERACTION
    achieved = inter / (ms / 1e3)
    return {"bound": "alu", "kernel": "k_small_loop", "achieved": achieved / 1e9, "peak": peak_rate / 1e9,
            "unit": "Ginteractions/s", "frac": achieved / peak_rate,
            "traffic": recorded_traffic("paper_2009_14005_gb300/csrc/fga_small.cu", summary,
                                        extra=("paper_2009_14005_gb300/csrc/fga_epi.cuh",)),
            "peak_source": "%d SMs x %d FP32 lanes x %.0f MHz (sm_max_mhz, %s) / %d FP32 "
                           "instructions per interaction" % (sms, FP32_LANES_PER_SM, sm_mhz, peak_src,
                                                             FP32_INSTR_PER_INTERACTION),
            "launches": 1, "interactions_per_launch": inter, "mean_launch_ms": ms,
            "timing": "CUDA events around the one launch of fga_step(%d) (all iterations in one "
                      "thread-block cluster), best of 3, outside the timed region" % iters}


def run_ours(a):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as fga

    w = workload(a)
    pairs = make_pairs(shard_seeds(rank, world, a.pairs), a)
    dev = [(torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")) for X, Y, _, _ in pairs]
    host = [(torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()) for X, Y, _, _ in pairs]
    gts = [(np.asarray(Rg), np.asarray(tg), float(np.linalg.norm(X.max(0) - X.min(0))))
           for X, Y, Rg, tg in pairs]
    # timed registrations run as a user calls them (no per-launch events, the
    # iteration loop as one CUDA graph); the force kernel's launch times come
    # from one extra registration with profile = 1 outside the timed region
    p = lib_params(fga, a)
    p.profile = 0
    p_prof = lib_params(fga, a)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    for k in range(a.warmup):
        Xd, Yd = dev[k % len(dev)]
        fga.fga_register(Xd, Yd, p)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = fga.fga_launch_count()
    m = time_registrations(fga, dev, p, a.steps, flush, stream, gts=gts)
    torch.cuda.synchronize()
    barrier(world)
    launches = fga.fga_launch_count() - launches0
    clk = clocks.stop()
    step_ms = m["step_ms"]
    t_local = sum(step_ms)
    t_max, inter_all = reduce_max_sum(t_local, float(m["inter"]), world)
    _, pair_terms_all = reduce_max_sum(t_local, float(m["pair_terms"]), world)
    value = inter_all / (t_max / 1e3)

    # end to end through the same C call with pinned host inputs
    e2e_t, e2e_i, h2d, d2h = 0.0, 0, 0, 0
    for k in range(a.e2e_steps):
        Xh, Yh = host[k % len(host)]
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R, t, st = fga.fga_register(Xh, Yh, p, stream=stream)
        e2e_t += time.perf_counter() - t0
        e2e_i += st["interactions"]
        h2d, d2h = st["h2d_bytes"], st["d2h_bytes"]
    e2e_tmax, e2e_iall = reduce_max_sum(1e3 * e2e_t, float(e2e_i), world)

    # planar-bh: theta 0.3 and 0.7, and the tiled all-pairs sum, on the same pairs
    sweep = {}
    if a.workload == "planar-bh" and not a.no_sweep:
        for th in (0.3, 0.7):
            q = lib_params(fga, a)
            q.theta = th
            fga.fga_register(*dev[0], q)
            s = time_registrations(fga, dev, q, a.sweep_steps, flush, stream)
            tl = sum(s["step_ms"])
            tm, ia = reduce_max_sum(tl, float(s["inter"]), world)
            sweep["theta_%.1f" % th] = {
                "value": ia / (tm / 1e3), "unit": "interactions/s", "steps": a.sweep_steps,
                "registrations_per_s": a.sweep_steps * world / (tm / 1e3), "ms_per_step": tm / a.sweep_steps,
                "k_bh_frac": None, "_s": s, "_tl": tl}
        q = lib_params(fga, a)
        q.method = fga.FGA_DIRECT
        q.max_iter = 5
        fga.fga_register(*dev[0], q)
        s = time_registrations(fga, dev, q, a.sweep_steps, flush, stream)
        tl = sum(s["step_ms"])
        tm, ia = reduce_max_sum(tl, float(s["inter"]), world)
        sweep["all_pairs"] = {"value": ia / (tm / 1e3), "unit": "interactions/s", "steps": a.sweep_steps,
                              "iterations": 5, "ms_per_step": tm / a.sweep_steps,
                              "note": "tiled all-pairs sum (Eq. 6) on the same pairs; 5 iterations per "
                                      "registration, N * M terms per iteration",
                              "_s": s, "_tl": tl}

    # per-launch times of the force kernel: one profiled registration of the first pair
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, _, stp = fga.fga_register(dev[0][0], dev[0][1], p_prof, stream=stream)
    e1.record(stream)
    e1.synchronize()
    prof_step_ms = e0.elapsed_time(e1)

    if rank != 0:
        return 0
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    kname = "k_bh" if w["method"] == "bh" else "k_direct"
    roof = roofline_of(kname, stp["interactions"], stp["force_ms"], stp["force_launches"], prof_step_ms,
                       peaks, peak_src, sms, "%s_%s.md" % (kname, a.workload))
    roof["timing"] = ("CUDA events around every force launch of one extra registration of the first "
                      "pair (fga_params.profile = 1), outside the timed region")
    if w["method"] != "bh":
        loop = small_loop_roofline(fga, dev[0], p, w["iters"], stream, peaks, peak_src, sms,
                                   "k_small_loop_%s.md" % a.workload)
        if loop is not None:
            # the timed registrations ran every iteration in one cluster launch:
            # that kernel is the step's dominant one; the separate-launch force
            # kernel stays as context
            loop["share_of_step"] = loop["mean_launch_ms"] / max(float(np.median(step_ms)), 1e-9)
            loop["separate_launches"] = {k: roof[k] for k in ("kernel", "achieved", "frac",
                                                              "mean_launch_ms", "launches")}
            roof = loop
    line = {"metric": "pair-interactions/s", "value": value, "unit": "interactions/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(a),
            "registrations_per_s": a.steps * world / (t_max / 1e3),
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "e2e": {"value": e2e_iall / (e2e_tmax / 1e3) if e2e_tmax > 0 else None,
                    "unit": "interactions/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_tmax / max(a.e2e_steps, 1)},
            "gpu_launches": launches, "roofline": roof, "clocks": clk,
            "ground_truth_error": gt_summary(m)}
    for key, v in sweep.items():
        s, tl = v.pop("_s"), v.pop("_tl")
        kn = "k_direct" if key == "all_pairs" else "k_bh"
        r = roofline_of(kn, s["inter"], s["force_ms"], s["force_launches"], tl, peaks, peak_src, sms,
                        "%s_%s.md" % (kn, a.workload))
        v["roofline_frac"] = r["frac"]
        v["mean_launch_ms"] = r["mean_launch_ms"]
        v.pop("k_bh_frac", None)
        line[key] = v
    if w["method"] == "bh":
        line["direct_equivalent"] = direct_equivalent(pair_terms_all, t_max)
    if world == 1 and not a.no_cpu_baseline:
        i, t, cores = cpu_sample(pairs[0], a, w["cpu_iters"])
        line["cpu_baseline"] = {"value": i / t, "unit": "interactions/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "FP64 C oracle (OpenMP), normalisation + %s masses + tree + "
                                          "%d of %d iterations on the first %dk x %dk pair (%.1f s; a sample shorter than 3 s is repeated)"
                                          % (w["masses"], w["cpu_iters"], w["iters"], w["n"] // 1000,
                                             w["n"] // 1000, t)}
        if a.workload == "sphere-direct":
            line["cpu_baseline"]["single_thread"] = cpu_single_thread(pairs[0], a)
        if w["method"] == "bh":
            line["cpu_baseline"]["direct_subsample"] = cpu_direct_sample(pairs[0], a)
    print(json.dumps(line), flush=True)
    return 0


def run_ours_batch(a):
    """One step = fga_register_batch over a whole batch of resident pairs."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as fga

    batches = make_pairs(shard_seeds(rank, world, a.pairs), a)
    dev = [[(torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")) for X, Y, _, _ in b]
           for b in batches]
    host = [[(torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()) for X, Y, _, _ in b]
            for b in batches]
    p = lib_params(fga, a)
    p.profile = 0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    tuned = fga.autotune(p, stream=stream)  # tiles and crossover for this GPU (untimed)
    for k in range(a.warmup):
        fga.fga_register_batch(dev[k % len(dev)], p, stream=stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = fga.fga_launch_count()
    step_ms, inter, regs, setup_ms = [], 0, 0, []
    for k in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, st = fga.fga_register_batch(dev[k % len(dev)], p, stream=stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        inter += st["interactions"]
        regs += len(res)
        setup_ms.append(st["elapsed_ms"] - st["force_ms"])  # preparation before the iteration graph
    torch.cuda.synchronize()
    barrier(world)
    launches = fga.fga_launch_count() - launches0
    clk = clocks.stop()
    t_local = sum(step_ms)
    t_max, inter_all = reduce_max_sum(t_local, float(inter), world)
    _, regs_all = reduce_max_sum(t_local, float(regs), world)
    value = inter_all / (t_max / 1e3)

    # the force kernel alone: one profiled call (plain launches, events around each)
    pp = lib_params(fga, a)
    pp.profile = 1
    flush.zero_()
    _, pst = fga.fga_register_batch(dev[0], pp, stream=stream)
    torch.cuda.synchronize()

    # the same batch, one fga_register call per pair (the one-pair path)
    seq_ms = 0.0
    flush.zero_()
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for Xd, Yd in dev[0]:
        fga.fga_register(Xd, Yd, p, stream=stream)
    s1.record(stream)
    s1.synchronize()
    seq_ms = s0.elapsed_time(s1)

    # end to end: pinned host inputs through the same C call
    e2e_t, e2e_i, h2d, d2h = 0.0, 0, 0, 0
    for k in range(a.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, st = fga.fga_register_batch(host[k % len(host)], p, stream=stream)
        e2e_t += time.perf_counter() - t0
        e2e_i += st["interactions"]
        h2d, d2h = st["h2d_bytes"], st["d2h_bytes"]
    e2e_tmax, e2e_iall = reduce_max_sum(1e3 * e2e_t, float(e2e_i), world)

    if rank != 0:
        return 0
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_rate = sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / FP32_INSTR_PER_INTERACTION
    launch_inter = pst["interactions"] / max(pst["force_launches"], 1)
    launch_s = pst["force_ms"] / 1e3 / max(pst["force_launches"], 1)
    achieved = launch_inter / launch_s if launch_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_batch_force", "achieved": achieved / 1e9,
            "peak": peak_rate / 1e9, "unit": "Ginteractions/s", "frac": achieved / peak_rate,
            "traffic": recorded_traffic("paper_2009_14005_gb300/csrc/fga_batch.cu",
                                        "k_batch_force_%s.md" % a.workload),
            "peak_source": "%d SMs x %d FP32 lanes x %.0f MHz (sm_max_mhz, %s) / %d FP32 "
                           "instructions per interaction" % (sms, FP32_LANES_PER_SM, sm_mhz, peak_src,
                                                             FP32_INSTR_PER_INTERACTION),
            "launches": pst["force_launches"], "interactions_per_launch": launch_inter,
            "mean_launch_ms": 1e3 * launch_s,
            "share_of_step": pst["force_ms"] / max(t_local / a.steps, 1e-9)}
    nb = len(dev[0])
    line = {"metric": "pair-interactions/s", "value": value, "unit": "interactions/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(a),
            "registrations_per_s": regs_all / (t_max / 1e3),
            "one_pair_path": {"registrations_per_s": nb / (seq_ms / 1e3), "ms_per_batch": seq_ms,
                              "note": "the same %d pairs, one fga_register call each" % nb},
            "setup_ms_per_step": float(np.mean(setup_ms)),
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "e2e": {"value": e2e_iall / (e2e_tmax / 1e3) if e2e_tmax > 0 else None,
                    "unit": "interactions/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_tmax / max(a.e2e_steps, 1)},
            "gpu_launches": launches, "roofline": roof, "clocks": clk,
            "autotuned": tune_summary(tuned)}
    if world == 1 and not a.no_cpu_baseline:
        i, t, cores = cpu_sample(batches[0], a, workload(a)["cpu_iters"])
        line["cpu_baseline"] = {"value": i / t, "unit": "interactions/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "FP64 C oracle (OpenMP), normalisation + tree + %d of %d "
                                          "iterations on the first pair of the batch (%d x %d, %.1f s; a sample shorter than 3 s is repeated)"
                                          % (workload(a)["cpu_iters"], workload(a)["iters"], len(batches[0][0][0]),
                                             len(batches[0][0][1]), t)}
    print(json.dumps(line), flush=True)
    return 0


def run_ours_grid(a):
    """One step = one fga_register_batch over all cells of the parameter grid."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as fga

    w = workload(a)
    X, Y, R_gt, t_gt = synth.box_pair(rank, n=1000, deg=30.0)  # every rank its own pair (weak scaling)
    Xd, Yd = torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")
    Xh, Yh = torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()
    cells = [fga.params(method=fga.FGA_DIRECT, G=float(g), eps=float(e), eta=float(h), max_iter=w["iters"])
             for g, e, h in grid_cells(w["n"])]
    base = fga.params(method=fga.FGA_DIRECT, max_iter=w["iters"])
    batch = [(Xd, Yd, None, None, c) for c in cells]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    tuned = fga.autotune(base, stream=stream)
    for _ in range(a.warmup):
        fga.fga_register_batch(batch, base, stream=stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = fga.fga_launch_count()
    step_ms, inter = [], 0
    for k in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, st = fga.fga_register_batch(batch, base, stream=stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        inter += st["interactions"]
    torch.cuda.synchronize()
    barrier(world)
    launches = fga.fga_launch_count() - launches0
    clk = clocks.stop()
    t_local = sum(step_ms)
    t_max, inter_all = reduce_max_sum(t_local, float(inter), world)
    value = inter_all / (t_max / 1e3)

    # the map the grid is for: rotation error of every cell against the ground truth
    import math
    err = np.array([math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(r["R"].T @ R_gt) - 1) / 2))))
                    for r in res])
    best = int(np.argmin(err))

    # the force kernel alone: one profiled call on the first 1000 cells
    pp = fga.params(method=fga.FGA_DIRECT, max_iter=w["iters"], profile=1)
    _, pst = fga.fga_register_batch(batch[:1000], pp, stream=stream)
    # the one-pair path on a sample of cells
    sample = cells[:: max(1, len(cells) // 200)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in sample:
        fga.fga_register(Xd, Yd, c, stream=stream)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    # e2e: host inputs through the same call
    e2e_t, h2d = 0.0, 0
    hbatch = [(Xh, Yh, None, None, c) for c in cells]
    for _ in range(a.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_h, st_h = fga.fga_register_batch(hbatch, base, stream=stream)
        e2e_t += time.perf_counter() - t0
        h2d = st_h["h2d_bytes"]
    e2e_tmax, e2e_iall = reduce_max_sum(1e3 * e2e_t, float(inter / max(a.steps, 1) * a.e2e_steps), world)

    if rank != 0:
        return 0
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_rate = sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / FP32_INSTR_PER_INTERACTION
    launch_inter = pst["interactions"] / max(pst["force_launches"], 1)
    launch_s = pst["force_ms"] / 1e3 / max(pst["force_launches"], 1)
    achieved = launch_inter / launch_s if launch_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_batch_force", "achieved": achieved / 1e9,
            "peak": peak_rate / 1e9, "unit": "Ginteractions/s", "frac": achieved / peak_rate,
            "traffic": recorded_traffic("paper_2009_14005_gb300/csrc/fga_batch.cu",
                                        "k_batch_force_%s.md" % a.workload),
            "peak_source": "%d SMs x %d FP32 lanes x %.0f MHz (sm_max_mhz, %s) / %d FP32 "
                           "instructions per interaction" % (sms, FP32_LANES_PER_SM, sm_mhz, peak_src,
                                                             FP32_INSTR_PER_INTERACTION),
            "launches": pst["force_launches"], "interactions_per_launch": launch_inter,
            "mean_launch_ms": 1e3 * launch_s,
            "measured_on": "fga_register_batch of the first 1000 cells, events around each force launch"}
    n = len(cells)
    line = {"metric": "pair-interactions/s", "value": value, "unit": "interactions/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(a),
            "registrations_per_s": n * a.steps * world / (t_max / 1e3),
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "grid_map": {"cells_within_1deg": float((err < 1.0).mean()),
                         "cells_within_0.1deg": float((err < 0.1).mean()),
                         "best": {"G": cells[best].G, "eps": cells[best].eps, "eta": cells[best].eta,
                                  "rot_err_deg": float(err[best])},
},
            "one_pair_path": {"registrations_per_s": len(sample) / seq_s,
                              "note": "%d cells of the grid, one fga_register call each" % len(sample)},
            "e2e": {"value": e2e_iall / (e2e_tmax / 1e3) if e2e_tmax > 0 else None,
                    "unit": "interactions/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": (8 * 12 + 64) * n,
                    "ms_per_step": e2e_tmax / max(a.e2e_steps, 1)},
            "gpu_launches": launches, "roofline": roof, "clocks": clk, "autotuned": tune_summary(tuned)}
    if world == 1 and not a.no_cpu_baseline:
        i, t, cores = cpu_sample([(X, Y, None, None)], a, w["cpu_iters"])
        line["cpu_baseline"] = {"value": i / t, "unit": "interactions/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "FP64 C oracle (OpenMP), %d of %d iterations of one cell "
                                          "(1000 x 1000, %.1f s; a sample shorter than 3 s is repeated)" % (w["cpu_iters"], w["iters"], t)}
    print(json.dumps(line), flush=True)
    return 0


def tune_summary(rep):
    return {"direct_max_n": rep["direct_max_n"],
            "direct_tiles": ["%dx%d" % (b, q) for b, q in zip(rep["direct_bs"], rep["direct_qpt"])],
            "sizes": list(rep["sizes"]),
            "direct_us_per_point": [round(x, 5) for x in rep["direct_us_per_point"]],
            "bh_us_per_point": [round(x, 5) for x in rep["bh_us_per_point"]],
            "tune_ms": rep["elapsed_ms"]}


def replay_served(fga, p, trace, inputs, warm):
    """Replays a request trace through a server in real time; returns
    (results, wall seconds from the first arrival to the last result)."""
    with fga.Server(p, iters_per_tick=4) as srv:
        for X, Y in warm:
            srv.submit(X, Y)
        srv.drain()
        results = []
        t0 = time.perf_counter()
        for (t_arr, *_), (X, Y) in zip(trace, inputs):
            while time.perf_counter() - t0 < t_arr:
                results.extend(srv.poll(256, wait_ms=1))
            srv.submit(X, Y)
            results.extend(srv.poll(256, wait_ms=0))
        results.extend(srv.drain())
        wall = time.perf_counter() - t0
        st = srv.stats()
    return results, wall, st


def replay_one_pair(fga, p, trace, inputs, stream):
    """The same trace through the one-pair path: FIFO, one fga_register call
    per request. Returns (latencies ms, wall seconds, interactions)."""
    lat, inter = [], 0
    t0 = time.perf_counter()
    for (t_arr, *_), (X, Y) in zip(trace, inputs):
        while time.perf_counter() - t0 < t_arr:
            time.sleep(0.0002)
        R, t, st = fga.fga_register(X, Y, p, stream=stream)
        inter += st["interactions"]
        lat.append(1e3 * (time.perf_counter() - t0 - t_arr))
    return lat, time.perf_counter() - t0, inter


def run_ours_serve(a):
    """One step = one request of a Poisson trace replayed through the server."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2009_14005_gb300 as fga

    w = workload(a)
    trace = synth.serve_trace(shard_seeds(rank, world, 1)[0], a.steps + a.warmup, rate=w["rate"],
                              lo=w["lo"], hi=w["n"])
    warm_tr, trace = trace[:a.warmup], trace[a.warmup:]
    t_first = trace[0][0]
    trace = [(t - t_first, X, Y, R, tt) for t, X, Y, R, tt in trace]
    dev = [(torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")) for _, X, Y, _, _ in trace]
    warm = [(torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")) for _, X, Y, _, _ in warm_tr]
    host = [(torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()) for _, X, Y, _, _ in trace]
    torch.cuda.synchronize()
    p = lib_params(fga, a)
    p.profile = 0
    stream = torch.cuda.current_stream()
    tuned = fga.autotune(p, stream=stream)  # tiles and crossover for this GPU (untimed)

    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    launches0 = fga.fga_launch_count()
    res, wall, sst = replay_served(fga, p, trace, dev, warm)
    launches = fga.fga_launch_count() - launches0
    clk = clocks.stop()
    ok = [r for r in res if r["status"] in (fga.FGA_OK, fga.FGA_EDEGENERATE)]
    lat = [r["done_ms"] - r["submit_ms"] for r in ok]
    inter = sum(r["interactions"] for r in ok)
    t_max, inter_all = reduce_max_sum(1e3 * wall, float(inter), world)
    _, regs_all = reduce_max_sum(1e3 * wall, float(len(ok)), world)
    value = inter_all / (t_max / 1e3)

    # e2e: the same trace with pinned host inputs (copies inside the server)
    res_h, wall_h, _ = replay_served(fga, p, trace, host, warm)
    inter_h = sum(r["interactions"] for r in res_h)
    e2e_tmax, e2e_iall = reduce_max_sum(1e3 * wall_h, float(inter_h), world)
    h2d = sum(4 * (X.numel() + Y.numel()) for X, Y in host) // max(len(host), 1)

    # the one-pair-per-launch path on the same trace
    base_lat, base_wall, base_inter = replay_one_pair(fga, p, trace, dev, stream)

    # the dominant kernel timed alone: one profiled batch of the trace's first pairs
    pp = lib_params(fga, a)
    pp.profile = 1
    sample = dev[:min(32, len(dev))]
    _, pst = fga.fga_register_batch(sample, pp, stream=stream)
    torch.cuda.synchronize()

    if rank != 0:
        return 0
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_rate = sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / FP32_INSTR_PER_INTERACTION
    launch_inter = pst["interactions"] / max(pst["force_launches"], 1)
    launch_s = pst["force_ms"] / 1e3 / max(pst["force_launches"], 1)
    achieved = launch_inter / launch_s if launch_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_batch_force", "achieved": achieved / 1e9,
            "peak": peak_rate / 1e9, "unit": "Ginteractions/s", "frac": achieved / peak_rate,
            "traffic": recorded_traffic("paper_2009_14005_gb300/csrc/fga_batch.cu",
                                        "k_batch_force_%s.md" % a.workload),
            "peak_source": "%d SMs x %d FP32 lanes x %.0f MHz (sm_max_mhz, %s) / %d FP32 "
                           "instructions per interaction" % (sms, FP32_LANES_PER_SM, sm_mhz, peak_src,
                                                             FP32_INSTR_PER_INTERACTION),
            "launches": pst["force_launches"], "interactions_per_launch": launch_inter,
            "mean_launch_ms": 1e3 * launch_s,
            "measured_on": "fga_register_batch of the trace's first %d pairs, events around each "
                           "force launch" % len(sample)}
    line = {"metric": "pair-interactions/s", "value": value, "unit": "interactions/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(a),
            "registrations_per_s": regs_all / (t_max / 1e3),
            "p50_ms": float(np.percentile(lat, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat else None,
            "failed": len(res) - len(ok),
            "server": {k: sst[k] for k in ("ticks", "pair_iterations", "busy_ms")},
            "one_pair_path": {"registrations_per_s": len(trace) / base_wall,
                              "interactions_per_s": base_inter / base_wall,
                              "p50_ms": float(np.percentile(base_lat, 50)),
                              "p99_ms": float(np.percentile(base_lat, 99)),
                              "note": "same trace, FIFO, one fga_register call per request"},
            "e2e": {"value": e2e_iall / (e2e_tmax / 1e3) if e2e_tmax > 0 else None,
                    "unit": "interactions/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 8 * 12 + 64,
                    "ms_per_step": e2e_tmax / max(a.steps, 1),
                    "p50_ms": float(np.percentile([r["done_ms"] - r["submit_ms"] for r in res_h], 50)),
                    "p99_ms": float(np.percentile([r["done_ms"] - r["submit_ms"] for r in res_h], 99))},
            "gpu_launches": launches, "roofline": roof, "clocks": clk,
            "autotuned": tune_summary(tuned)}
    if world == 1 and not a.no_cpu_baseline:
        X, Y = trace[0][1], trace[0][2]
        i, t, cores = cpu_sample([(X, Y, None, None)], a, w["cpu_iters"])
        line["cpu_baseline"] = {"value": i / t, "unit": "interactions/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "FP64 C oracle (OpenMP), normalisation + tree + %d of %d "
                                          "iterations on the trace's first request (%d x %d, %.1f s; a sample shorter than 3 s is repeated)"
                                          % (w["cpu_iters"], w["iters"], len(X), len(Y), t)}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    a = parse_args(argv)
    if a.impl == "reference":
        return run_reference(a)
    if workload(a)["gen"] == "batch":
        return run_ours_batch(a)
    if workload(a)["gen"] == "serve":
        return run_ours_serve(a)
    if workload(a)["gen"] == "grid":
        return run_ours_grid(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
