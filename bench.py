"""Benchmark: converged SPH particles/s for the density / smoothing-length solve on GB300.

One step = one pass of the whole hot path on one batch of input already resident in HBM:
sph_sort (fixed-point Morton keys, radix sort, gather, cell tables) followed by
sph_density_solve (all density passes, h updates and compactions until every particle is
in its band, then the scatter to caller order).

Default workload (--config c5, the largest configuration): 67,108,864 particles, 4,096
Plummer clumps (scale radii log-uniform in [1e-3, 1e-2], 70 % of the particles) plus a
uniform background in the periodic unit box, Nngb = 64 +- 2, and 8 snapshots drifting by
N(0, 1e-4^2) per coordinate.  Snapshot 0 is solved cold, untimed; each step replays the next
snapshot warm-started from the previous one's h, with the pass loop in a CUDA graph.
--config c1|c2|c3 time one cold solve of those sets, c4 the 20,000 batched groups.

Printed (one JSON line, rank 0): value = converged particles/s over all ranks, the FP32 +
compensated path; e2e = the same through the C ABI with the inputs in pinned host memory and
the host<->device copies inside the timed region; roofline of the density kernel (FP32 ALU
bound, against a measured FP32 FMA rate) with the step's HBM rate from algorithmic bytes; the
plain FP64 GPU solve beside it; the FP64 CPU oracle timed on this host on a bounded sample
(cpu_baseline).  ``--impl reference`` times only the oracle.

Multi-GPU: one process per GPU (torchrun), each solving its own replica of the workload
(the single periodic system is not sharded: replicas only), value = all particles / max time.
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

METRIC = "converged SPH particles/s (rho+h)"
UNIT = "particles/s"
# FP32 operations the method needs per in-h pair, the figure the scope table fixes (30): 3
# differences, r^2 (3 mul + 2 add), 1 compare, q (sqrt + 1 mul), w (7), -q w' (5), m*w (1),
# three sums (3), the integer count (1), and the two per-pair scalings of the sums' constant
# factors that a scalar loop would spend (the GPU applies them once per target).
FLOP_PER_PAIR = 30
# algorithmic HBM bytes of one sort + solve (the scope table's per-particle figures): keys,
# radix passes, gather, cell table, solve set-up and scatter per particle, and the record,
# h state and outputs per particle evaluation of every pass
BYTES_PER_PARTICLE = 200
BYTES_PER_EVALUATION = 80
KNN_METRIC = "kNN SPH particles/s (h = K-th neighbour distance, rho at h)"
INTERACT_METRIC = "SPH interaction-pass particles/s (rho, velocity mean, dispersion, div, curl at h)"
# FP32 operations per in-h pair of the interaction pass (FMA = 2): the distance test (3
# differences, r^2: 1 mul + 2 FMA), q (1 mul, sqrt), w and g = -w'/q (7), u = v_j - v_i (3),
# m w and m g (2), S0 (1), S1 (3 FMA), |u|^2 (1 mul + 2 FMA) and S2 (1 FMA), d . u (1 mul + 2
# FMA) and D (1 FMA), d x u (3 mul + 3 FMA) and C (3 FMA)
FLOP_PER_INTERACT_PAIR = 58
# algorithmic HBM bytes per particle of one interaction call: the velocity gather (24 B read,
# 16 B record written), the solve set-up (h read, sorted h, FP32 h, todo: 28 B), the target's
# position record, velocity record and FP64 velocity (16 + 16 + 24 B) and the outputs (9
# doubles + a count: 76 B)
BYTES_PER_INTERACT_PARTICLE = 200
# one neighbour-list entry: a squared distance from three offsets (3 subtractions, 3 multiplies,
# 2 additions); the radius compare and the selection are not counted
FLOP_PER_LIST_ENTRY = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default="c5",
                    help="c5 snapshot replay (the headline), c1|c2|c3 single cold solve, c4 batched groups")
    ap.add_argument("--n", type=int, default=0, help="override the particle count")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle targets (0 = auto)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tuning (profiling runs)")
    ap.add_argument("--kernel", default="m4", choices=["m4", "c6"],
                    help="c6: the paper's Wendland C6 kernel at Nngb = 295 +- 5")
    ap.add_argument("--interact", action="store_true",
                    help="time the interaction pass (sph_interact: velocity mean, dispersion, "
                         "divergence and curl at the converged h) instead of the solve")
    ap.add_argument("--knn", type=int, default=0,
                    help="K > 0: time the k-nearest-neighbour h (sph_knn_solve) instead of the "
                         "N_w solve; the paper's K is 295")
    return ap.parse_args()


def workload(args):
    from paper_1612_06090_gb300 import inputs

    kw = {"n": args.n} if args.n else {}
    if args.kernel == "c6":
        kw.update(nngb=295.0, tol=5.0)
    wl = inputs.make(args.config, **kw)
    desc = {
        "c1": "uniform periodic box",
        "c2": "64 Plummer spheres (a=0.01, 70%) + uniform background, periodic unit box",
        "c3": "log-normal density field (64^3 Gaussian, P(k)~k^-2, sigma_ln=2), periodic unit box",
        "c5": "4096 Plummer clumps (a log-uniform in [1e-3,1e-2], 70%) + background, periodic unit box",
    }[args.config]
    kname = "Wendland C6 kernel" if args.kernel == "c6" else "M4 kernel"
    return wl, f"{args.config}: {wl.n:,} particles, {desc}, Nngb={wl.nngb:g}+-{wl.tol:g}, {kname}"


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "native" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks during the timed region --------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    # the raw samples go to $SPH_BENCH_CLOCKS_DIR (default: the system temporary directory);
    # the JSON line carries their summary
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        d = os.environ.get("SPH_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---- the CPU oracle on a bounded sample --------------------------------------------------------

def cpu_baseline(wl, n_targets, kernel="m4"):
    import numpy as np

    import oracle

    rng = np.random.default_rng(99)
    tg = np.sort(rng.choice(wl.n, size=min(n_targets, wl.n), replace=False))
    t0 = time.perf_counter()
    r = oracle.solve(wl.pos, wl.mass, wl.h0[tg], box=wl.box, periodic=wl.periodic, nngb=wl.nngb,
                     tol=wl.tol, targets=tg, kernel="wendland_c6" if kernel == "c6" else "m4")
    dt = time.perf_counter() - t0
    return {"value": len(tg) / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{len(tg):,} random targets of the same workload solved against all "
                      f"{wl.n:,} particles (FP64, bucket grids, OpenMP dynamic over the todo list); "
                      f"{dt:.1f} s wall incl. grid builds",
            "seconds": dt, "passes": r["stats"]["passes"]}


def cpu_baseline_knn(wl, n_targets, k, kernel="m4"):
    import numpy as np

    import oracle

    rng = np.random.default_rng(98)
    tg = np.sort(rng.choice(wl.n, size=min(n_targets, wl.n), replace=False))
    t0 = time.perf_counter()
    oracle.knn(wl.pos, wl.mass, k, box=wl.box, periodic=wl.periodic, targets=tg,
               kernel="wendland_c6" if kernel == "c6" else "m4")
    dt = time.perf_counter() - t0
    return {"value": len(tg) / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{len(tg):,} random targets of the same workload, K = {k}: every distance to "
                      f"all {wl.n:,} particles sorted (qsort), then rho at h (FP64, OpenMP over "
                      f"targets); {dt:.1f} s wall",
            "seconds": dt}


def cpu_baseline_interact(wl, vel, h, n_targets=32):
    """The oracle's interaction sums on sampled targets of the same workload at the GPU's h, by
    brute force over all particles (a grid over tens of millions of particles costs a sort per
    level).  The oracle hands targets to its threads in chunks of 16."""
    import numpy as np

    import oracle

    k = min(n_targets, wl.n)
    tg = np.sort(np.random.default_rng(97).choice(wl.n, size=k, replace=False))
    t0 = time.perf_counter()
    oracle.interact(wl.pos, wl.mass, vel, h[tg], box=wl.box, periodic=wl.periodic, targets=tg, mode="brute")
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": min(oracle.threads(), -(-k // 16)), "kind": "oracle",
            "sample": f"{k} random targets of the same workload at the GPU's converged h: neighbours by "
                      f"brute force over all {wl.n:,} particles, then the sums (FP64, OpenMP over "
                      f"targets); {dt:.1f} s wall",
            "seconds": dt}


def cpu_baseline_replay(wl0, wl1, n_targets=0):
    """The oracle on sampled targets of the c5 replay: each target is solved cold on snapshot 0
    (untimed), then the timed part solves it on snapshot 1 warm-started from that solution, by
    brute force against all particles (a grid over 67 M particles costs a sort per level and
    call).  One brute-force evaluation scans all particles (about a second), and the oracle
    hands targets to its threads in chunks of 16, so the default sample of 8 targets runs on
    one thread: about 10 s timed after about 40 s untimed."""
    import numpy as np

    import oracle

    k = min(n_targets or 8, wl0.n)
    tg = np.sort(np.random.default_rng(96).choice(wl0.n, size=k, replace=False))
    cold = oracle.solve(wl0.pos, wl0.mass, wl0.h0[tg], nngb=wl0.nngb, tol=wl0.tol, targets=tg, mode="brute")
    t0 = time.perf_counter()
    r = oracle.solve(wl1.pos, wl1.mass, cold["h"], nngb=wl1.nngb, tol=wl1.tol, targets=tg, mode="brute")
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": min(oracle.threads(), -(-k // 16)), "kind": "oracle",
            "sample": f"{k} random targets of snapshot 1, warm-started from their own snapshot-0 solution "
                      f"(solved first, untimed), each solved by brute force against all {wl1.n:,} "
                      f"particles (FP64, OpenMP over targets); {r['stats']['passes']} passes, {dt:.1f} s wall",
            "seconds": dt}


def cpu_baseline_batch(wl, n_groups):
    """The oracle on a bounded sample of the c4 groups, each group solved on its own."""
    import numpy as np

    import oracle

    rng = np.random.default_rng(97)
    pick = np.sort(rng.choice(wl.n_groups, size=min(wl.n_groups, n_groups), replace=False))
    t0 = time.perf_counter()
    cnt = 0
    for gi in pick:
        a, e = int(wl.offsets[gi]), int(wl.offsets[gi + 1])
        oracle.solve(wl.pos[:, a:e], wl.mass[a:e], wl.h0[a:e], box=(0, 0, 0), periodic=False,
                     nngb=float(wl.nngb[gi]), tol=float(wl.tol[gi]))
        cnt += e - a
    dt = time.perf_counter() - t0
    return {"value": cnt / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{len(pick)} random groups ({cnt:,} particles) solved one after another "
                      f"(FP64, bucket grids; a group's particles go to the threads in chunks of 16, "
                      f"so a small group keeps few of them busy); {dt:.1f} s wall",
            "seconds": dt, "particles": cnt}


def run_reference_batch(args):
    """Reference arm of the c4 batch: the oracle over a random sample of whole groups."""
    from paper_1612_06090_gb300 import inputs

    wl = inputs.make("c4")
    n, G = wl.n, wl.n_groups
    desc = (f"c4: {G:,} open Plummer groups (a=1, truncated at 20a), sizes dN/dN ~ N^-2 on [32, 200000], "
            f"{n:,} particles in total, Nngb=32+-1, M4 kernel")
    k = args.cpu_sample or 2000
    for _ in range(args.warmup):
        cpu_baseline_batch(wl, max(8, k // 8))
    runs = [cpu_baseline_batch(wl, k) for _ in range(args.steps)]
    per_step = statistics.mean(r["seconds"] for r in runs)
    value = runs[-1]["particles"] / per_step
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "n": n, "groups": G, "sample_groups": min(k, G)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": runs[-1]["cores"], "kind": "oracle",
                         "sample": runs[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_replay(args):
    """Reference arm of the c5 replay: each step solves sampled targets of snapshot 1,
    warm-started from their own snapshot-0 solution (solved first, untimed), by brute force
    over all particles.  The per-step sample is sized so that all steps stay within minutes."""
    import numpy as np

    import oracle
    from paper_1612_06090_gb300 import inputs

    kw = {"n": args.n} if args.n else {}
    series = inputs.clumpy_snapshot_series(2, **kw)
    wl0 = next(series)
    wl1 = next(series)
    n = wl0.n
    desc = (f"c5: {n:,} particles, 4096 Plummer clumps (a log-uniform in [1e-3,1e-2], 70%) + background, "
            f"periodic unit box, Nngb=64+-2, M4 kernel; 8 snapshots drifting N(0,1e-4^2), each replayed "
            f"warm-started from the previous snapshot's h")
    # a warm solve of one target costs a few brute-force scans of all particles (about a second
    # each) and the oracle hands targets to its threads in chunks of 16: two targets per step,
    # the same two every step, keep the whole run near a minute and a half on one thread
    k = min(args.cpu_sample or 2, n)
    tg = np.sort(np.random.default_rng(96).choice(n, size=k, replace=False))
    cold = oracle.solve(wl0.pos, wl0.mass, wl0.h0[tg], nngb=wl0.nngb, tol=wl0.tol, targets=tg, mode="brute")

    def warm(j):
        t0 = time.perf_counter()
        r = oracle.solve(wl1.pos, wl1.mass, cold["h"], nngb=wl1.nngb, tol=wl1.tol, targets=tg, mode="brute")
        return time.perf_counter() - t0, r

    for j in range(args.warmup):
        warm(j)
    times = []
    for j in range(args.steps):
        dt, r = warm(args.warmup + j)
        times.append(dt)
    per_step = statistics.mean(times)
    value = k / per_step
    sample = (f"{k} random targets of snapshot 1 (the same every step), warm-started from their own "
              f"snapshot-0 solution (solved first, untimed), each solved by brute force against all "
              f"{n:,} particles (FP64, OpenMP over targets in chunks of 16); {per_step:.2f} s per step")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "n": n, "sample_targets_per_step": k},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(oracle.threads(), -(-k // 16)),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference(args):
    rank, world = dist_init(args)
    if rank != 0:
        return
    if not args.knn and args.config in ("c4", "c5"):
        line = run_reference_batch(args) if args.config == "c4" else run_reference_replay(args)
        line["n_gpus"] = world
        print(json.dumps(line), flush=True)
        return
    wl, desc = workload(args)
    if args.knn:
        n_t = args.cpu_sample or 1024
        for _ in range(args.warmup):
            cpu_baseline_knn(wl, max(64, n_t // 8), args.knn, args.kernel)
        times, last = [], None
        for _ in range(args.steps):
            last = cpu_baseline_knn(wl, n_t, args.knn, args.kernel)
            times.append(last["seconds"])
        value = min(n_t, wl.n) / statistics.mean(times)
        line = {
            "impl": "reference", "metric": KNN_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "n": wl.n, "k": args.knn, "sample_targets": min(n_t, wl.n)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    n_t = args.cpu_sample or max(1024, wl.n // 16)
    for _ in range(args.warmup):
        cpu_baseline(wl, max(256, n_t // 8), args.kernel)
    times = []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(wl, n_t, args.kernel)
        times.append(last["seconds"])
    per_step = statistics.mean(times)
    value = min(n_t, wl.n) / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "n": wl.n, "sample_targets": min(n_t, wl.n)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- the CUDA path ------------------------------------------------------------------------

def run_native(args):
    import numpy as np
    import torch

    from paper_1612_06090_gb300 import binding as B

    rank, world = dist_init(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl, desc = workload(args)
    n = wl.n
    stream = torch.cuda.current_stream()

    pos = torch.as_tensor(wl.pos, device=dev)
    mass = torch.as_tensor(wl.mass, device=dev)
    h0 = torch.as_tensor(wl.h0, device=dev)
    h = torch.empty_like(h0)
    rho = torch.empty_like(h0)
    nw = torch.empty_like(h0)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def make(prec):
        s = B.Solver(n, stream=stream, precision=prec, box=wl.box, nngb=wl.nngb, tol=wl.tol,
                     kernel=B.SPH_KERNEL_WENDLAND_C6 if args.kernel == "c6" else B.SPH_KERNEL_M4)
        s.n = n  # sorted through the raw ABI below
        return s

    def step(s, stats_out=None):
        h.copy_(h0)
        st = s._check(B.sph_sort(s.ctx, n, pos.data_ptr(), mass.data_ptr()))
        stats = B.SphStats()
        st = B.sph_density_solve(s.ctx, h.data_ptr(), rho.data_ptr(), cnt.data_ptr(), nw.data_ptr(), stats)
        if st != B.SPH_OK:
            raise B.SphError(st, B.sph_last_error(s.ctx))
        if stats_out is not None:
            stats_out.append(stats.to_dict())

    def timed(s, steps, warmup):
        for _ in range(warmup):
            step(s)
        torch.cuda.synchronize()
        stats = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()  # evict L2 between steps (outside the per-step events)
            ev[k][0].record(stream)
            step(s, stats)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - w0
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, stats, wall

    # ---- FP32 + compensated: the headline ----
    s32 = make(B.SPH_PREC_FP32_KAHAN)
    s32._check(B.sph_sort(s32.ctx, n, pos.data_ptr(), mass.data_ptr()))
    # one-time per (GPU, size, precision); outside the timed region
    tuning = s32.tuning() if args.no_autotune else s32.autotune(h0)
    with ClockSampler(local) as clk:
        ms32, st32, wall32 = timed(s32, args.steps, args.warmup)
    clocks = clk.summary()
    ms_step = statistics.mean(ms32)
    t_max = max_over_ranks(ms_step, world)
    value = world * n / (t_max / 1e3)

    # roofline of the density kernel from its own events (library-recorded on this stream)
    dens_ms = sum(s["density_ms"] for s in st32)
    dens_launch = sum(s["density_launches"] for s in st32)
    pairs = sum(s["pair_evals"] for s in st32)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak_tflops, probe = probe_fp32_peak(stream.cuda_stream)
    achieved = pairs * FLOP_PER_PAIR / (dens_ms / 1e3) / 1e12 if dens_ms > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_density<2> (FP32 pair loop)", "achieved": achieved,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": None,
            "traffic_note": "no ncu capture of this configuration is kept; the default c5 replay line carries one",
            "peak_note": "measured: dependent-FMA probe (libsph_probe.so), timed alone with CUDA events",
            "peak_probe": probe,
            "flop_per_pair": FLOP_PER_PAIR, "pairs_per_step": pairs // max(1, len(st32)),
            "density_ms_per_step": dens_ms / max(1, len(st32)),
            "density_launches_per_step": dens_launch / max(1, len(st32)),
            "density_share_of_step": dens_ms / max(1e-9, sum(ms32))}
    launches = sum(s["kernel_launches"] for s in st32)

    # ---- plain FP64 GPU solve at the same accuracy target ----
    fp64 = None
    if args.fp64_steps > 0:
        s64 = make(B.SPH_PREC_FP64)
        ms64, st64, _ = timed(s64, args.fp64_steps, 1)
        t64 = max_over_ranks(statistics.mean(ms64), world)
        fp64 = {"value": world * n / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64,
                "density_ms_per_step": sum(s["density_ms"] for s in st64) / len(st64)}
        # agreement of the two GPU precisions on this workload
        h.copy_(h0)
        s32_ref = s64.solve(h0)
        h64 = s32_ref["h"].cpu().numpy()
        s64.close()
        r32 = s32.solve(h0)
        h32 = r32["h"].cpu().numpy()
        rho32 = r32["rho"].cpu().numpy()
        rho64 = s32_ref["rho"].cpu().numpy()
        same = np.abs(h32 - h64) <= 1e-5 * h64
        fp64["fp32_vs_fp64"] = {
            "same_trajectory_frac": float(same.mean()),
            "max_rel_rho_err_same_trajectory": float(np.max(np.abs(rho32[same] - rho64[same]) / rho64[same])),
            "max_rel_h_err": float(np.max(np.abs(h32 - h64) / h64)),
        }

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        hp = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in
              (("pos", pos), ("mass", mass), ("h0", h0))}
        hp["pos"].copy_(torch.as_tensor(wl.pos))
        hp["mass"].copy_(torch.as_tensor(wl.mass))
        hp["h0"].copy_(torch.as_tensor(wl.h0))
        outp = {"h": torch.empty(n, dtype=torch.float64).pin_memory(),
                "rho": torch.empty(n, dtype=torch.float64).pin_memory(),
                "count": torch.empty(n, dtype=torch.int32).pin_memory()}
        dpos, dmass, dh = torch.empty_like(pos), torch.empty_like(mass), torch.empty_like(h0)

        def e2e_step():
            dpos.copy_(hp["pos"], non_blocking=True)
            dmass.copy_(hp["mass"], non_blocking=True)
            dh.copy_(hp["h0"], non_blocking=True)
            s32._check(B.sph_sort(s32.ctx, n, dpos.data_ptr(), dmass.data_ptr()))
            st = B.sph_density_solve(s32.ctx, dh.data_ptr(), rho.data_ptr(), cnt.data_ptr(), 0, None)
            if st != B.SPH_OK:
                raise B.SphError(st, B.sph_last_error(s32.ctx))
            outp["h"].copy_(dh, non_blocking=True)
            outp["rho"].copy_(rho, non_blocking=True)
            outp["count"].copy_(cnt, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        for _ in range(args.warmup):
            e2e_step()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier(world)
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": world * n / te, "unit": UNIT, "ms_per_step": te * 1e3,
               "h2d_bytes_per_step": n * (24 + 8 + 8), "d2h_bytes_per_step": n * (8 + 8 + 4)}

    cpu = None
    if rank == 0 and world >= 1 and not args.no_cpu and world == 1:
        cpu = cpu_baseline(wl, args.cpu_sample or max(2048, n // 8), args.kernel)
        cpu.pop("seconds", None)
        cpu.pop("passes", None)

    s32.close()
    if rank == 0:
        st0 = st32[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n": n, "precision": "FP32 pairs + Kahan sums, FP64 h update",
                       "l2": "flushed between steps (256 MiB write, outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "passes": st0["passes"], "todo_per_pass": st0["todo_per_pass"],
                       "sort_ms": st0["sort_ms"], "solve_ms": st0["solve_ms"], "tuning": tuning,
                       "pairs_per_pass": st0["pairs_per_pass"], "pair_tests": st0["pair_tests"],
                       "density_ms_per_pass": [round(v, 3) for v in st0["density_ms_per_pass"]],
                       "wall_s_timed_region": wall32},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_gpu": fp64,
            "gpu_launches": launches, "clocks": clocks,
            "paper_context": "paper speed-ups optimised vs original CPU code: 2.6x IVB, 13.7x KNC, 19.1x KNL",
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_knn(args):
    """k-nearest-neighbour smoothing lengths (Sec. IV-D): one step = sort + sph_knn_solve on
    the workload, h = distance to the K-th nearest particle and rho at that h."""
    import numpy as np
    import torch

    from paper_1612_06090_gb300 import binding as B

    rank, world = dist_init(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl, desc = workload(args)
    n, K = wl.n, args.knn
    kern = B.SPH_KERNEL_WENDLAND_C6 if args.kernel == "c6" else B.SPH_KERNEL_M4
    stream = torch.cuda.current_stream()
    pos = torch.as_tensor(wl.pos, device=dev)
    mass = torch.as_tensor(wl.mass, device=dev)
    # starting search radius 0: the library estimates one per particle from the cell table
    h0_np = np.zeros(n)
    h0 = torch.as_tensor(h0_np, device=dev)
    h = torch.empty_like(h0)
    rho = torch.empty_like(h0)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def make(prec):
        s = B.Solver(n, stream=stream, precision=prec, box=wl.box, nngb=max(wl.nngb, 64.0), tol=wl.tol,
                     kernel=kern)
        s.n = n
        return s

    def step(s, stats_out=None):
        h.copy_(h0)
        s._check(B.sph_sort(s.ctx, n, pos.data_ptr(), mass.data_ptr()))
        stats = B.SphStats()
        st = B.sph_knn_solve(s.ctx, K, h.data_ptr(), rho.data_ptr(), cnt.data_ptr(), 0, stats)
        if st != B.SPH_OK:
            raise B.SphError(st, B.sph_last_error(s.ctx))
        if stats_out is not None:
            stats_out.append(stats.to_dict())

    def timed(s, steps, warmup):
        for _ in range(warmup):
            step(s)
        torch.cuda.synchronize()
        stats = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            step(s, stats)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return [a.elapsed_time(b) for a, b in ev], stats, time.perf_counter() - w0

    s32 = make(B.SPH_PREC_FP32_KAHAN)
    with ClockSampler(local) as clk:
        ms32, st32, wall32 = timed(s32, args.steps, args.warmup)
    clocks = clk.summary()
    t_max = max_over_ranks(statistics.mean(ms32), world)
    value = world * n / (t_max / 1e3)

    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak_tflops, probe = probe_fp32_peak(stream.cuda_stream)
    knn_ms = sum(s_["density_ms"] for s_ in st32)
    listed = sum(s_["pair_evals"] for s_ in st32)
    achieved = listed * FLOP_PER_LIST_ENTRY / (knn_ms / 1e3) / 1e12 if knn_ms > 0 else 0.0
    roof = {"bound": "alu", "kernel": "k_knn<FP32> (neighbour lists + warp radix select)",
            "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": None,
            "peak_note": "measured: dependent-FMA probe (libsph_probe.so), timed alone with CUDA events",
            "peak_probe": probe,
            "flop_per_list_entry": FLOP_PER_LIST_ENTRY,
            "list_entries_per_step": listed // max(1, len(st32)),
            "candidates_streamed_per_step": sum(s_["pair_tests"] for s_ in st32) // max(1, len(st32)),
            "knn_ms_per_step": knn_ms / max(1, len(st32)),
            "knn_share_of_step": knn_ms / max(1e-9, sum(ms32))}
    launches = sum(s_["kernel_launches"] for s_ in st32)

    fp64 = None
    if args.fp64_steps > 0:
        s64 = make(B.SPH_PREC_FP64)
        ms64, st64, _ = timed(s64, args.fp64_steps, 1)
        t64 = max_over_ranks(statistics.mean(ms64), world)
        r64 = s64.knn(K, h0)
        r32 = s32.knn(K, h0)
        h64, h32 = r64["h"].cpu().numpy(), r32["h"].cpu().numpy()
        rho64, rho32 = r64["rho"].cpu().numpy(), r32["rho"].cpu().numpy()
        fp64 = {"value": world * n / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64,
                "fp32_vs_fp64": {"max_rel_h_err": float(np.max(np.abs(h32 - h64) / h64)),
                                 "max_rel_rho_err": float(np.max(np.abs(rho32 - rho64) / rho64))}}
        s64.close()

    e2e = None
    if not args.no_e2e:
        hp = {"pos": torch.as_tensor(wl.pos).pin_memory(), "mass": torch.as_tensor(wl.mass).pin_memory(),
              "h0": torch.as_tensor(h0_np).pin_memory()}
        outp = {"h": torch.empty(n, dtype=torch.float64).pin_memory(),
                "rho": torch.empty(n, dtype=torch.float64).pin_memory(),
                "count": torch.empty(n, dtype=torch.int32).pin_memory()}
        dpos, dmass, dh = torch.empty_like(pos), torch.empty_like(mass), torch.empty_like(h0)

        def e2e_step():
            dpos.copy_(hp["pos"], non_blocking=True)
            dmass.copy_(hp["mass"], non_blocking=True)
            dh.copy_(hp["h0"], non_blocking=True)
            s32._check(B.sph_sort(s32.ctx, n, dpos.data_ptr(), dmass.data_ptr()))
            st = B.sph_knn_solve(s32.ctx, K, dh.data_ptr(), rho.data_ptr(), cnt.data_ptr(), 0, None)
            if st != B.SPH_OK:
                raise B.SphError(st, B.sph_last_error(s32.ctx))
            outp["h"].copy_(dh, non_blocking=True)
            outp["rho"].copy_(rho, non_blocking=True)
            outp["count"].copy_(cnt, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        for _ in range(args.warmup):
            e2e_step()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier(world)
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": world * n / te, "unit": UNIT, "ms_per_step": te * 1e3,
               "h2d_bytes_per_step": n * (24 + 8 + 8), "d2h_bytes_per_step": n * (8 + 8 + 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_knn(wl, args.cpu_sample or 2048, K, args.kernel)
        cpu.pop("seconds", None)
    s32.close()
    if rank == 0:
        st0 = st32[-1]
        line = {
            "metric": KNN_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n": n, "k": K,
                       "precision": "FP32 squared distances and radix select, FP32+Kahan density at h",
                       "start": "search radii estimated from the cell table (h_in = 0)",
                       "l2": "flushed between steps (256 MiB write, outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "selection_passes": st0["passes"], "todo_per_pass": st0["todo_per_pass"],
                       "sort_ms": st0["sort_ms"], "solve_ms": st0["solve_ms"],
                       "list_entries_per_pass": st0["pairs_per_pass"],
                       "knn_ms_per_pass": [round(v, 3) for v in st0["density_ms_per_pass"]],
                       "wall_s_timed_region": wall32},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_gpu": fp64,
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_interact(args):
    """The interaction pass: one step = sph_interact over every particle of the workload at its
    converged h (solved once, untimed): velocity records, work items and the interaction kernel
    (velocity mean, dispersion, divergence and curl over the neighbours of Eq. 1)."""
    import numpy as np
    import torch

    from paper_1612_06090_gb300 import binding as B
    from paper_1612_06090_gb300 import inputs

    rank, world = dist_init(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl, desc = workload(args)
    n = wl.n
    kern = B.SPH_KERNEL_WENDLAND_C6 if args.kernel == "c6" else B.SPH_KERNEL_M4
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    vel_np = inputs.velocities(wl.pos, inputs.CONFIG_SEEDS[args.config] + 100)
    gen_s = time.perf_counter() - t_gen
    pos = torch.as_tensor(wl.pos, device=dev)
    mass = torch.as_tensor(wl.mass, device=dev)
    vel = torch.as_tensor(vel_np, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    out = {"rho": torch.empty(n, dtype=torch.float64, device=dev),
           "vmean": torch.empty((3, n), dtype=torch.float64, device=dev),
           "sigma2": torch.empty(n, dtype=torch.float64, device=dev),
           "div": torch.empty(n, dtype=torch.float64, device=dev),
           "curl": torch.empty((3, n), dtype=torch.float64, device=dev),
           "count": torch.empty(n, dtype=torch.int32, device=dev)}

    def make(prec):
        s = B.Solver(n, stream=stream, precision=prec, box=wl.box, nngb=wl.nngb, tol=wl.tol, kernel=kern,
                     use_graph=True)
        s.sort(pos, mass)
        return s

    s32 = make(B.SPH_PREC_FP32_KAHAN)
    r = s32.solve(torch.as_tensor(wl.h0, device=dev))
    if r["status"] != B.SPH_OK:
        raise B.SphError(r["status"], "the untimed solve did not converge")
    h = r["h"]

    def step(s, hh, vv, stats_out=None):
        stats = B.SphStats()
        st = B.sph_interact(s.ctx, hh.data_ptr(), vv.data_ptr(), out["rho"].data_ptr(), out["vmean"].data_ptr(),
                            out["sigma2"].data_ptr(), out["div"].data_ptr(), out["curl"].data_ptr(),
                            out["count"].data_ptr(), stats)
        if st != B.SPH_OK:
            raise B.SphError(st, B.sph_last_error(s.ctx))
        if stats_out is not None:
            stats_out.append(stats.to_dict())

    def timed(s, steps, warmup):
        for _ in range(warmup):
            step(s, h, vel)
        torch.cuda.synchronize()
        stats = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            step(s, h, vel, stats)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return [a.elapsed_time(b) for a, b in ev], stats, time.perf_counter() - w0

    with ClockSampler(local) as clk:
        ms32, st32, wall32 = timed(s32, args.steps, args.warmup)
    clocks = clk.summary()
    t_max = max_over_ranks(statistics.mean(ms32), world)
    value = world * n / (t_max / 1e3)
    res32 = {k: v.cpu().numpy() for k, v in out.items()}

    peak_tflops, probe = probe_fp32_peak(stream.cuda_stream)
    k_ms = sum(s_["density_ms"] for s_ in st32) / max(1, len(st32))
    pairs = sum(s_["pair_evals"] for s_ in st32) // max(1, len(st32))
    achieved = pairs * FLOP_PER_INTERACT_PAIR / (k_ms / 1e3) / 1e12 if k_ms > 0 else 0.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_gbs = BYTES_PER_INTERACT_PARTICLE * n / (t_max / 1e3) / 1e9
    prof = profiled_interact_traffic()
    roof = {"bound": "alu", "kernel": "k_interact<FP32> (item set-up + staging + pair sums)",
            "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": prof["kernel_dram_bytes_per_launch"] * n / prof["capture_particles"] if prof else None,
            "traffic_note": "DRAM bytes of one interaction kernel launch: ncu on the 8,388,608-particle set "
                            "(profiles/interact_c5_8M.md), scaled by particle count",
            "peak_note": "measured: dependent-FMA probe (libsph_probe.so), timed alone with CUDA events",
            "peak_probe": probe, "flop_per_pair": FLOP_PER_INTERACT_PAIR, "pairs_per_step": pairs,
            "candidate_tests_per_step": sum(s_["pair_tests"] for s_ in st32) // max(1, len(st32)),
            "kernel_ms_per_step": k_ms, "kernel_timing": "CUDA events around work-item set-up and the "
            "interaction kernel inside each call", "kernel_share_of_step": k_ms / max(1e-9, t_max),
            "hbm_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak, "hbm_frac": hbm_gbs / hbm_peak,
            "hbm_note": f"algorithmic bytes {BYTES_PER_INTERACT_PARTICLE} B per particle over the step time; "
                        "peak = measured copy bandwidth (MEASURED_PEAKS.json)"}
    launches = sum(s_["kernel_launches"] for s_ in st32)

    fp64 = None
    if args.fp64_steps > 0:
        s64 = make(B.SPH_PREC_FP64)
        ms64, _, _ = timed(s64, args.fp64_steps, 1)
        t64 = max_over_ranks(statistics.mean(ms64), world)
        res64 = {k: v.cpu().numpy() for k, v in out.items()}
        sc = np.sqrt(np.maximum(res64["sigma2"], 0.0)) + 1e-300
        fp64 = {"value": world * n / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64,
                "fp32_vs_fp64": {"max_rel_rho_err": float(np.max(np.abs(res32["rho"] / res64["rho"] - 1.0))),
                                 "count_equal_frac": float(np.mean(res32["count"] == res64["count"])),
                                 "median_rel_sigma2_err": float(np.median(np.abs(res32["sigma2"] - res64["sigma2"])
                                                                          / (sc * sc))),
                                 "median_abs_vmean_err_over_sigma": float(np.median(
                                     np.max(np.abs(res32["vmean"] - res64["vmean"]), axis=0) / sc))}}
        s64.close()

    # ---- end to end: every step uploads h and the velocities from pinned host memory and
    # downloads the nine outputs and the count; the copies run on their own streams, a step's
    # upload during the previous step's pass and its download during the next (double-buffered)
    e2e = None
    if not args.no_e2e:
        hp = {"h": h.cpu().pin_memory(), "vel": torch.as_tensor(vel_np).pin_memory()}
        hout = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()} for _ in range(2)]
        din = [{"h": torch.empty_like(h), "vel": torch.empty_like(vel)} for _ in range(2)]
        dout = [{k: torch.empty_like(v) for k, v in out.items()} for _ in range(2)]
        up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        ev_host = [torch.cuda.Event() for _ in range(2)]
        for e in ev_out + ev_host:
            e.record(stream)

        def upload(g):
            b = g % 2
            with torch.cuda.stream(up):
                up.wait_event(ev_out[b])
                din[b]["h"].copy_(hp["h"], non_blocking=True)
                din[b]["vel"].copy_(hp["vel"], non_blocking=True)
                ev_in[b].record(up)

        def e2e_step(g):
            b = g % 2
            upload(g + 1)
            stream.wait_event(ev_in[b])
            stream.wait_event(ev_host[b])
            o = dout[b]
            st = B.sph_interact(s32.ctx, din[b]["h"].data_ptr(), din[b]["vel"].data_ptr(), o["rho"].data_ptr(),
                                o["vmean"].data_ptr(), o["sigma2"].data_ptr(), o["div"].data_ptr(),
                                o["curl"].data_ptr(), o["count"].data_ptr(), None)
            if st != B.SPH_OK:
                raise B.SphError(st, B.sph_last_error(s32.ctx))
            ev_out[b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev_out[b])
                for k in o:
                    hout[b][k].copy_(o[k], non_blocking=True)
                ev_host[b].record(down)

        upload(0)
        for g in range(args.warmup):
            e2e_step(g)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            e2e_step(args.warmup + k)
        torch.cuda.synchronize()
        barrier(world)
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": world * n / te, "unit": UNIT, "ms_per_step": te * 1e3,
               "h2d_bytes_per_step": n * (8 + 24), "d2h_bytes_per_step": n * (9 * 8 + 4),
               "path": "pinned host h and velocities -> sph_interact on the sorted positions -> rho, vmean, "
                       "sigma2, div, curl, count back to pinned host memory; the copies run on their own "
                       "streams, a step's upload during the previous step's pass and its download during the "
                       "next; wall clock around the timed steps, which hold as many uploads and downloads as "
                       "steps"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_interact(wl, vel_np, h.cpu().numpy(), args.cpu_sample or 32)
        cpu.pop("seconds", None)
    s32.close()
    if rank == 0:
        st0 = st32[-1]
        line = {
            "metric": INTERACT_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc + "; velocities: smooth periodic flow (6 Fourier modes, rms 1) + "
                       "N(0, 0.3^2) per component", "n": n,
                       "precision": "FP32 offsets, velocities and pair terms, Kahan sums, FP64 outputs",
                       "h": "converged h of an untimed FP32 solve of the same workload",
                       "l2": "inputs (positions, velocities) larger than L2, and L2 flushed between steps "
                             "(256 MiB write, outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "velocity_generation_s": gen_s, "solve_ms": st0["solve_ms"],
                       "wall_s_timed_region": wall32},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_gpu": fp64,
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def roofline_from(stats_list, peak, kernel):
    """Density-stage roofline from solve statistics against the measured FP32 FMA rate."""
    dens_ms = sum(s["density_ms"] for s in stats_list)
    pairs = sum(s["pair_evals"] for s in stats_list)
    ach = pairs * FLOP_PER_PAIR / (dens_ms / 1e3) / 1e12 if dens_ms > 0 else 0.0
    return {"bound": "alu", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None, "flop_per_pair": FLOP_PER_PAIR,
            "pairs_per_step": pairs // max(1, len(stats_list)),
            "density_ms_per_step": dens_ms / max(1, len(stats_list))}


def run_batch(args):
    """Config c4: 20,000 independent open Plummer groups in one batched solve (a CUDA graph
    runs the pass loop; every kernel covers all groups) against one solve per group."""
    import numpy as np
    import torch

    from paper_1612_06090_gb300 import binding as B
    from paper_1612_06090_gb300 import inputs

    rank, world = dist_init(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = inputs.make("c4")
    n, G = wl.n, wl.n_groups
    desc = (f"c4: {G:,} open Plummer groups (a=1, truncated at 20a), sizes dN/dN ~ N^-2 on [32, 200000], "
            f"{n:,} particles in total, Nngb=32+-1, M4 kernel")
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    off, pos, mass, h0 = T(wl.offsets, torch.int64), T(wl.pos), T(wl.mass), T(wl.h0)
    nngb, tol = T(wl.nngb), T(wl.tol)
    s = B.Solver(n, precision=B.SPH_PREC_FP32_KAHAN, use_graph=True)
    # a finer grouping once the todo list is sparse suits the batch's long tail of scattered halo
    # targets (measured 47.3 -> 43.8 ms of density per solve); sph_autotune needs one sorted set,
    # so the batch takes it by hand
    s.set_tuning(sparse_shift=2)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        r = s.batch_solve(off, pos, mass, h0, nngb, tol)
    torch.cuda.synchronize()
    barrier(world)
    ms, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = s.batch_solve(off, pos, mass, h0, nngb, tol)
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
            stats.append(r["stats"])
    barrier(world)
    t = max_over_ranks(statistics.mean(ms), world)
    value = world * n / (t / 1e3)
    # the same groups solved one call per group, on a random subset (each group copied to its
    # own contiguous arrays beforehand; the copies are not timed)
    rng = np.random.default_rng(7)
    subset = np.sort(rng.choice(G, size=min(G, 300), replace=False))
    loop_particles, loop_time = 0, 0.0
    one = B.Solver(int(np.diff(wl.offsets).max()), precision=B.SPH_PREC_FP32_KAHAN, use_graph=False)
    one.set_tuning(sparse_shift=2)
    for gi in subset:
        a, e = int(wl.offsets[gi]), int(wl.offsets[gi + 1])
        args_g = (T([0, e - a], torch.int64), T(wl.pos[:, a:e]), T(wl.mass[a:e]), T(wl.h0[a:e]),
                  T(wl.nngb[gi:gi + 1]), T(wl.tol[gi:gi + 1]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one.batch_solve(*args_g)
        torch.cuda.synchronize()
        loop_time += time.perf_counter() - t0
        loop_particles += e - a
    # density roofline from one host-driven batched solve (per-pass kernel events)
    s2 = B.Solver(n, precision=B.SPH_PREC_FP32_KAHAN, use_graph=False)
    s2.set_tuning(sparse_shift=2)
    r2 = s2.batch_solve(off, pos, mass, h0, nngb, tol)
    fp32_peak, _ = probe_fp32_peak(torch.cuda.current_stream().cuda_stream)
    roof = roofline_from([r2["stats"]], fp32_peak, "k_density<2> (FP32 pair loop)")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        pick = np.sort(rng.choice(G, size=min(G, 400), replace=False))
        t0 = time.perf_counter()
        cnt = 0
        for gi in pick:
            a, e = int(wl.offsets[gi]), int(wl.offsets[gi + 1])
            oracle.solve(wl.pos[:, a:e], wl.mass[a:e], wl.h0[a:e], box=(0, 0, 0), periodic=False, nngb=32.0,
                         tol=1.0)
            cnt += e - a
        dt = time.perf_counter() - t0
        cpu = {"value": cnt / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"{len(pick)} random groups ({cnt:,} particles) solved one after another, "
                         f"{dt:.1f} s"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n": n, "groups": G, "mode": "batched, CUDA-graph pass loop",
                       "passes": stats[-1]["passes"], "l2": "flushed between steps"},
            "looped": {"value": loop_particles / loop_time, "unit": UNIT,
                       "sample": f"{len(subset)} random groups, one sph_batch_solve call each"},
            "roofline": roof, "cpu_baseline": cpu, "gpu_launches": sum(x["kernel_launches"] for x in stats),
            "clocks": clk.summary()}), flush=True)


def profiled_replay_traffic():
    """DRAM bytes of one c5 replay step from the committed ncu summary (measured on the 8M-particle
    replay and scaled by particle count), while the kernel sources are the ones it was captured
    from; else None."""
    import hashlib
    import re

    try:
        text = open(os.path.join(ROOT, "profiles", "replay_c5_launches.md")).read()
        src = b"".join(open(os.path.join(ROOT, "paper_1612_06090_gb300", "csrc", f), "rb").read()
                       for f in ("sph_density.cu", "sph_items.cuh", "sph_common.cuh", "sph_solve.cu", "sph_sort.cu"))
        want = re.search(r"kernel_source_sha256_16: (\w+)", text).group(1)
        if hashlib.sha256(src).hexdigest()[:16] != want:
            return None
        get = lambda k: float(re.search(k + r": ([0-9.eE+]+)", text).group(1))  # noqa: E731
        return {"capture_particles": int(get("capture_particles")),
                "density_dram_bytes_per_step": get("density_dram_bytes_per_step"),
                "step_dram_bytes_per_step": get("step_dram_bytes_per_step")}
    except Exception:
        return None


def profiled_interact_traffic():
    """DRAM bytes of one interaction kernel launch from the committed ncu summary (measured on
    8.4M particles, to be scaled by particle count), while the kernel sources are the ones it was
    captured from; else None."""
    import hashlib
    import re

    try:
        text = open(os.path.join(ROOT, "profiles", "interact_c5_8M.md")).read()
        src = b"".join(open(os.path.join(ROOT, "paper_1612_06090_gb300", "csrc", f), "rb").read()
                       for f in ("sph_interact.cu", "sph_items.cuh", "sph_common.cuh"))
        if hashlib.sha256(src).hexdigest()[:16] != re.search(r"kernel_source_sha256_16: (\w+)", text).group(1):
            return None
        get = lambda k: float(re.search(k + r": ([0-9.eE+]+)", text).group(1))  # noqa: E731
        return {"capture_particles": int(get("capture_particles")),
                "kernel_dram_bytes_per_launch": get("kernel_dram_bytes_per_launch")}
    except Exception:
        return None


def probe_fp32_peak(stream_handle):
    """FP32 FMA rate of this GPU from the dependent-FMA probe (libsph_probe.so): the larger of
    the scalar and the two-wide FMA forms, each timed alone with CUDA events."""
    import ctypes

    from paper_1612_06090_gb300 import build as _build

    L = ctypes.CDLL(_build.PROBE_PATH)
    L.sph_probe_fp32_fma.restype = ctypes.c_int
    L.sph_probe_fp32_fma.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    best = {}
    for packed in (0, 1):
        tf, ms = ctypes.c_double(), ctypes.c_double()
        rc = L.sph_probe_fp32_fma(ctypes.c_void_p(stream_handle or None), 8, 1 << 15, packed,
                                  ctypes.byref(tf), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError(f"sph_probe_fp32_fma failed ({rc})")
        best["packed" if packed else "scalar"] = {"tflops": tf.value, "ms": ms.value}
    return max(v["tflops"] for v in best.values()), best


def hbm_algorithmic_bytes(n, todo_per_pass):
    """Compulsory HBM bytes of one sort + solve: 200 B per particle (sort, gather, scatter and
    solve set-up) plus 80 B per particle evaluated in each pass."""
    return BYTES_PER_PARTICLE * n + BYTES_PER_EVALUATION * sum(todo_per_pass)


def run_replay(args):
    """Config c5, the default: 67,108,864 particles in 4,096 Plummer clumps plus a background,
    8 snapshots drifting by N(0, 1e-4^2) per coordinate.  Snapshot 0 is solved cold (untimed);
    then every step replays the next snapshot s = 1..7 (cyclically, restarting from the
    snapshot-0 solution after snapshot 7): sph_sort of its positions and sph_density_solve
    warm-started from snapshot s-1's h, the pass loop running as a CUDA graph with its loop
    condition on the device."""
    import numpy as np
    import torch

    from paper_1612_06090_gb300 import binding as B
    from paper_1612_06090_gb300 import inputs

    rank, world = dist_init(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    kw = {"n": args.n} if args.n else {}
    n_snap = 8
    t_gen = time.perf_counter()
    pos_d, pos_h, host0 = [], [], {}
    for wl in inputs.clumpy_snapshot_series(n_snap, **kw):
        s_i = wl.meta["snapshot"]
        pos_d.append(torch.as_tensor(wl.pos, device=dev))
        if s_i <= 1:
            host0[s_i] = wl  # the CPU baseline solves sampled targets of snapshots 0 and 1
        if not args.no_e2e and s_i >= 1:
            pos_h.append(torch.as_tensor(wl.pos).pin_memory())
    gen_s = time.perf_counter() - t_gen
    wl0 = host0[0]
    n = wl0.n
    desc = (f"c5: {n:,} particles, 4096 Plummer clumps (a log-uniform in [1e-3,1e-2], 70%) + background, "
            f"periodic unit box, Nngb=64+-2, M4 kernel; 8 snapshots drifting N(0,1e-4^2), each replayed "
            f"warm-started from the previous snapshot's h")
    mass = torch.as_tensor(wl0.mass, device=dev)
    h0 = torch.as_tensor(wl0.h0, device=dev)
    h = torch.empty_like(h0)
    rho = torch.empty_like(h0)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def solver(prec, graph):
        s_ = B.Solver(n, stream=stream, precision=prec, box=wl0.box, nngb=wl0.nngb, tol=wl0.tol,
                      use_graph=graph)
        s_.n = n  # sorted through the raw ABI below
        return s_

    def step(slv, s_i, stats_out=None):
        slv._check(B.sph_sort(slv.ctx, n, pos_d[s_i].data_ptr(), mass.data_ptr()))
        st = B.SphStats()
        code = B.sph_density_solve(slv.ctx, h.data_ptr(), rho.data_ptr(), cnt.data_ptr(), 0, st)
        if code != B.SPH_OK:
            raise B.SphError(code, B.sph_last_error(slv.ctx))
        if stats_out is not None:
            stats_out.append(st.to_dict())

    # ---- snapshot 0, cold (untimed); its solution starts every pass through the cycle ----
    s32 = solver(B.SPH_PREC_FP32_KAHAN, True)
    h.copy_(h0)
    cold = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step(s32, 0, cold)
    torch.cuda.synchronize()
    cold_ms = (time.perf_counter() - t0) * 1e3
    h_snap0 = h.clone()
    # autotune on the first replay step (warm start), once per (GPU, size, precision)
    tuning = s32.tuning()
    if not args.no_autotune:
        s32._check(B.sph_sort(s32.ctx, n, pos_d[1].data_ptr(), mass.data_ptr()))
        tuning = s32.autotune(h_snap0)

    def snap_of(g):
        return 1 + g % (n_snap - 1)

    def timed(slv, steps, warmup, g0=0, nvtx_name="replay_timed"):
        """warmup + steps replay steps from global step index g0; CUDA events around each
        step's sort + solve, on the library's stream."""
        saved = {}
        for g in range(g0, g0 + warmup):
            if snap_of(g) == 1:
                h.copy_(h_snap0)
            step(slv, snap_of(g))
            if snap_of(g) == 1 and "h1" not in saved:
                saved["h1"], saved["rho1"] = h.clone(), rho.clone()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stats = []
        barrier(world)
        torch.cuda.synchronize()
        # an NVTX range names the timed steps for profilers (ncu --nvtx --nvtx-include)
        torch.cuda.nvtx.range_push(nvtx_name)
        w0 = time.perf_counter()
        for k in range(steps):
            g = g0 + warmup + k
            if snap_of(g) == 1:
                h.copy_(h_snap0)  # restart the cycle (outside the step events)
            flush.zero_()  # evict L2 between steps (outside the step events)
            ev[k][0].record(stream)
            step(slv, snap_of(g), stats)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - w0
        torch.cuda.nvtx.range_pop()
        if "h1" not in saved:
            # no warm-up step replayed snapshot 1: replay it once more, untimed, for the
            # FP32 / FP64 comparison
            h.copy_(h_snap0)
            step(slv, 1)
            saved["h1"], saved["rho1"] = h.clone(), rho.clone()
        return [a.elapsed_time(b) for a, b in ev], stats, wall, saved

    # ---- the headline: FP32 + compensated sums, graph pass loop ----
    with ClockSampler(local) as clk:
        ms32, st32, wall32, saved = timed(s32, args.steps, args.warmup)
    clocks = clk.summary()
    ms_step = statistics.mean(ms32)
    t_max = max_over_ranks(ms_step, world)
    value = world * n / (t_max / 1e3)
    launches = sum(x["kernel_launches"] for x in st32)

    # ---- the same replay with the host-driven pass loop: per-pass density-kernel events ----
    sh = solver(B.SPH_PREC_FP32_KAHAN, False)
    sh._check(B.sph_set_tuning(sh.ctx, B.SphTuning(**tuning)))
    msh, sth, _, _ = timed(sh, n_snap - 1, 1, g0=0, nvtx_name="replay_host_loop")
    sh.close()
    dens_ms = statistics.mean(x["density_ms"] for x in sth)
    pairs = statistics.mean(x["pair_evals"] for x in sth)
    sweeps = statistics.mean(x["pair_tests"] for x in sth)

    # ---- roofline: the density kernel (FP32 ALU) and the step's HBM rate ----
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp32_peak, probe = probe_fp32_peak(stream.cuda_stream)
    achieved = pairs * FLOP_PER_PAIR / (dens_ms / 1e3) / 1e12 if dens_ms > 0 else 0.0
    todo_mean = [statistics.mean(x["todo_per_pass"][k] if k < len(x["todo_per_pass"]) else 0 for x in st32)
                 for k in range(max(x["passes"] for x in st32))]
    alg_bytes = statistics.mean(hbm_algorithmic_bytes(n, x["todo_per_pass"]) for x in st32)
    hbm_gbs = alg_bytes / (t_max / 1e3) / 1e9
    prof = profiled_replay_traffic()
    scale = n / prof["capture_particles"] if prof else None
    roof = {"bound": "alu", "kernel": "k_density<2> (FP32 pair loop, all passes of a replay step)",
            "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
            "traffic": prof["density_dram_bytes_per_step"] * scale if prof else None,
            "traffic_note": ("DRAM bytes of the density kernel per replay step: ncu on the 8,388,608-particle "
                             "replay (profiles/replay_c5_launches.md), scaled by particle count"),
            "peak_note": "measured: dependent-FMA probe (libsph_probe.so, best of scalar and two-wide "
                         "FMA), timed alone with CUDA events in this run",
            "peak_probe": probe, "flop_per_pair": FLOP_PER_PAIR,
            "pairs_per_step": pairs, "candidate_tests_per_step": sweeps,
            "density_ms_per_step": dens_ms,
            "density_share_of_step": dens_ms / statistics.mean(msh),
            "density_timing": "CUDA events around each density launch in the host-loop replay of "
                              "the same 7 snapshots (identical kernels and work)",
            "hbm_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak, "hbm_frac": hbm_gbs / hbm_peak,
            "hbm_bytes_per_step": alg_bytes,
            "hbm_note": f"algorithmic bytes {BYTES_PER_PARTICLE} B per particle + {BYTES_PER_EVALUATION} B "
                        "per particle evaluation, over the graph-loop step time; peak = measured "
                        "copy bandwidth (MEASURED_PEAKS.json)",
            "hbm_ncu_bytes_per_step": prof["step_dram_bytes_per_step"] * scale if prof else None,
            "hbm_ncu_gbs": prof["step_dram_bytes_per_step"] * scale / (t_max / 1e3) / 1e9 if prof else None,
            "hbm_ncu_note": "DRAM bytes of every kernel of a replay step, ncu on the 8,388,608-particle replay "
                            "(per-kernel, serialised) scaled by particle count, over the graph-loop step time"}

    # ---- plain FP64 GPU solve of the first replay step, same start ----
    fp64 = None
    if args.fp64_steps > 0:
        s64 = solver(B.SPH_PREC_FP64, True)
        h.copy_(h_snap0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st64 = []
        e0.record(stream)
        step(s64, 1, st64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = max_over_ranks(e0.elapsed_time(e1), world)
        s64.close()
        h64, rho64 = h.cpu().numpy(), rho.cpu().numpy()
        h32, rho32 = saved["h1"].cpu().numpy(), saved["rho1"].cpu().numpy()
        same = np.abs(h32 - h64) <= 1e-5 * h64
        fp64 = {"value": world * n / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64, "steps": 1,
                "passes": st64[0]["passes"], "step": "snapshot 1 from the snapshot-0 solution (graph loop)",
                "fp32_vs_fp64": {
                    "same_trajectory_frac": float(same.mean()),
                    "max_rel_rho_err_same_trajectory": float(np.max(np.abs(rho32[same] - rho64[same]) / rho64[same])),
                    "max_rel_h_err": float(np.max(np.abs(h32 - h64) / h64))}}

    # ---- end to end through the C ABI: host buffers in, results back, copies timed ----
    # Every step copies its snapshot's positions and the masses from pinned host memory and its
    # h, rho and count back, inside the timed region.  The copies run on their own streams and
    # overlap the neighbouring steps' solves (double-buffered device inputs and outputs); the
    # warm-start h stays on the device from one step to the next, as a replaying caller keeps it.
    e2e = None
    if not args.no_e2e:
        hmass = torch.as_tensor(wl0.mass).pin_memory()
        hout = [{"h": torch.empty(n, dtype=torch.float64).pin_memory(),
                 "rho": torch.empty(n, dtype=torch.float64).pin_memory(),
                 "count": torch.empty(n, dtype=torch.int32).pin_memory()} for _ in range(2)]
        dpos = [torch.empty_like(pos_d[0]) for _ in range(2)]
        dmass = [torch.empty_like(mass) for _ in range(2)]
        dres = [{"h": torch.empty_like(h0), "rho": torch.empty_like(h0),
                 "count": torch.empty(n, dtype=torch.int32, device=dev)} for _ in range(2)]
        dh = torch.empty_like(h0)
        up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        ev_host = [torch.cuda.Event() for _ in range(2)]
        for e in ev_out + ev_host:
            e.record(stream)

        def upload(g):
            b = g % 2
            with torch.cuda.stream(up):
                up.wait_event(ev_out[b])  # the solve that last read these buffers is done
                dpos[b].copy_(pos_h[snap_of(g) - 1], non_blocking=True)
                dmass[b].copy_(hmass, non_blocking=True)
                ev_in[b].record(up)

        def e2e_step(g):
            b = g % 2
            upload(g + 1)  # the next step's inputs travel while this step solves
            stream.wait_event(ev_in[b])
            if snap_of(g) == 1:
                dh.copy_(h_snap0)  # the cycle restarts from the snapshot-0 solution
            s32._check(B.sph_sort(s32.ctx, n, dpos[b].data_ptr(), dmass[b].data_ptr()))
            stream.wait_event(ev_host[b])  # the results two steps back have reached the host
            code = B.sph_density_solve(s32.ctx, dh.data_ptr(), dres[b]["rho"].data_ptr(),
                                       dres[b]["count"].data_ptr(), 0, None)
            if code != B.SPH_OK:
                raise B.SphError(code, B.sph_last_error(s32.ctx))
            dres[b]["h"].copy_(dh)
            ev_out[b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev_out[b])
                for k in ("h", "rho", "count"):
                    hout[b][k].copy_(dres[b][k], non_blocking=True)
                ev_host[b].record(down)

        upload(0)
        for g in range(args.warmup):
            e2e_step(g)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            e2e_step(args.warmup + k)
        torch.cuda.synchronize()
        barrier(world)
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": world * n / te, "unit": UNIT, "ms_per_step": te * 1e3,
               "h2d_bytes_per_step": n * (24 + 8), "d2h_bytes_per_step": n * (8 + 8 + 4),
               "path": "pinned host positions and masses -> sph_sort + sph_density_solve (warm start from "
                       "the device-resident h) -> h, rho, count back to pinned host memory; the copies run on "
                       "their own streams, a step's upload during the previous step's solve and its download "
                       "during the next; wall clock around the timed steps, which hold as many uploads and "
                       "downloads as steps"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_replay(host0[0], host0[1], args.cpu_sample)
        cpu.pop("seconds", None)

    s32.close()
    if rank == 0:
        st0 = st32[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "n": n, "precision": "FP32 pairs + Kahan sums, FP64 h update",
                       "loop": "CUDA graph (conditional while node; the loop condition is set on the device)",
                       "l2": "inputs (1.6 GB of positions per snapshot) larger than L2, and L2 flushed "
                             "between steps (256 MiB write, outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "snapshots_per_cycle": n_snap - 1, "cold_snapshot0_ms": cold_ms,
                       "cold_passes": cold[0]["passes"], "input_generation_s": gen_s,
                       "replay_passes": [x["passes"] for x in st32], "todo_per_pass_mean": todo_mean,
                       "sort_ms": statistics.mean(x["sort_ms"] for x in st32), "tuning": tuning,
                       "ms_per_step_each": [round(v, 2) for v in ms32],
                       "host_loop_ms_per_step": statistics.mean(msh),
                       "host_loop_density_ms_per_pass": [round(v, 3) for v in sth[0]["density_ms_per_pass"]],
                       "host_loop_pairs_per_pass": sth[0]["pairs_per_pass"],
                       "wall_s_timed_region": wall32},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_gpu": fp64,
            "gpu_launches": launches, "clocks": clocks,
            "paper_context": "paper speed-ups optimised vs original CPU code: 2.6x IVB, 13.7x KNC, 19.1x KNL",
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.knn:
        run_knn(args)
    elif args.interact:
        run_interact(args)
    elif args.config == "c4":
        run_batch(args)
    elif args.config == "c5":
        run_replay(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
