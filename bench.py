#!/usr/bin/env python
"""Throughput benchmark of the BiCGStab 7-point path on GB300.

Workload (default): the nonsymmetric variable-coefficient 7-point system on a
600 x 595 x 1536 mesh (548,352,000 cells; the mesh of the paper's Sec. V run),
float32 storage and arithmetic, x0 = 0, iteration-bounded solves of 100
BiCGStab steps.  A benchmark *step* is one such solve: the start residual,
100 steps of three fused kernels, the float64 true residual and the copy of x
out.  Inputs are seeded synthetic data (SplitMix64, see ``synth``) and stay
resident in HBM; the ~31 GB working set is far larger than L2, so no L2
flush is needed between steps.

Prints one JSON line: ``value`` = cell-iterations/s over all ranks, with the
dominant kernel's roofline, per-kernel HBM rates, an end-to-end figure
through the C ABI with host buffers, the FP64 oracle timed on the host cores
(``cpu_baseline``) and the SM clocks seen during the timed region.

``--impl reference`` times the FP64 CPU oracle instead (rank 0 only), on a
bounded slab of the same workload per step.

Multi-GPU: the path does not shard; ``--gpus N`` under torchrun runs N
independent replicas (one system per GPU, weak scaling).
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-iters/s & HBM GB/s (BiCGStab 7-pt, 600×595×1536); p99 solve latency"
# Algorithmic HBM bytes per cell per launch of each step kernel:
# sweep 1: 6 coefficients + r, p_old, s_old, r0 read + p, s written
# sweep 2: 6 coefficients + r, s read + y written
# update : x, p, r, s, y, r0 read + x, r written


def bytes_per_cell(storage, variant=0):
    """Algorithmic HBM bytes per cell of each step kernel: w_c = w_v = storage
    size, w_x = 8 for float64 storage else 4 (12 w_c + 15 w_v + 2 w_x per step).
    Variant 1 (two passes): the q/y pass reads 6 coefficients + r, s, r0 and
    writes y; the fused pass reads 6 coefficients + r, s, y, p, r0, x and
    writes x, r, p, s (12 w_c + 12 w_v + 2 w_x per step)."""
    w = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[storage]
    wx = 8 if storage == "f64" else 4
    if variant == 1:
        k = {"spmv_p_dot": 6 * w + 8 * w + 2 * wx, "spmv_q_dots": 6 * w + 4 * w}
    else:
        k = {"spmv_p_dot": 6 * w + 6 * w, "spmv_q_dots": 6 * w + 3 * w,
             "update_dots": 5 * w + wx + w + wx}
    return k, sum(k.values())
def bytes_per_cell9(storage, variant=0):
    """The same for the 2D 9-point operator: 8 coefficients per sweep
    (16 w_c + 15 w_v + 2 w_x per step; variant 1: 16 w_c + 12 w_v + 2 w_x)."""
    w = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[storage]
    wx = 8 if storage == "f64" else 4
    if variant == 1:
        k = {"spmv_p_dot": 8 * w + 8 * w + 2 * wx, "spmv_q_dots": 8 * w + 4 * w}
    else:
        k = {"spmv_p_dot": 8 * w + 6 * w, "spmv_q_dots": 8 * w + 3 * w,
             "update_dots": 5 * w + wx + w + wx}
    return k, sum(k.values())


FLOPS_PER_CELL = 44          # Table I of the paper
FLOPS_PER_CELL_9PT = 52      # Table I's dots and AXPYs with two 16-flop 9-point matvecs
PAPER_CS1_CELL_ITERS = 548352000 / 28.1e-6   # Sec. V, CS-1, mixed 16/32-bit


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="solve",
                    choices=["solve", "solve9", "refined", "batched", "serve", "speedup",
                             "accuracy"],
                    help="solve: FP32 600x595x1536 (default); refined: 512^3 BF16/FP16 vs FP32 "
                         "storage with FP64 refinement; batched: 512 systems; serve: request stream")
    ap.add_argument("--edge", type=int, default=512, help="refined: cube edge")
    ap.add_argument("--edge2d", type=int, default=22800,
                    help="solve9: edge of the square 2D mesh (Sec. IV-A's largest: 22800)")
    ap.add_argument("--systems", type=int, default=512, help="batched: number of systems")
    ap.add_argument("--bthreads", type=int, default=0,
                    help="batched: threads per block (0 = autotuned)")
    ap.add_argument("--bzchunk", type=int, default=0, help="batched: z planes per block (0 = autotuned)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="batched: 0 chosen by the autotuner, 1 one persistent launch, -1 one "
                         "launch per kernel")
    ap.add_argument("--bfixed-variant", action="store_true",
                    help="batched: run the handles' variant (default: the autotuner may pick "
                         "the other one)")
    ap.add_argument("--requests", type=int, default=20000, help="serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=40.0, help="serve: arrivals per second")
    ap.add_argument("--serve-deadline", type=float, default=540.0,
                    help="serve: stop submitting after this many seconds")
    ap.add_argument("--serve-held-gb", type=float, default=60.0,
                    help="serve: most input bytes held for unfinished requests")
    ap.add_argument("--pool", type=int, default=48, help="speedup: requests solved both ways")
    ap.add_argument("--no-serve", action="store_true", help="default line without the stream")
    ap.add_argument("--no-speedup", action="store_true", help="default line without the speedup")
    ap.add_argument("--no-refined", action="store_true",
                    help="default line without the 512^3 refined solves")
    ap.add_argument("--no-batched", action="store_true",
                    help="default line without the 512-system batched solve")
    ap.add_argument("--cpu-all-nz", type=int, default=12,
                    help="z planes of each slab of the all-core oracle baseline")
    ap.add_argument("--serve-storage", default="bf16", choices=["bf16", "f16"],
                    help="speedup: storage of the served form")
    ap.add_argument("--serve-inner-tol", type=float, default=0.0,
                    help="speedup: inner tolerance of the served form (0 = server default)")
    ap.add_argument("--serve-three-pass", action="store_true",
                    help="speedup/serve: inner steps as Algorithm 1's three passes")
    ap.add_argument("--serve-steps-per-tick", type=int, default=0,
                    help="speedup: batched steps between the server's host checks (0 = default)")
    ap.add_argument("--nx", type=int, default=600)
    ap.add_argument("--ny", type=int, default=595)
    ap.add_argument("--nz", type=int, default=1536)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--variant", type=int, default=0,
                    help="0: Algorithm 1, three reductions per step; 1: two (merged passes)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-nz", type=int, default=24)
    ap.add_argument("--cpu-sample-iters", type=int, default=10)
    ap.add_argument("--bx", type=int, default=0, help="sweep tile width in threads (0 = tuned)")
    ap.add_argument("--by", type=int, default=0, help="sweep tile rows (0 = tuned)")
    ap.add_argument("--zchunk", type=int, default=0, help="z planes per block (0 = tuned)")
    ap.add_argument("--stages", type=int, default=0,
                    help="cp.async pipeline depth of the step sweeps (0 = tuned, 1 = none)")
    ap.add_argument("--step-cells", type=int, default=0,
                    help="cells per thread in the pipelined sweeps (0 = tuned; 8 for 16-bit)")
    ap.add_argument("--pipe-kinds", type=int, default=0,
                    help="sweeps using the pipeline: bit 0 p/s sweep, bit 1 q/y sweep (0 = tuned)")
    ap.add_argument("--tma", action="store_true",
                    help="pipelined sweeps stage with TMA tensor copies instead of cp.async")
    ap.add_argument("--residual-f64", action="store_true",
                    help="float64-accuracy residual sweeps in binary64 (default: double words)")
    ap.add_argument("--ref-sample-nz", type=int, default=8)
    ap.add_argument("--ref-sample-iters", type=int, default=5)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources that define the profiled step kernels (their device code and
# launch configuration); host-side drivers and tile defaults are not included
# the sources of the kernels profiles/traffic.json holds (the single-system step
# sweeps, the update and the true residual; the batched kernels are not among them)
KERNEL_SOURCES = ("s7_common.cuh", "s7_sweep.cuh", "s7_sweep9.cuh", "s7_step.cuh",
                  "s7_engine.cuh", "s7_resid.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2010_03660_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n_cells, table="kernels"):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to a launch over n_cells; None if absent or taken on other kernel code.
    `table`: "kernels" (3D 7-point) or "kernels_9pt" (2D 9-point)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    k = d.get(table, {}).get(kernel)
    if not k:
        return None
    return k["dram_bytes_per_launch"] * n_cells / k["cells"]


def combine_ranks(elapsed_ms, iters, pg, device):
    """Replicas: the job time is the slowest rank's, the work is every rank's
    (max of the times, sum of the iterations).  pg is torch.distributed or None."""
    if pg is None:
        return float(elapsed_ms), float(iters)
    import torch
    t = torch.tensor([float(elapsed_ms), float(iters)], dtype=torch.float64, device=device)
    tmax = t.clone()
    pg.all_reduce(tmax, op=pg.ReduceOp.MAX)
    tsum = t.clone()
    pg.all_reduce(tsum, op=pg.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "s7_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle
# ---------------------------------------------------------------------------

def oracle_sample(nx, ny, nz_sample, iters, seed=0, window=False):
    """The FP64 oracle on a slab of the same recipe; returns (cell-iters/s, desc,
    seconds) and, with `window`, also the wall-clock start and end of the solve."""
    import synth
    from oracle import bicgstab as ob
    p = synth.varcoef(nx, ny, nz_sample, seed=seed)
    w0 = time.time()
    t0 = time.perf_counter()
    r = ob.bicgstab(nx, ny, nz_sample, p.coef, p.b, tol=0.0, maxit=iters, storage="f32")
    dt = time.perf_counter() - t0
    w1 = time.time()
    desc = ("%dx%dx%d slab of the same coefficient recipe (seed %d), FP64 NumPy oracle "
            "(Algorithm 1), %d iterations incl. Jacobi scaling" % (nx, ny, nz_sample, seed,
                                                                 r.iters))
    if window:
        return p.n * r.iters, desc, dt, w0, w1
    return p.n * r.iters / dt, desc, dt


def _oracle_job(a):
    """One oracle solve in a worker process (spawned: no CUDA state)."""
    nx, ny, nz, iters, seed = a
    return oracle_sample(nx, ny, nz, iters, seed, window=True)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def oracle_baseline(nx, ny, nz_sample, iters, procs):
    """The FP64 oracle, as it stands, on `procs` host cores: one independent
    slab solve per worker process (seeds 0..procs-1), each process limited
    to one thread (BLAS included), started with spawn.  Returns cell-iters/s
    over the common wall-clock window (first start to last end) and the
    sample description."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    jobs = [(nx, ny, nz_sample, iters, seed) for seed in range(procs)]
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_job, jobs)
    work = sum(r[0] for r in res)
    t0 = min(r[3] for r in res)
    t1 = max(r[4] for r in res)
    desc = ("%d independent %dx%dx%d slabs of the same coefficient recipe (seeds 0..%d), "
            "FP64 NumPy oracle (Algorithm 1), %d iterations each, one process per core, "
            "one thread per process" % (procs, nx, ny, nz_sample, procs - 1, iters))
    return work / (t1 - t0), desc, t1 - t0


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    # each step is the oracle on a bounded slab of the workload; value is the
    # median of its cell-iters/s and ms_per_step the measured time of one
    # such sampled step (not the full-size step it stands for)
    vals, secs = [], []
    desc = ""
    for s in range(args.warmup + args.steps):
        v, desc, dt = oracle_sample(args.nx, args.ny, min(args.ref_sample_nz, args.nz),
                                    min(args.ref_sample_iters, args.iters))
        if s >= args.warmup:
            vals.append(v)
            secs.append(dt)
    value = statistics.median(vals)
    ms_per_step = statistics.median(secs) * 1e3
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-iters/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args),
        "cpu_baseline": {"value": value, "unit": "cell-iters/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "cell-iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "step_sample": desc,
    }
    print(json.dumps(out))


def config_of(args):
    return {"workload": "bicgstab_%s_%dx%dx%d_%dit%s" % (args.storage, args.nx, args.ny, args.nz,
                                                          args.iters,
                                                          "_merged" if args.variant else ""),
            "variant": "two reductions per step" if args.variant else "Algorithm 1",
            "nx": args.nx, "ny": args.ny, "nz": args.nz, "cells": args.nx * args.ny * args.nz,
            "iters_per_step": args.iters, "storage": args.storage,
            "coefficients": "per-cell off-diagonals -U[0.5,1.5], diag = sum|off| + U[0.01,0.1]",
            "rhs": "N(0,1)", "x0": "0", "stop": "iteration-bounded (tol 0)",
            "true_residual": "binary64" if args.residual_f64 else "double words (binary32 pairs)",
            "l2": "inputs larger than L2 (working set ~%d GB), no flush" %
                  round(args.nx * args.ny * args.nz * 60 / 1e9),
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import synth
    import paper_2010_03660_gb300 as s7

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    s7.lib()

    nx, ny, nz, iters = args.nx, args.ny, args.nz, args.iters
    n = nx * ny * nz
    raw = np.float64 if args.storage == "f64" else np.float32
    t0 = time.time()
    prob = synth.varcoef(nx, ny, nz, seed=rank, dtype=raw)
    gen_s = time.time() - t0
    coef_d = {k: torch.from_numpy(v).to(dev) for k, v in prob.coef.items()}
    op = s7.stencil7_create(nx, ny, nz, coef_d, storage=args.storage, bx=args.bx, by=args.by,
                            zchunk=args.zchunk, variant=args.variant, stages=args.stages,
                            pipe_kinds=args.pipe_kinds, step_cells=args.step_cells,
                            residual_f64=args.residual_f64, tma=args.tma)
    del coef_d
    torch.cuda.empty_cache()
    b = torch.from_numpy(prob.b).to(dev)
    x = torch.zeros(n, dtype=b.dtype, device=dev)

    def step():
        x.zero_()
        return s7.bicgstab_solve(op, b, x, tol=0.0, maxit=iters, history=True)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    s7.stencil7_profile(op, True)
    sampler = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    done_iters = 0
    for _ in range(args.steps):
        res = step()
        done_iters += res.iters
    ev1.record()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    prof = s7.stencil7_profile(op, False)
    elapsed_ms, total_iters = combine_ranks(ev0.elapsed_time(ev1), done_iters, pg, dev)
    value = n * total_iters / (elapsed_ms / 1e3)

    peak, peak_kind = measured_peaks()
    bpc, iter_bpc = bytes_per_cell(args.storage, args.variant)
    kern = {}
    for k, (ms, cnt) in prof.items():
        if cnt == 0:
            continue
        avg = ms / cnt
        e = {"launches": int(cnt), "avg_ms": avg, "share": None}
        if k in bpc:
            gbs = bpc[k] * n / (avg / 1e3) / 1e9
            e.update({"alg_bytes_per_launch": bpc[k] * n, "gbs": gbs,
                      "frac": gbs / peak})
        kern[k] = e
    tot_ms = sum(v["avg_ms"] * v["launches"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["avg_ms"] * v["launches"] / tot_ms if tot_ms else None
    dom = max((k for k in kern if k in bpc),
              key=lambda k: kern[k]["avg_ms"] * kern[k]["launches"])
    table = {"f32": "kernels", "bf16": "kernels_bf16"}.get(args.storage)
    traffic = (ncu_traffic(dom, n, table) if table and args.variant == 0 and not args.stages
               and not args.pipe_kinds and not args.step_cells else None)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak,
                "unit": "GB/s", "frac": kern[dom]["gbs"] / peak, "peak_kind": peak_kind,
                "traffic": traffic}
    iter_ms = elapsed_ms / (done_iters if done_iters else 1)
    hbm_gbs = iter_bpc * n * total_iters / (elapsed_ms / 1e3) / 1e9
    launches = int(sum(c for _, c in prof.values()))

    # end to end through the C ABI with pinned host buffers (rank-local)
    op.close()
    del b, x
    torch.cuda.empty_cache()
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, s7, prob, dev)

    extras = {}
    if rank == 0 and world == 1:
        del prob
        extras = run_extras(args)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            v, desc, _ = oracle_baseline(nx, ny, min(args.cpu_sample_nz, nz),
                                         args.cpu_sample_iters, 1)
            cpu = {"value": v, "unit": "cell-iters/s", "cores": 1, "kind": "oracle",
                   "sample": desc, "cpu_model": cpu_model()}
            ncores = os.cpu_count() or 1
            v, desc, _ = oracle_baseline(nx, ny, min(args.cpu_all_nz, nz), args.cpu_sample_iters,
                                         ncores)
            cpu_all = {"value": v, "unit": "cell-iters/s", "cores": ncores, "kind": "oracle",
                       "sample": desc, "cpu_model": cpu_model()}
        except Exception as e:          # reported, the GPU line stands
            cpu = cpu or {"error": repr(e)}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "cell-iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
            "data": "synthetic (seeded SplitMix64 variable-coefficient 7-point system)",
            "config": config_of(args),
            "hbm_gbs": hbm_gbs, "hbm_frac": hbm_gbs / peak / world,
            "gflops": FLOPS_PER_CELL * value / 1e9,
            "ms_per_iter": iter_ms,
            "roofline": roofline, "kernels": kern,
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks,
            "context": {"paper_cs1_cell_iters_per_s": PAPER_CS1_CELL_ITERS,
                        "final_rel_resid": float(res.hist[-1]) if res.hist is not None else None,
                        "input_gen_s": gen_s},
        }
        out.update(extras)
        print(json.dumps(out))
    if pg:
        pg.destroy_process_group()


def run_extras(args):
    """The rest of the headline metric, measured after the main line in the
    same run: the served request stream (p50/p99 latency), the served
    mixed-precision form against the plain FP32 form to 1e-8, 512^3 refined
    solves with their solution error, and the 512-system batched solve.  A
    failure in one of them is reported in its object; the main line stands."""
    import torch
    out = {}
    blocks = []
    if not args.no_serve:
        blocks.append(("serve", lambda: serve_block(args)))
    if not args.no_speedup:
        blocks.append(("speedup", lambda: {s: speedup_block(args, s) for s in ("bf16", "f16")}))
    if not args.no_refined:
        blocks.append(("refined", lambda: refined_block(args)))
    if not args.no_batched:
        blocks.append(("batched", lambda: batched_block(args, systems=512, steps=3, variant=0,
                                                        schedule=0)))
    for name, fn in blocks:
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:
            out[name] = {"error": repr(e)}
        if isinstance(out[name], dict):
            out[name]["bench_s"] = time.perf_counter() - t0
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def kernel_table(prof, bpc, n, peak):
    """Per-kernel launches, average time, share and algorithmic GB/s."""
    kern = {}
    for k, (ms, cnt) in prof.items():
        if cnt == 0:
            continue
        avg = ms / cnt
        e = {"launches": int(cnt), "avg_ms": avg, "share": None}
        if k in bpc:
            gbs = bpc[k] * n / (avg / 1e3) / 1e9
            e.update({"alg_bytes_per_launch": bpc[k] * n, "gbs": gbs, "frac": gbs / peak})
        kern[k] = e
    tot_ms = sum(v["avg_ms"] * v["launches"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["avg_ms"] * v["launches"] / tot_ms if tot_ms else None
    return kern


def run_solve9(args):
    """BiCGStab on the 2D 9-point operator (Sec. IV-A) at its largest mesh,
    iteration-bounded like the 3D solve line."""
    import torch
    import synth
    import paper_2010_03660_gb300 as s7

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s7.lib()
    nx = ny = args.edge2d
    n = nx * ny
    iters = args.iters
    raw = np.float64 if args.storage == "f64" else np.float32
    prob = synth.varcoef9(nx, ny, seed=rank, dtype=raw)
    coef_d = {k: torch.from_numpy(v).to(dev) for k, v in prob.coef.items()}
    op = s7.stencil9_create(nx, ny, coef_d, storage=args.storage, bx=args.bx,
                            zchunk=args.zchunk, variant=args.variant)
    del coef_d
    torch.cuda.empty_cache()
    b = torch.from_numpy(prob.b).to(dev)
    x = torch.zeros(n, dtype=b.dtype, device=dev)
    del prob

    def step():
        x.zero_()
        return s7.bicgstab_solve(op, b, x, tol=0.0, maxit=iters, history=True)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    s7.stencil7_profile(op, True)
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    done = 0
    for _ in range(args.steps):
        res = step()
        done += res.iters
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = s7.stencil7_profile(op, False)
    op.close()
    elapsed_ms = ev0.elapsed_time(ev1)
    value = n * done / (elapsed_ms / 1e3)
    peak, peak_kind = measured_peaks()
    bpc, iter_bpc = bytes_per_cell9(args.storage, args.variant)
    kern = kernel_table(prof, bpc, n, peak)
    dom = max((k for k in kern if k in bpc), key=lambda k: kern[k]["avg_ms"] * kern[k]["launches"])
    hbm_gbs = iter_bpc * n * done / (elapsed_ms / 1e3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "cell-iters/s & HBM GB/s (BiCGStab 9-pt 2D, %dx%d)" % (nx, ny),
            "value": value, "unit": "cell-iters/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.storage,
            "data": "synthetic (seeded SplitMix64 variable-coefficient 9-point 2D system)",
            "config": {"workload": "bicgstab9_%s_%dx%d_%dit%s" % (args.storage, nx, ny, iters,
                                                                  "_merged" if args.variant else ""),
                       "cells": n, "iters_per_step": iters, "storage": args.storage,
                       "coefficients": "per-cell off-diagonals -U[0.5,1.5] (8 directions), "
                                       "diag = sum|off| + U[0.01,0.1]",
                       "stop": "iteration-bounded (tol 0)",
                       "l2": "inputs larger than L2 (working set ~%d GB), no flush"
                             % round(n * 68 / 1e9)},
            "hbm_gbs": hbm_gbs, "hbm_frac": hbm_gbs / peak,
            "gflops": FLOPS_PER_CELL_9PT * value / 1e9, "ms_per_iter": elapsed_ms / done,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"],
                         "peak": peak, "unit": "GB/s", "frac": kern[dom]["gbs"] / peak,
                         "peak_kind": peak_kind,
                         "traffic": ncu_traffic(dom, n, "kernels_9pt")
                         if (args.storage == "f32" and args.variant == 0) else None},
            "kernels": kern, "gpu_launches": int(sum(c for _, c in prof.values())),
            "clocks": clocks,
            "context": {"final_rel_resid": float(res.hist[-1])}}))


def run_e2e(args, s7, prob, dev):
    import torch
    n = prob.n
    pin = {k: torch.from_numpy(v).pin_memory() for k, v in prob.coef.items()}
    bh = torch.from_numpy(prob.b).pin_memory()
    xh = torch.zeros(n, dtype=bh.dtype).pin_memory()
    times = []
    iters = 0
    for s in range(1 + args.e2e_steps):
        xh.zero_()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        op = s7.stencil7_create(prob.nx, prob.ny, prob.nz, pin, storage=args.storage,
                                residual_f64=args.residual_f64)
        r = s7.bicgstab_solve(op, bh, xh, tol=0.0, maxit=args.iters, history=True)
        op.close()
        ev1.record()
        torch.cuda.synchronize()
        if s >= 1:
            times.append(ev0.elapsed_time(ev1))
            iters = r.iters
    es = bh.element_size()
    h2d = 7 * n * pin["diag"].element_size() + 2 * n * es
    d2h = n * es + (iters + 1) * 8
    ms = statistics.median(times)
    return {"value": n * iters / (ms / 1e3), "unit": "cell-iters/s", "ms_per_step": ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "includes": "stencil7_create from pinned host coefficients + bicgstab_solve with "
                        "pinned host b/x (%d iterations) + destroy" % args.iters}


# ---------------------------------------------------------------------------
# other workloads (not the default line)
# ---------------------------------------------------------------------------

def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    outs = []
    ev0.record()
    for _ in range(steps):
        outs.append(fn())
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps, outs


def batched_block(args, systems=None, steps=None, variant=None, schedule=None):
    """512 systems, cube edges log-uniform in [16,128] (seed 1), per-system
    coefficients of the variable-coefficient recipe, FP32, tol 1e-6: one
    batched solve (block shape and fusion schedule chosen by the library's
    autotuner on the untimed first solve), timed over `steps`
    repetitions, against the same systems solved one after another.
    Systems are generated on the device (the host generator's coefficients,
    bit for bit)."""
    import torch
    import synth
    from synth import device as sd
    import paper_2010_03660_gb300 as s7
    systems = args.systems if systems is None else systems
    steps = max(1, args.steps if steps is None else steps)
    variant = args.variant if variant is None else variant
    schedule = args.schedule if schedule is None else schedule
    dev = torch.device("cuda", torch.cuda.current_device())
    edges = synth.batched_edges(systems, seed=1)
    ops, bs = [], []
    for j, e in enumerate(edges):
        coef, b = sd.varcoef(e, e, e, synth.system_seed(1, j), dev, b_dtype="f32")
        torch.cuda.synchronize()   # the library reads the inputs on its own stream
        ops.append(s7.stencil7_create(e, e, e, coef, storage="f32", variant=variant))
        bs.append(b)
        del coef
    cells = [e ** 3 for e in edges]
    xs = [torch.zeros_like(b) for b in bs]

    def fn():
        for x in xs:
            x.zero_()
        return s7.bicgstab_solve_batched(ops, bs, xs, tol=1e-6, maxit=2000, schedule=schedule,
                                         threads=args.bthreads, zchunk=args.bzchunk,
                                         choose_variant=not args.bfixed_variant)
    ms, outs = _timed(fn, steps, 1)
    r = outs[-1]
    ci = sum(c * it for c, it in zip(cells, r.iters))
    # the same systems one after another through bicgstab_solve
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_ci = 0
    for op, b, x, c in zip(ops, bs, xs, cells):
        x.zero_()
        rs = s7.bicgstab_solve(op, b, x, tol=1e-6, maxit=2000, history=False, true_resid=False)
        seq_ci += c * rs.iters
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    pol = r.policy
    out = {"workload": "batched_%d_systems" % systems,
           "value": ci / (ms / 1e3), "unit": "cell-iters/s",
           "schedule": {1: "persistent", -1: "launch per kernel"}[pol["schedule"]]
           + (" (chosen by the autotuner)" if schedule == 0 else ""),
           "variant": "two reductions per step" if pol["variant"] else "Algorithm 1",
           "policy": dict(pol, variant_chosen_by_autotuner=not args.bfixed_variant,
                          handles_variant=variant),
           "dtype": "f32", "ms_per_batch_solve": ms, "systems": len(ops),
           "total_cells": int(sum(cells)), "iters_min_max": [min(r.iters), max(r.iters)],
           "all_converged": r.rc == 0, "hbm_gbs": 116 * ci / (ms / 1e3) / 1e9,
           "sequential_single_solves": {"s": seq_s, "cell_iters_per_s": seq_ci / seq_s},
           "speedup_vs_sequential": (seq_s * 1e3) / ms, "repetitions": steps}
    for op in ops:
        op.close()
    del bs, xs
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    import torch
    import paper_2010_03660_gb300 as s7
    s7.lib()
    torch.cuda.set_device(0)
    out = batched_block(args)
    out.update({"metric": "batched cell-iters/s (512 systems, edges 16..128, FP32, tol 1e-6)",
                "higher_is_better": True, "data": "synthetic (seed 1)"})
    print(json.dumps(out))


def _quantiles(v):
    v = np.asarray(v, dtype=np.float64)
    return {"min": float(v.min()), "median": float(np.median(v)), "max": float(v.max()),
            "iqr": float(np.percentile(v, 75) - np.percentile(v, 25))}


def serve_block(args, requests=None, rate=None, deadline_s=None, storage=None):
    """The served request stream: Poisson arrivals of solve requests, mesh
    edges log-uniform in [32,384] with aspect ratios log-uniform in [0.5,2],
    tolerances drawn from {1e-4,1e-6,1e-8}, BF16 storage + float64-accuracy
    refinement, 150 GB admission budget.  Every request is its own system
    (its own seed), generated on the device at its arrival time and submitted
    from device memory.  Latency = completion - submission (the server's host
    monotonic clock); p50/p99 over the requests after the warm-up ones.
    Submission stops at `deadline_s`; the requests submitted until then are
    all waited for and reported."""
    import threading
    import torch
    import synth
    from synth import device as sd
    import paper_2010_03660_gb300 as s7
    requests = args.requests if requests is None else requests
    rate = args.rate if rate is None else rate
    deadline_s = args.serve_deadline if deadline_s is None else deadline_s
    storage = args.serve_storage if storage is None else storage
    dev = torch.device("cuda", torch.cuda.current_device())
    reqs = synth.request_stream(requests, rate=rate, seed=3)
    srv = s7.Server(storage=storage, hbm_budget_bytes=150 << 30)
    ids = [None] * len(reqs)
    lag = [0.0] * len(reqs)
    state = {"submitted": 0, "done": False, "error": None, "inflight": 0, "held": 0}
    lock = threading.Lock()
    # inputs held for submitted, unfinished requests (7 float32 arrays, b and
    # x in float64): past the limit the producer waits for completions, so
    # an overloaded stream shows up as arrival lag instead of running the
    # device out of memory
    held_limit = int(args.serve_held_gb * 1e9)
    arr0 = reqs[0].arrival
    t_start = time.perf_counter()

    def producer():
        try:
            torch.cuda.set_device(dev)
            gs = torch.cuda.Stream(dev)
            with torch.cuda.stream(gs):
                for j, q in enumerate(reqs):
                    if time.perf_counter() - t_start > deadline_s:
                        break
                    delay = (q.arrival - arr0) - (time.perf_counter() - t_start)
                    if delay > 0:
                        time.sleep(delay)
                    need = 44 * q.nx * q.ny * q.nz
                    while state["inflight"] and state["inflight"] + need > held_limit:
                        time.sleep(0.001)
                    with lock:
                        state["inflight"] += need
                        state["held"] = max(state["held"], state["inflight"])
                    coef, b = sd.varcoef(q.nx, q.ny, q.nz, q.seed, dev)
                    x = torch.empty_like(b)
                    gs.synchronize()
                    lag[j] = time.perf_counter() - t_start - (q.arrival - arr0)
                    ids[j] = srv.submit(q.nx, q.ny, q.nz, coef, b, x, q.tol)
                    state["submitted"] = j + 1
        except Exception as e:      # reported in the output, the stream stops
            state["error"] = repr(e)
        finally:
            state["done"] = True

    th = threading.Thread(target=producer, daemon=True)
    th.start()
    lat, statuses, over, cells, tols = [], [], [], [], []
    for j in range(len(reqs)):
        while ids[j] is None and not (state["done"] and state["submitted"] <= j):
            time.sleep(0.0005)
        if ids[j] is None:
            break
        r = srv.wait(ids[j], timeout=900)
        q = reqs[j]
        lat.append(r["latency"])
        statuses.append(r["status"])
        over.append(r["resid"] / q.tol)
        cells.append(q.nx * q.ny * q.nz)
        tols.append(q.tol)
        srv.release(ids[j])
        with lock:
            state["inflight"] -= 44 * q.nx * q.ny * q.nz
    th.join()
    wall = time.perf_counter() - t_start
    st = srv.stats()
    srv.close()
    torch.cuda.empty_cache()
    n = len(lat)
    warm = min(500, n // 10)
    lw = np.array(lat[warm:]) if n > warm else np.array(lat)
    out = {"workload": "serve_%d_requests_at_%g_per_s" % (n, rate),
           "requests_in_stream": requests, "requests_run": n, "warmup_requests": warm,
           "rate_per_s": rate, "storage": storage, "budget_gb": 150 * 2 ** 30 / 1e9,
           "p50_s": float(np.percentile(lw, 50)), "p99_s": float(np.percentile(lw, 99)),
           "mean_s": float(lw.mean()), "max_s": float(lw.max()),
           "completed": int(st["completed"]), "failed": int(st["failed"]),
           "statuses_ok": int(sum(1 for s_ in statuses if s_ == 0)),
           "max_resid_over_tol": float(max(over)) if over else None,
           "wall_s": wall, "cell_iters_per_s": st["cell_iters"] / wall,
           "mean_cells": float(np.mean(cells)) if cells else 0.0,
           "mem_peak_gb": st["mem_peak"] / 1e9,
           "arrival_lag_p99_s": float(np.percentile(lag[:n], 99)) if n else None,
           "arrival_lag_max_s": float(np.max(lag[:n])) if n else None,
           "inputs_held_peak_gb": state["held"] / 1e9,
           "stopped_by_deadline": n < requests,
           "inputs": "each request its own seeded system (SplitMix64, seed 3 stream), generated "
                     "on the device at arrival and submitted from device memory",
           "latency": "completion - submission, host monotonic clock"}
    if state["error"]:
        out["error"] = state["error"]
    return out


def run_serve(args):
    import torch
    import paper_2010_03660_gb300 as s7
    s7.lib()
    torch.cuda.set_device(0)
    out = serve_block(args)
    out.update({"metric": "p99 solve latency (serving, %s + FP64 refinement)"
                % args.serve_storage.upper(), "value": out["p99_s"], "unit": "s",
                "higher_is_better": False, "data": "synthetic (seed 3)"})
    print(json.dumps(out))


def speedup_block(args, storage, requests=None, reps=None):
    """The same requests to relative residual 1e-8 two ways: one after another
    with FP32 storage + float64-accuracy refinement (the plain form, at the
    faster of two inner tolerances), and all at once through the server
    (`storage` + refinement, continuous batching).  Inputs are device-resident
    for both forms (generated on the device, each request its own seed);
    both include operator creation.  The plain and served forms alternate
    `reps` times; the ratio is of the medians, with every sample reported."""
    import torch
    import synth
    from synth import device as sd
    import paper_2010_03660_gb300 as s7
    requests = args.pool if requests is None else requests
    reps = max(5, args.steps if reps is None else reps)
    dev = torch.device("cuda", torch.cuda.current_device())
    reqs = synth.request_stream(requests, rate=1.0, seed=3)
    pool = []
    for q in reqs:
        coef, b = sd.varcoef(q.nx, q.ny, q.nz, q.seed, dev)
        pool.append((q.nx, q.ny, q.nz, coef, b))
    torch.cuda.synchronize()
    cells = sum(nx * ny * nz for nx, ny, nz, _, _ in pool)

    def plain(inner_tol):
        its = 0
        for nx, ny, nz, coef, b in pool:
            op = s7.stencil7_create(nx, ny, nz, coef, storage="f32", keep_true=True)
            x = torch.zeros_like(b)
            r = s7.bicgstab_solve_refined(op, b, x, tol=1e-8, max_outer=60, inner_maxit=400,
                                          inner_tol=inner_tol)
            its += r.inner_total
            op.close()
        torch.cuda.synchronize()
        return its

    def served():
        with s7.Server(storage=storage, hbm_budget_bytes=150 << 30,
                       inner_tol=args.serve_inner_tol, three_pass=args.serve_three_pass,
                       steps_per_tick=args.serve_steps_per_tick) as srv:
            xs = [torch.empty_like(b) for _, _, _, _, b in pool]
            ids = [srv.submit(nx, ny, nz, coef, b, x, 1e-8)
                   for (nx, ny, nz, coef, b), x in zip(pool, xs)]
            return [srv.wait(i, timeout=600) for i in ids]

    plain(1e-2)                   # warm-up (module loading, pool)
    served()
    t_inner = {}
    for inner_tol in (1e-2, 1e-5):
        t0 = time.perf_counter()
        its_k = plain(inner_tol)
        t_inner[inner_tol] = (time.perf_counter() - t0, its_k)
    best = min(t_inner, key=lambda k: t_inner[k][0])
    its = t_inner[best][1]
    tp, ts = [], []
    res = None
    for _ in range(reps):
        t0 = time.perf_counter()
        plain(best)
        tp.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        res = served()
        ts.append(time.perf_counter() - t0)
    ratios = [a / b for a, b in zip(tp, ts)]
    t_plain, t_served = statistics.median(tp), statistics.median(ts)
    value = t_plain / t_served
    lo = float(np.percentile(ratios, 25))
    return {"workload": "speedup_%d_requests_to_1e-8" % len(pool), "served_storage": storage,
            "value": value, "unit": "x", "requests": len(pool), "total_cells": cells,
            "plain_fp32_s": t_plain, "served_s": t_served,
            "plain_fp32_samples_s": tp, "served_samples_s": ts,
            "ratio_per_pair": ratios, "ratio_spread": _quantiles(ratios),
            "clears_1_5x_by_more_than_spread": bool(lo > 1.5 and min(ratios) > 1.5),
            "plain_fp32_inner_tol": best,
            "plain_fp32_s_by_inner_tol": {str(k): v[0] for k, v in t_inner.items()},
            "plain_inner_iters": its,
            "served_inner_iters": int(sum(r["inner_iters"] for r in res)),
            "served_all_ok": all(r["status"] == 0 for r in res),
            "served_max_resid": max(r["resid"] for r in res),
            "reps": reps, "inputs": "device-resident, each request its own seeded system"}


def run_speedup(args):
    import torch
    import paper_2010_03660_gb300 as s7
    s7.lib()
    torch.cuda.set_device(0)
    out = speedup_block(args, args.serve_storage)
    out.update({"metric": "speedup to relative residual 1e-8: served %s + FP64 refinement vs "
                          "sequential FP32 + FP64 refinement" % args.serve_storage.upper(),
                "higher_is_better": True, "data": "synthetic (seed 3)"})
    print(json.dumps(out))


def refined_block(args, edge=None, storages=("bf16", "f16"), reps=3):
    """512^3 (seed 2) refined to relative residual 1e-10 with 16-bit storage:
    the time of the solve on b ~ N(0,1) (median of `reps`), its steps and
    certified float64-accuracy residual, and the solution error against the
    exact solution of a manufactured system: x* ~ N(0,1) (seeded), b* = A x*
    computed by the FP64 oracle on the host from the same raw float32
    coefficients, so x* solves A x = b* to float64 rounding."""
    import torch
    import synth
    from synth import device as sd
    import paper_2010_03660_gb300 as s7
    from oracle import stencil
    e = args.edge if edge is None else edge
    n = e ** 3
    dev = torch.device("cuda", torch.cuda.current_device())
    coef, b = sd.varcoef(e, e, e, 2, dev)
    torch.cuda.synchronize()       # the library reads the inputs on its own stream
    # the manufactured system, on the host, by the oracle
    t0 = time.perf_counter()
    ph = synth.varcoef(e, e, e, seed=2)
    xs = synth.random_vector(n, 2, 9, np.float64)
    bs = stencil.apply(e, e, e, ph.coef, xs)
    del ph
    oracle_s = time.perf_counter() - t0
    bs_d = torch.from_numpy(bs).to(dev)
    del bs
    out = {"workload": "refined_%d^3_to_1e-10" % e, "cells": n,
           "error_reference": "x* ~ N(0,1) seeded, b* = A x* by the FP64 oracle on the host "
                              "(raw float32 coefficients, float64 arithmetic)",
           "oracle_host_s": oracle_s, "runs": {}}
    for storage in storages:
        op = s7.stencil7_create(e, e, e, coef, storage=storage, keep_true=True)
        times, r = [], None
        for k in range(reps + 1):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            r = s7.bicgstab_solve_refined(op, b, x, tol=1e-10, max_outer=60, inner_maxit=200,
                                          inner_tol=1e-2)
            torch.cuda.synchronize()
            if k:
                times.append(time.perf_counter() - t1)
        rn, bn = s7.stencil7_residual(op, b, r.x)
        xm = torch.zeros_like(bs_d)
        rm = s7.bicgstab_solve_refined(op, bs_d, xm, tol=1e-10, max_outer=60, inner_maxit=200,
                                       inner_tol=1e-2)
        xsd = torch.from_numpy(xs).to(dev)
        err = float(torch.linalg.norm(rm.x - xsd) / torch.linalg.norm(xsd))
        err_inf = float((rm.x - xsd).abs().max() / xsd.abs().max())
        del xsd
        out["runs"][storage] = {
            "s": statistics.median(times), "samples_s": times, "status": r.status,
            "outer": r.outer, "inner_iters": r.inner_total, "true_resid": rn / bn,
            "manufactured": {"status": rm.status, "outer": rm.outer,
                             "inner_iters": rm.inner_total, "resid": float(rm.hist[-1]),
                             "rel_error_2norm": err, "rel_error_max": err_inf}}
        op.close()
    del coef, b, bs_d
    torch.cuda.empty_cache()
    return out


def run_refined(args):
    """512^3, seed 2: refined solves to 1e-8 and 1e-10 with BF16, FP16 and FP32
    storage (FP32 arithmetic, FP64 outer residual on the true operator)."""
    import torch
    import synth
    import paper_2010_03660_gb300 as s7
    from oracle import stencil
    s7.lib()
    e = args.edge
    p = synth.varcoef(e, e, e, seed=2)
    dev = torch.device("cuda:0")
    b = torch.from_numpy(p.b.astype(np.float64)).to(dev)
    coef = {k: torch.from_numpy(v).to(dev) for k, v in p.coef.items()}
    runs = {}
    rng = np.random.default_rng(0)
    idx = rng.integers(0, p.n, 2000)
    for storage, inner_tol in (("bf16", 1e-2), ("f16", 1e-2), ("f16", 1e-3), ("f32", 1e-5),
                               ("f32", 1e-2)):
        op = s7.stencil7_create(e, e, e, coef, storage=storage, keep_true=True,
                                variant=args.variant, residual_f64=args.residual_f64)
        for tol in (1e-8, 1e-10):
            def fn():
                return s7.bicgstab_solve_refined(op, b, tol=tol, max_outer=80, inner_maxit=200,
                                                 inner_tol=inner_tol)
            ms, outs = _timed(fn, args.steps, min(args.warmup, 2))
            r = outs[-1]
            rr = torch.empty_like(b)
            rn, bn = s7.stencil7_residual(op, b, r.x, rr)
            # the certified residual, verified on sampled rows by the oracle
            cf, _ = synth.varcoef_at(e, e, e, idx, seed=2)
            xg = r.x
            def x_at(j):
                return xg[torch.from_numpy(np.asarray(j)).to(dev)].cpu().numpy()
            ax, mag = stencil.apply_at(e, e, e, cf, x_at, idx)
            ref = p.b.astype(np.float64)[idx] - ax
            got = rr[torch.from_numpy(idx).to(dev)].cpu().numpy()
            row_err = float(np.max(np.abs(got - ref) / (mag + np.abs(p.b[idx]))))
            runs["%s_in%g_tol%g" % (storage, inner_tol, tol)] = {
                "ms": ms, "outer": r.outer, "inner_iters": r.inner_total, "status": r.status,
                "true_resid": rn / bn, "oracle_row_check": row_err, "inner_tol": inner_tol,
                "inner_cell_iters_per_s": p.n * r.inner_total / (ms / 1e3)}
        op.close()
    base = min(runs["f32_in1e-05_tol1e-08"]["ms"], runs["f32_in0.01_tol1e-08"]["ms"])
    out = {"metric": "time to relative residual 1e-10, mixed precision (BF16 storage) + FP64 refinement",
           "value": runs["bf16_in0.01_tol1e-10"]["ms"] / 1e3, "unit": "s", "higher_is_better": False,
           "workload": "refined_%d^3%s" % (e, "_merged" if args.variant else ""),
           "dtype": "bf16/f16/f32 storage, f32 arithmetic, f64 outer",
           "data": "synthetic (seed 2)", "runs": runs,
           "speedup_vs_best_fp32_storage_to_1e-8": {
               k: base / runs["%s_tol1e-08" % k]["ms"] for k in ("bf16_in0.01", "f16_in0.01",
                                                                 "f16_in0.001")},
           "manufactured_solution_error": refined_block(args, edge=e)["runs"],
           "steps": args.steps}
    print(json.dumps(out))


def run_accuracy(args):
    """Residual histories of plain BiCGStab (no refinement) with FP32, BF16 and
    FP16 storage on a 100 x 400 x 100 synthetic system (the mesh of the
    paper's mixed-precision experiment, Sec. VI-B), and of the refined solve."""
    import torch
    import synth
    import paper_2010_03660_gb300 as s7
    s7.lib()
    from oracle import bicgstab as ob
    nx, ny, nz = 100, 400, 100
    p = synth.varcoef(nx, ny, nz, seed=4)
    dev = torch.device("cuda:0")
    coef = {k: torch.from_numpy(v).to(dev) for k, v in p.coef.items()}
    b = torch.from_numpy(p.b).to(dev)
    # the FP64 oracle's solution of the true (float32-coefficient) system
    t0 = time.perf_counter()
    orc_ref = ob.bicgstab(nx, ny, nz, p.coef, p.b.astype(np.float64), tol=1e-13, maxit=5000,
                          storage="f64")
    oracle_s = time.perf_counter() - t0
    x_ref = orc_ref.x
    nref = np.linalg.norm(x_ref)

    def err(x):
        x = x.double().cpu().numpy()
        return {"rel_error_2norm": float(np.linalg.norm(x - x_ref) / nref),
                "rel_error_max": float(np.max(np.abs(x - x_ref)) / np.max(np.abs(x_ref)))}
    curves = {}
    for storage in ("f32", "bf16", "f16"):
        with s7.stencil7_create(nx, ny, nz, coef, storage=storage, keep_true=True) as op:
            r = s7.bicgstab_solve(op, b, tol=1e-12, maxit=60)
            rn, bn = s7.stencil7_residual(op, b, r.x)
            curves[storage] = {"hist": [float(v) for v in r.hist], "status": r.status,
                               "min_recurrence": float(min(r.hist)),
                               "true_resid_raw": rn / bn, "error_vs_oracle": err(r.x)}
            rr = s7.bicgstab_solve_refined(op, b.double(), tol=1e-10, max_outer=40,
                                           inner_maxit=100, inner_tol=1e-2)
            curves[storage]["refined_outer_hist"] = [float(v) for v in rr.hist]
            curves[storage]["refined_error_vs_oracle"] = err(rr.x)
    ref = np.array(curves["f32"]["hist"])
    for k in ("bf16", "f16"):
        h = np.array(curves[k]["hist"])
        m = min(len(h), len(ref))
        dev_ = np.abs(h[:m] - ref[:m]) / ref[:m]
        curves[k]["tracks_fp32_until"] = int(np.argmax(dev_ > 0.1)) if np.any(dev_ > 0.1) else m
    out = {"metric": "mixed-precision accuracy: residual histories, 100x400x100",
           "value": curves["bf16"]["true_resid_raw"], "unit": "relative residual (bf16, plain)",
           "higher_is_better": False, "workload": "accuracy_100x400x100",
           "data": "synthetic (seed 4)", "curves": curves,
           "error_reference": "FP64 oracle (Algorithm 1) on the true float32-coefficient "
                              "system to relative residual 1e-13 (%d steps, %.0f s on the host)"
                              % (orc_ref.iters, oracle_s)}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "solve9":
        run_solve9(args)
    elif args.workload == "refined":
        run_refined(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "speedup":
        run_speedup(args)
    elif args.workload == "accuracy":
        run_accuracy(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
