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
# algorithmic HBM bytes per cell per launch of each kernel (float32 storage):
# sweep 1: 6 coefficients + r, p_old, s_old, r0 read + p, s written
# sweep 2: 6 coefficients + r, s read + y written
# update : x, p, r, s, y, r0 read + x, r written
BYTES_PER_CELL = {"spmv_p_dot": 48, "spmv_q_dots": 36, "update_dots": 32}
ITER_BYTES_PER_CELL = 116
FLOPS_PER_CELL = 44          # Table I of the paper
PAPER_CS1_CELL_ITERS = 548352000 / 28.1e-6   # Sec. V, CS-1, mixed 16/32-bit


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=600)
    ap.add_argument("--ny", type=int, default=595)
    ap.add_argument("--nz", type=int, default=1536)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-nz", type=int, default=24)
    ap.add_argument("--cpu-sample-iters", type=int, default=10)
    ap.add_argument("--bx", type=int, default=0, help="sweep tile width in threads (0 = tuned)")
    ap.add_argument("--by", type=int, default=0, help="sweep tile rows (0 = tuned)")
    ap.add_argument("--zchunk", type=int, default=0, help="z planes per block (0 = tuned)")
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


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2010_03660_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n_cells):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to a launch over n_cells; None if absent or taken on other kernel code."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k:
        return None
    return k["dram_bytes_per_launch"] * n_cells / k["cells"]


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

def oracle_sample(nx, ny, nz_sample, iters, seed=0):
    """The FP64 oracle on a slab of the same recipe; returns (cell-iters/s, desc)."""
    import synth
    from oracle import bicgstab as ob
    p = synth.varcoef(nx, ny, nz_sample, seed=seed)
    t0 = time.perf_counter()
    r = ob.bicgstab(nx, ny, nz_sample, p.coef, p.b, tol=0.0, maxit=iters, storage="f32")
    dt = time.perf_counter() - t0
    desc = ("%dx%dx%d slab of the same coefficient recipe (seed %d), FP64 NumPy oracle "
            "(Algorithm 1), %d iterations incl. Jacobi scaling" % (nx, ny, nz_sample, seed,
                                                                 r.iters))
    return p.n * r.iters / dt, desc, dt


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    vals = []
    desc = ""
    for s in range(args.warmup + args.steps):
        v, desc, _ = oracle_sample(args.nx, args.ny, min(args.ref_sample_nz, args.nz),
                                   min(args.ref_sample_iters, args.iters))
        if s >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    n = args.nx * args.ny * args.nz
    ms_per_step = n * args.iters / value * 1e3
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
    }
    print(json.dumps(out))


def config_of(args):
    return {"workload": "bicgstab_%s_%dx%dx%d_%dit" % (args.storage, args.nx, args.ny, args.nz,
                                                        args.iters),
            "nx": args.nx, "ny": args.ny, "nz": args.nz, "cells": args.nx * args.ny * args.nz,
            "iters_per_step": args.iters, "storage": args.storage,
            "coefficients": "per-cell off-diagonals -U[0.5,1.5], diag = sum|off| + U[0.01,0.1]",
            "rhs": "N(0,1)", "x0": "0", "stop": "iteration-bounded (tol 0)",
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
                            zchunk=args.zchunk)
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
    elapsed_ms = ev0.elapsed_time(ev1)
    t = torch.tensor([elapsed_ms, float(done_iters)], dtype=torch.float64, device=dev)
    if pg:
        tmax = t.clone()
        pg.all_reduce(tmax, op=pg.ReduceOp.MAX)
        tsum = t.clone()
        pg.all_reduce(tsum, op=pg.ReduceOp.SUM)
        elapsed_ms = float(tmax[0])
        total_iters = float(tsum[1])
    else:
        total_iters = float(done_iters)
    value = n * total_iters / (elapsed_ms / 1e3)

    peak, peak_kind = measured_peaks()
    kern = {}
    for k, (ms, cnt) in prof.items():
        if cnt == 0:
            continue
        avg = ms / cnt
        e = {"launches": int(cnt), "avg_ms": avg, "share": None}
        if k in BYTES_PER_CELL:
            gbs = BYTES_PER_CELL[k] * n / (avg / 1e3) / 1e9
            e.update({"alg_bytes_per_launch": BYTES_PER_CELL[k] * n, "gbs": gbs,
                      "frac": gbs / peak})
        kern[k] = e
    tot_ms = sum(v["avg_ms"] * v["launches"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["avg_ms"] * v["launches"] / tot_ms if tot_ms else None
    dom = max((k for k in kern if k in BYTES_PER_CELL),
              key=lambda k: kern[k]["avg_ms"] * kern[k]["launches"])
    traffic = ncu_traffic(dom, n)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak,
                "unit": "GB/s", "frac": kern[dom]["gbs"] / peak, "peak_kind": peak_kind,
                "traffic": traffic}
    iter_ms = elapsed_ms / (done_iters if done_iters else 1)
    hbm_gbs = ITER_BYTES_PER_CELL * n * total_iters / (elapsed_ms / 1e3) / 1e9
    launches = int(sum(c for _, c in prof.values()))

    # end to end through the C ABI with pinned host buffers (rank-local)
    e2e = None
    if not args.no_e2e:
        op.close()
        del b, x
        torch.cuda.empty_cache()
        e2e = run_e2e(args, s7, prob, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, _ = oracle_sample(nx, ny, min(args.cpu_sample_nz, nz), args.cpu_sample_iters)
        cpu = {"value": v, "unit": "cell-iters/s", "cores": 1, "kind": "oracle", "sample": desc}

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
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
            "context": {"paper_cs1_cell_iters_per_s": PAPER_CS1_CELL_ITERS,
                        "final_rel_resid": float(res.hist[-1]) if res.hist is not None else None,
                        "input_gen_s": gen_s},
        }
        print(json.dumps(out))
    if pg:
        pg.destroy_process_group()


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
        op = s7.stencil7_create(prob.nx, prob.ny, prob.nz, pin, storage=args.storage)
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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
