#!/usr/bin/env python
"""Benchmark of the DVM source iteration (linearized BGK, arXiv:1704.03126 Sec. II.A) on GB300.

Workload: force-driven flow through the rough channel -- 128 x 128 cells, periodic along x1, diffuse
plates with one 26 x 32 block per wall, 32 x 32 trapezoid velocities on [-5, 5]^2 -- at Kn = 0.1, 1
and 10, the three instances advanced together.  One step = one source iteration of all three
(transport sweep with fused moments and wall fluxes, mass projection, residual, flow rate), i.e.
3 x 14720 gas cells x 1024 velocities = 45.2 M cell-velocity updates.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

KNS = (0.1, 1.0, 10.0)
METRIC = "DVM cell-velocity updates/s (rough channel 128x128, 32x32 velocities, Kn 0.1/1/10)"
UNIT = "updates/s"
# FP32 / FP64 operations per interior cell-velocity update of the sweep kernel:
# right-hand side 3 FMA, two upwind combinations 2 x (FMA + MUL), update 2 FMA + MUL, moments 4 FMA
FLOPS_PER_UPDATE = 25
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--skip-extras", action="store_true", help="only the timed steps (profiling runs)")
    ap.add_argument("--single", action="store_true", help="time only the selected precision")
    ap.add_argument("--min-warmup-s", type=float, default=1.0,
                    help="keep warming up for at least this long (clock sampling); 0 for profiling")
    return ap.parse_args()


def workload_config(precision):
    return {
        "workload": "rough channel 128x128 (blocks 26x32 on both walls, x1 periodic), 32x32 trapezoid "
                    "velocities |v|<=5, Kn 0.1/1/10 batched; force-driven (F=1)",
        "instances_per_step": len(KNS),
        "precision": "fp32 store / fp64 accumulate" if precision == "fp32" else "fp64",
        "l2": "flushed between timed steps (256 MiB write)",
        "data": "synthetic staircase geometry",
    }


def instances():
    from paper_1704_03126_gb300 import inputs
    return [inputs.rough_instance(kn) for kn in KNS]


def updates_per_step(insts):
    return sum(int((inst.mask == 0).sum()) * inst.quad[1] ** 2 for inst in insts)


# ------------------------------------------------------------------------------ clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1704_03126_gb300 import dvm

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    insts = instances()
    upd = updates_per_step(insts)

    def make(precision):
        return [dvm.Solver(inst.mask, True, False, kn=inst.kn, quad=inst.quad, precision=precision,
                           stream=stream.cuda_stream) for inst in insts]

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed_steps(batch, steps, warmup, sampler=None):
        t_end = time.perf_counter() + args.min_warmup_s
        w = 0
        while w < warmup or time.perf_counter() < t_end:  # at least `warmup` steps and ~1 s of load
            batch.iterate(1)
            w += 1
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        sweep_ms, fin_ms = [], []
        for k in range(steps):
            flush.zero_()  # evict L2 between timed steps (outside the events)
            ev0[k].record(stream)
            batch.iterate(1)
            ev1[k].record(stream)
            s_ms, f_ms = batch.timing()
            sweep_ms.append(s_ms)
            fin_ms.append(f_ms)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        total = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        return total, sweep_ms, fin_ms, w

    results = {}
    sampler = ClockSampler(local_rank)
    sampler.start()
    precisions = [args.precision] + ([] if args.single else ["fp64" if args.precision == "fp32" else "fp32"])
    for precision in precisions:
        solvers = make(precision)
        batch = dvm.Batch(solvers)
        total_ms, sweep_ms, fin_ms, wsteps = timed_steps(batch, args.steps, args.warmup)
        if world > 1:
            t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_ms = float(t.item())
        results[precision] = dict(total_ms=total_ms, sweep_ms=float(np.mean(sweep_ms)),
                                  fin_ms=float(np.mean(fin_ms)), warmup_steps=wsteps,
                                  kernels_per_step=batch.kernels_per_sweep(), batch=batch, solvers=solvers)
        if precision == args.precision:
            clocks = sampler.stop()
    main = results[args.precision]
    ms_per_step = main["total_ms"] / args.steps
    value = world * args.steps * upd / (main["total_ms"] / 1e3)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32: 152 SMs x 128 FMA lanes; FP64 on GB300: 2 FMA per SM per clock (measured 1.9); 2 flops per FMA
    peak = {"fp32": 152 * 128 * 2 * sm_max_mhz * 1e6 / 1e12, "fp64": 152 * 2 * 2 * sm_max_mhz * 1e6 / 1e12}

    def roofline(prec):
        r = results[prec]
        achieved = FLOPS_PER_UPDATE * upd / (r["sweep_ms"] / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak[prec], "unit": "TFLOP/s",
                "frac": achieved / peak[prec], "traffic": None,
                "kernel": f"sweep_kernel ({prec})", "flops_per_update": FLOPS_PER_UPDATE,
                "peak_note": ("FP32 FMA units x max SM clock" if prec == "fp32"
                              else "FP64 units (2 FMA/SM/clk) x max SM clock") + ", derived (of unit counts)",
                "sweep_ms": r["sweep_ms"], "finalize_ms": r["fin_ms"]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic", "config": workload_config(args.precision),
        "roofline": roofline(args.precision),
        "clocks": clocks,
        "gpu_launches": args.steps * (main["kernels_per_step"] + len(KNS)),
    }
    other = "fp64" if args.precision == "fp32" else "fp32"
    if other in results:
        out[other] = {"value": world * args.steps * upd / (results[other]["total_ms"] / 1e3),
                      "ms_per_step": results[other]["total_ms"] / args.steps, "roofline": roofline(other)}
    hbm = float(peaks.get("hbm_gbs", 6762.6)) * 1e9
    vals = {p: world * args.steps * upd / (results[p]["total_ms"] / 1e3) for p in results}
    out["effective_hbm_fraction"] = {
        "note": "updates/s x bytes a non-fused sweep would move (write + read h) / measured HBM copy bandwidth",
        **{p: vals[p] * (8 if p == "fp32" else 16) / hbm for p in vals},
    }

    if not args.skip_extras:
        out["e2e"] = e2e(args, insts, stream, dvm, torch)
        out["converge"] = converge(results, insts, torch)
    if rank == 0 and not args.skip_extras:
        out["cpu_baseline"] = cpu_baseline(insts)
    for r in results.values():
        r["batch"].close()
        for s in r["solvers"]:
            s.close()
    return out


def e2e(args, insts, stream, dvm, torch, sweeps=50, reps=3):
    """Public API with host buffers: create from the host mask (H2D), `sweeps` sweeps, flow rate and
    fields back to the host (D2H), destroy -- for every instance; wall clock."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(reps):
        for inst in insts:
            s = dvm.Solver(inst.mask, True, False, kn=inst.kn, quad=inst.quad, precision=args.precision,
                           stream=stream.cuda_stream)
            s.iterate(sweeps)
            q, _ = s.flowrate()
            f = s.fields()
            s.close()
            h2d += inst.mask.nbytes
            d2h += 8 + sum(a.nbytes for a in f.values())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    upd = updates_per_step(insts) * sweeps * reps
    return {"value": upd / dt, "unit": UNIT, "h2d_bytes_per_step": h2d // (reps * sweeps),
            "d2h_bytes_per_step": d2h // (reps * sweeps),
            "note": f"per instance: dvm_create from host mask, {sweeps} sweeps, dvm_flowrate + dvm_fields to host, "
                    f"dvm_destroy; {reps} repetitions"}


def converge(results, insts, torch, tol=None):
    """Time to converge: each instance alone (plain) vs the three batched, from h = 0."""
    out = {}
    for prec, r in results.items():
        t = 1e-10 if prec == "fp64" else 1e-6
        per = {}
        t_plain = 0.0
        for inst, s in zip(insts, r["solvers"]):
            s.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, iters, est = s.solve(tol=t, max_iter=200000, raise_on_noconv=False)
            dt = time.perf_counter() - t0
            t_plain += dt
            per[f"kn{inst.kn:g}"] = {"iterations": iters, "seconds": dt, "Q": s.flowrate()[0], "status": int(st)}
        for s in r["solvers"]:
            s.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r["batch"].run(tol=t, max_iter=200000)
        t_batch = time.perf_counter() - t0
        out[prec] = {"tol": t, "plain": per, "plain_total_s": t_plain, "batched_total_s": t_batch,
                     "batched_Q": [s.flowrate()[0] for s in r["solvers"]]}
    return out


def cpu_baseline(insts, budget_s=12.0):
    """The FP64 oracle as it stands, on the host cores: sweeps of the Kn = 1 instance."""
    import oracle

    inst = insts[1]
    p = oracle.Problem.make(inst.mask, True, False, oracle.delta_from_kn(inst.kn), inst.quad)
    K = inst.quad[1] ** 2
    h = np.zeros((K, p.ny, p.nx))
    t0 = time.perf_counter()
    oracle.solve(p, tol=0.0, max_iter=1, h0=h, inplace=True)
    first = time.perf_counter() - t0
    n = max(1, int(budget_s / max(first, 1e-3)))
    t0 = time.perf_counter()
    oracle.solve(p, tol=0.0, max_iter=n, h0=h, inplace=True)
    dt = time.perf_counter() - t0
    upd = int((inst.mask == 0).sum()) * K * n
    return {"value": upd / dt, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "kind": "oracle",
            "sample": f"{n} source-iteration sweeps of the Kn=1 rough-channel instance (FP64, C + OpenMP), "
                      f"{dt:.1f} s"}


# ------------------------------------------------------------------------------ reference arm

def run_reference(args):
    """The oracle timed as it stands on the host cores: one step = one sweep of each instance."""
    import oracle

    insts = instances()
    probs = [oracle.Problem.make(i.mask, True, False, oracle.delta_from_kn(i.kn), i.quad) for i in insts]
    states = [np.zeros((i.quad[1] ** 2, p.ny, p.nx)) for i, p in zip(insts, probs)]
    upd = updates_per_step(insts)
    for _ in range(args.warmup):
        for p, h in zip(probs, states):
            oracle.solve(p, tol=0.0, max_iter=1, h0=h, inplace=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for p, h in zip(probs, states):
            oracle.solve(p, tol=0.0, max_iter=1, h0=h, inplace=True)
    dt = time.perf_counter() - t0
    value = args.steps * upd / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config("fp64"), "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps, each one FP64 oracle sweep of all three instances"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        print(json.dumps(run_reference(args)), flush=True)
        return 0
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        import torch
        torch.distributed.barrier()
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
