#!/usr/bin/env python
"""Benchmark of the DVM source iteration (linearized BGK, arXiv:1704.03126 Sec. II.A) on GB300.

Default workload (--workload batched): 64 seeded instances -- sides 64 to 256, rough channels or
periodic disk media, Kn log-uniform in [0.01, 10], cubic velocity grids of 16 to 48 nodes per axis
(Eq. nonuniform_v) -- advanced together, FP32 storage with FP64 moments.  One step = one source
iteration of every instance (transport sweep with fused moments and wall fluxes, mass projection,
residual, flow rate).  The same JSON line carries, under "workloads", the rough channel (FP32 and FP64)
and the porous medium, each with its own roofline, end-to-end rate, time to converge and oracle
baseline.

  rough    force-driven flow through the rough channel -- 128 x 128 cells, periodic along x1, diffuse
           plates with one 26 x 32 block per wall, 32 x 32 trapezoid velocities on [-5, 5]^2 -- at
           Kn = 0.1, 1 and 10, the three instances advanced together (45.2 M updates per step).
Other workloads (--workload), one JSON line each:
  porous   periodic disk medium 256 x 256 (porosity 0.6, radii 8-20), cubic 48 x 48 velocities,
           Kn = 0.05, 0.5, 5 advanced together (FP32 storage).
  adjoint  porous 256 x 256 (porosity 0.5), cubic 32 x 32, Kn = 1, FP64: one step = one transposed
           (adjoint) sweep; gradient checked against central differences of forward solves.
  couette  Couette flow of Sec. II on the paper's grid: top plate moving with U = 1, no force, 1500
           columns (aspect 5, dx1 = H / 300); bottom wall a Weierstrass-Mandelbrot staircase (D = 1.5,
           eps = 2 %) resolved by 60 rows across its band and 100 above, or smooth (100 rows); cubic
           32 x 32 velocities, Kn = 0.1, 1, 10: six instances advanced together; reports
           Q* = Q_rough / Q_smooth per Kn from the converged solves.
  permeability  Sec. III's curves: three synthetic media 256 x 256 (irregular, square and circular
           solids, porosity about 0.6, both axes periodic), cubic 32 x 32 velocities, Kn = 0.02 ... 2:
           21 instances advanced together.  Extras: k_inf extrapolated from Kn = 0.005, 0.01, 0.02
           solved on the media refined twice (512 x 512, Gauss-Hermite 12 x 12), then H* and
           k_a / k_inf against Kn* per medium.

The sweep kernel of every launch is chosen by the library's autotuner before the timed region.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

KNS = (0.1, 1.0, 10.0)
PERM_FIT_KNS = (0.005, 0.01, 0.02)  # k_inf is extrapolated to Kn = 0 from these (refined grid)
PERM_KNS = (0.02, 0.05, 0.1, 0.2, 0.5, 1.0, 2.0)
PERM_FIT_QUAD = ("gh", 12, 0.0)
PERM_FIT_REFINE = 2
FD_DIR_CELLS = 1024  # cells of the adjoint workload's directional finite-difference check
ANDERSON_DEPTH = 6  # depth of the mixed iteration reported beside the plain one (time to converge)
POROUS_KNS = (0.05, 0.5, 5.0)
METRICS = {
    "rough": "DVM cell-velocity updates/s (rough channel 128x128, 32x32 velocities, Kn 0.1/1/10)",
    "porous": "DVM cell-velocity updates/s (porous 256x256 phi 0.6, cubic 48x48 velocities, Kn 0.05/0.5/5)",
    "batched": "DVM cell-velocity updates/s (64 mixed instances, one batched launch per kernel)",
    "adjoint": "adjoint sweep cell-velocity updates/s (porous 256x256 phi 0.5, cubic 32x32, Kn 1, FP64)",
    "couette": "DVM cell-velocity updates/s (Couette on the paper's grid, 1500 x (60+100) WM-rough and "
               "1500 x 100 smooth, cubic 32x32, Kn 0.1/1/10)",
    "permeability": "DVM cell-velocity updates/s (3 porous media 256x256 x 7 Kn in 0.02-2, cubic 32x32)",
}
METRIC = METRICS["rough"]
UNIT = "updates/s"
# FP32 / FP64 floating-point operations per interior cell-velocity update of the sweep kernel, counted
# from its source: right-hand side 3 FMA, two upwind combinations 2 x 2 FMA, update FMA + MUL, moments
# 4 FMA (FMA = 2 flops): 25.  The ncu instruction counts of the sweep (profiles/) confirm the count.
FLOPS_PER_UPDATE = {"fp32": 25, "fp64": 25}
# DRAM bytes (read + write) of one sweep-kernel launch from ncu, keyed by (workload, precision, kernel,
# shape), each with the hash of the sweep kernels' sources it was measured on (kernel_source_hash);
# a figure whose hash no longer matches is reported as null
NCU_TRAFFIC = {
    ("batched", "fp32", "rows", 16): {"bytes": 719.50e6, "src": "6b0e8aadf3bbbe1b"},
    ("porous", "fp32", "rows", 16): {"bytes": 73.49e6, "src": "6b0e8aadf3bbbe1b"},
    ("rough", "fp32", "rows", 8): {"bytes": 14.41e6, "src": "6b0e8aadf3bbbe1b"},
    ("rough", "fp32", "rows", 16): {"bytes": 14.41e6, "src": "6b0e8aadf3bbbe1b"},
    ("rough", "fp64", "rows", 8): {"bytes": 20.99e6, "src": "6b0e8aadf3bbbe1b"},
    ("batched", "fp64", "rows", 16): {"bytes": 1122.46e6, "src": "6b0e8aadf3bbbe1b"},
}
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
    ap.add_argument("--workload", default="batched", choices=sorted(METRICS))
    ap.add_argument("--schedule", default="autotune",
                    help="sweep kernel: autotune, rows, rows<cw> (chunk width), columns1, columns2, columns4")
    ap.add_argument("--fd-cells", type=int, default=16, help="adjoint workload: cells checked by central differences")
    ap.add_argument("--anderson", type=int, default=0,
                    help="mix the timed iterates with Anderson mixing of this depth (0 = the paper's plain "
                         "iteration; needs --precision fp64, times that precision only)")
    ap.add_argument("--persistent", action="store_true",
                    help="time the main workload in the persistent launch (row sweep; profiling runs)")
    return ap.parse_args()


WORKLOAD_TEXT = {
    "rough": "rough channel 128x128 (blocks 26x32 on both walls, x1 periodic), 32x32 trapezoid velocities "
             "|v|<=5, Kn 0.1/1/10 batched; force-driven (F=1)",
    "porous": "periodic disk medium 256x256 (seeded non-overlapping disks, radii 8-20, porosity 0.6), cubic "
              "48x48 velocities |v|<=4, Kn 0.05/0.5/5 batched; force-driven (F=1)",
    "batched": "64 seeded instances: side 64-256, rough or porous, Kn log-uniform 0.01-10, cubic 16-48 "
               "velocities; one launch per kernel per sweep",
    "adjoint": "periodic disk medium 256x256 (porosity 0.5, seed 1), cubic 32x32 velocities, Kn 1, FP64; "
               "transposed sweeps of the adjoint iteration at the converged forward state",
    "couette": "Couette flow, top plate U = 1, no force, x1 periodic, 1500 columns (aspect 5, dx1 = H/300): "
               "Weierstrass-Mandelbrot staircase bottom (D 1.5, gamma 1.5, n1 -4, eps 2%, truncated at the "
               "grid Nyquist frequency, zero mean) on 60 rows across its band + 100 rows above, and smooth "
               "plates on 100 rows; cubic 32x32 velocities |v|<=4, Kn 0.1/1/10 batched",
    "permeability": "three seeded periodic media 256x256, porosity about 0.6 (irregular: thresholded "
                    "Gaussian-filtered noise, width 20 cells; squares: sides 32-80; disks: radii 20-48), cubic "
                    "32x32 velocities |v|<=4, Kn 0.02/0.05/0.1/0.2/0.5/1/2, force-driven (F=1); 21 instances "
                    "batched",
}


def workload_config(precision, workload="rough"):
    return {
        "workload": WORKLOAD_TEXT[workload],
        "instances_per_step": len(instances(workload)),
        "precision": "fp32 store / fp64 accumulate" if precision == "fp32" else "fp64",
        "l2": "flushed between timed steps (256 MiB write)",
        "data": "synthetic staircase geometry",
    }


_INSTANCES = {}


def instances(workload="rough"):
    from paper_1704_03126_gb300 import inputs
    if workload not in _INSTANCES:
        if workload == "rough":
            _INSTANCES[workload] = [inputs.rough_instance(kn) for kn in KNS]
        elif workload == "porous":
            _INSTANCES[workload] = [inputs.porous_instance(kn) for kn in POROUS_KNS]
        elif workload == "batched":
            _INSTANCES[workload] = inputs.batched_instances(64)
        elif workload == "permeability":
            masks = {kind: inputs.medium_mask(kind, 256) for kind in inputs.MEDIA}
            _INSTANCES[workload] = [
                inputs.Instance(f"{kind}256_phi0.6_cubic32_kn{kn:g}", masks[kind][0], True, True, kn, ("cubic", 32, 4.0),
                                {"porosity": masks[kind][1], "medium": kind})
                for kind in inputs.MEDIA for kn in PERM_KNS]
        elif workload == "couette":
            _INSTANCES[workload] = [inputs.couette_instance(kn, rough=rough, grid="paper")
                                    for rough in (True, False) for kn in KNS]
        else:
            _INSTANCES[workload] = [inputs.porous_instance(1.0, nv=32, porosity=0.5, seed=1)]
    return _INSTANCES[workload]


def drive(inst):
    """Grid, body force and top-plate speed of an instance (square cells, force-driven flow unless it
    says otherwise)."""
    x = inst.extra
    return {"ly": float(x.get("ly", 1.0)), "force": float(x.get("force", 1.0)),
            "top_wall_u1": float(x.get("top_u", 0.0)), "dx1": float(x.get("dx1", 0.0)),
            "row_heights": x.get("row_heights")}


def solver(dvm, inst, precision, stream, anderson=0):
    return dvm.Solver(inst.mask, inst.periodic_x, inst.periodic_y, kn=inst.kn, quad=inst.quad,
                      precision=precision, stream=stream, anderson=anderson, **drive(inst))


def oracle_problem(oracle, inst):
    d = drive(inst)
    rows = d["row_heights"]
    if rows is None and d["dx1"] > 0.0:
        rows = np.full(inst.mask.shape[0], d["ly"] / inst.mask.shape[0])
    return oracle.Problem.make(inst.mask, inst.periodic_x, inst.periodic_y, oracle.delta_from_kn(inst.kn), inst.quad,
                               force=d["force"], ly=d["ly"], top_u=d["top_wall_u1"], dy=rows,
                               dx1=d["dx1"] if rows is not None else None)


def apply_schedule(batch, spec):
    """Pick the batch's sweep kernel: the library autotuner (5 timed sweeps per candidate) or a fixed one."""
    if spec == "autotune":
        kind, v, ms = batch.autotune(5)
        return {"kernel": kind, "shape": v, "tuned_sweep_ms": ms, "by": "autotuner"}
    if spec.startswith("rows"):
        batch.set_schedule("rows", int(spec[4:] or 0))
    else:
        batch.set_schedule("columns", int(spec[len("columns"):]))
    kind, v = batch.schedule()
    return {"kernel": kind, "shape": v, "by": "fixed"}


def max_over_ranks(ms, world, device="cpu"):
    """Max of a per-rank time over the ranks (the slowest rank sets the job's time)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, updates, total_ms):
    """Whole-job throughput: every rank runs `steps` steps of `updates` each (replicas, weak scaling)."""
    return world * steps * updates / (total_ms / 1e3)


def updates_per_step(insts):
    return sum(int((inst.mask == 0).sum()) * inst.quad[1] ** 2 for inst in insts)


# ------------------------------------------------------------------------------ clocks

def physical_gpu_id(cuda_index):
    """The nvidia-smi --id of CUDA device `cuda_index`: "GPU-<uuid>" from torch's device properties,
    else the PCI bus id, else the index itself."""
    try:
        import torch
        props = torch.cuda.get_device_properties(cuda_index)
        uuid = str(getattr(props, "uuid", "") or "")
        if uuid:
            return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        bus = getattr(props, "pci_bus_id", None)
        if bus is not None:
            dom = getattr(props, "pci_domain_id", 0)
            dev = getattr(props, "pci_device_id", 0)
            return f"{dom:08x}:{bus:02x}:{dev:02x}.0"
    except Exception:
        pass
    return str(cuda_index)


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        # nvidia-smi numbers the GPUs of the whole machine and ignores CUDA_VISIBLE_DEVICES: name the
        # device by its UUID (from the CUDA runtime, which sees only the visible GPUs)
        self.gpu = physical_gpu_id(gpu_index)
        self.proc = None
        # raw samples go to a scratch file; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"dvm_bench_clocks_{os.getpid()}.csv")

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
                "reasons": sorted(reasons), "samples": len(sm), "gpu_id": self.gpu}


# ------------------------------------------------------------------------------ our arm

def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def device_peaks(dvm):
    """FMA ceilings measured live on this GPU (dvm_probe_peaks, about 0.2 s each) and its L2 size."""
    out = {}
    for kind in ("fp32", "fp32x2", "fp64"):
        tf, l2, sms = dvm.probe_peaks(kind, 0.2)
        out[kind] = tf
    out["l2_bytes"] = l2
    out["sms"] = sms
    return out


def kernel_source_hash(csrc=None):
    """Hash of the sweep kernels' code (comments and blank lines removed): a recorded DRAM-traffic figure
    holds only for this hash."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_1704_03126_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.startswith("dvm_sweep") or name in ("dvm_device.cuh", "dvm_kernels.h"):
            text = open(os.path.join(csrc, name), encoding="utf-8").read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            text = re.sub(r"//[^\n]*", "", text)
            code = "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())
            h.update(name.encode())
            h.update(code.encode())
    return h.hexdigest()[:16]


def roofline(upd, sweep_ms, fin_ms, prec, sched, hbm_gbs, alu_peaks, workload):
    """Roofline of the dominant kernel (the sweep) for one launch of `upd` cell-velocity updates.

    bound hbm, "effective, fused": the algorithmic bytes of the method per update -- the source
    iteration writes h^{n+1} once and reads it once for its moments, 2 s bytes (s = 4 FP32, 8 FP64) --
    over the sweep kernel's CUDA-event time, against the measured HBM copy bandwidth.  The fused kernel
    keeps h on chip, so its DRAM traffic (`traffic`, from ncu) is far below those bytes; the ALU fraction
    against the measured FMA rate is given beside it."""
    bpu = 8 if prec == "fp32" else 16
    achieved = upd * bpu / (sweep_ms / 1e3) / 1e9
    kname = (f"sweep_kernel, chunk width {sched['shape']}" if sched["kernel"] == "rows"
             else f"cols_kernel, {sched['shape']} thread(s) per column")
    rec = NCU_TRAFFIC.get((workload, prec, sched["kernel"], sched["shape"]))
    src = kernel_source_hash()
    traffic = rec["bytes"] if rec is not None and rec["src"] == src else None
    alu_key = "fp32" if prec == "fp32" else "fp64"
    alu_ach = FLOPS_PER_UPDATE[prec] * upd / (sweep_ms / 1e3) / 1e12
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
            "traffic": traffic,
            "basis": f"effective, fused: {bpu} B per cell-velocity update (write + read of h that a non-fused "
                     f"iteration needs) x {upd} updates per launch / sweep-kernel CUDA-event time; peak = "
                     f"MEASURED_PEAKS hbm_gbs (of measured)",
            "traffic_note": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of this kernel build"
                             if traffic is not None else
                             "null: no ncu capture of this launch configuration for the current kernel sources"),
            "kernel": f"{kname} ({prec})", "schedule": sched, "sweep_ms": sweep_ms, "finalize_ms": fin_ms,
            "updates_per_launch": upd, "kernel_src": src,
            "alu": {"achieved": alu_ach, "peak": alu_peaks[alu_key], "unit": "TFLOP/s",
                    "frac": alu_ach / alu_peaks[alu_key], "flops_per_update": FLOPS_PER_UPDATE[prec],
                    "peak_note": f"{alu_key.upper()} FMA chains measured live by dvm_probe_peaks (of measured)"}}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1704_03126_gb300 import dvm

    torch.cuda.set_device(local_rank)
    # a stream of our own (the default stream's handle is 0, which the library would replace by a
    # private stream): the solvers, the L2 flush and the CUDA events all run on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peaks = load_peaks()
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    alu = device_peaks(dvm)
    torch.cuda.synchronize()

    def timed_steps(batch, steps, warmup):
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
            batch.enqueue(1)  # no host round trip inside the timed region
            ev1[k].record(stream)
            if k % 16 == 15 or k == steps - 1:
                # the sweep/finalize events of a step are re-recorded by the next one: read them
                # for a sample of steps (this waits for the stream, outside the measured events)
                torch.cuda.synchronize()
                s_ms, f_ms = batch.timing()
                sweep_ms.append(s_ms)
                fin_ms.append(f_ms)
        torch.cuda.synchronize()
        batch.check()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        total = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        return total, float(np.mean(sweep_ms)), float(np.mean(fin_ms)), w

    def measure(workload, precision, steps, warmup, sampler=None):
        insts = instances(workload)
        upd = updates_per_step(insts)
        solvers = [solver(dvm, inst, precision, stream.cuda_stream, anderson=args.anderson) for inst in insts]
        batch = dvm.Batch(solvers)
        sched = apply_schedule(batch, args.schedule)
        if args.persistent and workload == args.workload and precision == args.precision:
            batch.set_schedule("rows", sched["shape"] if sched["kernel"] == "rows" else 0)
            batch.set_persistent(True)
            sched = dict(sched, persistent=True)
        total_ms, sweep_ms, fin_ms, wsteps = timed_steps(batch, steps, warmup)
        clocks = sampler.stop() if sampler is not None else None
        total_ms = max_over_ranks(total_ms, world, device="cuda")
        persistent_ok = args.anderson == 0 and not any(
            i.extra.get("top_u", 0.0) or i.extra.get("row_heights") is not None for i in insts)
        return dict(workload=workload, precision=precision, insts=insts, upd=upd, solvers=solvers, batch=batch,
                    sched=sched, total_ms=total_ms, sweep_ms=sweep_ms, fin_ms=fin_ms, warmup_steps=wsteps,
                    kernels_per_step=batch.kernels_per_sweep(), steps=steps, clocks=clocks,
                    value=job_value(world, steps, upd, total_ms), persistent_ok=persistent_ok,
                    roofline=roofline(upd, sweep_ms, fin_ms, precision, sched, hbm_gbs, alu, workload))

    def measure_persistent(m, steps, warmup):
        """The same batch and steps in the persistent launch (one launch per step: every member's sweep
        and finalize, scheduled on the device)."""
        b = m["batch"]
        b.set_schedule("rows", m["sched"]["shape"] if m["sched"]["kernel"] == "rows" else 0)
        b.set_persistent(True)
        total_ms, sweep_ms, _, _ = timed_steps(b, steps, warmup)
        total_ms = max_over_ranks(total_ms, world, device="cuda")
        on, blocks = b.persistent()
        return {"value": job_value(world, steps, m["upd"], total_ms), "ms_per_step": total_ms / steps,
                "launch_ms": sweep_ms, "blocks": blocks, "kernels_per_step": b.kernels_per_sweep() + 1,
                "effective_hbm_frac": m["upd"] * (8 if m["precision"] == "fp32" else 16) / (sweep_ms / 1e3) / 1e9 / hbm_gbs,
                "note": "one launch per step (arming + scheduler kernels): every member's sweep tiles and "
                        "finalize chunks; launch_ms = CUDA-event time of that launch"}

    def close(m):
        m["batch"].close()
        for s in m["solvers"]:
            s.close()

    def extras(m, cpu=True, budget_s=12.0):
        """e2e, time to converge, the CPU oracle beside it."""
        big = len(m["insts"]) > 6
        r = {}
        r["e2e"] = e2e(args, m["insts"], m["precision"], stream, dvm, torch, max_iter=10000 if big else 200000)
        if m["workload"] == "permeability":
            r["curves"] = curves({m["precision"]: m}, m["insts"], torch)
        else:
            r["converge"] = converge({m["precision"]: m}, m["insts"], torch, max_iter=10000 if big else 200000,
                                     dvm=dvm, stream=stream.cuda_stream)
        if cpu and rank == 0:
            r["cpu_baseline"] = cpu_baseline(m["insts"], m["workload"], budget_s=budget_s)
        return r

    sampler = ClockSampler(local_rank)
    sampler.start()
    main = measure(args.workload, args.precision, args.steps, args.warmup, sampler)
    out = {
        "metric": METRICS[args.workload], "value": main["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["total_ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": dict(workload_config(args.precision, args.workload), anderson_depth=args.anderson),
        "roofline": main["roofline"],
        "clocks": main["clocks"],
        # per step: the arming kernel, the sweep and the two finalize kernels (and three mixing kernels)
        "gpu_launches": args.steps * (main["kernels_per_step"] + 1),
        "device_peaks_measured": alu,
    }
    if not args.skip_extras:
        out.update(extras(main))
    if main["persistent_ok"] and not args.skip_extras and args.workload in ("batched", "rough", "porous"):
        out["persistent"] = measure_persistent(main, args.steps, args.warmup)
    close(main)
    # the other configurations of the method, each with its own roofline, e2e and oracle baseline
    # (same steps and warm-up; the default line's workload is the 64-instance batch)
    if not args.single and not args.skip_extras and args.anderson == 0:
        others = {"batched": [("batched", "fp64"), ("rough", "fp32"), ("rough", "fp64"), ("porous", "fp32")],
                  "rough": [("rough", "fp64" if args.precision == "fp32" else "fp32")]}.get(args.workload, [])
        out["workloads"] = {}
        cpu_done = {}
        for wl, prec in others:
            s2 = ClockSampler(local_rank)
            s2.start()
            m = measure(wl, prec, args.steps, args.warmup, s2)
            rec = {"metric": METRICS[wl], "value": m["value"], "unit": UNIT, "ms_per_step": m["total_ms"] / args.steps,
                   "dtype": "f32" if prec == "fp32" else "f64", "config": workload_config(prec, wl),
                   "roofline": m["roofline"], "clocks": m["clocks"],
                   "gpu_launches": args.steps * (m["kernels_per_step"] + 1)}
            if wl == args.workload:
                # the same batch in FP64 storage: timed steps only (its solve to 1e-10 would take minutes);
                # the oracle baseline is the main line's
                ex = {"cpu_baseline": out.get("cpu_baseline"),
                      "note": "timed steps of the default batch in FP64 storage (no converge or e2e run)"}
                if m["persistent_ok"]:
                    ex["persistent"] = measure_persistent(m, args.steps, args.warmup)
            else:
                ex = extras(m, cpu=wl not in cpu_done, budget_s=8.0)
                if "cpu_baseline" in ex:
                    cpu_done[wl] = ex["cpu_baseline"]
                else:
                    ex["cpu_baseline"] = cpu_done.get(wl)
            rec.update(ex)
            out["workloads"][f"{wl}_{prec}"] = rec
            close(m)
    return out


def e2e(args, insts, precision, stream, dvm, torch, max_iter=200000):
    """Time to solution through the public API with host buffers, in the line's metric: create every
    instance from its host mask (H2D: mask, tables, the launch graphs), one batched solve to the
    converge tolerance (dvm_batch_run; FP32 storage includes its refinement), flow rates and fields
    back to the host (D2H), destroy.  updates = the sweeps each instance ran x its cell-velocity
    updates per sweep; value = updates / wall time of all of it.  The breakdown gives each part."""
    tol = 1e-10 if precision == "fp64" else 1e-6
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sols = [solver(dvm, inst, precision, stream.cuda_stream) for inst in insts]
    t1 = time.perf_counter()
    batch = dvm.Batch(sols)
    t2 = time.perf_counter()
    status = batch.run(tol=tol, max_iter=max_iter)
    t3 = time.perf_counter()
    out = [(s.flowrate()[0], s.fields()) for s in sols]
    sweeps = [s.info()["iterations"] for s in sols]
    t4 = time.perf_counter()
    batch.close()
    for s in sols:
        s.close()
    torch.cuda.synchronize()
    t5 = time.perf_counter()
    upd = sum(int((inst.mask == 0).sum()) * inst.quad[1] ** 2 * n for inst, n in zip(insts, sweeps))
    steps = max(1, max(sweeps))
    h2d = sum(inst.mask.nbytes for inst in insts)
    d2h = sum(8 + sum(a.nbytes for a in f.values()) for _, f in out)
    return {"value": upd / (t5 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d // steps, "d2h_bytes_per_step": d2h // steps,
            "seconds": t5 - t0, "tol": tol, "converged": int((np.asarray(status) == 0).sum()),
            "sweeps": {"max": max(sweeps), "total": sum(sweeps)},
            "breakdown_s": {"create": t1 - t0, "batch_graphs": t2 - t1, "solve": t3 - t2, "readback": t4 - t3,
                            "destroy": t5 - t4},
            "note": "dvm_create from host masks, dvm_batch_create, dvm_batch_run to tol, dvm_flowrate + dvm_fields "
                    "to host, destroy; per-step bytes = all bytes / the most sweeps of an instance"}


def converge(results, insts, torch, max_iter=200000, dvm=None, stream=None):
    """Time to converge: each instance alone (plain, automatic sweep kernel) vs all of them batched
    (the timed launch), from h = 0, to the same tolerance; for up to six instances also the batch with
    mixed iterates (Anderson depth ANDERSON_DEPTH)."""
    out = {}
    for prec, r in results.items():
        t = 1e-10 if prec == "fp64" else 1e-6
        per = {}
        t_plain = 0.0
        for inst, s in zip(insts, r["solvers"]):
            s.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, iters, est = s.solve(tol=t, max_iter=max_iter, raise_on_noconv=False)
            dt = time.perf_counter() - t0
            t_plain += dt
            per[inst.name] = {"iterations": iters, "seconds": dt, "Q": s.flowrate()[0], "status": int(st)}
        for s in r["solvers"]:
            s.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status = r["batch"].run(tol=t, max_iter=max_iter)
        t_batch = time.perf_counter() - t0
        bq = [s.flowrate()[0] for s in r["solvers"]]
        pq = [v["Q"] for v in per.values()]
        out[prec] = {"tol": t, "max_iter": max_iter, "plain_total_s": t_plain, "batched_total_s": t_batch,
                     "converged_plain": sum(v["status"] == 0 for v in per.values()),
                     "converged_batched": int((np.asarray(status) == 0).sum()), "instances": len(insts),
                     "max_rel_dQ_batched_vs_plain": max(abs(a - b) / max(abs(b), 1e-300) for a, b in zip(bq, pq))}
        # the same batch in one persistent launch per 64 sweeps (device-side scheduler, row sweep)
        if dvm is not None and r.get("persistent_ok"):
            pb = dvm.Batch(r["solvers"])
            pb.set_schedule("rows", r["sched"]["shape"] if r["sched"]["kernel"] == "rows" else 0)
            pb.set_persistent(True)
            for s in r["solvers"]:
                s.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pst = pb.run(tol=t, max_iter=max_iter)
            t_p = time.perf_counter() - t0
            pqs = [s.flowrate()[0] for s in r["solvers"]]
            out[prec]["persistent"] = {
                "batched_total_s": t_p, "converged": int((np.asarray(pst) == 0).sum()), "blocks": pb.persistent()[1],
                "max_rel_dQ_vs_per_kernel_batch": max(abs(a - b) / max(abs(b), 1e-300) for a, b in zip(pqs, bq))}
            pb.close()
        # the batched run again with mixed iterates (an extension of the paper's plain iteration; FP64
        # storage only)
        if len(insts) <= 6 and dvm is not None and prec == "fp64":
            aa = [solver(dvm, s_inst, prec, stream, anderson=ANDERSON_DEPTH) for s_inst in insts]
            ab = dvm.Batch(aa)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st_aa = ab.run(tol=t, max_iter=max_iter)
            t_aa = time.perf_counter() - t0
            out[prec]["anderson"] = {
                "depth": ANDERSON_DEPTH, "batched_total_s": t_aa,
                "converged": int((np.asarray(st_aa) == 0).sum()),
                "iterations": [s.info()["iterations"] for s in aa],
                "max_rel_dQ_vs_plain": max(abs(s.flowrate()[0] - b) / max(abs(b), 1e-300) for s, b in zip(aa, pq))}
            ab.close()
            for s in aa:
                s.close()
        if len(insts) <= 6 and dvm is not None and prec == "fp32":
            # the FP32 path's stated error: each converged Q against the same instance in FP64 storage
            ref = [solver(dvm, s_inst, "fp64", stream) for s_inst in insts]
            rb = dvm.Batch(ref)
            st64 = rb.run(tol=1e-11, max_iter=max_iter)
            q64 = [s.flowrate()[0] for s in ref]
            u64 = [s.fields()["u1"] for s in ref]
            rb.close()
            for s in ref:
                s.close()
            f_err = []
            for s, u in zip(r["solvers"], u64):
                u32 = s.fields()["u1"]
                gas = np.isfinite(u)
                f_err.append(float(np.abs(u32[gas] - u[gas]).max() / np.abs(u[gas]).max()))
            out[prec]["vs_fp64"] = {
                "fp64_tol": 1e-11, "fp64_converged": int((np.asarray(st64) == 0).sum()), "Q_fp64": q64,
                "rel_err_Q": [abs(a - b) / abs(b) for a, b in zip(bq, q64)],
                "max_abs_err_u1_over_max_u1": f_err}
        if len(insts) <= 6:
            out[prec]["plain"] = per
            out[prec]["batched_Q"] = bq
        if any(i.extra.get("top_u", 0.0) != 0.0 for i in insts):
            out[prec]["Q_star"] = couette_q_star(insts, bq)
            out[prec]["profiles"] = couette_profiles(insts, r["solvers"])
    return out


def curves(results, insts, torch, max_iter=200000):
    """Sec. III: the timed batch (curve points) converged in one run; the fit points of every medium
    (refined grid, Gauss-Hermite velocities) as a second batch; then per medium k_inf, H* and
    k_a / k_inf against Kn*.  The Knudsen number solved on both grids shows their agreement."""
    from paper_1704_03126_gb300 import inputs
    from paper_1704_03126_gb300 import permeability as perm
    out = {}
    for prec, r in results.items():
        tol = 1e-10 if prec == "fp64" else 1e-6
        for s in r["solvers"]:
            s.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status = r["batch"].run(tol=tol, max_iter=max_iter)
        dt = time.perf_counter() - t0
        fit_masks, fit_kns, owners = [], [], []
        for kind in inputs.MEDIA:
            m = next(i.mask for i in insts if i.extra.get("medium") == kind)
            for kn in PERM_FIT_KNS:
                fit_masks.append(inputs.refine_mask(m, PERM_FIT_REFINE))
                fit_kns.append(kn)
                owners.append(kind)
        t0 = time.perf_counter()
        fka, fit_iters, fit_status = perm.solve_batch(fit_masks, fit_kns, PERM_FIT_QUAD, prec, tol, max_iter)
        dt_fit = time.perf_counter() - t0
        media = {}
        for kind in inputs.MEDIA:
            idx = [i for i, inst in enumerate(insts) if inst.extra.get("medium") == kind]
            ka = {insts[i].kn: r["solvers"][i].flowrate()[1] for i in idx}
            iters = {insts[i].kn: r["solvers"][i].info()["iterations"] for i in idx}
            fsel = [j for j, o in enumerate(owners) if o == kind]
            res = perm.curve_from_values(PERM_KNS, [ka[k] for k in PERM_KNS], [fit_kns[j] for j in fsel],
                                         [fka[j] for j in fsel], insts[idx[0]].extra["porosity"])
            res["iterations"] = {f"{k:g}": iters[k] for k in sorted(iters)}
            res["fit_iterations"] = {f"{fit_kns[j]:g}": fit_iters[j] for j in fsel}
            both = sorted(set(PERM_KNS) & set(PERM_FIT_KNS))
            res["grid_check"] = {f"{k:g}": {"coarse_cubic32": ka[k], "refined_gh12": fka[fsel[PERM_FIT_KNS.index(k)]]}
                                 for k in both}
            media[kind] = res
        out[prec] = {"tol": tol, "max_iter": max_iter, "curve_batch_s": dt, "fit_batch_s": dt_fit,
                     "instances": len(insts) + len(fit_kns),
                     "converged": int((np.asarray(status) == 0).sum()) + sum(s == 0 for s in fit_status),
                     "fit": f"k_inf from Kn {PERM_FIT_KNS} on the media refined {PERM_FIT_REFINE}x, {PERM_FIT_QUAD}",
                     "media": media}
    return out


PROFILE_POINTS = (0.02, 0.05, 0.1, 0.25, 0.5, 0.75, 0.9, 0.95, 0.98)


def couette_profiles(insts, solvers):
    """Mean streamwise velocity u1_bar(x2) (average over x1, solid cells as zero; the plate moves at
    x2 = H = 1, the mean bottom is x2 = 0) at PROFILE_POINTS for Kn 0.1 and 1, the cases of the paper's
    velocity-profile comparison (Sec. II.B)."""
    from paper_1704_03126_gb300 import couette
    out = {}
    for inst, s in zip(insts, solvers):
        if inst.kn not in (0.1, 1.0):
            continue
        x = inst.extra
        ly = float(x.get("ly", 1.0))
        y, ub = couette.mean_profile(s.fields()["u1"], inst.mask, ly, x.get("row_heights"), y0=1.0 - ly)
        kind = "rough" if x.get("eps", 0.0) > 0.0 else "smooth"
        out[f"{kind}_kn{inst.kn:g}"] = {"x2": list(PROFILE_POINTS),
                                         "u1_bar": couette.profile_at(y, ub, PROFILE_POINTS).tolist()}
    return out


def couette_q_star(insts, q):
    """Q* = Q_r / Q_s of Sec. II at each Kn: flow rate over the rough wall over that of smooth plates."""
    rough = {i.kn: v for i, v in zip(insts, q) if i.extra.get("eps", 0.0) > 0.0}
    smooth = {i.kn: v for i, v in zip(insts, q) if i.extra.get("eps", 0.0) == 0.0}
    return {f"{kn:g}": {"Q_r": rough[kn], "Q_s": smooth[kn], "Q_star": rough[kn] / smooth[kn]}
            for kn in sorted(rough) if kn in smooth}


def cpu_baseline(insts, workload="rough", budget_s=12.0):
    """The FP64 oracle as it stands, on the host cores: sweeps of one instance of the workload (the
    middle Knudsen number, or the first batched instance)."""
    import oracle

    inst = insts[1] if len(insts) in (3, 6) else insts[0]
    p = oracle_problem(oracle, inst)
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
            "sample": f"{n} source-iteration sweeps of instance {inst.name} (FP64, C + OpenMP), {dt:.1f} s",
            "one_thread": oracle_one_thread(workload, budget_s / 4)}


def oracle_one_thread(workload, budget_s):
    """The same oracle sample on one host thread (a fresh interpreter with OMP_NUM_THREADS=1)."""
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench, json; "
            f"r = bench.cpu_baseline_sample(bench.instances({workload!r}), {workload!r}, {budget_s!r}); "
            f"print(json.dumps(r))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"error": str(e)[:200]}


def cpu_baseline_sample(insts, workload="rough", budget_s=3.0):
    """updates/s of the oracle on the sample cpu_baseline uses, with the threads OpenMP is given."""
    import oracle

    inst = insts[1] if len(insts) in (3, 6) else insts[0]
    p = oracle_problem(oracle, inst)
    K = inst.quad[1] ** 2
    h = np.zeros((K, p.ny, p.nx))
    t0 = time.perf_counter()
    oracle.solve(p, tol=0.0, max_iter=1, h0=h, inplace=True)
    first = time.perf_counter() - t0
    n = max(1, int(budget_s / max(first, 1e-3)))
    t0 = time.perf_counter()
    oracle.solve(p, tol=0.0, max_iter=n, h0=h, inplace=True)
    dt = time.perf_counter() - t0
    return {"value": int((inst.mask == 0).sum()) * K * n / dt, "unit": UNIT, "cores": 1,
            "sample": f"{n} sweeps of instance {inst.name} on one thread, {dt:.1f} s"}


def run_adjoint(args, rank, world, local_rank):
    """Adjoint workload: converged FP64 forward state, then the adjoint iteration (transposed sweeps)
    timed with CUDA events on the solver's stream; checked against central differences of forward
    solves (cells drawn with SplitMix64 seed 7, step 1e-3 delta, solves to 1e-12, all perturbed solves
    in one batch) and one directional difference over all sampled cells at once."""
    import torch

    from paper_1704_03126_gb300 import dvm, inputs

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    inst = instances("adjoint")[0]
    upd = updates_per_step([inst])
    delta = dvm.kn_to_delta(inst.kn)
    tol = 1e-12

    def solver(store, sched=None):
        s = dvm.Solver(inst.mask, inst.periodic_x, inst.periodic_y, delta=delta, quad=inst.quad,
                       precision="fp64", store_distribution=store, stream=stream.cuda_stream)
        if sched is not None:
            s.set_schedule(*sched)
        return s

    if args.schedule == "autotune":
        probe = solver(False)
        b = dvm.Batch([probe])
        kind, v, _ = b.autotune(3)
        b.close()
        probe.close()
        sched = (kind, v)
    else:
        sched = (("rows", int(args.schedule[4:] or 0)) if args.schedule.startswith("rows")
                 else ("columns", int(args.schedule[7:])))
    sol = solver(True, sched)
    sampler = ClockSampler(local_rank)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sol.solve(tol=tol, max_iter=100000)  # warm-up (graphs, clocks)
    sol.reset()
    torch.cuda.synchronize()
    e0.record(stream)
    st, f_iters, _ = sol.solve(tol=tol, max_iter=100000)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    q0 = sol.flowrate()[0]
    sol.adjoint(tol=tol, max_iter=100000)  # warm-up of the adjoint graph
    torch.cuda.synchronize()
    e0.record(stream)
    grad, q_id, a_iters = sol.adjoint(tol=tol, max_iter=100000)
    e1.record(stream)
    torch.cuda.synchronize()
    adj_ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    sched = sol.schedule()

    # central differences: all perturbed solves in one batch
    cells = inputs.sample_gas_cells(inst.mask, args.fd_cells, seed=7)
    base = np.where(inst.mask == 0, delta, 0.0)
    rng = np.random.default_rng(7)
    dirn = np.zeros(inst.mask.size)
    dirn[cells] = rng.standard_normal(len(cells))
    fields = []
    step = 1e-3 * delta
    for c in cells:
        for sgn in (1.0, -1.0):
            d = base.copy().ravel()
            d[c] += sgn * step
            fields.append(d.reshape(inst.mask.shape))
    eps_dir = 1e-3
    for sgn in (1.0, -1.0):
        fields.append((base.ravel() * (1.0 + sgn * eps_dir * dirn)).reshape(inst.mask.shape))
    # one directional difference over FD_DIR_CELLS seeded cells (the adjoint configuration's check size)
    cells_dir = inputs.sample_gas_cells(inst.mask, FD_DIR_CELLS, seed=11)
    dirn2 = np.zeros(inst.mask.size)
    dirn2[cells_dir] = np.random.default_rng(11).standard_normal(len(cells_dir))
    for sgn in (1.0, -1.0):
        fields.append((base.ravel() * (1.0 + sgn * eps_dir * dirn2)).reshape(inst.mask.shape))
    qs = []
    t0 = time.perf_counter()
    chunk = 48
    fd_tol = 1e-12
    for k in range(0, len(fields), chunk):
        sols = [solver(False, sched) for _ in fields[k:k + chunk]]
        for s, f in zip(sols, fields[k:k + chunk]):
            s.set_delta_field(f)
        dvm.batch_solve(sols, tol=fd_tol, max_iter=100000)
        qs.extend(s.flowrate()[0] for s in sols)
        for s in sols:
            s.close()
    fd_s = time.perf_counter() - t0
    qs = np.array(qs)
    fd = (qs[0:2 * len(cells):2] - qs[1:2 * len(cells):2]) / (2 * step)
    g = grad.ravel()[cells]
    gscale = np.abs(grad).max()
    dir_fd = (qs[-4] - qs[-3]) / (2 * eps_dir)
    dir_adj = float((grad.ravel() * base.ravel() * dirn).sum())
    dir2_fd = (qs[-2] - qs[-1]) / (2 * eps_dir)
    dir2_adj = float((grad.ravel() * base.ravel() * dirn2).sum())
    value = a_iters * upd / (adj_ms / 1e3)
    alu = device_peaks(dvm)
    peak64 = alu["fp64"]
    achieved = FLOPS_PER_UPDATE["fp64"] * value / 1e12
    out = {
        "metric": METRICS["adjoint"], "value": value, "unit": UNIT, "n_gpus": world, "steps": a_iters,
        "warmup": 1, "ms_per_step": adj_ms / a_iters, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config("fp64", "adjoint"),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                     "frac": achieved / peak64, "traffic": None,
                     "kernel": f"transposed sweep, {sched[0]} kernel (fp64), whole adjoint iteration incl. bookkeeping",
                     "flops_per_update": FLOPS_PER_UPDATE["fp64"],
                     "peak_note": "FP64 FMA chains measured live by dvm_probe_peaks (of measured)"},
        "clocks": clocks,
        "device_peaks_measured": alu,
        # per adjoint sweep: transposed sweep, seam sums, two finalize kernels; plus arm, reset, gradient
        "gpu_launches": 4 * a_iters + 3,
        "adjoint_vs_plain": {"tol": tol, "forward_iterations": f_iters, "forward_ms": fwd_ms,
                             "adjoint_iterations": a_iters, "adjoint_ms": adj_ms,
                             "forward_updates_per_s": f_iters * upd / (fwd_ms / 1e3),
                             "Q": q0, "Q_identity_rel_err": abs(q_id - q0) / abs(q0)},
        "fd_check": {"cells": int(len(cells)), "step": "1e-3 delta", "forward_tol": fd_tol,
                     "max_abs_err_over_max_grad": float(np.abs(fd - g).max() / gscale),
                     "median_rel_err": float(np.median(np.abs(fd - g) / np.maximum(np.abs(g), 1e-300))),
                     "directional_rel_err": abs(dir_fd - dir_adj) / abs(dir_adj),
                     "directional_cells": int(len(cells_dir)),
                     "directional_over_cells_rel_err": abs(dir2_fd - dir2_adj) / abs(dir2_adj), "seconds": fd_s,
                     "solves": len(fields)},
    }
    sol.close()
    return out


# ------------------------------------------------------------------------------ reference arm

def run_reference(args):
    """The oracle timed as it stands on the host cores: one step = one sweep of each instance."""
    import oracle

    insts = instances(args.workload if args.workload != "adjoint" else "rough")
    if len(insts) > 6:
        # a bounded sample of the batch (every eighth instance): the rate is a per-update figure
        insts = insts[::8]
    probs = [oracle_problem(oracle, i) for i in insts]
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
        "metric": METRICS[args.workload if args.workload != "adjoint" else "rough"], "value": value,
        "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the same config as our arm's line for this workload (the oracle itself computes in FP64: dtype)
        "config": dict(workload_config(args.precision, args.workload if args.workload != "adjoint" else "rough"),
                       anderson_depth=args.anderson),
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps, each one FP64 oracle sweep of every instance"
                                   + (f" of a sample of {len(insts)} (every eighth)" if args.workload == "batched" else "")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    if args.anderson > 0 and args.precision != "fp64":
        raise SystemExit("--anderson needs --precision fp64 (mixing runs on FP64 storage only)")
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
    out = (run_adjoint if args.workload == "adjoint" else run_ours)(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
