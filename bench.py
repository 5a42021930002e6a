#!/usr/bin/env python
"""Benchmark of the regularized PonD finite-volume step on GB300.

Workload: the 2D four-quadrant Riemann problem on the D2Q16 lattice, 1024 x 1024 cells on
the unit square, quadrant states drawn from seed 0 (rho, p log-uniform in [0.1, 10], Mach
up to 3), gamma 1.4, transmissive boundaries, CFL 0.2.  A step is one full time step of
the grid (face corrector + cell update).  The headline runs the populations in FP32 (frames
as float-float pairs); the plain FP64 path is measured on the same GPU and reported beside
it.  Before timing, the autotuner picks the face and cell kernel variants on the workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica (seed + rank): the step has no
data-path exchange in this single-GPU build, so N GPUs run N independent problems.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s (MLUPS) and % HBM roofline, FP32+learned vs plain FP64, same accuracy"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
N_SMS, FP32_LANES = 152, 128
# ncu dram read + write of one face-kernel launch at 1024^2, for the tile variants measured
# on the current kernel (profiles/face_kernel_quadrants1024_fp32.md); other variants: null
FACE_KERNEL_DRAM_BYTES = {
    "face 8x8 cells, 128 threads, 4 CTA/SM, centre cells in shared scratch": 134.708e6 + 136.232e6,
    "face 8x8 cells, 128 threads, 4 CTA/SM, centre cells and moment sums in shared scratch": 134.678e6 + 136.447e6,
    "face 8x8 cells, 128 threads, 4 CTA/SM, centre cells in shared scratch, TMA staging": 134.782e6 + 136.415e6,
    "face 8x8 cells, 128 threads, 4 CTA/SM, centre cells and moment sums in shared scratch, TMA staging":
        134.643e6 + 133.277e6,
}
# FP32 operations of one corrector pass at one D2Q16 face (per-face overhead included),
# counted by ncu on one launch of the headline face variant at 1024^2 (level-2 scratch, TMA
# staging): FFMA x 2 + FFMA2 x 4 + FMUL + FMUL2 x 2 + FADD + FADD2 x 2 = 8.417 GFLOP over
# 2,099,200 faces x 1.028 passes (profiles/face_kernel_quadrants1024_fp32.md); used for the
# ALU roofline.  (The scalar kernel of earlier builds executed 4550 per pass.)
FLOPS_PER_FACE_PASS = 3900.0
# algorithmic bytes per cell-update of the FP32 D2Q16 layout: the face kernel reads the
# cell state (8 + 6 FP32 coefficients + 3 float-float frame words = 80 B) and two face predictors
# (2 x 24 B) and writes two faces (2 x (16 x 4 + 24) B)
FACE_KERNEL_BYTES_PER_CELL = 80 + 48 + 176
# algorithmic bytes per cell-update of the whole FP32 D2Q16 step in the population layout of
# the method: the 16 f and 16 g populations in FP32 (128 B), the FP64 cell frame (24 B) and
# the cell's two FP32 face gauges (24 B), each read once and written once
STEP_BYTES_PER_CELL = 352


def replica_seed(base_seed, rank):
    """Each rank advances its own replica of the workload (seed + rank)."""
    return base_seed + rank


def max_over_ranks(x, world, device=None):
    """The slowest rank's time (the job's time); every rank gets the same value."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(cells_per_rank, steps, seconds, world):
    """Whole-job throughput: the updates of all ranks over the slowest rank's time."""
    return world * cells_per_rank * steps / seconds / 1e6


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class _NvmlPoller:
    """Reads the SM clock and the clock-event reasons through NVML's C API every millisecond
    from a thread, so that a timed region of a few milliseconds still gets samples (the
    nvidia-smi loop samples every 100 ms at best).  Read-only queries; None if NVML is not
    loadable."""

    SM = 1  # NVML_CLOCK_SM
    # clock-event reason bits of the NVML API
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}

    def __init__(self, index, period_s=0.001):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if isinstance(index, str):
            rc = self.lib.nvmlDeviceGetHandleByUUID(index.encode(), ctypes.byref(self.h))
        else:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h))
        if rc != 0:
            raise RuntimeError("no NVML handle for device %s" % index)
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ctypes.byref(mx)) == 0 else None
        self.period = period_s
        self.samples = []
        self.stop = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def read(self):
        c, r = self.ct.c_uint(0), self.ct.c_ulonglong(0)
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.ct.byref(c)) != 0:
            return None
        if self.reasons_fn(self.h, self.ct.byref(r)) != 0:
            return None
        return float(c.value), int(r.value)

    def _run(self):
        while not self.stop.is_set():
            v = self.read()
            if v is not None:
                self.samples.append(v)
            time.sleep(self.period)

    def start(self):
        self.thread.start()

    def finish(self):
        self.stop.set()
        self.thread.join(timeout=2.0)
        self.lib.nvmlShutdown()


class ClockSampler:
    """Samples the SM clock and throttle reasons while the timed region runs: NVML polled in
    process every millisecond (the samples reported), and the nvidia-smi loop beside it,
    whose samples are used when NVML cannot be loaded."""

    def __init__(self, local, interval_ms=100):
        self.index = self.device_id(local)
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.skip = 0
        self.nvml = None

    @staticmethod
    def device_id(local):
        """The CUDA device's UUID ("GPU-..."), which nvidia-smi and NVML accept whatever
        CUDA_VISIBLE_DEVICES says; else the index that CUDA_VISIBLE_DEVICES maps it to."""
        try:
            import torch
            u = str(torch.cuda.get_device_properties(local).uuid)
            if u:
                return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
        if local < len(vis) and vis[local].strip().isdigit():
            return int(vis[local])
        return local

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to start: let its first sample arrive, so that the
            # samples after this point fall inside the timed region that follows
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.skip = len(self.lines)
        except Exception:
            self.proc = None
        try:
            self.nvml = _NvmlPoller(self.index)
            self.nvml.start()
        except Exception:
            self.nvml = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.nvml:
            self.nvml.finish()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, sm_max_default):
        """Median SM clock and the throttle reasons seen in the samples taken during the timed
        region: NVML's when it was loadable, else nvidia-smi's (the samples before the region
        when the region was shorter than one interval)."""
        if self.nvml and self.nvml.samples:
            sm = [c for c, _ in self.nvml.samples]
            reasons = sorted(nm for nm, bit in _NvmlPoller.BITS.items()
                             if any(r & bit for _, r in self.nvml.samples))
            return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm),
                    "sm_max_mhz": self.nvml.max_mhz or sm_max_default, "reasons": reasons,
                    "samples": len(sm), "samples_in_region": len(sm),
                    "source": "NVML polled in process every 1 ms during the timed region"}
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        in_region = self.lines[self.skip:]
        for ln in in_region or self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": sm_max_default, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms), "samples_in_region": len(in_region), "source": "nvidia-smi -lms %d" % self.interval_ms}


def cpu_baseline(pb_full, steps, target_s=12.0):
    """The FP64 oracle as it stands, single thread, on a bounded square patch of the workload."""
    import oracle as O
    from paper_2203_05477_gb300 import inputs as I
    n = pb_full.nx
    side = 96
    i0 = n // 2 - side // 2
    sub = lambda a: a.reshape(n, n)[i0:i0 + side, i0:i0 + side].ravel()
    patch = I.Problem(2, side, side, 0, side * pb_full.dx, 0, side * pb_full.dy, pb_full.gamma,
                      sub(pb_full.rho), sub(pb_full.ux), sub(pb_full.uy), sub(pb_full.p))
    s = O.make_solver(2, side, side, dx=patch.dx, dy=patch.dy, gamma=patch.gamma, tau=1e-5, cfl=0.2,
                      tol=1e-10, max_iter=16)
    s.set_primitive(patch.rho, patch.ux, patch.uy, patch.p)
    done, t0 = 0, time.perf_counter()
    while done < steps and (time.perf_counter() - t0) < target_s:
        s.step(1)
        done += 1
    el = time.perf_counter() - t0
    return {"value": side * side * done / el / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "%dx%d centre patch of the workload, %d steps, FP64, single thread, %.1f s" % (side, side, done, el)}


def host_cpu():
    """Core count and CPU model of this host (the cores the CPU baselines run on)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "model": model}


def _oracle_patch_worker(job):
    """One process: the FP64 oracle as it stands on one side x side patch of the quadrant
    workload for `steps` steps; returns (cell-updates, seconds)."""
    n, seed, i0, j0, side, steps = job
    import oracle as O
    from paper_2203_05477_gb300 import inputs as I
    pb = I.quadrants_2d(n, seed=seed)
    sub = lambda a: a.reshape(n, n)[j0:j0 + side, i0:i0 + side].ravel()
    s = O.make_solver(2, side, side, dx=pb.dx, dy=pb.dy, gamma=pb.gamma, tau=1e-5, cfl=0.2, tol=1e-10, max_iter=16)
    s.set_primitive(sub(pb.rho), sub(pb.ux), sub(pb.uy), sub(pb.p))
    t0 = time.perf_counter()
    s.step(steps)
    return side * side * steps, time.perf_counter() - t0


def cpu_baseline_parallel(n, seed, side=64, steps=8):
    """The single-thread oracle run as one process per host core, each on its own patch of
    the workload (patches along the domain's diagonal, all crossing the quadrant fronts):
    whole-host throughput = all processes' cell-updates over the wall time of the slowest."""
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context
    cores = os.cpu_count() or 1
    jobs = []
    for k in range(cores):
        c = int((k + 0.5) * (n - side) / cores)
        jobs.append((n, seed, c, n - side - c, side, steps))
    with ProcessPoolExecutor(max_workers=cores, mp_context=get_context("spawn")) as pool:
        list(pool.map(_oracle_patch_worker, [(n, seed, 0, 0, 8, 1)] * cores))   # start-up and build outside the timing
        t0 = time.perf_counter()
        res = list(pool.map(_oracle_patch_worker, jobs))
        wall = time.perf_counter() - t0
    updates = sum(r[0] for r in res)
    return {"value": updates / wall / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d processes of the single-thread oracle, each on its own %dx%d patch of the workload for %d steps, "
                      "FP64, %.1f s wall" % (cores, side, side, steps, wall)}


def cpu_baseline_sod(target_s=15.0):
    """Configuration 1 on the oracle as it stands, single thread: the 400-cell Sod tube, FP64,
    CFL 0.5, run to t = 0.2."""
    import oracle as O
    from paper_2203_05477_gb300 import inputs as I
    pb = I.sod_400()
    s = O.make_solver(1, pb.nx, dx=pb.dx, gamma=pb.gamma, tau=1e-5, cfl=0.5, t_end=0.2, tol=1e-10, max_iter=16)
    s.set_primitive(pb.rho, pb.ux, None, pb.p)
    t0 = time.perf_counter()
    steps = s.step(100000)
    el = time.perf_counter() - t0
    return {"value": pb.ncell * steps / el / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle", "steps": steps,
            "latency_ms": 1e3 * el, "sample": "the whole run to t = 0.2 (%d steps), FP64, single thread" % steps}


TUBE_BYTES_PER_CELL = 96  # state (3+3 FP32 + 2 float-float frame words) and face predictor (2 FP32), read and written


def bench_tubes(args, n_tubes=4096, seed=0, rank=0):
    """The batched-tube workload: 4096 D1Q4 tubes of 200-8000 cells (seeded states with density
    and pressure ratios up to 1e5 and velocity jumps up to Mach 20), FP32, one launch per call."""
    import torch
    import paper_2203_05477_gb300 as pond
    from paper_2203_05477_gb300 import inputs as I
    bt = I.tube_batch(n_tubes, seed=replica_seed(seed, rank))
    rho, ux, p = I.tube_batch_fields(bt)
    s = pond.BatchSolver(bt.lengths, bt.gammas, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16)
    s.set_primitive(rho, ux, None, p)
    # tuned over the full step count: as tubes stop, the longest tubes set the launch's
    # length, so a short window from the initial state does not rank the variants right
    tune = None if args.no_tune else s.autotune(steps=args.tube_steps, cache=args.tune_cache)
    tv = tune["tube"] if tune else 0
    if args.tube_variant is not None:
        tv = s.variants().index(args.tube_variant)
        s.set_variants(0, 0, tv)
    s.step(max(1, args.warmup))
    d0 = s.sync()
    torch.cuda.synchronize()
    steps = args.tube_steps
    _, done0 = s.status()
    ms, _ = s.step_timed(steps)
    d1 = s.sync()
    status, done1 = s.status()
    ncell = int(bt.lengths.sum())
    updates = float((bt.lengths * (done1 - done0)).sum())  # tubes that stopped count their steps only
    mlups = updates / (ms * 1e-3) / 1e6
    gbs = TUBE_BYTES_PER_CELL * updates / (ms * 1e-3) / 1e9
    out = {"workload": "tubes_4096_seed%d" % seed, "cells": ncell, "steps": steps, "value": mlups, "unit": "MLUPS",
           "ms_per_step": ms / steps, "hbm_gbs": gbs, "bytes_per_cell_update": TUBE_BYTES_PER_CELL,
           "launches": 1, "passes_per_face": (d1["face_iters"] - d0["face_iters"]) / max(1, d1["face_solves"] - d0["face_solves"]),
           "tubes_stopped": int(status.sum()), "cell_updates": updates,
           "note": "tubes that reach a non-physical state stop and are reported; throughput counts performed updates",
           "variant": s.variants()[tv], "autotune_ms": tune["ms"] if tune else None}
    s.close()
    return out


# executed FP32 FLOP per node-pass of the semi-Lagrangian kernels (FFMA x 2 + FADD + FMUL, packed
# forms x 2), counted by ncu on the sl_vs_fv workloads: sl_kernel<float> (D1Q4) 4.124 GFLOP per
# launch over 4.19 M node-passes, sl2_kernel<float> (D2Q16) 41.17 GFLOP over 2.10 M
SL_FLOPS_PER_NODE_PASS = {1: 983.0, 2: 19.6e3}


def time_schemes(pb, cfl, steps):
    import paper_2203_05477_gb300 as pond
    out = {}
    for scheme in ("fv", "sl"):
        s = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=cfl, max_iter=16, scheme=scheme)
        s.set_primitive()
        s.step(5)
        d0 = s.sync()
        ms = s.step_timed(steps)
        d1 = s.sync()
        t = (ms[0] + ms[1]) / steps
        out[scheme] = {"ms_per_step": t, "mlups": pb.ncell / (t * 1e-3) / 1e6,
                       "passes": (d1["face_iters"] - d0["face_iters"]) / max(1, d1["face_solves"] - d0["face_solves"]),
                       "status_ok": d1["status"] == pond.POND_OK}
        if scheme == "sl":
            # the whole step is one kernel: its executed FLOP rate (ALU roofline)
            node_passes = (d1["face_iters"] - d0["face_iters"]) / steps
            out[scheme]["tflops"] = SL_FLOPS_PER_NODE_PASS[pb.dim] * node_passes / (t * 1e-3) / 1e12
        s.close()
    out["fv_over_sl"] = out["fv"]["ms_per_step"] / out["sl"]["ms_per_step"]
    return out


def bench_sl_vs_fv(args, seed=0, rank=0):
    """The paper's cost comparison of its two realizations (Sec. IV: the finite-volume step
    costs about 20% more than the semi-Lagrangian one): the same smooth periodic field
    advanced by each scheme in FP32, device time per step, on D1Q4 (4 M cells, 200 steps)
    and on D2Q16 (1024 x 1024 cells, 50 steps)."""
    from paper_2203_05477_gb300 import inputs as I
    n1, n2 = 1 << 22, 1024
    out = {"d1": {"workload": "smooth_periodic_1d_%d" % n1, "steps": 200},
           "d2": {"workload": "smooth_periodic_2d_%dx%d" % (n2, n2), "steps": 50}}
    out["d1"].update(time_schemes(I.smooth_periodic(1, n1, 1, seed=replica_seed(seed, rank), amp=0.15), 0.3, 200))
    out["d2"].update(time_schemes(I.smooth_periodic(2, n2, n2, seed=replica_seed(seed, rank), amp=0.15), 0.2, 50))
    return out


# algorithmic bytes per cell and step of the D3Q64 kernels with FP32 populations and
# float-float frames: cell state 27 coefficients + 4 frame words (140 B), the faces of a
# cell 3 x (30 coefficients + 4 frame words) (456 B).  The face kernel reads the state and
# the face predictors and writes the faces; the cell kernel reads state and faces and
# writes the state.
D3_FACE_BYTES_PER_CELL = 140 + 3 * 32 + 456
D3_CELL_BYTES_PER_CELL = 140 + 456 + 140
# executed FP32 FLOP per face-pass of face3_kernel<float> (FFMA x 2 + FADD + FMUL), counted by
# ncu on the 64^3 spherical explosion (profiles/face3_kernel_blast64_fp32.md)
D3_FLOPS_PER_FACE_PASS = 33.6e3


def bench_d3q64(args, n=128, steps=20, fp64_steps=3, rank=0):
    """The D3Q64 finite-volume step (Sec. V's three-dimensional extension) on the spherical
    explosion in a box, n^3 cells, FP32 (and FP64): device time per step through
    pond_step_timed, face and cell kernels apart."""
    import paper_2203_05477_gb300 as pond
    from paper_2203_05477_gb300 import inputs as I
    pb = I.spherical_blast_3d(n)
    out = {"workload": "spherical_blast_3d_%d" % n, "cells": pb.ncell, "steps": steps}
    for prec, k in (("fp32", steps), ("fp64", fp64_steps)):
        s = pond.Solver3(pb, precision=prec, tau=1e-5, cfl=0.3, max_iter=16)
        s.set_primitive()
        tune = None if args.no_tune or prec == "fp64" else s.autotune(steps=2, cache=args.tune_cache)
        s.step(2)
        d0 = s.sync()
        ms_face, ms_cell = s.step_timed(k)
        d1 = s.sync()
        t = (ms_face + ms_cell) / k
        out[prec] = {"mlups": pb.ncell / (t * 1e-3) / 1e6, "ms_per_step": t, "face_ms": ms_face / k,
                     "cell_ms": ms_cell / k, "steps": k,
                     "passes_per_face": (d1["face_iters"] - d0["face_iters"]) / max(1, d1["face_solves"] - d0["face_solves"]),
                     "status_ok": d1["status"] == pond.POND_OK}
        if tune is not None:
            names = s.variants()
            out[prec]["variants"] = [names[tune["face"]], [n for n in names if n.startswith("cell3")][tune["cell"]]]
            out[prec]["autotune_ms"] = tune["ms"]
        s.close()
        if prec == "fp32":
            out[prec]["face_passes_per_step"] = (d1["face_iters"] - d0["face_iters"]) / k
    f32 = out["fp32"]
    f32["face_gbs"] = D3_FACE_BYTES_PER_CELL * pb.ncell / (f32["face_ms"] * 1e-3) / 1e9
    f32["cell_gbs"] = D3_CELL_BYTES_PER_CELL * pb.ncell / (f32["cell_ms"] * 1e-3) / 1e9
    f32["face_tflops"] = D3_FLOPS_PER_FACE_PASS * f32["face_passes_per_step"] / (f32["face_ms"] * 1e-3) / 1e12
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_3d(pb)
    return out


def cpu_baseline_3d(pb, side=12, steps=3, target_s=10.0):
    """The FP64 oracle, single thread, on a side^3 patch of the 3D workload that crosses the
    explosion's spherical front."""
    import oracle as O
    from paper_2203_05477_gb300 import inputs as I
    n = pb.nx
    c0 = n // 2 + int(0.4 * n / 2) - side // 2, n // 2 - side // 2, n // 2 - side // 2
    sub = lambda a: np.asarray(a).reshape(n, n, n)[c0[2]:c0[2] + side, c0[1]:c0[1] + side, c0[0]:c0[0] + side].ravel()
    patch = I.Problem3(side, side, side, 0, side * pb.dx, 0, side * pb.dy, 0, side * pb.dz, pb.gamma,
                       sub(pb.rho), sub(pb.ux), sub(pb.uy), sub(pb.uz), sub(pb.p))
    s = O.make_solver(3, side, side, side, dx=patch.dx, dy=patch.dy, dz=patch.dz, gamma=patch.gamma, tau=1e-5,
                      cfl=0.3, tol=1e-10, max_iter=16)
    s.set_primitive3(patch.rho, patch.ux, patch.uy, patch.uz, patch.p)
    done, t0 = 0, time.perf_counter()
    while done < steps and (time.perf_counter() - t0) < target_s:
        s.step(1)
        done += 1
    el = time.perf_counter() - t0
    return {"value": side ** 3 * done / el / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "%d^3 patch across the spherical front, %d steps, FP64, single thread, %.1f s" % (side, done, el)}


def bench_sod(args):
    """Configuration 1: the 400-cell Sod tube on the D1Q4 lattice, FP64 (and FP32), CFL 0.5,
    run to t = 0.2.  The whole problem fits in L2, so the figures are the latency of the run
    and steps per second (graph replay of pond_step), not an HBM fraction."""
    import torch
    import paper_2203_05477_gb300 as pond
    from paper_2203_05477_gb300 import inputs as I
    pb = I.sod_400()
    out = {"workload": "sod_400_t0.2", "cells": pb.ncell}
    for prec in ("fp64", "fp32"):
        s = pond.Solver(pb, precision=prec, tau=1e-5, cfl=0.5, t_end=0.2, max_iter=16)
        s.set_primitive()
        tuned = s.autotune(steps=20)
        names = s.variants()
        s.step(2000)                      # steps after t_end are no-ops; find the step count
        n_steps = s.sync()["steps"]
        reps = []
        for _ in range(3):
            s.set_primitive()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.step(n_steps)
            e1.record(s.stream)
            e1.synchronize()
            reps.append(e0.elapsed_time(e1))
        d = s.sync()
        ms = statistics.median(reps)
        out[prec] = {"steps": int(n_steps), "latency_ms": ms, "steps_per_s": n_steps / (ms * 1e-3),
                     "mlups": pb.ncell * n_steps / (ms * 1e-3) / 1e6, "t": d["t"], "status_ok": d["status"] == pond.POND_OK,
                     "variants": [names[tuned["face"]], [nm for nm in names if nm.startswith("cell")][tuned["cell"]]]}
        s.close()
    return out


def train_predictor(args):
    """The learned face-gauge predictor, trained on the GPU from pairs the plain FP32 solver
    collects on another seed of the quadrant workload (256^2, 100 steps)."""
    import torch
    import paper_2203_05477_gb300 as pond
    from paper_2203_05477_gb300 import inputs as I
    t0 = time.perf_counter()
    tr = pond.Solver(I.quadrants_2d(256, seed=args.seed + 101), precision="fp32", tau=1e-5, cfl=0.2)
    tr.set_primitive()
    pairs = tr.gauge_collect(100, cap=300_000, every=2)
    perm = torch.randperm(pairs.shape[0], device=pairs.device)
    losses = tr.gauge_train(pairs[perm].contiguous(), epochs=6, batch=4096, lr=2e-3)
    params = tr.gauge_params()
    tr.close()
    return params, {"pairs": int(pairs.shape[0]), "epochs": 6, "loss_first": float(losses[0]),
                    "loss_last": float(losses[-1]), "seconds": time.perf_counter() - t0}


def timed_run(pb, params, steps, warmup, learned, variants=None, tune=True):
    """FP32 steps of one 2D workload (optionally with the learned predictor), device time of
    `steps` graph-replayed steps after `warmup` steps; stops early at a non-physical state."""
    import torch
    import paper_2203_05477_gb300 as pond
    s = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16)
    s.set_primitive()
    if learned:
        s.set_gauge_params(params)
        s.gauge_enable(True)
    tuned = None
    if variants is not None:
        s.set_variants(*variants)
    elif tune:
        tuned = s.autotune(steps=2)
    s.step(warmup)
    d0 = s.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    e1.synchronize()
    d1 = s.sync()
    ms = e0.elapsed_time(e1)
    out = {"steps": steps, "mlups": pb.ncell * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
           "passes_per_face": (d1["face_iters"] - d0["face_iters"]) / max(1, d1["face_solves"] - d0["face_solves"]),
           "nonconverged_faces": d1["nonconverged"] - d0["nonconverged"], "status_ok": d1["status"] == pond.POND_OK}
    if tuned is not None:
        names = s.variants()
        out["variants"] = [names[tuned["face"]], [n for n in names if n.startswith("cell")][tuned["cell"]],
                           [n for n in names if n.startswith("step")][tuned["tube"]]]
    s.close()
    return out


def bench_equilibration(pb, steps=50):
    """The equilibration alternative of Sec. II.C against Grad's projection on the same
    workload, FP32, both on the face tile and cell block the equilibration kernels are
    compiled for (face variant 0, cell variant 0): device time per step and passes."""
    import torch
    import paper_2203_05477_gb300 as pond
    out = {}
    for name, eq in (("grad", False), ("equilibration", True)):
        s = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16)
        s.set_primitive()
        s.set_variants(0, 0)
        if eq:
            s.set_equilibration(True)
        s.step(5)
        d0 = s.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        d1 = s.sync()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "mlups": pb.ncell / (ms * 1e-3) / 1e6,
                     "passes_per_face": (d1["face_iters"] - d0["face_iters"]) / max(1, d1["face_solves"] - d0["face_solves"]),
                     "status_ok": d1["status"] == pond.POND_OK}
        s.close()
    out["cost_ratio"] = out["equilibration"]["ms_per_step"] / out["grad"]["ms_per_step"]
    out["note"] = "%d steps of the workload, FP32, face 32x4 cells / 2 CTA per SM, cell 256 threads for both" % steps
    return out


def first_nonphysical_step(pb, limit):
    """Steps the plain FP32 solver takes on a workload before a non-physical state (0: none)."""
    import paper_2203_05477_gb300 as pond
    s = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16)
    s.set_primitive()
    for k in range(1, limit + 1):
        s.step(1)
        if s.sync()["nonphysical"]:
            s.close()
            return k
    s.close()
    return 0


def bench_interface_and_jet(args, params, hbm_peak):
    """Configurations 4 and 5 at their stated sizes, FP32 with and without the learned
    predictor: the shocked perturbed interface (4096 x 1024) over `c4_steps` of its 20 000
    steps, and the Mach-80 jet (4096^2), which the method as read takes to a non-physical
    state within its first steps: it is timed over the steps before that state."""
    from paper_2203_05477_gb300 import inputs as I
    c4 = I.shocked_interface_2d(4096, 1024, seed=args.seed)
    out = {"c4": {"workload": "shocked_interface_4096x1024_seed%d" % args.seed, "cells": c4.ncell,
                  "note": "%d of the stated 20000 steps (the whole 20000-step run stays physical: --c4-steps 20000)"
                          % args.c4_steps}}
    plain = timed_run(c4, params, args.c4_steps, 5, False)
    out["c4"]["fp32"] = plain
    out["c4"]["fp32_learned"] = timed_run(c4, params, args.c4_steps, 5, True)
    out["c4"]["fp32"]["hbm_frac_step"] = 352 * plain["mlups"] * 1e6 / (hbm_peak * 1e9)
    c5 = I.jet_2d(4096, seed=args.seed)
    stop = first_nonphysical_step(c5, 40)
    out["c5"] = {"workload": "jet_4096_seed%d" % args.seed, "cells": c5.ncell, "first_nonphysical_step": stop}
    if stop != 1:
        k = (stop - 1) if stop else 40
        out["c5"]["fp32"] = timed_run(c5, params, k, 0, False)
        out["c5"]["fp32_learned"] = timed_run(c5, params, k, 0, True)
        out["c5"]["note"] = "timed over the %d steps before the first non-physical state (graph-replayed, autotuned)" % k
    return out


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle (the paper ships no code) on host cores."""
    if rank != 0:
        return
    from paper_2203_05477_gb300 import inputs as I
    import oracle as O
    n = args.n
    pb = I.quadrants_2d(n, seed=args.seed)
    side = 48
    i0 = n // 2 - side // 2
    sub = lambda a: a.reshape(n, n)[i0:i0 + side, i0:i0 + side].ravel()
    patch = I.Problem(2, side, side, 0, side * pb.dx, 0, side * pb.dy, pb.gamma, sub(pb.rho), sub(pb.ux), sub(pb.uy), sub(pb.p))
    s = O.make_solver(2, side, side, dx=patch.dx, dy=patch.dy, gamma=patch.gamma, tau=1e-5, cfl=0.2, tol=1e-10, max_iter=16)
    s.set_primitive(patch.rho, patch.ux, patch.uy, patch.p)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    el = time.perf_counter() - t0
    val = side * side * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "quadrants_2d_1024_seed%d" % args.seed,
                                            "sample": "%dx%d centre patch per step" % (side, side)},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": "%dx%d centre patch of the workload per step, FP64, single thread" % (side, side)},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--tube-steps", type=int, default=1000)
    ap.add_argument("--no-tune", action="store_true", help="skip the kernel-variant autotuner (use the defaults)")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file: choices found there are reused without timing (profiling runs)")
    ap.add_argument("--workload", default="quadrants", choices=["quadrants", "tubes", "d3q64", "sl", "learned"],
                    help="tubes / d3q64 / sl / learned: only that measurement (profiling cases)")
    ap.add_argument("--d3-n", type=int, default=128, help="cells per side of the D3Q64 measurement")
    ap.add_argument("--c4-steps", type=int, default=200, help="timed steps of the 4096 x 1024 interface leg")
    ap.add_argument("--tube-variant", default=None,
                    help="run the tube workload with this tube-kernel variant (its full name) instead of the tuner's")
    ap.add_argument("--face-variant", default=None,
                    help="run the headline with this face-kernel variant (its full name) instead of the tuner's")
    ap.add_argument("--quick", action="store_true",
                    help="FP32 timed steps only (no e2e, FP64 or CPU legs): the profiling case")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    import paper_2203_05477_gb300 as pond
    from paper_2203_05477_gb300 import _build, inputs as I

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    pk, pk_kind = peaks()
    if args.workload == "tubes":
        if rank == 0:
            print(json.dumps(bench_tubes(args)), flush=True)
        return
    if args.workload == "d3q64":
        if rank == 0:
            print(json.dumps(bench_d3q64(args, n=args.d3_n)), flush=True)
        return
    if args.workload == "sl":
        if rank == 0:
            print(json.dumps(bench_sl_vs_fv(args)), flush=True)
        return
    if args.workload == "learned":
        # the learned predictor on the headline workload: training, then FP32 steps with it
        if rank == 0:
            params, train = train_predictor(args)
            pbl = I.quadrants_2d(args.n, seed=args.seed)
            out = timed_run(pbl, params, args.steps, args.warmup, True, tune=not args.no_tune)
            out["train"] = train
            print(json.dumps(out), flush=True)
        return
    n = args.n
    pb = I.quadrants_2d(n, seed=replica_seed(args.seed, rank))
    ncell = n * n

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks_(x):
        return max_over_ranks(x, world, device="cuda")

    # ---- headline: FP32 populations, float-float frames
    s = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16)
    s.set_primitive()
    # the autotuner times every compiled face/cell variant on this state and restores it
    tune = None if args.no_tune else s.autotune(steps=3, cache=args.tune_cache)
    fv, cv, sv = (tune["face"], tune["cell"], tune["tube"]) if tune else (0, 0, 0)
    variant_names = s.variants()
    if args.face_variant is not None:
        fv = variant_names.index(args.face_variant)
        s.set_variants(fv, cv, sv)
    s.step(args.warmup)
    d0 = s.sync()
    l0 = s.launch_count()
    stream = s.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        ms_face, ms_cell = s.step_timed(args.steps)
        e1.record(stream)
        barrier()
    el_ms = max_over_ranks_(e0.elapsed_time(e1))
    d1 = s.sync()
    launches = s.launch_count() - l0
    value = aggregate_mlups(ncell, args.steps, el_ms * 1e-3, world)
    face_passes = d1["face_iters"] - d0["face_iters"]
    faces = d1["face_solves"] - d0["face_solves"]
    status_ok = d1["status"] == pond.POND_OK
    s.close()

    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "value": value, "unit": "MLUPS", "ms_per_step": el_ms / args.steps,
                              "face_variant": variant_names[fv], "tune_ms": None if tune is None else tune["ms"],
                              "face_ms": ms_face / args.steps, "cell_ms": ms_cell / args.steps,
                              "passes_per_face": face_passes / max(faces, 1), "status_ok": status_ok}), flush=True)
        return

    # ---- the same workload through the public API with host buffers (e2e)
    pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (pb.rho, pb.ux, pb.uy, pb.p)]
    outs = [torch.empty(ncell, dtype=torch.float64).pin_memory() for _ in range(4)]
    s2 = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16)
    s2.set_variants(fv, cv, sv)
    barrier()
    t0 = time.perf_counter()
    s2.set_primitive(*[a.numpy() for a in pin])
    s2.step(args.steps)
    s2.lib.pond_moments(s2.h, *[o.data_ptr() for o in outs], None, 0)
    barrier()
    e2e_s = max_over_ranks_(time.perf_counter() - t0)
    s2.close()
    e2e = {"value": world * ncell * args.steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 4 * 8 * ncell / args.steps, "d2h_bytes_per_step": 4 * 8 * ncell / args.steps,
           "note": ("pond_set_primitive from pinned host arrays, %d steps, pond_moments to pinned host; "
                    "the steps replay the captured step graph (pond_step), while the device-timed value "
                    "records an event after every kernel (pond_step_timed) to time face and cell kernels "
                    "apart, so e2e can come out slightly above it" % args.steps)}

    # ---- FP32 with the learned face-gauge predictor (trained here on another seed)
    learned, params, train = None, None, None
    if not args.no_learned:
        params, train = train_predictor(args)
        sl = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, max_iter=16)
        sl.set_variants(fv, cv)
        sl.set_primitive()
        sl.set_gauge_params(params)
        sl.gauge_enable(True)
        sl.step(args.warmup)
        dl0 = sl.sync()
        l0e, l1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        l0e.record(sl.stream)
        lf, lc = sl.step_timed(args.steps)
        l1e.record(sl.stream)
        barrier()
        dl1 = sl.sync()
        lms = max_over_ranks_(l0e.elapsed_time(l1e))
        learned = {"value": world * ncell * args.steps / (lms * 1e-3) / 1e6, "unit": "MLUPS",
                   "passes_per_face": (dl1["face_iters"] - dl0["face_iters"]) / max(1, dl1["face_solves"] - dl0["face_solves"]),
                   "predictor_and_face_ms": lf / args.steps, "cell_ms": lc / args.steps, "train": train,
                   "status_ok": dl1["status"] == pond.POND_OK}
        sl.close()

    # ---- plain FP64 on the same GPU
    s3 = pond.Solver(pb, precision="fp64", tau=1e-5, cfl=0.2, max_iter=16)
    s3.set_primitive()
    tune64 = None if args.no_tune else s3.autotune(steps=2, cache=args.tune_cache)
    s3.step(2)
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(s3.stream)
    s3.step(args.fp64_steps)
    f1.record(s3.stream)
    barrier()
    fp64_value = world * ncell * args.fp64_steps / (max_over_ranks_(f0.elapsed_time(f1)) * 1e-3) / 1e6
    s3.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    clocks = clk.summary(pk.get("sm_max_mhz", 2070.0))
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = N_SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    face_ms_avg = ms_face / args.steps
    flops = FLOPS_PER_FACE_PASS * face_passes / args.steps
    achieved = flops / (face_ms_avg * 1e-3) / 1e12
    hbm_peak = pk.get("hbm_gbs", FALLBACK_HBM_GBS)
    face_gbs = FACE_KERNEL_BYTES_PER_CELL * ncell / (face_ms_avg * 1e-3) / 1e9
    step_gbs = STEP_BYTES_PER_CELL * value * 1e6 / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "quadrants_2d_1024_seed%d" % args.seed, "lattice": "D2Q16", "cells": ncell,
                   "precision": "fp32 populations, float-float frames", "cfl": 0.2, "tau": 1e-5,
                   "corrector": "tol 1e-6, max 16 passes", "l2": "working set %.0f MB > L2" % (
                       (ncell * (80 + 2 * 88)) / 1e6), "parallelism": "replicas" if world > 1 else "single",
                   "value_path": "plain FP32 corrector (the faster path here); FP32 + learned predictor in "
                                 "fp32_learned_mlups, plain FP64 in fp64_mlups"},
        "fp32_learned_mlups": None if learned is None else learned["value"],
        "fp64_mlups": fp64_value,
        "hbm_frac_step": step_gbs / hbm_peak,
        "passes_per_face": face_passes / max(faces, 1),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": FACE_KERNEL_DRAM_BYTES.get(variant_names[fv]),
                     "kernel": ("face_kernel<2,float> (%s)" % variant_names[fv]) if sv == 0 else
                               ("step_kernel<2,float> (%s; faces and cell update)" % [nm for nm in variant_names if nm.startswith("step")][sv]),
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_mhz,
                     "face_ms": face_ms_avg, "cell_ms": ms_cell / args.steps,
                     "hbm_gbs": face_gbs, "hbm_frac": face_gbs / hbm_peak,
                     "step_hbm_gbs": step_gbs, "step_bytes_per_cell": STEP_BYTES_PER_CELL,
                     "hbm_peak": hbm_peak, "hbm_peak_source": pk_kind},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pb, steps=20)
        line["cpu_baseline"]["host"] = host_cpu()
    line["fp64"] = {"value": fp64_value, "unit": "MLUPS", "steps": args.fp64_steps, "speedup_fp32": value / fp64_value}
    line["fp32_learned"] = learned
    line["corrector"] = {"passes_per_face": face_passes / max(faces, 1), "status_ok": status_ok}
    line["autotune"] = None if tune is None else {
        "face": variant_names[fv], "cell": [nm for nm in variant_names if nm.startswith("cell")][cv],
        "step": [nm for nm in variant_names if nm.startswith("step")][sv],
        "step_ms": {nm: round(ms, 4) for nm, ms in tune["ms"].items() if nm.startswith("step")},
        "fp64": None if tune64 is None else {"face": tune64["face"], "cell": tune64["cell"]}}
    line["sod_c1"] = bench_sod(args)
    line["equilibration_ablation"] = bench_equilibration(pb)
    if params is not None:
        line.update(bench_interface_and_jet(args, params, hbm_peak))
    tubes = bench_tubes(args, rank=rank)
    tubes["hbm_frac"] = tubes["hbm_gbs"] / hbm_peak
    line["tubes"] = tubes
    line["sl_vs_fv"] = bench_sl_vs_fv(args, rank=rank)
    d3 = bench_d3q64(args, n=args.d3_n, rank=rank)
    d3["fp32"]["cell_hbm_frac"] = d3["fp32"]["cell_gbs"] / hbm_peak
    d3["fp32"]["face_alu_frac"] = d3["fp32"]["face_tflops"] / fp32_peak
    for leg in ("d1", "d2"):
        line["sl_vs_fv"][leg]["sl"]["alu_frac"] = line["sl_vs_fv"][leg]["sl"]["tflops"] / fp32_peak
    line["d3q64"] = d3
    if not args.no_cpu_baseline:
        line["cpu_parallel"] = cpu_baseline_parallel(args.n, args.seed)
        line["cpu_sod_c1"] = cpu_baseline_sod()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
