#!/usr/bin/env python
"""Throughput benchmark of the PSC lattice-Boltzmann + JKR-DEM step on GB300.

A step is one pass of the whole hot path over the workload: bin the particles into lattice
tiles, the fused PSC collide-stream kernel (solid fractions, weights, collision, streaming,
force/torque reduction) and, when the DEM library is built, the DEM sub-steps. The default
workload is the 2048 x 2048 D2Q9 channel with 5000 mobile discs (FP32, 10 DEM sub-steps per
LBM step). The metric is million lattice updates per second (MLUPS), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload on its own
GPU (the method shards by domain, but one replica per GPU is what is measured here); the
timed region is bracketed by a barrier and a device synchronisation, and the slowest rank's
time is used. ``--impl reference`` times the FP64 CPU oracle on the host cores instead (rank
0 only), each step a bounded sub-box of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
KERNEL_FILES = ["psc_kernels.cuh", "psc_pair.cuh", "lattice.cuh", "psc_internal.h", "psc_f32.cu"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--storage", default=None)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dem", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-d3", action="store_true", help="skip the D3Q19 workloads (c3, c3dense, c5, c5dense)")
    ap.add_argument("--d3", default="c3,c3dense,c5,c5dense", help="D3Q19 workloads to time")
    return ap.parse_args(argv)


# ------------------------------------------------------------------- distributed helpers
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(value, world, device=None):
    """Max of a float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and str(device).startswith("cuda"):
            dist.barrier(device_ids=[device.index if hasattr(device, "index") else 0])
        else:
            dist.barrier()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        return self.summary()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------- workload
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_FILES:
        with open(os.path.join(ROOT, "paper_1901_09745_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, storage):
    """DRAM bytes per collide-stream launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get("%s/%s" % (workload, storage))
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["bytes_per_launch"])


WORKLOAD_TEXT = {
    "c2": "D2Q9 2048x2048 channel (walls y), tau 0.7, 5000 mobile discs r~U(4,8) in a band of "
          "solid fraction 0.40, velocities N(0,1e-3), JKR DEM 10 sub-steps per LBM step",
    "c3": "D3Q19 256^3 periodic, tau 0.6, 2000 static spheres r=6, body force 1e-6",
    "c3dense": "D3Q19 256^3 periodic, tau 0.6, 5563 static spheres r=6 (solid fraction 0.3)",
    "c5": "D3Q19 512^3 channel (walls z), tau 0.55, 50000 spheres r~U(3,8) (random sequential addition, "
          "solid fraction 0.31)",
    "c5dense": "D3Q19 512^3 channel (walls z), tau 0.55, 71830 spheres r~U(3,8) at solid fraction 0.45 "
               "(growth and relaxation, many near-contacts), JKR DEM 10 sub-steps per LBM step",
    "c4": "D3Q19 128^3 periodic, tau 0.7, 200 static spheres r=5, body force 1e-6, 500 steps, "
          "checkpoint every 50",
}
DEFAULT_STORAGE = {"c2": "f32", "c3": "f32", "c3dense": "f32", "c5": "f16", "c5dense": "f16", "c4": "f32",
                   "c1": "f64"}
BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}
TIMING_EVERY = 16


def dem_defaults(w):
    """Contact-model parameters of the coupled workloads, in lattice units: E = 2, Poisson
    ratio 0.3, the workload's surface energy (2e-4 for the 2D channel, 2e-2 for the 512^3
    channels), particle/fluid density ratio 3, friction 0.3, critical rolling angle 0.01,
    normal damping 0.3."""
    return dict(E=2.0, poisson=0.3, gamma=w["dem"].get("gamma", 2e-4), density=3.0, mu_f=0.3, theta_crit=0.01,
                alpha_n=0.3, k_t_scale=1.0, eta_t_scale=1.0, dt_dem=1.0 / w["dem"]["substeps"],
                gravity=(0.0, 0.0, 0.0), adhesive=1)


# ---------------------------------------------------------------------------- ours
def run_ours(args, rank, local_rank, world):
    import torch
    import paper_1901_09745_gb300 as P
    import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    P.lib()
    w = synth.workload(args.workload)
    storage = args.storage or DEFAULT_STORAGE.get(args.workload, "f32")
    nx, ny, nz = w["n"]
    ncell = nx * ny * nz
    use_dem = (w.get("dem") is not None) and (not args.no_dem) and hasattr(P.lib(), "dem_create")
    # a stream of our own: the library queues on it and the timing events are recorded on it
    # (events on the legacy default stream would not order with a non-blocking context stream)
    stream = torch.cuda.Stream(device=dev)

    ctx = P.lbm_create(w["lattice"], nx, ny, nz, bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                       storage=storage, stream=stream.cuda_stream)
    P.lbm_set_particles(ctx, w["X"], w["U"], w["Om"], w["r"])
    dem = None
    if use_dem:
        dem = P.dem_create(ctx, **dem_defaults(w))
    substeps = w["dem"]["substeps"] if use_dem else 0

    def one_step():
        if dem is not None:
            P.lbm_coupled_step(ctx, dem, 1, substeps)
        else:
            P.lbm_step(ctx, 1)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize(dev)
    launches0 = P.lbm_get_info(ctx)["launches"]   # counts the DEM's launches too

    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    # the collide-stream kernels' own duration, from CUDA events around every TIMING_EVERY-th
    # step of the timed run (the other steps replay the step's CUDA graph)
    P.lbm_kernel_timing(ctx, max(1, min(TIMING_EVERY, args.steps // 4)))
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        one_step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    k_ms, k_n = P.lbm_kernel_timing(ctx, 0)
    launches1 = P.lbm_get_info(ctx)["launches"]
    ms_max = reduce_max(ms, world, dev)

    # end to end through the C ABI with host (pinned) buffers, copies inside the timed region
    n = len(w["r"])
    hX = torch.from_numpy(np.ascontiguousarray(w["X"])).pin_memory()
    hU = torch.from_numpy(np.ascontiguousarray(w["U"])).pin_memory()
    hO = torch.from_numpy(np.ascontiguousarray(w["Om"])).pin_memory()
    hR = torch.from_numpy(np.ascontiguousarray(w["r"])).pin_memory()
    hF = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    hT = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    h0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.lbm_set_particles(ctx, hX, hU, hO, hR)
        one_step()
        P.lbm_get_forces(ctx, hF, hT)
    torch.cuda.synchronize(dev)
    e2e_s = reduce_max(time.perf_counter() - h0, world, dev)
    P.lbm_destroy(ctx)

    # the collide-stream kernel alone on the same grid and particles, per storage form
    storage_cmp = {}
    if rank == 0:
        for st in ("f32", "f16", "bf16"):
            c2 = P.lbm_create(w["lattice"], nx, ny, nz, bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                              storage=st, stream=stream.cuda_stream)
            P.lbm_set_particles(c2, w["X"], w["U"], w["Om"], w["r"])
            P.lbm_step(c2, 5)
            P.lbm_kernel_timing(c2, 1)
            P.lbm_step(c2, 200)
            kms, kn = P.lbm_kernel_timing(c2, 0)
            P.lbm_destroy(c2)
            us = kms / max(kn, 1) * 1e3
            byt = 2.0 * w["lattice"] * BYTES[st] * ncell
            storage_cmp[st] = {"kernel_us": round(us, 2), "kernel_mlups": round(ncell / us, 1),
                               "bytes_per_cell": 2 * w["lattice"] * BYTES[st],
                               "GBs": round(byt / (us * 1e-6) / 1e9, 1)}

    adjoint = adjoint_timing(P, torch, stream) if (rank == 0 and not args.no_adjoint) else None
    # where the coupled step's time goes: the step, and the DEM call alone (events on the
    # context stream, after the timed region)
    breakdown = None
    if rank == 0 and use_dem:
        cpl = coupled_timing(P, torch, stream, w, storage, steps=300)
        sep = cpl["separate_calls_ms_per_step"]
        breakdown = {"coupled_us": round(cpl["ms_per_step"] * 1e3, 2),
                     "separate_calls_us": round(sep * 1e3, 2),
                     "dem_call_us": round(cpl["dem_ms_per_call"] * 1e3, 2),
                     "lbm_step_with_binning_us": round((sep - cpl["dem_ms_per_call"]) * 1e3, 2),
                     "dem_substeps": cpl["dem_substeps"], "contacts": cpl["contacts"],
                     "note": "coupled_us: lbm_coupled_step (the plain-fluid tiles beside the DEM call); "
                             "separate_calls_us: lbm_step then dem_step"}
    peak0, _ = load_peaks()
    d3 = (d3_workloads(P, torch, stream, [v for v in args.d3.split(",") if v], peak0)
          if (rank == 0 and not args.no_d3) else None)

    if rank != 0:
        return None
    q, sbytes = w["lattice"], BYTES[storage]
    mlups = ncell * args.steps * world / (ms_max * 1e-3) / 1e6
    peak, peak_kind = load_peaks()
    bytes_per_launch = 2.0 * q * sbytes * ncell
    k_avg_s = (k_ms / max(k_n, 1)) * 1e-3
    achieved = bytes_per_launch / k_avg_s / 1e9
    traffic = recorded_traffic(args.workload, storage)
    line = {
        "metric": "PSC collide-stream + DEM step throughput (MLUPS)",
        "value": round(mlups, 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": storage,
        "data": "synthetic (seeded packings, see synth/)",
        "config": {"workload": "%s: %s" % (args.workload, WORKLOAD_TEXT.get(args.workload, "")),
                   "cells": ncell, "particles": n, "dem_substeps": substeps,
                   "dem": "on" if use_dem else "not built",
                   "l2": "inputs larger than L2: %.0f MB of populations read+written per step"
                         % (bytes_per_launch / 1e6),
                   "parallelism": "replicas (one independent domain per GPU)"},
        "roofline": {"bound": "hbm", "kernel": "k_collide_stream with k_fluid_pair and k_collide_overflow "
                                               "(one collide-stream step)", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_us": round(k_avg_s * 1e6, 2), "launches_timed": k_n,
                     # the measured DRAM bytes of a step (ncu) over the same duration
                     "dram_achieved": round(traffic / k_avg_s / 1e9, 1) if traffic else None,
                     "dram_frac": round(traffic / k_avg_s / 1e9 / peak, 4) if traffic else None},
        "e2e": {"value": round(ncell * e2e_steps * world / e2e_s / 1e6, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": int(n * 10 * 8), "d2h_bytes_per_step": int(n * 6 * 8),
                "steps": e2e_steps,
                "path": "per step: lbm_set_particles from page-locked host tensors (copied into the "
                        "library's page-locked staging buffer, read by the upload kernel), lbm_coupled_step "
                        "(lbm_step + dem_step), lbm_get_forces into page-locked host tensors (written by "
                        "the download kernel, with the status words)"},
        "gpu_launches": int(launches1 - launches0),
        "storage_compare": {"note": "collide-stream kernels only (fluid + PSC tiles), static particles, "
                                    "same grid; error against FP64 reported by the test suite",
                            **storage_cmp},
        "clocks": clocks,
    }
    if adjoint is not None:
        line["adjoint"] = adjoint
    if breakdown is not None:
        line["breakdown"] = breakdown
    if d3:
        line["workloads"] = d3
    return line


def collide_stream_us(P, w, storage, stream, steps):
    """Mean duration (us) of one collide-stream step (its kernels, CUDA events on the
    launching stream) on workload w with static particles, after 3 warm-up steps."""
    nx, ny, nz = w["n"]
    ctx = P.lbm_create(w["lattice"], nx, ny, nz, bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                       storage=storage, stream=stream.cuda_stream)
    P.lbm_set_particles(ctx, w["X"], w["U"], w["Om"], w["r"])
    P.lbm_step(ctx, 3)
    P.lbm_kernel_timing(ctx, 1)
    P.lbm_step(ctx, steps)
    kms, kn = P.lbm_kernel_timing(ctx, 0)
    info = P.lbm_get_info(ctx)
    P.lbm_destroy(ctx)
    return kms / max(kn, 1) * 1e3, kn, info


def d3_workloads(P, torch, stream, names, peak):
    """The D3Q19 workloads the metric's FP16-against-FP32 comparison is defined on: per
    workload and storage the collide-stream step's duration, MLUPS and fraction of the
    measured copy bandwidth (algorithmic bytes 2 Q s per cell); for the dense channel also
    the coupled step (collide-stream + 10 DEM sub-steps)."""
    import synth
    out = {}
    for name in names:
        w = synth.workload(name)
        nx, ny, nz = w["n"]
        ncell = nx * ny * nz
        big = ncell > 5e7
        rec = {"workload": "%s: %s" % (name, WORKLOAD_TEXT.get(name, "")), "cells": ncell,
               "particles": int(len(w["r"])), "solid_fraction": round(w["solid_fraction"], 4),
               "default_storage": DEFAULT_STORAGE[name], "storage": {}}
        for st in ("f32", "f16", "bf16"):
            us, kn, info = collide_stream_us(P, w, st, stream, 20 if big else 50)
            byt = 2.0 * w["lattice"] * BYTES[st] * ncell
            gbs = byt / (us * 1e-6) / 1e9
            rec["storage"][st] = {"kernel_us": round(us, 2), "launches_timed": kn,
                                  "kernel_mlups": round(ncell / us, 1), "bytes_per_cell": 2 * w["lattice"] * BYTES[st],
                                  "GBs": round(gbs, 1), "frac": round(gbs / peak, 4),
                                  "overflow_tiles": int(info["overflow_tiles"]),
                                  "max_tile_candidates": int(info["max_tile_candidates"])}
        s32, s16 = rec["storage"]["f32"]["kernel_us"], rec["storage"]["f16"]["kernel_us"]
        rec["f16_over_f32_time"] = round(s16 / s32, 3)
        d = rec["storage"][DEFAULT_STORAGE[name]]
        rec["roofline"] = {"bound": "hbm", "storage": DEFAULT_STORAGE[name], "achieved": d["GBs"], "peak": peak,
                           "unit": "GB/s", "frac": d["frac"], "traffic": None,
                           "algorithmic_bytes_per_launch": 2.0 * w["lattice"] * BYTES[DEFAULT_STORAGE[name]] * ncell,
                           "avg_launch_us": d["kernel_us"]}
        if w.get("dem") is not None:
            rec["coupled"] = coupled_timing(P, torch, stream, w, DEFAULT_STORAGE[name], steps=10)
        out[name] = rec
        del w
    return out


def coupled_timing(P, torch, stream, w, storage, steps):
    """Coupled step (collide-stream + DEM sub-steps) on a D3Q19 workload: time per step with
    CUDA events on the context's stream, the DEM's share, its counters, and the adhesion
    scale against the drag (pull-off force F_C = 3 pi gamma R of the smallest pair against
    the mean hydrodynamic force)."""
    nx, ny, nz = w["n"]
    sub = w["dem"]["substeps"]
    ctx = P.lbm_create(w["lattice"], nx, ny, nz, bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                       storage=storage, stream=stream.cuda_stream)
    P.lbm_set_particles(ctx, w["X"], w["U"], w["Om"], w["r"])
    prm = dem_defaults(w)
    dem = P.dem_create(ctx, **prm)
    for _ in range(3):
        P.lbm_coupled_step(ctx, dem, 1, sub)
        P.lbm_step(ctx, 1)
        P.dem_step(dem, sub)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        P.lbm_coupled_step(ctx, dem, 1, sub)
    ev[1].record(stream)
    for _ in range(steps):
        P.dem_step(dem, sub)
    ev[2].record(stream)
    for _ in range(steps):
        P.lbm_step(ctx, 1)
        P.dem_step(dem, sub)
    ev[3].record(stream)
    torch.cuda.synchronize()
    F, T = P.lbm_get_forces(ctx)
    info = P.dem_get_info(dem)
    pairs, _ = P.dem_get_contacts(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)
    ms = ev[0].elapsed_time(ev[1]) / steps
    dem_ms = ev[1].elapsed_time(ev[2]) / steps
    separate_ms = ev[2].elapsed_time(ev[3]) / steps
    ncell = nx * ny * nz
    rmin = float(np.min(w["r"]))
    FC = 3.0 * np.pi * prm["gamma"] * (rmin / 2.0)
    return {"storage": storage, "ms_per_step": round(ms, 4), "mlups": round(ncell / (ms * 1e3), 1),
            "dem_ms_per_call": round(dem_ms, 4), "separate_calls_ms_per_step": round(separate_ms, 4),
            "dem_substeps": sub, "contacts": int(len(pairs)),
            "dem_overflows": int(info["overflows"]), "dem_solve_failures": int(info["solve_failures"]),
            "skin_violations": int(info["skin_violations"]),
            "pull_off_force_min": FC, "mean_abs_drag": float(np.mean(np.linalg.norm(F, axis=1)))}


def adjoint_timing(P, torch, stream):
    """Adjoint/forward time on the adjoint workload (D3Q19 128^3, 200 static spheres, 500
    steps, checkpoint every 50), FP32 storage: the forward is T plain steps (forces every
    step); the adjoint call runs the same T steps with checkpoints, re-runs each segment and
    sweeps back. Both timed with CUDA events on the context's stream after one untimed call
    (which also sizes the adjoint workspace)."""
    import synth
    w = synth.workload("c4")
    T, K = w["steps"], w["checkpoint"]
    ncell = int(np.prod(w["n"]))
    ctx = P.lbm_create(19, *w["n"], bc=w["bc"], tau=w["tau"], body_force=w["body_force"], storage="f32",
                       stream=stream.cuda_stream)
    P.lbm_set_particles(ctx, w["X"], w["U"], w["Om"], w["r"])
    P.lbm_adjoint_drag(ctx, T, K)
    P.lbm_step(ctx, 20)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    P.lbm_step(ctx, T)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ev[2].record(stream)
    J, dX, dF = P.lbm_adjoint_drag(ctx, T, K)
    ev[3].record(stream)
    torch.cuda.synchronize()
    P.lbm_destroy(ctx)
    fwd, adj = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    q, s = 19, 4
    return {"workload": "c4: " + WORKLOAD_TEXT["c4"], "storage": "f32",
            "fwd_ms": round(fwd, 3), "adjoint_ms": round(adj, 3), "ratio": round(adj / fwd, 3),
            "fwd_mlups": round(ncell * T / (fwd * 1e-3) / 1e6, 1),
            "bytes_per_cell_step": {"forward": 2 * q * s, "adjoint_min": 7 * q * s},
            "ratio_at_roofline": 3.5,
            "note": "adjoint = forward with checkpoints (2Qs) + segment re-run (2Qs) + reverse sweep "
                    "(reads state and adjoint, writes adjoint: 3Qs) per cell and step",
            "J": J, "max_abs_dJdX": float(np.max(np.abs(dX))), "dJdF": [float(v) for v in dF]}


# ------------------------------------------------------------------------ CPU oracle
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample(workload, box, seed_offset=0):
    """A bounded sub-box of the workload (same solid fraction and radius distribution);
    seed_offset draws a different packing (the disjoint samples of the all-core runs)."""
    import synth
    w = synth.workload(workload)
    scale = box / float(w["n"][0])
    return synth.workload(workload, scale=scale, seed_offset=seed_offset)


def _oracle_worker(task):
    """One host process: build its own seeded sub-box, run `steps` oracle steps (or as many
    as fit in `budget_s`), return (lattice updates, seconds)."""
    workload, box, seed_offset, steps, budget_s = task
    import oracle as O
    ws = oracle_sample(workload, box, seed_offset)
    p = O.make_params(ws["lattice"], *ws["n"], bc=ws["bc"], tau=ws["tau"], body_force=ws["body_force"])
    f = O.equilibrium(p, 1.0, (0, 0, 0)).copy()
    ncell = int(np.prod(ws["n"]))
    O.run(p, f, 1, ws["X"], ws["U"], ws["Om"], ws["r"])          # warm
    if steps is None:
        t = time.perf_counter()
        O.run(p, f, 2, ws["X"], ws["U"], ws["Om"], ws["r"])
        t1 = (time.perf_counter() - t) / 2.0
        steps = int(max(2, min(5000, budget_s / max(t1, 1e-6))))
    t = time.perf_counter()
    O.run(p, f, steps, ws["X"], ws["U"], ws["Om"], ws["r"])
    return ncell * steps, time.perf_counter() - t, "x".join(map(str, ws["n"])), steps


def _oracle_pool(tasks):
    """Run the tasks in `len(tasks)` processes started with spawn (a process forked after
    the GPU was used would inherit its state)."""
    import multiprocessing as mp
    import oracle as O
    O.lib()                       # build the oracle once, before the workers load it
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        return pool.map(_oracle_worker, tasks)


def cpu_baseline(workload, budget_s=8.0):
    """The FP64 oracle as it stands on the host cores: one process on one sub-box, then one
    process per core, each on its own seeded sub-box of the same solid fraction and radii
    (the oracle itself is single-threaded and is not changed for this)."""
    box = 256 if workload in ("c2",) else 48
    cores = host_cores()
    one = _oracle_pool([(workload, box, 0, None, budget_s)])[0]
    allc = _oracle_pool([(workload, box, k, None, budget_s) for k in range(cores)])
    mlups_1 = one[0] / one[1] / 1e6
    mlups_all = sum(r[0] for r in allc) / max(r[1] for r in allc) / 1e6
    return {"value": round(mlups_all, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "value_1core": round(mlups_1, 3),
            "sample": "%s sub-boxes %s (same solid fraction and radii; a different seeded packing per "
                      "process), static particles, no DEM, FP64; %d processes x ~%d steps, value = all "
                      "lattice updates / slowest process time; value_1core = one process alone"
                      % (workload, one[2], cores, int(np.mean([r[3] for r in allc])))}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step one LBM step of a 512^2 (2D) or 64^3 (3D)
    sub-box of the workload in every host process (one per core, disjoint seeded
    sub-boxes); the time of a step is the slowest process's."""
    if rank != 0:
        return None
    box = 512 if args.workload == "c2" else 64
    cores = host_cores()
    steps = max(1, args.steps)
    res = _oracle_pool([(args.workload, box, k, steps, None) for k in range(cores)])
    total_lu = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    mlups = total_lu / t / 1e6
    cb = {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
          "sample": "%d processes, each %d LBM steps of its own %s sub-box of %s (static particles, FP64)"
                    % (cores, steps, res[0][2], args.workload)}
    return {"metric": "PSC collide-stream + DEM step throughput (MLUPS)", "value": round(mlups, 3),
            "unit": "MLUPS", "impl": "reference", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": t / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s: %s" % (args.workload, WORKLOAD_TEXT.get(args.workload, ""))},
            "cpu_baseline": cb,
            "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return 0
    import torch
    init_dist(world, "nccl" if torch.cuda.is_available() else "gloo")
    line = run_ours(args, rank, local_rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
