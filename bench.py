#!/usr/bin/env python
"""Throughput of the full moving-solid D2Q9 step on one GB300.

Workload (default): the precision-study domain, 8192 x 4096 fully periodic
nodes, 2000 non-overlapping disks (radii uniform in 8..20, constant
prescribed velocities with components uniform in +-0.05, seeded), tau drawn
once in [0.55, 1.0].  One step = forces on every disk (conventional and
Galilean-invariant momentum exchange, FP64 reduction) + fused
advection/bounce-back/BGK collision + disk motion + re-rasterisation with
covered/fresh node handling.

Prints one JSON line.  ``value`` is MLUPS (lattice nodes updated per second,
all nodes of the domain, summed over ranks) with every input resident in HBM;
``e2e`` repeats the measurement through the C ABI with host buffers (initial
populations uploaded from pinned host memory inside the timed region, force
records read back to the host every 50 steps).  ``roofline`` relates the
fused advection-collision kernel's algorithmic bytes to the measured HBM copy
bandwidth.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS for stream+collide+GIMEM vs HBM roofline; time-to-drag at 1e-4 rel err"
STORAGE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f32"}
FALLBACK_HBM_GBS = 6800.0
CPU_CROP = (1024, 512)


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp16", "fp64"], default="fp32")
    ap.add_argument("--nx", type=int, default=8192)
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--ndisk", type=int, default=2000)
    ap.add_argument("--collision", choices=["bgk", "mrt"], default="bgk",
                    help="collision model of the main measurement (MRT: the rates of Sec. IV; "
                         "on the 8192 x 4096 workload MRT turns unstable near step 300, so "
                         "use --steps 200)")
    ap.add_argument("--boundary", choices=["halfway", "interpolated"], default="halfway",
                    help="fluid-solid boundary of the main measurement (interpolated: the "
                         "linear interpolated bounce-back of the paper's simulations)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="launch variant of the advection-collision pass (0-5, see lbm.h); "
                         "default: the autotuner's choice")
    ap.add_argument("--overlap", type=int, default=-1, choices=[-1, 0, 1],
                    help="force kernel beside (1) or before (0) the advection-collision kernel; "
                         "default: the autotuner's choice")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e pass, the other precisions and the CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--sed-steps", type=int, default=400)
    ap.add_argument("--precision-horizon", type=int, default=500)
    ap.add_argument("--batch-cases", type=int, default=512)
    ap.add_argument("--warm-start", action="store_true",
                    help="train the warm-start network and measure time to converged drag")
    ap.add_argument("--ws-train", type=int, default=1024)
    ap.add_argument("--ws-test", type=int, default=256)
    ap.add_argument("--ws-epochs", type=int, default=100)
    ap.add_argument("--ws-save", type=str, default="",
                    help="with --warm-start: write the trained parameters here (npz)")
    ap.add_argument("--ws-rho-weight", type=float, default=1.0,
                    help="weight of the density channel in the training loss (the target is "
                         "scaled by it)")
    ap.add_argument("--ws-load", type=str, default="",
                    help="with --warm-start: evaluate these parameters instead of training")
    ap.add_argument("--ws-bench-cases", type=int, default=96,
                    help="held-out channels of the default line's time-to-drag entry")
    ap.add_argument("--batch-converge", type=int, default=0, metavar="STEPS",
                    help="run the 512-channel sweep until every case retires or STEPS steps")
    ap.add_argument("--unet", action="store_true",
                    help="time the warm-start network's forward pass and training step")
    ap.add_argument("--galilean", type=int, default=0, metavar="STEPS",
                    help="free-disk sedimentation in frames moving at V (Sec. III.A), driven by "
                         "Eq. 5 and by Eq. 4: trajectory deviations from V = 0 after STEPS steps")
    ap.add_argument("--galilean-boundary", choices=["halfway", "interpolated"], default="halfway",
                    help="disk boundary of --galilean")
    ap.add_argument("--galilean-frames", type=str, default="0,0.001,0.002,0.01,0.02",
                    help="frame velocities V of --galilean, comma-separated, the first 0")
    ap.add_argument("--galilean-gravity", type=float, default=0.0,
                    help="gravity of --galilean in lattice units (net of buoyancy: g (1 - rho_f/rho_s)); "
                         "0 keeps the net gravity 7.4e-6; the paper's 980 cm/s^2 at its scales "
                         "(dx = 0.4/120 cm, nu = 0.01 cm^2/s, tau 0.6) is 4.03e-4")
    ap.add_argument("--galilean-density", type=float, default=1.5,
                    help="solid/fluid density ratio of --galilean (the paper's 1.003 and 1.03 "
                         "need the interpolated boundary)")
    ap.add_argument("--precision-full", type=int, default=0, metavar="STEPS",
                    help="precision study to STEPS steps on a 2048 x 1024 variant of the workload "
                         "whose disks share one velocity (no overlaps)")
    ap.add_argument("--batch-only", action="store_true",
                    help="measure only the cylinder-sweep batch and print its record")
    ap.add_argument("--batch-warmup", type=int, default=100)
    return ap.parse_args()


def workload(a):
    import workloads as W
    return W.precision_study(nx=a.nx, ny=a.ny, ndisk=a.ndisk)


def workload_name(a):
    return (f"precision-study domain {a.nx}x{a.ny} periodic, {a.ndisk} moving disks r 8-20, "
            f"|v| components <= 0.05")


# ------------------------------------------------------------ distributed

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def kernel_source_hash():
    """Hash of the single-domain advection-collision kernel's sources."""
    h = hashlib.sha256()
    for name in ("k_stream_collide.cu", "k_stream_collide.cuh"):
        with open(os.path.join(ROOT, "paper_1303_0625_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(precision, nx, ny, variant):
    """DRAM bytes per step of the advection-collision pass (the fused kernel,
    plus the slow-node kernels when the variant defers them) from the
    committed ncu summary, if it was taken on the current kernel source with
    the same inline or deferred slow-node path."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh).get(precision)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sha256_16") != kernel_source_hash():
        return None
    if bool(rec.get("deferred", False)) != (variant >= 3):
        return None
    # captured on a smaller domain: traffic scales with the node count
    return rec["dram_bytes_per_launch"] * (nx * ny) / (rec["nx"] * rec["ny"])


def algorithmic_bytes(precision, cells):
    """Per launch of the advection-collision kernel: every node reads and
    writes its nine populations once and reads its 2-byte flags word."""
    return cells * (18 * STORAGE_BYTES[precision] + 2)


# ------------------------------------------------------------ our path

def run_ours(a, ws, rank, local):
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    w = workload(a)
    cells = w["nx"] * w["ny"]
    peaks, peak_kind = measured_peaks()

    def measure(precision, steps, warmup, sample_clocks, collision=0, boundary=0):
        lat = G.Lattice.from_workload(w, precision=G.PRECISION_NAMES[precision], device=local,
                                      stream=stream.cuda_stream, force_ring=512,
                                      collision=collision, boundary=boundary)
        if collision:
            variant = -1  # MRT has one launch shape
        elif a.variant >= 0:
            lat.set_kernel_variant(a.variant)
            variant = a.variant
            if a.overlap >= 0:
                lat.set_force_overlap(a.overlap)
        else:
            # node width and slow-node path of the fused pass, and where the
            # force kernel runs
            variant = lat.autotune(4)
        lat.step(warmup)
        lat.sync()
        lat.set_timing(True)
        launches0 = lat.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(local)
        barrier(ws)
        torch.cuda.synchronize()
        if sample_clocks:
            clocks.__enter__()
            time.sleep(0.3)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if sample_clocks:
            clocks.__exit__(None, None, None)
        lat.sync()  # raises on an unstable run
        ms = e0.elapsed_time(e1)
        k1_ms, k1_n = lat.timing()
        launches = lat.launch_count() - launches0
        nfluid = int((lat.owner() < 0).sum())
        overlap = lat.force_overlap()
        lat.close()
        return dict(ms=ms, k1_avg_ms=k1_ms / max(k1_n, 1), launches=launches, nfluid=nfluid,
                    clocks=clocks.summary() if sample_clocks else None, variant=variant,
                    overlap=overlap)

    interp = a.boundary == "interpolated"
    main = measure(a.precision, a.steps, a.warmup, rank == 0,
                   collision=1 if a.collision == "mrt" else 0,
                   boundary=G.LBM_INTERPOLATED if interp else 0)
    t_max = max_over_ranks(main["ms"], ws)
    value = cells * a.steps * ws / (t_max / 1e3) / 1e6
    bytes_launch = algorithmic_bytes(a.precision, cells)
    achieved = bytes_launch / (main["k1_avg_ms"] / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    traffic = (None if a.collision == "mrt" or interp  # the record is the half-way BGK pass's
               else captured_traffic(a.precision, a.nx, a.ny, main["variant"]))
    kernels = ("k_stream_collide + k_boundary_update" if main["variant"] >= 3 or interp
               else "k_stream_collide")
    if a.collision == "mrt":
        kernels = "k_stream_collide (MRT)"
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": kernels, "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": bytes_launch,
                "bytes_per_node": 18 * STORAGE_BYTES[a.precision] + 2,
                "avg_launch_ms": round(main["k1_avg_ms"], 5),
                "kernel_variant": main["variant"],
                "force_kernel": "beside it (second stream)" if main["overlap"] else "before it",
                "frac_counts": "all nodes of the domain",
                # the method's own work: the fluid nodes only
                "frac_fluid_nodes": round(main["nfluid"] * (18 * STORAGE_BYTES[a.precision] + 2)
                                          / (main["k1_avg_ms"] / 1e3) / 1e9 / peak, 4),
                # the whole step (forces, motion and re-rasterisation included)
                "step_frac": round(bytes_launch / (t_max / a.steps / 1e3) / 1e9 / peak, 4),
                "share_of_step": round(main["k1_avg_ms"] / (main["ms"] / a.steps), 4)}
    line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(t_max / a.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[a.precision], "data": "synthetic",
            "config": {"workload": workload_name(a), "nx": a.nx, "ny": a.ny, "disks": a.ndisk,
                       "tau": round(w["tau"], 6), "precision": a.precision,
                       "storage": {"fp64": "f64", "fp32": "f32 (f - w_i)",
                                   "fp16": "f16 (f - w_i)"}[a.precision],
                       "force_reduction": "f64, both forms every step",
                       "collision": a.collision,
                       "boundary": a.boundary,
                       "l2": "inputs larger than L2 (populations "
                             f"{2 * 9 * cells * STORAGE_BYTES[a.precision] / 1e9:.2f} GB)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "fluid_nodes": main["nfluid"]},
            "roofline": roofline, "gpu_launches": main["launches"], "clocks": main["clocks"]}
    if not a.no_extras and rank == 0:
        line["e2e"] = run_e2e(a, w, local, stream)
        modes = {}
        for prec in ("fp16", "fp64", "fp32"):
            if prec == a.precision:
                continue
            k = max(20, a.steps // 4) if prec != "fp64" else max(10, a.steps // 20)
            m = measure(prec, k, 3, False)
            b = algorithmic_bytes(prec, cells)
            modes[prec] = {"mlups": round(cells * k / (m["ms"] / 1e3) / 1e6, 1), "steps": k,
                           "kernel_gbs": round(b / (m["k1_avg_ms"] / 1e3) / 1e9, 1),
                           "kernel_frac_of_hbm": round(b / (m["k1_avg_ms"] / 1e3) / 1e9 / peak, 4),
                           "ms_per_step": round(m["ms"] / k, 5)}
        # MRT (Sec. IV's rates) on the same workload, FP32 deviation storage
        k = max(20, a.steps // 4)
        m = measure("fp32", k, 3, False, collision=1)
        b = algorithmic_bytes("fp32", cells)
        modes["fp32_mrt"] = {"mlups": round(cells * k / (m["ms"] / 1e3) / 1e6, 1), "steps": k,
                             "kernel_gbs": round(b / (m["k1_avg_ms"] / 1e3) / 1e9, 1),
                             "kernel_frac_of_hbm": round(b / (m["k1_avg_ms"] / 1e3) / 1e9 / peak, 4),
                             "ms_per_step": round(m["ms"] / k, 5)}
        # the interpolated boundary of the paper's simulations (Sec. IV, ref. [40])
        m = measure("fp32", k, 3, False, boundary=G.LBM_INTERPOLATED)
        modes["fp32_interpolated"] = {
            "mlups": round(cells * k / (m["ms"] / 1e3) / 1e6, 1), "steps": k,
            "kernel_gbs": round(b / (m["k1_avg_ms"] / 1e3) / 1e9, 1),
            "kernel_frac_of_hbm": round(b / (m["k1_avg_ms"] / 1e3) / 1e9 / peak, 4),
            "ms_per_step": round(m["ms"] / k, 5)}
        for name, rec in modes.items():  # the whole step against the roofline of its storage
            prec = "fp32" if name.startswith("fp32") else name
            rec["step_frac"] = round(algorithmic_bytes(prec, cells) / (rec["ms_per_step"] / 1e3)
                                     / 1e9 / peak, 4)
        line["modes"] = modes
        line["batch"] = run_batch(a, local, stream, peak)
        line["sedimentation"] = run_sedimentation(a, local, stream, peak)
        line["precision_study"] = run_precision_study(a, w, local, stream)
        line["warm_start"] = run_warm_start_bench(a, local)
        line["cpu_baseline"] = run_cpu_baseline(a, w, a.cpu_seconds)
    elif rank == 0:
        line["e2e"] = None
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(a, local, stream, peak):
    """The cylinder sweep: 512 independent channels (nx 128..1024, ny
    64..512, one fixed disk of radius ny/10 each, Poiseuille inlet, Re
    1..100, tau 0.6, FP32) in one batch: tile shape from the autotuner,
    `every`-step blocks replayed as CUDA graphs with the convergence test
    (drag change below 1e-7 per 100 steps) in each block.  Reports the
    aggregate MLUPS over the steps the active cases took, and the fused
    kernel's bandwidth over the active tiles."""
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G
    import workloads as W

    ws = W.cylinder_sweep(a.batch_cases)
    cells = np.array([w["nx"] * w["ny"] for w in ws], dtype=np.int64)
    t0 = time.time()
    b = G.Batch.from_workloads(ws, precision=G.LBM_FP32_DEV, force_ring=4, device=local,
                               stream=stream.cuda_stream)
    setup_s = time.time() - t0
    variant, tile_rows, persistent = b.autotune(4)
    b.set_convergence(every=100, tol=1e-7, max_steps=2_000_000)
    b.run(a.batch_warmup)
    steps = a.batch_steps
    _, s0, _ = b.state()
    n0 = b.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    active = b.run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st, s1, _ = b.state()
    launches = b.launch_count() - n0
    updates = float((cells * (s1 - s0)).sum())
    # the fused kernel alone, events around every launch
    b.set_timing(True)
    _, s2, _ = b.state()
    b.run(200)
    _, s3, _ = b.state()
    k_ms, k_n = b.timing()
    b.set_timing(False)
    live = cells[(s3 - s2) > 0]
    bytes_launch = float(live.sum()) * (18 * 4 + 2)
    gbs = bytes_launch / (k_ms / max(k_n, 1) / 1e3) / 1e9 if k_n else 0.0
    out = {"workload": f"cylinder sweep: {len(ws)} channels, nx 128..1024, ny 64..512 (even), "
                       "one fixed disk r = ny/10, Poiseuille inlet, Re 1..100, tau 0.6, fp32",
           "cases": len(ws), "cells": int(cells.sum()), "setup_s": round(setup_s, 2),
           "kernel_variant": variant, "tile_rows": tile_rows, "persistent": bool(persistent),
           "steps": steps, "ms": round(ms, 3), "ms_per_step": round(ms / steps, 5),
           "mlups": round(updates / (ms / 1e3) / 1e6, 1), "active_after": active,
           "converged": int((st == G.LBM_CASE_CONVERGED).sum()), "gpu_launches": launches,
           "kernel_gbs": round(gbs, 1), "kernel_frac_of_hbm": round(gbs / peak, 4),
           "kernel_avg_ms": round(k_ms / max(k_n, 1), 5)}
    b.close()
    return out


def run_sedimentation(a, local, stream, peak):
    """Freely moving particles: 200 disks of radius 10 (density ratio 1.5)
    settling under gravity 1e-5 in a 2048 x 8192 box with walls, tau 0.7,
    FP32 populations, FP64 Newton-Euler motion with lubrication below a gap
    of 2.  MLUPS over a bounded number of steps from rest."""
    import torch

    import paper_1303_0625_gb300 as G
    import workloads as W

    w = W.sedimentation()
    cells = w["nx"] * w["ny"]
    lat = G.Lattice.from_workload(w, precision=G.LBM_FP32_DEV, device=local,
                                  stream=stream.cuda_stream, force_ring=64)
    variant = lat.autotune(4)
    lat.step(a.warmup)
    lat.sync()
    steps = a.sed_steps
    y0 = lat.solids()[:, 1].copy()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n0 = lat.launch_count()
    torch.cuda.synchronize()
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat.sync()
    launches = lat.launch_count() - n0
    lat.set_timing(True)
    lat.step(50)
    k_ms, k_n = lat.timing()
    dy = lat.solids()[:, 1] - y0
    lat.close()
    bytes_launch = algorithmic_bytes("fp32", cells)
    gbs = bytes_launch / (k_ms / k_n / 1e3) / 1e9
    return {"workload": "sedimentation: 2048 x 8192 walled box, 200 free disks r 10, density "
                        "ratio 1.5, g 1e-5, tau 0.7, fp32 populations, fp64 rigid-body motion",
            "steps": steps, "ms_per_step": round(ms / steps, 5),
            "mlups": round(cells * steps / (ms / 1e3) / 1e6, 1), "kernel_variant": variant,
            "kernel_gbs": round(gbs, 1), "kernel_frac_of_hbm": round(gbs / peak, 4),
            "gpu_launches": launches,
            "mean_descent": round(float(-dy.mean()), 6)}


def run_precision_study(a, w, local, stream):
    """Force error of the deviation-storage modes against the FP64 mode on
    the precision-study workload (the FP64 mode matches the FP64 oracle to
    1e-12 in the parity tests).  Per horizon: the largest error over all
    disks and both force forms, relative to the larger of the force's
    magnitude and the one-sided pressure force 2 rho0 r / 3 (torque: times r).
    The horizon stops below the step where this overlapping-disk workload
    produces a non-finite density in every mode (about 550)."""
    import numpy as np

    import paper_1303_0625_gb300 as G

    horizons = [1, 10, 100, a.precision_horizon]
    n = horizons[-1]
    radii = np.array([s["r"] for s in w["solids"]])
    rec = {}
    for prec in ("fp64", "fp32", "fp16"):
        lat = G.Lattice.from_workload(w, precision=G.PRECISION_NAMES[prec], device=local,
                                      stream=stream.cuda_stream, force_ring=n)
        rec[prec] = lat.step_record(n)  # [n][nsolid][2][3]
        lat.sync()
        lat.close()
    ref = rec["fp64"]
    f0 = 2.0 * radii / 3.0
    scale = np.empty_like(ref)
    fmag = np.abs(ref).max(axis=0, keepdims=True)
    scale[..., :2] = np.maximum(fmag[..., :2], f0[None, :, None, None])
    scale[..., 2:] = np.maximum(fmag[..., 2:], (f0 * radii)[None, :, None, None])
    # each force's error relative to its own series' largest magnitude (no
    # floor): the error of the net force itself; median and worst over solids
    own = np.abs(ref).max(axis=0, keepdims=True)
    out = {"reference": "fp64 mode on the GPU", "horizons": horizons,
           "scale": "larger of the series' magnitude and 2 rho0 r / 3 (torque: times r)"}
    for prec in ("fp32", "fp16"):
        err = np.abs(rec[prec] - ref) / scale
        out[prec] = [float("%.3g" % err[h - 1].max()) for h in horizons]
        rel_own = np.abs(rec[prec] - ref) / np.where(own > 0, own, 1.0)
        per_solid = [rel_own[:h].max(axis=(0, 2, 3)) for h in horizons]  # worst up to h
        out[prec + "_own_scale_median_worst"] = [
            [float("%.3g" % np.median(v)), float("%.3g" % v.max())] for v in per_solid]
    return out


def run_precision_full(a, local):
    """Force error of the FP32 and FP16 deviation modes against the FP64 mode
    up to a.precision_full steps, on the precision-study recipe with one
    shared disk velocity (no overlaps, so every horizon is computable):
    horizons 1, 10, 100, 1000 and on to the last; same error scales as
    run_precision_study."""
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G
    import workloads as W

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    w = W.precision_study_common_velocity()
    n = a.precision_full
    horizons = sorted({h for h in (1, 10, 100, 1000, 5000, 10000, n) if h <= n})
    radii = np.array([s["r"] for s in w["solids"]])
    f0 = 2.0 * radii / 3.0
    t0 = time.time()
    recs = {}
    for prec in ("fp64", "fp32", "fp16"):
        lat = G.Lattice.from_workload(w, precision=G.PRECISION_NAMES[prec], device=local,
                                      stream=stream.cuda_stream, force_ring=1024)
        lat.set_graph(100)
        rows, done = [], 0
        for h in horizons:  # the record of each horizon's step
            lat.step(h - done - 1)
            rows.append(lat.step_record(1)[0])
            done = h
        lat.sync()
        lat.close()
        recs[prec] = np.array(rows)  # [horizons][nsolid][2][3]
    ref = recs["fp64"]
    out = {"workload": f"{w['nx']}x{w['ny']} periodic, {len(w['solids'])} disks r 8-20 sharing "
                       f"one velocity, tau {w['tau']:.6f}",
           "reference": "fp64 mode on the GPU", "horizons": horizons,
           "seconds": round(time.time() - t0, 1)}
    for prec in ("fp32", "fp16"):
        err = np.abs(recs[prec] - ref)
        scale = np.empty_like(ref)
        fmag = np.abs(ref).max(axis=0, keepdims=True)
        scale[..., :2] = np.maximum(fmag[..., :2], f0[None, :, None, None])
        scale[..., 2:] = np.maximum(fmag[..., 2:], (f0 * radii)[None, :, None, None])
        out[prec] = [float("%.3g" % (err[k] / scale[0]).max()) for k in range(len(horizons))]
    return out


def run_batch_converge(a, local):
    """The 512-channel sweep run the way it is meant to be used: 100-step
    graph blocks with the convergence test (drag change below 1e-7 per 100
    steps), converged cases retiring, until every case has retired or the
    step budget is spent.  Reports the wall time, the retired counts and the
    aggregate MLUPS over the steps the cases actually took."""
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G
    import workloads as W

    torch.cuda.set_device(local)
    ws = W.cylinder_sweep(a.batch_cases)
    cells = np.array([w["nx"] * w["ny"] for w in ws], dtype=np.int64)
    b = G.Batch.from_workloads(ws, precision=G.LBM_FP32_DEV, force_ring=4, device=local)
    shape = b.autotune(4)
    b.set_convergence(every=100, tol=1e-7, max_steps=2_000_000)
    _, s0, _ = b.state()
    t0 = time.perf_counter()
    done, marks = 0, []
    while done < a.batch_converge:
        n = min(10_000, a.batch_converge - done)
        active = b.run(n)
        done += n
        marks.append([done, int(active), round(time.perf_counter() - t0, 2)])
        if active == 0:
            break
    wall = time.perf_counter() - t0
    st, s1, _ = b.state()
    upd = float((cells * (s1 - s0)).sum())
    b.close()
    conv = st == G.LBM_CASE_CONVERGED
    return {"metric": "cylinder sweep run to convergence (drag change < 1e-7 per 100 steps)",
            "cases": len(ws), "launch_shape": list(shape), "budget_steps": a.batch_converge,
            "batch_steps": done, "wall_s": round(wall, 2),
            "converged": int(conv.sum()), "active": int((st == G.LBM_CASE_ACTIVE).sum()),
            "unstable": int((st == G.LBM_CASE_UNSTABLE).sum()),
            "capped": int((st == G.LBM_CASE_CAPPED).sum()),
            "steps_to_converge_pct_0_50_90_100": [int(np.percentile(s1[conv], q)) for q in (0, 50, 90, 100)]
            if conv.any() else None,
            "aggregate_mlups": round(upd / wall / 1e6, 1),
            "active_after_steps": marks[::10] + ([marks[-1]] if len(marks) % 10 != 1 else [])}


def run_unet(a, local, H=128, W=256, B=16, levels=4, base=32):
    """Forward pass and training step of the warm-start U-Net (BF16 tensor
    cores, FP32 accumulation) on a batch of B synthetic 128 x 256 inputs:
    time per call (CUDA events) and algorithmic TFLOP/s of the convolutions
    (forward 2 H W Cout Cin k^2 per sample and layer; a training step counts
    three times the forward)."""
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G
    from paper_1303_0625_gb300 import lbm as L

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flops = 0.0
    cin = 8
    ch = [base << l for l in range(levels)]
    for l, c in enumerate(ch):
        hw = (H >> l) * (W >> l)
        flops += 2 * hw * 9 * (cin * c + c * c)
        cin = c
    for l in range(levels - 2, -1, -1):
        hw = (H >> l) * (W >> l)
        flops += 2 * hw * 9 * ((ch[l + 1] + ch[l]) * ch[l] + ch[l] * ch[l])
    flops += 2 * H * W * ch[0] * 3
    rng = np.random.default_rng(0)
    x = torch.zeros((B, 8, H, W), device=dev)
    x[:, 0] = torch.from_numpy((rng.random((B, H, W)) < 0.1).astype(np.float32)).to(dev)
    x[:, 1] = 0.5
    y = torch.from_numpy(rng.normal(0, 0.3, (B, 3, H, W)).astype(np.float32)).to(dev)
    fl = 1.0 - x[:, 0].contiguous()
    out = torch.empty((B, 3, H, W), device=dev)
    stream = torch.cuda.Stream(device=dev)
    net = G.UNet(H, W, levels=levels, base=base, max_batch=B, seed=0, device=local,
                 stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, fn, mult in (("forward", lambda: L.lbm_unet_forward(net.handle, x, out, B, True), 1),
                           ("train_step", lambda: L.lbm_unet_train_step(net.handle, x, y, fl, B, 1e-4,
                                                                        True), 3)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        n = 10
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        res[name] = {"ms": round(ms, 3), "tflops": round(mult * flops * B / (ms / 1e3) / 1e12, 1)}
    net.close()
    return {"metric": "U-Net forward / training step throughput", "batch": B, "H": H, "W": W,
            "levels": levels, "base": base, "gflop_per_sample_forward": round(flops / 1e9, 2),
            **res}


WS_WEIGHTS = os.path.join(ROOT, "paper_1303_0625_gb300", "weights", "unet_channels_256x128.npz")


def evaluate_warm_start(net, test_all, local, rho_weight=1.0):
    """Time to converged drag on held-out channels, warm (net) against cold:
    steps and wall time (inference included) until every case's drag is within
    1e-4 of the drag its plain run converges to (within 1e-5 of one value
    for 5000 steps), same batch engine and GPU; cases without a steady state
    are left out and counted; prediction error on the held-out steady
    fields."""
    import numpy as np

    import paper_1303_0625_gb300 as G
    from paper_1303_0625_gb300 import warmstart as WS

    # the reference: the plain run until its drag stays within 1e-5 of one
    # value for 50 tests 100 steps apart (above the FP32 drag's round-off
    # noise; no oscillation passes it)
    ref = WS.steady(test_all, tol=WS.REF_TOL, cap=WS.REF_CAP, window=WS.REF_WINDOW, device=local)
    keep = np.flatnonzero(ref["state"] == G.LBM_CASE_CONVERGED)
    test = [test_all[k] for k in keep]
    d_star = ref["drag"][keep]
    cold = WS.time_to_drag(test, d_star, cap=WS.REF_CAP, device=local)
    warm = WS.time_to_drag(test, d_star, net=net, cap=WS.REF_CAP, rho_weight=rho_weight,
                           device=local)
    tdata = WS.dataset(test_all, ref, rho_weight=rho_weight)
    pred = WS.predict(net, tdata["x"]).cpu().numpy()
    m = tdata["fluid"][:, None]
    err = float(np.sqrt(((pred - tdata["y"]) ** 2 * m).sum() / ((tdata["y"] ** 2) * m).sum()))
    # per channel (independent of the channels' scales)
    err_c = [round(float(np.sqrt(((pred[:, c] - tdata["y"][:, c]) ** 2 * m[:, 0]).sum()
                                 / ((tdata["y"][:, c] ** 2) * m[:, 0]).sum())), 4)
             for c in range(3)]
    steps_c, steps_w = cold["steps"].astype(float), warm["steps"].astype(float)
    return {"test_cases": len(test_all), "test_steady": len(test),
            "excluded_unsteady": int(len(test_all) - len(test)),
            "cold": {"wall_s": round(cold["wall"], 3), "batch_steps": int(cold["batch_steps"]),
                     "median_case_steps": float(np.median(steps_c))},
            "warm": {"wall_s": round(warm["wall"], 3), "batch_steps": int(warm["batch_steps"]),
                     "median_case_steps": float(np.median(steps_w)),
                     "fallbacks": int(warm["fallback"].sum()),
                     "settled_elsewhere": int(warm["elsewhere"].sum())},
            "prediction_rel_l2": round(err, 4), "prediction_rel_l2_rho_ux_uy": err_c,
            "wall_speedup": round(cold["wall"] / warm["wall"], 3),
            "median_step_speedup": round(float(np.median(steps_c / np.maximum(steps_w, 1))), 3)}


WS_WORKLOAD = ("256x128 channels, 1-4 fixed disks r 6-16, Re 1..100, tau from Re (>= 0.53), "
               "velocity inlet / pressure outlet, fp32 batch engine")


def run_warm_start(a, local):
    """Learned warm start on 256 x 128 channels with 1-4 fixed disks and Re
    in 1..100: train the U-Net on steady fields the batch engine computes for
    a training set (or load parameters), then evaluate_warm_start on held-out
    cases.  --ws-save writes the trained parameters (FP16) with their
    provenance."""
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G
    import workloads as W
    from paper_1303_0625_gb300 import warmstart as WS

    torch.cuda.set_device(local)
    net = G.UNet(128, 256, levels=4, base=32, max_batch=16, seed=3, device=local)
    out = {"metric": "time-to-drag at 1e-4 rel err, warm vs cold start", "workload": WS_WORKLOAD}
    rho_weight = a.ws_rho_weight
    if a.ws_load:
        z = np.load(a.ws_load)
        net.set_params(z["params"].astype(np.float32))
        rho_weight = float(z["rho_weight"]) if "rho_weight" in z.files else 1.0
        out["parameters"] = a.ws_load
    else:
        t0 = time.time()
        train_cases = W.warm_start_channels(a.ws_train, seed_offset=5)
        runs = WS.steady(train_cases, device=local)
        data = WS.dataset(train_cases, runs, mirror=True, rho_weight=rho_weight)
        t_data = time.time() - t0
        t1 = time.time()
        losses = WS.train(net, data, epochs=a.ws_epochs, batch=16, lr=1e-3, lr_end=1e-5)
        out.update({"train_unstable": int((runs["state"] == G.LBM_CASE_UNSTABLE).sum()),
                    "train_capped": int((runs["state"] == G.LBM_CASE_CAPPED).sum()),
                    "train_cases": len(train_cases), "train_steady": int(len(data["index"])),
                    "train_samples": int(data["x"].shape[0]),
                    "data_seconds": round(t_data, 1), "train_seconds": round(time.time() - t1, 1),
                    "epochs": a.ws_epochs, "final_loss": float("%.4g" % losses[-1]),
                    "rho_weight": rho_weight})
        if a.ws_save:
            os.makedirs(os.path.dirname(os.path.abspath(a.ws_save)), exist_ok=True)
            np.savez(a.ws_save, params=net.params().astype(np.float16), levels=4, base=32,
                     height=128, width=256, inputs="lbm_case_input", rho_weight=rho_weight,
                     trained_on=f"{len(train_cases)} channels (seed offset 5), "
                                f"{int(data['x'].shape[0])} samples with mirrors, "
                                f"{a.ws_epochs} epochs, Adam 1e-3 -> 1e-5",
                     command=f"python bench.py --warm-start --ws-train {a.ws_train} "
                             f"--ws-test {a.ws_test} --ws-epochs {a.ws_epochs} "
                             f"--ws-rho-weight {rho_weight} --ws-save <path>")
            out["saved"] = a.ws_save
    test_all = W.warm_start_channels(a.ws_test, seed_offset=6)
    out.update(evaluate_warm_start(net, test_all, local, rho_weight))
    net.close()
    return out


def run_warm_start_bench(a, local):
    """The default line's time-to-drag entry: the shipped network parameters
    against the plain run on the first ws_bench_cases held-out channels."""
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G
    import workloads as W

    if not os.path.exists(WS_WEIGHTS):
        return {"unavailable": "no trained network parameters in the package"}
    torch.cuda.set_device(local)
    z = np.load(WS_WEIGHTS)
    net = G.UNet(int(z["height"]), int(z["width"]), levels=int(z["levels"]), base=int(z["base"]),
                 max_batch=16, seed=0, device=local)
    net.set_params(z["params"].astype(np.float32))
    t0 = time.time()
    out = {"metric": "time-to-drag at 1e-4 rel err, warm vs cold start", "workload": WS_WORKLOAD,
           "parameters": os.path.relpath(WS_WEIGHTS, ROOT), "trained_on": str(z["trained_on"])}
    rho_weight = float(z["rho_weight"]) if "rho_weight" in z.files else 1.0
    out.update(evaluate_warm_start(net, W.warm_start_channels(a.ws_bench_cases, seed_offset=6),
                                   local, rho_weight))
    out["seconds"] = round(time.time() - t0, 1)
    net.close()
    return out


def run_e2e(a, w, local, stream):
    """Same metric through the C ABI with host buffers: initial populations
    from pinned host memory, force records read back every 50 steps."""
    import numpy as np
    import torch

    import paper_1303_0625_gb300 as G
    from paper_1303_0625_gb300 import lbm as L

    nx, ny = w["nx"], w["ny"]
    lat = G.Lattice.from_workload(w, precision=G.PRECISION_NAMES[a.precision], device=local,
                                  stream=stream.cuda_stream, force_ring=512)
    f0 = torch.empty((9, ny, nx), dtype=torch.float64, pin_memory=True)
    lat.step(1)
    L.lbm_get_populations(lat.handle, f0.numpy())  # a valid state to upload
    if a.variant >= 0:  # the launch shape of the main measurement
        lat.set_kernel_variant(a.variant)
        if a.overlap >= 0:
            lat.set_force_overlap(a.overlap)
    else:
        lat.autotune(4)
    ns = lat.nsolid
    block = 50
    out = torch.empty((2, block, ns, 3), dtype=torch.float64, pin_memory=True)
    # a job of at least 400 steps: the initial state is uploaded once per job,
    # and a 20-step job would time mostly that copy
    steps = max(a.steps, 400)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.lbm_set_populations(lat.handle, f0.numpy())
    t_start = lat.t
    done = 0
    while done < steps:
        n = min(block, steps - done)
        lat.step(n)
        for form in (L.LBM_CME, L.LBM_GME):
            L.lbm_forces(lat.handle, form, t_start + done, n, out[form].numpy())
        done += n
    lat.sync()
    dt = time.perf_counter() - t0
    lat.close()
    h2d = 9 * nx * ny * 8
    d2h = 2 * steps * ns * 3 * 8
    return {"value": round(nx * ny * steps / dt / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": int(h2d / steps), "d2h_bytes_per_step": int(d2h / steps),
            "seconds": round(dt, 4), "steps": steps,
            "what": "C ABI with host buffers: FP64 initial populations uploaded from pinned host "
                    "memory once per job of max(steps, 400) steps, both force forms copied to "
                    "the host every 50 steps"}


# ------------------------------------------------------------ CPU oracle

def crop_workload(w):
    import workloads as W
    return W.crop_disks(w, *CPU_CROP)


def run_cpu_baseline(a, w, seconds):
    """The oracle as it stands on the host's cores: half the time on one
    thread, half with its per-node loops on every core (OpenMP)."""
    import oracle as O
    c = crop_workload(w)

    def timed(threads, budget):
        used = O.set_threads(threads)
        o = O.Oracle(c["nx"], c["ny"], c["tau"])
        for s in c["solids"]:
            o.add_disk(s["cx"], s["cy"], s["r"], s["vx"], s["vy"], s["omega"], s["rho_s"],
                       s["motion"])
        o.step(1)
        n = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget:
            o.step(1)
            n += 1
        dt = time.perf_counter() - t0
        return c["nx"] * c["ny"] * n / dt / 1e6, n, used

    one, n1, _ = timed(1, 0.5 * seconds)
    allc, n, cores = timed(0, 0.5 * seconds)
    O.set_threads(0)
    return {"value": round(allc, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "single_thread": {"value": round(one, 3), "cores": 1, "steps": n1},
            "sample": f"{n} steps of the {c['nx']}x{c['ny']} corner crop of the workload "
                      f"({len(c['solids'])} disks lying wholly inside), FP64 oracle, per-node "
                      f"loops on {cores} threads (OpenMP); single_thread: the same on one"}


def run_reference(a, ws, rank):
    if rank != 0:
        return
    w = workload(a)
    c = crop_workload(w)
    import oracle as O
    cores = O.set_threads(0)  # every host core for the per-node loops
    o = O.Oracle(c["nx"], c["ny"], c["tau"])
    for s in c["solids"]:
        o.add_disk(s["cx"], s["cy"], s["r"], s["vx"], s["vy"], s["omega"], s["rho_s"], s["motion"])
    o.step(a.warmup)
    t0 = time.perf_counter()
    o.step(a.steps)
    dt = time.perf_counter() - t0
    value = c["nx"] * c["ny"] * a.steps / dt / 1e6
    sample = (f"each step: one FP64 oracle step of the {c['nx']}x{c['ny']} corner crop of the "
              f"workload ({len(c['solids'])} disks lying wholly inside), per-node loops on "
              f"{cores} threads (OpenMP)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(dt / a.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "precision": "fp64 oracle",
                       "crop": list(CPU_CROP)},
            "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_galilean(a, local):
    """Galilean test of Sec. III.A on the paper's geometry: a channel 120 wide
    and 1200 long (periodic along its axis x, walls at y = -1/2 and 119.5),
    tau 0.6, a free disk of diameter 30 released at 0.19 of the width.  Fluid,
    walls and disk all start with the frame velocity V along the axis; the
    trajectory relative to the channel, x - x0 - V t, should not depend on V.
    Three series: Eq. 5 drives the disk, Eq. 4 drives it, and Eq. 5 with the
    covered/fresh momenta booked relative to the boundary velocity.
    Density ratio 1.5 and net gravity 7.4e-6 (terminal Reynolds number about
    9) by default: the paper's ratios 1.003 and 1.03 are unstable with half-way
    bounce-back and explicit coupling, and run with the interpolated boundary
    (--galilean-boundary interpolated --galilean-density 1.03 --galilean-frames
    0,0.01,0.02 --galilean-gravity 4.03e-4, the paper's gravity).  FP64.  A
    run that turns unstable is reported as such."""
    import numpy as np
    import torch
    import paper_1303_0625_gb300 as G
    import workloads as W
    torch.cuda.set_device(local)
    width, length, r, tau, every = 120, 1200, 15.0, 0.6, 500
    rs = a.galilean_density
    boundary = 1 if a.galilean_boundary == "interpolated" else 0
    g = a.galilean_gravity if a.galilean_gravity > 0 else 7.4e-6 / (1.0 - 1.0 / rs)
    gnet = g * (1.0 - 1.0 / rs)
    frames = tuple(float(v) for v in a.galilean_frames.split(","))
    assert frames[0] == 0.0, "the first frame velocity is the reference, 0"
    nu = (tau - 0.5) / 3.0
    traj, unstable = {}, {}
    t0 = time.perf_counter()
    series = ((0, 0, "eq5_gme"), (1, 0, "eq4_cme"), (0, 1, "eq5_gme_relative_changes"))
    for cme, relative, _ in series:
        for V in frames:
            w = dict(nx=length, ny=width, tau=tau, rho0=1.0, bc_x=W.PERIODIC, bc_y=W.WALL,
                     u0=(V, 0.0), wall_ux=(V, V), body_force=(0.0, 0.0), gravity=(-g, 0.0),
                     rho_w_mode=0, refill=1, motion_cme=cme, relative_changes=relative,
                     boundary=boundary,
                     solids=[dict(cx=0.6 * length, cy=0.19 * width - 0.5, r=r, vx=V, vy=0.0,
                                  omega=0.0, rho_s=rs, motion=1)])
            lat = G.Lattice.from_workload(w, precision=G.LBM_FP64, force_ring=8, device=local)
            rows = []
            try:
                for k in range(max(1, a.galilean // every)):
                    lat.step(every)
                    st = lat.solids()[0]
                    rows.append([st[0] - 0.6 * length - V * every * (k + 1), st[1], st[2] - V,
                                 st[3], st[4]])
                lat.sync()
            except G.LBMError as e:  # the method's instability, reported by the status word
                unstable[(cme, relative, V)] = f"{e} (within steps {len(rows) * every}.."\
                                               f"{(len(rows) + 1) * every})"
            lat.close()
            traj[(cme, relative, V)] = np.array(rows)
    out = {"metric": "trajectory relative to the channel vs frame velocity V (Sec. III.A)",
           "geometry": f"{length}x{width} channel, disk r {r}, tau {tau}, rho_s/rho_f {rs}, "
                       f"net gravity {gnet:.4g}, {a.galilean_boundary} boundary",
           "steps": max(1, a.galilean // every) * every,
           "seconds": round(time.perf_counter() - t0, 1)}
    for cme, relative, name in series:
        base = traj[(cme, relative, 0.0)]
        bad = {f"V={V}": unstable[(cme, relative, V)] for V in frames
               if (cme, relative, V) in unstable}
        if bad:
            out[name] = {"unstable": bad}
            continue
        rec = {"final_V0": [round(float(v), 5) for v in base[-1]],
               "terminal_Re_V0": round(float(2.0 * r * abs(base[-1][2]) / nu), 3)}
        for V in frames[1:]:
            dev = np.abs(traj[(cme, relative, V)] - base).max(axis=0)
            rec[f"V={V}"] = {"max_dx": round(float(dev[0]), 4), "max_dy": round(float(dev[1]), 4),
                             "max_dvx": float("%.3g" % dev[2]), "max_dvy": float("%.3g" % dev[3]),
                             "max_domega": float("%.3g" % dev[4])}
        out[name] = rec
    return out


def main():
    a = parse()
    ws, rank, local = dist_setup()
    if a.impl == "reference":
        run_reference(a, ws, rank)
    elif a.batch_converge:
        if rank == 0:
            print(json.dumps(run_batch_converge(a, local)), flush=True)
    elif a.unet:
        if rank == 0:
            print(json.dumps(run_unet(a, local)), flush=True)
    elif a.galilean:
        if rank == 0:
            print(json.dumps(run_galilean(a, local)), flush=True)
    elif a.precision_full:
        if rank == 0:
            print(json.dumps(run_precision_full(a, local)), flush=True)
    elif a.warm_start:
        if rank == 0:
            print(json.dumps(run_warm_start(a, local)), flush=True)
    elif a.batch_only:
        import torch
        torch.cuda.set_device(local)
        peaks, _ = measured_peaks()
        rec = run_batch(a, local, torch.cuda.Stream(), float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)))
        if rank == 0:
            print(json.dumps(rec), flush=True)
    else:
        run_ours(a, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
