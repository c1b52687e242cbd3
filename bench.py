#!/usr/bin/env python
"""FMM-IPM hot-path benchmark (one JSON line on rank 0).

A step is one pass of the whole hot path over the high-magnification map
workload (kappa_* = 0.45, gamma = 0.45, mean mu = 10; N* = 1.5e6 equal-mass
stars uniform in a disk; 2000^2-pixel map over 200 Einstein radii; ~1.1e8
image-plane cells): quadtree build + upward/downward FMM passes
(lens_fmm_build) and the chunked deflection + IPM map (lens_ipm_map).
``value`` is corner rays deflected per second (whole job), inputs resident
in HBM; ``e2e`` is the same metric through the C ABI with host buffers
(star upload and map download inside the timed region).

--impl reference times the CPU oracle (plain FP64 direct sum of Eq. 1) on the
host cores on a bounded sample of the same rays, in the same unit.
Under torchrun every rank computes its own independent map (seed = rank):
weak scaling, no collective on the data path.
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

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "FMM rays deflected/s at stated error vs GPU direct sum; IPM map time (1xGB300)"
FUSED = {"default": None, "fused": True, "separate": False}
UNIT = "rays/s"
# Fallbacks when the pipe micro-benchmark cannot run: unit counts x the
# maximum SM clock (float32: 152 SMs x 128 lanes x 2 flops; float64: the
# ratio the micro-benchmark measured on this GPU in development, 1/62)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = FP32_PEAK_TFLOPS / 62.0


def measure_pipe_peaks():
    """Run the pipe micro-benchmark (paper_2211_00354_gb300/pipe_peaks.cu,
    built by build()): float32 FMA, paired float32 FMA, float64 FMA and MUFU
    reciprocal rates on this GPU.  None if it is not built or fails."""
    from paper_2211_00354_gb300 import _build
    path = _build.PEAKS_BIN
    if not os.path.exists(path):
        try:
            path = _build.build_peaks()
        except Exception:
            return None
    try:
        out = subprocess.run([path], capture_output=True, text=True, timeout=120)
        if out.returncode != 0:
            return None
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=16)
    ap.add_argument("--leaf", type=int, default=8)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--n-stars", type=int, default=1_500_000)
    ap.add_argument("--npix", type=int, default=2000)
    ap.add_argument("--half-map", type=float, default=100.0)
    ap.add_argument("--h", type=float, default=0.063)
    ap.add_argument("--cap", type=int, default=64)
    ap.add_argument("--refine", type=int, default=0,
                    help="levels of 2x2 refinement of cells over the cap (0: they are dropped)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--shard", default="independent", choices=["independent", "strips"],
                    help="N>1: independent maps per rank (weak scaling) or one map split in "
                         "row strips with a final sum all-reduce (strong scaling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--next-rows", action="store_true",
                    help="also time image finding, the lensed Gaussian source, the lensing "
                         "potential and the map consumers on this workload")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--accuracy-rays", type=int, default=100_000,
                    help="corner rays compared with the CPU oracle (0: skip)")
    ap.add_argument("--workload", default="high_mag",
                    choices=["high_mag", "clustered", "critical", "nfw", "differentiation"],
                    help="high_mag: the high-magnification map (the default line); clustered: "
                         "1e6 lenses in Plummer clusters, 4096^2 map; critical: mu ~ 286 near a "
                         "critical curve, 8192^2 map in chunks; nfw: deflection of a 4096^2 grid "
                         "by a 1e7-particle elliptical NFW halo; differentiation: forward + "
                         "adjoint of a Gaussian-source light-curve loss (1e5 stars, 3e6 rays)")
    ap.add_argument("--map-path", default="default", choices=["default", "fused", "separate"],
                    help="the fused deflection + IPM kernel, the separate kernels, or the "
                         "library's default")
    ap.add_argument("--p-arms", default="8,24",
                    help="high_mag: also time whole maps at these orders (comma list, '' = none)")
    return ap.parse_args()


def workload(args, seed):
    from paper_2211_00354_gb300 import synth
    return synth.c2_high_mag(seed=seed, n=args.n_stars, npix=args.npix, half_map=args.half_map,
                             h=args.h)


def workload_name(args):
    return ("high-magnification map: N*=%d equal-mass stars uniform in a disk, kappa*=0.45, "
            "kappa_s=0, gamma=0.45 (mu=10), %d^2 map over %g ER, h=%g ER, p=%d, leaf=%d, %s"
            % (args.n_stars, args.npix, 2 * args.half_map, args.h, args.p, args.leaf,
               "FP32-bulk" if args.prec == "fp32" else "FP64"))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "lens_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_oracle_rays_per_s(f, budget_s, seed, reps=3):
    """Time the FP64 CPU oracle (direct sum of Eq. 1, OpenMP over the rays, one
    ray per scheduling unit) on random corner rays of the workload grid: a
    calibration run of 4 rays per thread, then `reps` samples of at least 16
    rays per thread sized to budget_s in all; the best rate of the samples."""
    import oracle
    from paper_2211_00354_gb300 import synth
    oracle.build()
    cores = oracle.threads()
    m0 = 4 * cores
    _, x = synth.subsample_grid_rays(seed + 100, f.grid, m0)
    t0 = time.perf_counter()
    oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    rate0 = m0 / max(time.perf_counter() - t0, 1e-9)
    m = int(max(16 * cores, min(1 << 17, rate0 * budget_s / reps)))
    best, spent = 0.0, 0.0
    for k in range(reps):
        _, x = synth.subsample_grid_rays(seed + 101 + k, f.grid, m)
        t0 = time.perf_counter()
        oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
        dt = time.perf_counter() - t0
        spent += dt
        best = max(best, m / dt)
    return best, m, spent, cores, reps


def cpu_oracle_ipm(seed, reps=3):
    """The oracle's IPM (the scalar first-order IPM, cell by cell on one core)
    on the plain-method map (500^2 cells, 100^2 pixels) and on a 200 x 200-
    pixel window of the high-magnification map (its shooting region, 1.1e6
    cells of h = 0.063 ER, cap 64 px), each on the oracle's own deflections:
    best of `reps` wall-clock runs."""
    import oracle
    from paper_2211_00354_gb300 import synth
    oracle.build()
    out = {}
    for name, f, cap in (("plain_map_100px", synth.c1_plain(seed), 0),
                         ("high_mag_window_200px", synth.c2_window(seed), 64)):
        g = f.grid
        y = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, g.corners().reshape(-1, 2))
        y = y.reshape(g.ny + 1, g.nx + 1, 2)
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.ipm_map(y, g.h, f.box, f.npx, f.npy, bbox_cap=cap)
            best = min(best, time.perf_counter() - t0)
        out[name] = {"s": best, "cells": g.n_cells, "cells_per_s": g.n_cells / best,
                     "npix": [f.npx, f.npy], "n_stars": f.n, "bbox_cap_px": cap}
    out["cores"] = 1
    out["kind"] = "oracle (scalar IPM, best of %d)" % reps
    return out


def run_reference(args):
    """The oracle as it stands on the host cores, on the bench workload's
    rays: each step deflects a fresh random sample of its corner rays,
    sized from a calibration run to args.cpu_seconds / steps and to at least
    16 rays per thread (every core busy for the whole step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2211_00354_gb300 import synth
    oracle.build()
    f = workload(args, args.seed)
    cores = oracle.threads()
    m0 = 4 * cores
    _, x = synth.subsample_grid_rays(args.seed + 100, f.grid, m0)
    t0 = time.perf_counter()
    oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
    rate0 = m0 / max(time.perf_counter() - t0, 1e-9)
    m = int(max(16 * cores, min(1 << 17, rate0 * args.cpu_seconds / max(1, args.steps))))
    for k in range(args.warmup):
        pass  # the oracle keeps no state between calls: nothing to warm up
    tot_rays, tot_s = 0, 0.0
    for k in range(args.steps):
        _, x = synth.subsample_grid_rays(args.seed + 200 + k, f.grid, m)
        t0 = time.perf_counter()
        oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, x)
        tot_s += time.perf_counter() - t0
        tot_rays += m
    value = tot_rays / tot_s
    sample = ("%d random corner rays of the workload grid per step (%d per thread), FP64 direct "
              "sum over all %d stars, OpenMP on %d threads" % (m, m // cores, f.n, cores))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# Sources whose code a kernel's ncu figures depend on (a figure recorded
# under profiles/ counts only while these files are unchanged).
PROFILE_SOURCES = {
    "k_ipm_cells": ("ipm.cu", "ipm_warp.cuh", "cx.cuh", "lens_internal.h"),
    "k_eval32": ("eval32.cu", "ipm_warp.cuh", "cx.cuh", "lens_internal.h"),
}


def host_cpu():
    """The host's machine type and CPU model (lscpu's "Model name", else
    /proc/cpuinfo's "model name"), for the CPU baseline."""
    import platform
    import subprocess
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.strip().startswith("Model name:"):
                model = l.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for l in open("/proc/cpuinfo"):
                if l.lower().startswith("model name"):
                    model = l.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"machine": platform.machine(), "model": model, "logical_cpus": os.cpu_count()}


def sources_sha(kernel):
    import hashlib
    h = hashlib.sha256()
    for fn in PROFILE_SOURCES[kernel]:
        with open(os.path.join(HERE, "paper_2211_00354_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_figures(kernel):
    """The machine-readable figures ('name: value' lines) of
    profiles/<kernel>_c2_reduced.md, or {} when the kernel's sources have
    changed since that capture (its 'source-sha256' line)."""
    import re
    try:
        txt = open(os.path.join(HERE, "profiles", kernel + "_c2_reduced.md")).read()
    except OSError:
        return {}
    m = re.search(r"source-sha256: ([0-9a-f]{64})", txt)
    if not m or m.group(1) != sources_sha(kernel):
        return {}
    out = {}
    for key in ("dram-bytes-per-corner-ray", "warp-instructions-per-update",
                "warp-instructions-per-ray", "issue-active-pct"):
        mm = re.search(re.escape(key) + r": ([0-9.eE+-]+)", txt)
        if mm:
            out[key] = float(mm.group(1))
    return out


def next_rows(args, f, g, stars, masses, prec, target, mp, hbm_peak):
    """Device times (CUDA events on the current stream, after one warm-up
    call) of the calls built on top of the map path, on the same workload:
    image finding and the lensed Gaussian source on the whole deflected
    grid (float64 corners, (nx+1)(ny+1) x 16 B read), the lensing potential
    at 2^20 rays of the target region, the finite-source map and a
    log-binned histogram of the map, the map with one level of critical-cell
    refinement (plan built once; beside the same map without it), and the map
    through three lens planes (the stars split in thirds, the shear on the
    nearest plane)."""
    import torch

    from paper_2211_00354_gb300 import lens

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    P = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=args.p, leaf_size=args.leaf,
                     prec=prec, target_box=target)
    y = P.deflect_grid(g)
    nray = y.shape[0] * y.shape[1]
    beta = (0.5 * (f.box[0] + f.box[1]) + 0.37, 0.5 * (f.box[2] + f.box[3]) - 0.21)
    t = timed(lambda: lens.find_images(y, g, beta, max_out=1 << 16))
    cells, _ = lens.find_images(y, g, beta, max_out=1 << 16)
    gbs = 16.0 * nray / t / 1e6
    out["find_images"] = {"ms": t, "cells": g.n_cells, "image_cells": int(cells.shape[0]),
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                       "unit": "GB/s", "frac": gbs / hbm_peak}}
    t = timed(lambda: lens.source_image(y, beta, 0.05))
    gbs = 24.0 * nray / t / 1e6
    out["source_image"] = {"ms": t, "rays": nray,
                           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                        "unit": "GB/s", "frac": gbs / hbm_peak}}
    del y
    gen = torch.Generator().manual_seed(args.seed + 11)
    u = torch.rand((1 << 20, 2), generator=gen, dtype=torch.float64)
    xr = torch.stack([target[0] + (target[1] - target[0]) * u[:, 0],
                      target[2] + (target[3] - target[2]) * u[:, 1]], dim=1).to(stars.device)
    t = timed(lambda: P.potential(xr), reps=3)
    out["potential"] = {"ms": t, "rays": 1 << 20, "rays_per_s": (1 << 20) / (t / 1e3)}
    # critical-cell refinement: cells over the 64-pixel cap split 2 x 2 once
    m2 = torch.empty_like(mp)
    t0 = timed(lambda: P.ipm_map(g, f.box, f.npx, f.npy, bbox_cap=64, out=m2), reps=3)
    t1 = timed(lambda: P.ipm_map(g, f.box, f.npx, f.npy, bbox_cap=64, out=m2, refine_levels=1),
               reps=3)
    _, st1 = P.ipm_map(g, f.box, f.npx, f.npy, bbox_cap=64, out=m2, refine_levels=1)
    out["refined_map"] = {"ms": t1, "ms_unrefined": t0, "refine_levels": 1,
                          "cells_refined": st1["cells_refined"],
                          "cells_dropped": st1["cells_dropped"]}
    P.close()
    # three lens planes
    K = 3
    part = torch.randperm(stars.shape[0], generator=gen).to(stars.device)
    planes = []
    for k in range(K):
        sel = part[k::K]
        planes.append((stars[sel].contiguous(), masses[sel].contiguous(), 0.0,
                       f.gamma if k == 0 else 0.0))
    beta = np.zeros((K, K))
    beta[0, 1], beta[0, 2], beta[1, 2] = 0.2, 0.35, 0.2
    t = timed(lambda: lens.multiplane_ipm_map(planes, beta, g, f.box, f.npx, f.npy, p=args.p,
                                              leaf_size=args.leaf, prec=prec, bbox_cap=64,
                                              out=m2), reps=1)
    _, stm = lens.multiplane_ipm_map(planes, beta, g, f.box, f.npx, f.npy, p=args.p,
                                     leaf_size=args.leaf, prec=prec, bbox_cap=64, out=m2)
    out["multiplane_map"] = {"ms": t, "planes": K, "rays": stm["rays"],
                             "rays_per_s": stm["rays"] / (t / 1e3), "chunks": stm["chunks"]}
    del m2
    t = timed(lambda: lens.map_source(mp, 5.0), reps=3)
    out["map_source"] = {"ms": t, "sigma_px": 5.0, "npix": [f.npx, f.npy]}
    t = timed(lambda: lens.map_histogram(mp.reshape(-1), 1e-2, 1e3, 256, log_bins=True))
    out["map_histogram"] = {"ms": t, "bins": 256, "values": f.npx * f.npy}
    return out


def config_line(args):
    """One JSON line for a workload other than the high-magnification map:
    W untimed warm-up steps, then K steps timed with CUDA events (L2 flushed
    before each), clocks sampled meanwhile.  Map workloads: a step is the
    plan build plus the whole map (value = corner rays/s); nfw: the plan
    build plus the deflection of the whole 4096^2 ray grid (rays/s);
    differentiation: the forward pass (plan build, deflection of 3e6 rays,
    2048-sample light curve) and the backward pass (light-curve gradient,
    adjoint FMM) of the squared light-curve loss (rays/s through both)."""
    import torch
    from paper_2211_00354_gb300 import autograd, lens, synth
    pipes = measure_pipe_peaks()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp32_peak = max(pipes["ffma_tflops"], pipes["ffma2_tflops"]) if pipes else FP32_PEAK_TFLOPS
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    w = args.workload
    if w == "clustered":
        f, p, leaf, cap = synth.c3_clustered(seed=args.seed), 16, 64, 64
        desc = ("clustered PBH field: 1e6 lenses in 1e3 Plummer clusters (a = 0.5 ER), log-normal "
                "masses, kappa*=0.2, kappa_s=0.3, gamma=0.3, 4096^2 map over 100 ER, n0 = 1, "
                "p=16, leaf=64, FP32-bulk, cap 64 px")
    elif w == "critical":
        # leaf 4: 29.5 near pairs per ray instead of 36.5 at leaf 8 (936 against
        # 993 ms a map); p 16 keeps the 2e-5 bound (p 12: 7.6e-5)
        f, p, leaf, cap = synth.c4_critical(seed=args.seed), 16, 4, 64
        desc = ("critical curve: 2e5 stars m ~ U[0.1,1], kappa_s=0.81, kappa*=0.01, gamma=0.17 "
                "(mu ~ 286), 8192^2 map over 2 ER, h = 2.44e-4 ER, p=16, leaf=4, FP32-bulk, cap 64 px")
    elif w == "nfw":
        # leaf 128, p 12: 2.3e5 boxes and 2.9e6 V-list pairs instead of 1.8e6
        # and 2.1e7 at leaf 16, ~200 rays per leaf instead of ~31 (13.3 against
        # 54.9 ms a step; max error 4.8e-7 on sampled rays, p 10: 1.9e-6)
        f, p, leaf, cap = synth.nfw_halo(seed=args.seed), 12, 128, 0
        desc = ("elliptical NFW halo (q = 0.7): 1e7 equal-mass particles, 4096^2 ray grid over "
                "+-2 r_s, p=12, leaf=128, FP32-bulk, deflection only")
    else:
        # p 24 for the float32-bulk step (its gradient within 2.5e-8, normwise,
        # of p 32's); the float64 form stays at p 32
        f, p, leaf, cap = synth.c5_differentiable(seed=args.seed), 24, 16, 0
        desc = ("differentiation: 1e5 stars m ~ U[0.5,1.5], kappa*=0.3, kappa_s=0.2, gamma=0.4, "
                "6000 x 500 cells of h = 0.01 ER (3e6 rays), 2048-sample Gaussian light curve "
                "(sigma 0.05 ER), p=24, leaf=16, FP32-bulk forward and adjoint (float64 "
                "translations); the float64 arm at p=32")
    g = f.grid
    box = (g.x0, g.x0 + g.nx * g.h, g.y0, g.y0 + g.ny * g.h)
    stars, masses = T(f.stars), T(f.masses)
    extra = {}
    if w in ("clustered", "critical"):
        mp = torch.empty((f.npy, f.npx), dtype=torch.float64, device=dev)

        def step():
            P = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=p, leaf_size=leaf,
                             prec=lens.FP32_BULK, target_box=box)
            _, st = P.ipm_map(g, f.box, f.npx, f.npy, bbox_cap=cap, out=mp)
            info = P.info()
            P.close()
            return st, info
    elif w == "nfw":
        # the work counters and the evaluation kernel's time come from one map
        # call over the same grid (the grid kernel with pixel output); a 1024^2
        # map keeps the grid in one chunk (chunks hold at most 64 cells per pixel)
        P = lens.LensFMM(stars, masses, 0.0, 0.0, p=p, leaf_size=leaf, prec=lens.FP32_BULK,
                         target_box=box)
        _, st_w = P.ipm_map(g, box, 1024, 1024)
        assert st_w["chunks"] == 1
        P.close()

        def step():
            P = lens.LensFMM(stars, masses, 0.0, 0.0, p=p, leaf_size=leaf, prec=lens.FP32_BULK,
                             target_box=box)
            P.deflect_grid(g)
            info = P.info()
            P.close()
            return st_w, info
    else:
        rays = T(g.corners().reshape(-1, 2))
        smp = T(synth.light_curve_track(2048, length=5.0))
        sig, wr = 0.05, g.h ** 2
        ft = synth.perturbed(f, seed=args.seed + 1, sd=0.01)
        with torch.no_grad():
            yt = autograd.deflect(T(ft.stars), T(ft.masses), ft.kappa_s, ft.gamma, rays, p=32,
                                  leaf_size=leaf, target_box=box)
            Tk = lens.light_curve(yt, wr, smp, sig)

        split = {"fwd": [], "bwd": []}

        def step(prec=lens.FP32_BULK, record=True):
            st_ = stars.detach().clone().requires_grad_(True)
            ms_ = masses.detach().clone().requires_grad_(True)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y = autograd.deflect(st_, ms_, f.kappa_s, f.gamma, rays,
                                 p=p if prec == lens.FP32_BULK else 32, leaf_size=leaf,
                                 prec=prec, target_box=box)
            loss = ((autograd.light_curve(y, wr, smp, sig) - Tk) ** 2).sum()
            e1.record(stream)
            loss.backward()
            e2.record(stream)
            if record:
                torch.cuda.synchronize()
                split["fwd"].append(e0.elapsed_time(e1))
                split["bwd"].append(e1.elapsed_time(e2))
            return {"rays": float(rays.shape[0])}, None
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    tot, stats, infos = 0.0, [], []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
        stats.append(st); infos.append(info)
    clk = clocks.stop()
    ms = tot / args.steps
    nrays = stats[-1]["rays"] if w != "nfw" else float((g.nx + 1) * (g.ny + 1))
    line = {"metric": METRIC, "value": nrays / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": desc, "n_stars": f.n, "grid": [g.nx, g.ny],
                       "l2": "flushed between steps (256 MiB write)"},
            "clocks": clk, "pipe_peaks": pipes}
    if w != "differentiation":
        st, info = stats[-1], infos[-1]
        K = args.steps
        ms_eval = sum(s_["ms_eval_kernel"] for s_ in stats) / K
        eval_flops = 10.0 * st["p2p_pairs"] + 8.0 * (p + 1) * (st["rays"] + st["m2p_evals"])
        tf = eval_flops / (ms_eval / 1e3) / 1e12
        line["eval_roofline"] = {"bound": "alu", "achieved": tf, "peak": fp32_peak,
                                 "unit": "TFLOP/s", "frac": tf / fp32_peak, "ms": ms_eval}
        line["roofline"] = dict(line["eval_roofline"], kernel="k_eval32 (fused L2P+P2P+M2P)",
                                traffic=None)
        line["phase_ms"] = {"build": sum(i_["ms_build"] for i_ in infos) / K,
                            "tree": sum(i_["ms_tree"] for i_ in infos) / K}
        line["work"] = {"rays": st["rays"], "p2p_pairs": st["p2p_pairs"],
                        "pairs_per_ray": st["p2p_pairs"] / max(st["rays"], 1.0)}
        line["tree"] = {k: info[k] for k in ("n_boxes", "n_active_leaves", "n_v", "n_x", "n_u",
                                             "n_w", "levels")}
        # the float64 far field (M2L over the V lists, P2L over X) of the build
        ms_far = sum(i_["ms_far_local"] for i_ in infos) / K
        if ms_far > 0 and pipes:
            ftf = 4.0 * (p + 1) ** 2 * info["n_v"] / (ms_far / 1e3) / 1e12
            line["far_field_roofline"] = {
                "bound": "fp64", "kernel": "k_far_local (M2L over V, P2L over X)", "achieved": ftf,
                "peak": pipes["dfma_tflops"], "unit": "TFLOP/s", "frac": ftf / pipes["dfma_tflops"],
                "ms": ms_far, "peak_source": "measured: pipe_peaks.cu DFMA",
                "work": "4 (p+1)^2 flops per V pair (P2L over X not counted)"}
            if ms_far > ms_eval:
                line["roofline"] = dict(line["far_field_roofline"], traffic=None)
        if w != "nfw":
            ms_ipm = sum(s_["ms_ipm_kernel"] for s_ in stats) / K
            ipm_bytes = 16.0 * st["rays"] + 8.0 * st["ipm_updates"]
            gbs = ipm_bytes / (ms_ipm / 1e3) / 1e9
            line["ipm_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                    "unit": "GB/s", "frac": gbs / hbm_peak, "ms": ms_ipm}
            if ms_ipm > max(ms_eval, ms_far):
                line["roofline"] = dict(line["ipm_roofline"], kernel="k_ipm_cells+k_ipm_ext",
                                        traffic=None)
            line["map_ms"] = ms
            line["phase_ms"].update({"deflect": st["ms_deflect"], "ipm": st["ms_ipm"],
                                     "eval_kernel": ms_eval, "ipm_kernels": ms_ipm})
            line["ledger"] = {k: st[k] for k in ("area_total", "area_in_map", "area_outside",
                                                 "area_dropped", "cells_dropped", "chunks")}
    else:
        line["config"]["parts"] = "forward (build + deflect + light curve) + backward (light-curve gradient + adjoint FMM)"
        n = args.steps
        line["phase_ms"] = {"forward": sum(split["fwd"][-n:]) / n, "backward": sum(split["bwd"][-n:]) / n}
        # the adjoint FMM alone (lens_deflect_adjoint on this step's plan and
        # rays, a random cotangent), against its near-field transpose: the
        # forward's ray-star pairs (counted by a one-chunk map over the same
        # grid) at ~14 float32 flops each (the complex 1/d and 1/d^2 per pair)
        PA = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=p, leaf_size=leaf,
                          prec=lens.FP32_BULK, target_box=box)
        _, st_a = PA.ipm_map(g, box, 1024, 1024)
        assert st_a["chunks"] == 1
        cot = torch.randn(rays.shape, dtype=torch.float64, device=dev,
                          generator=torch.Generator(device=dev).manual_seed(args.seed + 5))
        PA.adjoint(rays, cot)
        torch.cuda.synchronize()
        ea = torch.cuda.Event(enable_timing=True); eb = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(3):
            PA.adjoint(rays, cot)
        eb.record(stream)
        torch.cuda.synchronize()
        ms_adj = ea.elapsed_time(eb) / 3
        PA.close()
        atf = 14.0 * st_a["p2p_pairs"] / (ms_adj / 1e3) / 1e12
        line["adjoint_roofline"] = {
            "bound": "alu", "kernel": "lens_deflect_adjoint (P2P^T, L2P^T/M2P^T moments, "
            "transposed translations)", "achieved": atf, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": atf / fp32_peak, "ms": ms_adj, "pairs": st_a["p2p_pairs"],
            "work": "14 flops per ray-star pair of the near field (the transposed translations "
                    "and moments not counted)"}
        line["roofline"] = dict(line["adjoint_roofline"], traffic=None)
        # the float64 form of the same step (forward and adjoint in float64)
        for _ in range(2):
            step(lens.FP64, record=False)
        torch.cuda.synchronize()
        split["fwd"].clear(); split["bwd"].clear()
        for _ in range(args.steps):
            step(lens.FP64)
        line["fp64_arm"] = {"ms_per_step": (sum(split["fwd"]) + sum(split["bwd"])) / n,
                            "forward_ms": sum(split["fwd"]) / n, "backward_ms": sum(split["bwd"]) / n}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "high_mag":
        config_line(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2211_00354_gb300 import lens

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the pipe peaks first, in a process of their own (before this one
    # creates its CUDA context)
    pipes = measure_pipe_peaks() if local == 0 else None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2211_00354_gb300 import dist as ldist
    strips = world > 1 and args.shard == "strips"
    f = workload(args, args.seed if strips else args.seed + rank)
    g_full = f.grid
    g = g_full
    if strips:
        r0, nr = ldist.row_strips(g_full.ny, world)[rank]
        g = ldist.strip_grid(g_full, r0, nr)
    prec = lens.FP32_BULK if args.prec == "fp32" else lens.FP64
    target = (g_full.x0, g_full.x0 + g_full.nx * g_full.h, g_full.y0, g_full.y0 + g_full.ny * g_full.h)
    stars = torch.tensor(f.stars, device=dev)
    masses = torch.tensor(f.masses, device=dev)
    mp = torch.empty((f.npy, f.npx), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        P = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=args.p, leaf_size=args.leaf,
                         prec=prec, target_box=target)
        _, st = P.ipm_map(g, f.box, f.npx, f.npy, bbox_cap=args.cap, out=mp,
                          refine_levels=args.refine, fused=FUSED[args.map_path])
        if strips:
            ldist.allreduce_map(mp)  # the path's one exchange: sum of the strip maps
        info = P.info()
        return P, st, info

    for _ in range(args.warmup):
        P, _, _ = step()
        P.close()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    tot_ms, stats, infos = 0.0, [], []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        if not args.no_flush:
            flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P, st, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        tot_ms += e0.elapsed_time(e1)
        stats.append(st)
        infos.append(info)
        P.close()
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms = tot_ms / args.steps
    ms = ldist.max_over_ranks(ms, dev)
    rays_step = stats[-1]["rays"]
    total_rays = ldist.allreduce_ledger({"r": rays_step}, ("r",), dev)["r"] if world > 1 else rays_step
    value = total_rays / (ms / 1e3)

    # ---- kernel-level roofline (live CUDA events inside the library) -----
    K = args.steps
    ms_eval = sum(s["ms_eval_kernel"] for s in stats) / K
    ms_ipm = sum(s["ms_ipm_kernel"] for s in stats) / K
    pairs = stats[-1]["p2p_pairs"]
    m2p = stats[-1]["m2p_evals"]
    eval_flops = 10.0 * pairs + 8.0 * (args.p + 1) * (rays_step + m2p)
    launches = stats[-1]["chunks"]
    eval_tflops = eval_flops / (ms_eval / 1e3) / 1e12 if ms_eval > 0 else 0.0
    if pipes:
        fp32_peak = max(pipes["ffma_tflops"], pipes["ffma2_tflops"])
        fp32_src = "measured: pipe_peaks.cu, max of FFMA and paired FFMA2 (%.1f / %.1f TFLOP/s)" % (
            pipes["ffma_tflops"], pipes["ffma2_tflops"])
        fp64_peak = pipes["dfma_tflops"]
        fp64_src = "measured: pipe_peaks.cu DFMA"
    else:
        fp32_peak, fp32_src = FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
        fp64_peak, fp64_src = FP64_PEAK_TFLOPS, "derived: float32 peak / 62"
    # far field (M2L over the V lists): 2 (p+1)^2 float64 FMAs per V pair
    ms_far = sum(i_.get("ms_far_local", 0.0) for i_ in infos) / K
    far_flops = 4.0 * (args.p + 1) ** 2 * infos[-1]["n_v"]
    far_tflops = far_flops / (ms_far / 1e3) / 1e12 if ms_far > 0 else 0.0
    # IPM algorithmic bytes: the 16 B pixel-coordinate corner read per grid
    # ray plus 8 B (read + write of a float) per atomic map or difference
    # array update
    ipm_bytes = 16.0 * rays_step + 8.0 * stats[-1]["ipm_updates"]
    ipm_gbs = ipm_bytes / (ms_ipm / 1e3) / 1e9 if ms_ipm > 0 else 0.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # DRAM bytes per launch from the ncu figure per corner ray of the reduced
    # case (the traffic is the corner array, in proportion to the rays)
    pf_ipm, pf_eval = profile_figures("k_ipm_cells"), profile_figures("k_eval32")
    ipm_traffic = (pf_ipm["dram-bytes-per-corner-ray"] * rays_step / launches
                   if "dram-bytes-per-corner-ray" in pf_ipm else None)
    eval_traffic = (pf_eval["dram-bytes-per-corner-ray"] * rays_step / launches
                    if "dram-bytes-per-corner-ray" in pf_eval else None)
    # issue slots: warp instructions per map update (ncu, reduced case) x the
    # updates of this map, over the kernels' live time, against one warp
    # instruction per clock per SM sub-partition at the maximum SM clock
    issue_peak = 152 * 4 * 2.070e9
    ipm_issue = None
    if "warp-instructions-per-update" in pf_ipm and ms_ipm > 0:
        wi = pf_ipm["warp-instructions-per-update"] * stats[-1]["ipm_updates"]
        ipm_issue = {"bound": "issue", "kernel": "k_ipm_cells+k_ipm_ext",
                     "achieved": wi / (ms_ipm / 1e3), "peak": issue_peak, "unit": "warp-inst/s",
                     "frac": wi / (ms_ipm / 1e3) / issue_peak,
                     "warp_inst_per_update": pf_ipm["warp-instructions-per-update"],
                     "thread_inst_per_update": pf_ipm["warp-instructions-per-update"] * 32,
                     "issue_active_pct_ncu": pf_ipm.get("issue-active-pct"),
                     "peak_source": "152 SMs x 4 sub-partitions x 1 warp instruction/clock x 2.07 GHz"}
    fused_on = bool(stats[-1].get("fused", 0))
    ms_fused = sum(s_["ms_fused_kernel"] for s_ in stats) / K
    if fused_on:
        # one kernel deflects and maps (the seam cells' pass is ms_ipm): its
        # float32 work against the FP32 peak, and its map updates (8 B each,
        # the only algorithmic traffic once no corner array exists) against HBM
        f_tflops = eval_flops / (ms_fused / 1e3) / 1e12
        f_gbs = 8.0 * stats[-1]["ipm_updates"] / (ms_fused / 1e3) / 1e9
        roof = {"bound": "alu", "kernel": "k_eval32_map (fused deflection + IPM)",
                "achieved": f_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": f_tflops / fp32_peak, "traffic": None, "peak_source": fp32_src,
                "ms_per_launch": ms_fused / launches,
                "map_updates_gbs": f_gbs, "map_updates_frac_of_hbm": f_gbs / hbm_peak,
                "seam_pass_ms": ms_ipm}
    elif ms_eval >= ms_ipm:
        roof = {"bound": "alu", "kernel": "k_eval (fused L2P+P2P+M2P)",
                "achieved": eval_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": eval_tflops / fp32_peak, "traffic": eval_traffic,
                "peak_source": fp32_src, "ms_per_launch": ms_eval / launches}
    else:
        roof = {"bound": "hbm", "kernel": "k_ipm_cells+k_ipm_ext", "achieved": ipm_gbs,
                "peak": hbm_peak, "unit": "GB/s", "frac": ipm_gbs / hbm_peak, "traffic": ipm_traffic,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "ms_per_launch": ms_ipm / launches}

    # ---- accuracy of this configuration vs the GPU FP64 direct sum ------
    extra = {}
    acc_oracle = None
    if not args.no_accuracy and rank == 0:
        from paper_2211_00354_gb300 import synth
        _, xs = synth.subsample_grid_rays(args.seed + 7, g, 4096)
        xs_t = torch.tensor(xs, device=dev)
        P = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=args.p, leaf_size=args.leaf,
                         prec=prec, target_box=target)
        y = P.deflect(xs_t)
        P.close()
        y_ref = lens.direct_deflect(stars, masses, f.kappa_s, f.gamma, xs_t, prec=lens.FP64)
        a = torch.tensor([1 - f.kappa_s - f.gamma, 1 - f.kappa_s + f.gamma], device=dev,
                         dtype=torch.float64)
        al = a * xs_t - y_ref
        mag = al.norm(dim=1)
        err = (y - y_ref).norm(dim=1) / torch.clamp(mag, min=1e-3 * mag.pow(2).mean().sqrt())
        extra["error_vs_gpu_direct_fp64"] = {"max": float(err.max()),
                                             "p99.9": float(torch.quantile(err, 0.999)),
                                             "rays": 4096}
        if args.accuracy_rays > 0 and world == 1:
            # the same plan's deflections against the CPU oracle (FP64 direct
            # sum of Eq. 1) on a random subsample of the grid's corner rays
            import oracle
            oracle.build()
            _, xo = synth.subsample_grid_rays(args.seed + 9, g, args.accuracy_rays)
            xo_t = torch.tensor(xo, device=dev)
            P = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=args.p, leaf_size=args.leaf,
                             prec=prec, target_box=target)
            yg = P.deflect(xo_t).cpu().numpy()
            P.close()
            t0 = time.perf_counter()
            yo = oracle.deflect(f.stars, f.masses, f.kappa_s, f.gamma, xo)
            t_or = time.perf_counter() - t0
            acc_oracle = xo.shape[0] / t_or
            ab = np.array([1 - f.kappa_s - f.gamma, 1 - f.kappa_s + f.gamma])
            al = ab * xo - yo
            mg = np.hypot(al[:, 0], al[:, 1])
            eo = np.hypot(*(yg - yo).T) / np.maximum(mg, 1e-3 * np.sqrt(np.mean(mg ** 2)))
            extra["error_vs_oracle"] = {"max": float(eo.max()),
                                        "p99.9": float(np.quantile(eo, 0.999)),
                                        "normwise": float(np.linalg.norm(yg - yo) / np.linalg.norm(al)),
                                        "rays": int(xo.shape[0]), "oracle_s": t_or}

        def rel_err(yy):
            e = (yy - y_ref).norm(dim=1) / torch.clamp(mag, min=1e-3 * mag.pow(2).mean().sqrt())
            return float(e.max())

        # the FP64 form of the FMM (order 32) on the same field: plan build +
        # deflection of a 512-row band of the workload grid (device time),
        # and its error on the same 4096 corners
        band = ldist.strip_grid(g, g.ny // 2 - 256, 512)
        P64 = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=32, leaf_size=args.leaf,
                           prec=lens.FP64, target_box=target)
        build64 = P64.info()["ms_build"]
        P64.deflect_grid(band, nrows=8)  # warm-up
        t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        P64.deflect_grid(band)
        t1.record(stream)
        torch.cuda.synchronize()
        y64 = P64.deflect(xs_t)
        P64.close()
        extra["fmm_fp64"] = {"p": 32, "deflect_rays_per_s": band.n_rays / (t0.elapsed_time(t1) / 1e3),
                             "rays": band.n_rays, "build_ms": build64,
                             "error_vs_gpu_direct_fp64_max": rel_err(y64)}
        # the same map at other expansion orders: whole maps timed (one warm-up,
        # three timed), their error on the same 4096 corners
        arms = {}
        for pa in [int(t) for t in args.p_arms.split(",") if t.strip()]:
            if pa == args.p:
                continue
            msa, sta = [], None
            for it in range(4):
                flush.fill_(1)
                torch.cuda.synchronize()
                a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                PA = lens.LensFMM(stars, masses, f.kappa_s, f.gamma, p=pa, leaf_size=args.leaf,
                                  prec=prec, target_box=target)
                _, sta = PA.ipm_map(g, f.box, f.npx, f.npy, bbox_cap=args.cap, out=mp,
                                    fused=FUSED[args.map_path])
                a1.record(stream)
                torch.cuda.synchronize()
                if it > 0:
                    msa.append(a0.elapsed_time(a1))
                ya = PA.deflect(xs_t) if it == 3 else None
                PA.close()
            ea = sum(msa) / len(msa)
            fl = 10.0 * sta["p2p_pairs"] + 8.0 * (pa + 1) * (sta["rays"] + sta["m2p_evals"])
            arms[str(pa)] = {"map_ms": ea, "rays_per_s": sta["rays"] / (ea / 1e3),
                             "error_vs_gpu_direct_fp64_max": rel_err(ya),
                             "eval_kernel_ms": sta["ms_eval_kernel"],
                             "ipm_kernels_ms": sta["ms_ipm_kernel"],
                             "eval_tflops": fl / (sta["ms_eval_kernel"] / 1e3) / 1e12}
        extra["order_arms"] = arms
        # GPU direct-sum throughput on the same workload (FP32 and FP64 forms)
        _, xd = synth.subsample_grid_rays(args.seed + 8, g, 1 << 19)
        xd_t = torch.tensor(xd, device=dev)
        for name, pr, nr in (("direct_f32", lens.FP32_BULK, 1 << 19), ("direct_f64", lens.FP64, 1 << 15)):
            xx = xd_t[:nr].contiguous()
            lens.direct_deflect(stars, masses, f.kappa_s, f.gamma, xx[:256].contiguous(), prec=pr)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lens.direct_deflect(stars, masses, f.kappa_s, f.gamma, xx, prec=pr)
            e1.record(stream)
            torch.cuda.synchronize()
            extra[name + "_rays_per_s"] = nr / (e0.elapsed_time(e1) / 1e3)

    # ---- end to end through the C ABI with host buffers ---------------
    e2e = None
    if not args.no_e2e:
        h_stars = torch.tensor(f.stars).pin_memory()
        h_masses = torch.tensor(f.masses).pin_memory()
        h_map = torch.empty((f.npy, f.npx), dtype=torch.float64).pin_memory()
        d_stars = torch.empty_like(stars)
        d_masses = torch.empty_like(masses)
        e_ms = 0.0
        for it in range(1 + args.steps):
            if not args.no_flush:
                flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d_stars.copy_(h_stars, non_blocking=True)
            d_masses.copy_(h_masses, non_blocking=True)
            P = lens.LensFMM(d_stars, d_masses, f.kappa_s, f.gamma, p=args.p, leaf_size=args.leaf,
                             prec=prec, target_box=target)
            P.ipm_map(g, f.box, f.npx, f.npy, bbox_cap=args.cap, out=mp,
                      refine_levels=args.refine, fused=FUSED[args.map_path])
            if strips:
                ldist.allreduce_map(mp)
            h_map.copy_(mp, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            P.close()
            if it > 0:
                e_ms += e0.elapsed_time(e1)
        e_ms /= args.steps
        e_ms = ldist.max_over_ranks(e_ms, dev)
        e2e = {"value": total_rays / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h_stars.numel() * 8 + h_masses.numel() * 8),
               "d2h_bytes_per_step": int(h_map.numel() * 8), "ms_per_step": e_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, m, dt, cores, reps = cpu_oracle_rays_per_s(f, args.cpu_seconds, args.seed)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "best of %d samples of %d random corner rays of the workload grid (%d "
                         "per thread), FP64 direct sum over all %d stars, %.1f s in all"
                         % (reps, m, m // cores, f.n, dt),
               "ipm": cpu_oracle_ipm(args.seed), "host": host_cpu()}
        if acc_oracle is not None:
            cpu["accuracy_sample_rays_per_s"] = acc_oracle

    if rank == 0:
        if args.next_rows:
            extra["next_rows"] = next_rows(args, f, g, stars, masses, prec, target, mp, hbm_peak)
        info = infos[-1]
        st = stats[-1]
        mu_mean = float(mp[int(0.05 * f.npy):int(0.95 * f.npy), int(0.05 * f.npx):int(0.95 * f.npx)].mean())
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if strips else "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "n_stars": f.n, "cells": g.n_cells,
                       "grid": [g.nx, g.ny], "npix": [f.npx, f.npy], "p": args.p,
                       "leaf_size": args.leaf, "bbox_cap_px": args.cap,
                       "refine_levels": args.refine,
                       "l2": "flushed between steps (256 MiB write)" if not args.no_flush else "not flushed",
                       "parallelism": ("one map in %d row strips + map all-reduce" % world if strips
                                       else "independent map per GPU" if world > 1 else "1 GPU")},
            "map_ms": ms, "maps_per_s": (1 if strips else world) / (ms / 1e3),
            "omega_per_s": 10.0 * f.npx * f.npy * f.n * (1 if strips else world) / (ms / 1e3),
            "phase_ms": {"build": info["ms_build"], "tree": info["ms_tree"],
                         "deflect": st["ms_deflect"],
                         "ipm": st["ms_ipm"], "eval_kernel": ms_eval, "ipm_kernels": ms_ipm,
                         "fused_kernel": ms_fused},
            "map_path": "fused" if fused_on else "separate",
            "work": {"rays": rays_step, "p2p_pairs": pairs, "m2p_evals": m2p,
                     "ipm_updates": st["ipm_updates"], "cells_queued": st["cells_queued"],
                     "cells_ext": st["cells_ext"], "rays_evaluated": st["rays_evaluated"],
                     "pairs_per_ray": pairs / rays_step},
            "tree": {k: info[k] for k in ("n_boxes", "n_active_boxes", "n_active_leaves", "n_v",
                                          "n_x", "n_u", "n_w", "levels")},
            "ledger": {k: st[k] for k in ("area_total", "area_in_map", "area_outside",
                                           "area_dropped", "area_degenerate", "cells_dropped",
                                           "cells_refined")},
            "mean_mu_interior": mu_mean,
            "roofline": roof,
            "ipm_roofline": {"bound": "hbm", "achieved": ipm_gbs, "peak": hbm_peak,
                             "unit": "GB/s", "frac": ipm_gbs / hbm_peak},
            "ipm_issue_roofline": ipm_issue,
            "eval_roofline": {"bound": "alu", "achieved": eval_tflops, "peak": fp32_peak,
                              "unit": "TFLOP/s", "frac": eval_tflops / fp32_peak,
                              "peak_source": fp32_src},
            "far_field_roofline": {"bound": "fp64", "kernel": "k_far_local (M2L over V, P2L over X)",
                                   "achieved": far_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                                   "frac": far_tflops / fp64_peak if fp64_peak else None,
                                   "ms": ms_far, "peak_source": fp64_src,
                                   "work": "4 (p+1)^2 flops per V pair (P2L over X not counted)"},
            "pipe_peaks": pipes,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": int(sum(s_["launches"] for s_ in stats) / K
                                + sum(i_["build_launches"] for i_ in infos) / K),
            "wall_s": wall,
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
