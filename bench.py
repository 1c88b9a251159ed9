#!/usr/bin/env python
"""Benchmark of the adaptive black-hole ray tracer on GB300: rays/s of one adaptive render.

One step = one whole adaptive render of the workload (trace the base grid, I_bar_int, then per
level the criterion + interpolation + compaction kernel and the trace of the queued rays), on
inputs already resident (the job's parameters; no input arrays exist).  The L2 is flushed before
every step by writing a 512 MB buffer outside the CUDA-event-timed region.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
Under torchrun with N > 1 every rank renders its own image (replicas: no collective on the data
path); the time is the maximum over ranks and `value` counts the rays of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2103_07417_gb300 import workloads as W  # noqa: E402

# Algorithmic FLOPs per RK4 step of the trace kernel, counting +, -, *, /, sqrt, rsqrt and exp
# as one each (an FMA counts 2): 4 Hamiltonian right-hand sides of 97 (388), the RK4 stage and
# update arithmetic for 6 variables (81), the Keplerian emissivity (44), the polar-turn test (11)
# and the transfer segment (11).  The FP32 and FP64 kernels take the end point's radius from the
# right-hand side there, which is the next step's first stage; the double-float kernel (one rolled
# loop of stages) solves the radius quadratic separately (15 more).  The FP32 pass of the mixed
# path adds the swept-angle accumulation (28).
FLOPS_PER_STEP = {"trace_fp64": 535, "trace_fp32": 563, "trace_df": 550}
# Polarized synchrotron steps, counted from the kernel's formulas (+-10 %): the geodesic (495),
# parallel transport of the polarization covector at the 4 RK4 stages plus its update (1332), the
# synchrotron coefficients in the fluid frame (590) and the exact Stokes segment (590).
FLOPS_PER_STEP_POL = {"trace_fp64": 3007, "trace_fp32": 3035, "trace_df": 3007}
# Fluid-grid (GRMHD-like snapshot) steps, unpolarized: the geodesic and transfer as above (491)
# plus the grid emission instead of the analytic one: angles and cell coordinates (22), the
# trilinear interpolation of 8 fields from 8 cells (147), the Jacobian to Cartesian components and
# u, B (46), u^t from the normalisation (28), b^mu and b^2 (41), the two-temperature plasma state
# (29) and the thermal-synchrotron j_I, alpha_I (164).  The FP32 and FP64 kernels take 1/r and the
# Kerr-Schild F and L of the sample from the geodesic's right-hand side there; the double-float
# kernel evaluates them (18) and the radius (15) itself.
FLOPS_PER_STEP_GRID = {"trace_fp64": 968, "trace_fp32": 996, "trace_df": 1001}
# Algorithmic bytes of one grid sample: 8 cells x 8 FP32 fields (before any cache reuse).
GRID_BYTES_PER_SAMPLE = 256
# Peaks for "alu"-bound kernels, derived from unit counts and the maximum clock: FP32 = 152 SMs x
# 128 lanes x 2 flops x 2.07 GHz; FP64 = GB300's nominal dense FP64 rate.  The bench line's
# fraction uses the measured FMA throughput of this GPU (art_measure_alu_peaks) and quotes these.
PEAK_TFLOPS = {"trace_fp32": 152 * 128 * 2 * 2.07e9 / 1e12, "trace_fp64": 1.25,
               "trace_df": 152 * 128 * 2 * 2.07e9 / 1e12}
PEAK_SOURCE = {"trace_fp32": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
               "trace_df": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (FP32 pipes)",
               "trace_fp64": "nominal GB300 dense FP64"}
# HBM and BF16 denominators: the driver's measurement on this machine (MEASURED_PEAKS.json at the
# repository root), else the pool's earlier measurement.
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        out = {k: float(d[k]) for k in FALLBACK_PEAKS}
        out["source"] = "measured (MEASURED_PEAKS.json)"
        return out
    except (OSError, KeyError, ValueError):
        return {**FALLBACK_PEAKS, "source": "fallback (no MEASURED_PEAKS.json)"}


DTYPE = {"mixed": "f32+f64", "mixed_df": "f32+df32x2", "fp64": "f64", "fp32": "f32",
         "mixed_exact": "f32+df32x2+f64"}
METRIC = "rays/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grmhd_16385", choices=sorted(W.BENCH_WORKLOADS))
    ap.add_argument("--precision", default="mixed_exact",
                    choices=["mixed", "mixed_df", "mixed_exact", "fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-render measurement")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default kernel-form thresholds (skip the autotuner)")
    ap.add_argument("--no-mse", action="store_true",
                    help="skip the time-to-0.1%%-MSE measurement")
    ap.add_argument("--fp64-truth", action="store_true",
                    help="time to 0.1%%-MSE against a full FP64 trace (minutes at 16385^2) "
                         "instead of the full mixed-precision trace")
    ap.add_argument("--heldout", type=int, default=5,
                    help="held-out seeds of the time-to-0.1%%-MSE measurement")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training the block-proposal network and the learned path")
    ap.add_argument("--learn-jobs", type=int, default=2000,
                    help="seeded plain renders whose masks train the proposal network")
    ap.add_argument("--learn-epochs", type=int, default=2)
    ap.add_argument("--no-vis", action="store_true",
                    help="skip the visibility spectra of the 8193^2 grid workload")
    ap.add_argument("--contours", action="store_true",
                    help="IF / FE / MSE of the 8193^2 grid workload over a (R_rel, R_abs) log "
                         "grid (the paper's tolerance study), nothing else")
    ap.add_argument("--single", action="store_true",
                    help="one warm-up and one profiled render, nothing else (for profiler "
                         "captures): prints the stats and the per-launch records")
    ap.add_argument("--batch-only", action="store_true",
                    help="one warm-up and one batched render of the 256-image mixed-parameter batch, "
                         "nothing else (for profiler captures)")
    ap.add_argument("--cnn", action="store_true",
                    help="one forward and one gradient pass of the block-proposal network on a "
                         "seeded 1025 x 1025 lattice, nothing else (for profiler captures)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.device), "-lms", "100"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _base_pixels(params: dict, limit: int | None = None):
    """Pixel indices of the base grid of the workload (optionally an evenly spaced subset)."""
    import numpy as np
    levels = params["levels"]
    s0 = 1 << levels
    nx = s0 * (params["n0x"] - 1) + 1
    jj, ii = np.mgrid[0:params["n0y"], 0:params["n0x"]]
    pix = (jj * s0 * nx + ii * s0).ravel().astype(np.int64)
    if limit is not None and pix.size > limit:
        pix = pix[np.linspace(0, pix.size - 1, limit).astype(np.int64)]
    return pix


def _sampled_on_cpu(params: dict) -> bool:
    """Workloads whose full render takes the oracle too long: polarized ones (several ms per ray)
    and the 8193^2 grid render; the CPU legs trace base-level rays of them instead."""
    return params.get("stokes", 1) == 4 or params.get("emission") == "grid"


def cpu_baseline(params: dict, snap=None, reps: int = 3):
    """The FP64 oracle on the host cores, median of `reps` runs.  Unpolarized analytic
    workloads: one full adaptive render.  Polarized and grid ones: a bounded sample of the
    workload's base level (every 4th base ray: a few seconds per run)."""
    import oracle as O
    job = O.make_job(grid=snap, **params)
    runs = []
    if _sampled_on_cpu(params):
        pix = _base_pixels(params)[::4]
        for _ in range(reps):
            t0 = time.perf_counter()
            _, info = O.trace_pixels(job, pix)
            runs.append((time.perf_counter() - t0, pix.size, int(info["steps"].sum())))
        note = (f"every 4th ray of the {params['n0x']}x{params['n0y']} base level of the workload "
                f"({pix.size} rays)")
    else:
        for _ in range(reps):
            t0 = time.perf_counter()
            img, mask, st = O.render(job, None)
            runs.append((time.perf_counter() - t0, int(st["rays_traced"]), int(st["steps"])))
        note = "one full adaptive render of the workload"
    dt, rays, steps = sorted(runs)[len(runs) // 2]
    cores = O.get_threads()
    # one core: every 64th base-level ray (a bounded sample of a few seconds), median of reps
    pix1 = _base_pixels(params)[::64]
    O.set_threads(1)
    t1 = []
    try:
        for _ in range(reps):
            t0 = time.perf_counter()
            O.trace_pixels(job, pix1)
            t1.append(time.perf_counter() - t0)
    finally:
        O.set_threads(cores)
    dt1 = statistics.median(t1)
    return {"value": rays / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": note + f" by the FP64 oracle (OpenMP over rays, all host cores), median of {reps}",
            "seconds": dt, "rays": rays, "steps_per_s": steps / dt,
            "single_core": {"value": pix1.size / dt1, "unit": "rays/s", "cores": 1,
                            "sample": f"every 64th base-level ray ({pix1.size} rays), median of {reps}",
                            "seconds": dt1}}


def max_over_ranks(t_local: float, dist=None, device=None) -> float:
    """The slowest rank's time (an all-reduce MAX over the process group); t_local alone when
    the run has one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return t_local
    import torch
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(rays_per_step: int, steps: int, world: int, t_max: float) -> float:
    """Replicas: every rank renders its own copy of the workload, so the job traces
    rays_per_step x steps rays on each of `world` ranks within the slowest rank's time."""
    return rays_per_step * steps * world / t_max


def flip_distances(params: dict, ref_plane, mask_ref, mask, norm: float, cap: int = 2000):
    """For every point whose mask differs from the FP64 render's (at most `cap` of them): the
    relative distance of the FP64 render's decision from flipping, from the oracle's estimates
    (Eqs. epabs, eprel) on the FP64 image's level lattice around the point."""
    import numpy as np
    import oracle as O
    m0, m1 = mask_ref.cpu().numpy(), mask.cpu().numpy()
    jj, ii = np.nonzero(m0 != m1)
    N = params["levels"]
    img = None
    out = []
    for i, j in list(zip(ii, jj))[:cap]:
        if img is None:
            img = ref_plane.cpu().numpy()
        k = N
        while k > 0 and i % (1 << (N - k + 1)) == 0 and j % (1 << (N - k + 1)) == 0:
            k -= 1
        s = 1 << (N - k)
        # a window of the level-k lattice around the point (the stencil reaches 3 lattice steps)
        li, lj = i // s, j // s
        L = img[::s, ::s]
        x0, y0 = max(0, (li - 8) & ~1), max(0, (lj - 8) & ~1)
        x1, y1 = min(L.shape[1], li + 9), min(L.shape[0], lj + 9)
        win = np.ascontiguousarray(L[y0:y1, x0:x1])
        # keep the image's own edges where the window meets them (the edge rule depends on it)
        if x0 > 0 or y0 > 0 or x1 < L.shape[1] or y1 < L.shape[0]:
            if (win.shape[1] - 1) % 2 or (win.shape[0] - 1) % 2:
                win = win[: win.shape[0] - ((win.shape[0] - 1) % 2), : win.shape[1] - ((win.shape[1] - 1) % 2)]
        ny, nx = win.shape
        job = O.make_job(**W.job(n0x=(nx - 1) // 2 + 1, n0y=(ny - 1) // 2 + 1, levels=1,
                                 R_abs=params["R_abs"], R_rel=params["R_rel"],
                                 interp=params.get("interp", "linear"),
                                 edge_mode=params.get("edge_mode", "onesided")))
        m = np.zeros(win.shape, np.uint8)
        m[::2, ::2] = O.MASK_TRACED
        _, _, ea, er = O.refine_level(job, win, m, 1, norm)
        a = ea[lj - y0, li - x0] / params["R_abs"] - 1.0
        r = er[lj - y0, li - x0] / params["R_rel"] - 1.0
        if a > 0 and r > 0:
            out.append(float(min(a, r)))
        elif a <= 0 and r <= 0:
            out.append(float(max(-a, -r)))
        else:
            out.append(float(-a if a <= 0 else -r))
    return out


def accuracy(params: dict, img, mask, ref, rmask, rnorm, ctx=None):
    """The render against the FP64 render of the same workload, per plane (Stokes parameter, or
    subring n): the error sum (dI)^2 / (N Ibar^2) of the whole adaptive image (Ibar the mean
    total intensity of the FP64 render), the part of it on points whose mask differs, the number
    of such points and the FP64 estimate's distance from its tolerance at each (the criterion
    decided them differently because its inputs differ by rounding), and, when a context is
    given, the per-ray error over every traced ray against the FP64 trace of the same ray."""
    import torch
    from paper_2103_07417_gb300 import art
    planes = img.shape[0]
    stokes, subr = params.get("stokes", 1), params.get("subrings", 0)
    tot = sum(ref[n * stokes] for n in range(max(subr, 1)))
    m0 = float(tot.double().mean())
    n = img[0].numel()
    d2 = (img - ref).double() ** 2
    flip = mask != rmask
    whole = [float(d2[c].sum()) / (n * m0 * m0) for c in range(planes)]
    on_flips = [float(d2[c][flip].sum()) / (n * m0 * m0) for c in range(planes)]
    nflip = int(flip.sum())
    dist = flip_distances(params, ref[0], rmask, mask, rnorm) if nflip else []
    per_ray = None
    if ctx is not None:
        job64 = art.make_job(**{**params, "precision": "fp64"})
        pix = torch.nonzero(mask.reshape(-1) == art.MASK_TRACED).reshape(-1).to(torch.int32)
        out = torch.empty((pix.numel(), planes), dtype=torch.float64, device=img.device)
        ctx.art_trace_pixels(job64, pix, out)
        got = img.reshape(planes, -1)[:, pix.long()].T
        per_ray = [float(((got[:, c] - out[:, c]) ** 2).sum()) / (pix.numel() * m0 * m0)
                   for c in range(planes)]
        del out, got
    if stokes == 4:
        names = [f"{'IQUV'[c % 4]}" + (f"_n{c // 4}" if subr else "") for c in range(planes)]
    else:
        names = [f"I_n{c}" if subr else "I" for c in range(planes)]
    del d2
    return {"against": "the FP64 render of the same workload (equal to the FP64 oracle to 1e-6)",
            "planes": names, "image_bj": whole, "image_bj_on_mask_flips": on_flips,
            "mask_flips": nflip,
            "flips_fp64_estimate_distance": {"max": max(dist) if dist else None,
                                             "within_1e-9": sum(1 for x in dist if x <= 1e-9),
                                             "measured": len(dist)},
            "per_ray_bj": per_ray}


def run_reference(args, params, desc):
    """The reference arm: the FP64 oracle on the host cores.  Each step is a bounded sample of the
    workload: one full adaptive render (unpolarized analytic) or 2048 evenly spaced base-level
    rays (polarized, grid), so the whole run stays within a few minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    snap = W.grmhd_snapshot(seed=0) if params.get("emission") == "grid" else None
    job = O.make_job(grid=snap, **params)
    pol = _sampled_on_cpu(params)
    pix = _base_pixels(params, 2048) if pol else None

    def step():
        if pol:
            _, info = O.trace_pixels(job, pix)
            return pix.size, int(info["steps"].sum())
        _, _, st = O.render(job, None)
        return st["rays_traced"], st["steps"]

    for _ in range(args.warmup):
        step()
    times, rays, steps = [], 0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rays, steps = step()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = rays * args.steps / total
    sample = ("2048 evenly spaced base-level rays per step" if pol
              else "one full adaptive render per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "name": args.workload},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": O.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "geodesic_steps_per_s": steps * args.steps / total}
    print(json.dumps(line), flush=True)


def _roofline(ctx, recs, params, peaks):
    """Per-kind split of one render's launches and the roofline of its dominant trace kernel
    (CUDA events on the library's stream): algorithmic FLOPs per RK4 step (counted from the
    kernel's formulas) x the steps the kernel's launches executed, over their summed durations."""
    by_kind = {}
    for r in recs:
        d = by_kind.setdefault(r["kind"], {"launches": 0, "ms": 0.0, "steps": 0})
        d["launches"] += 1
        d["ms"] += r["ms"]
        d["steps"] += r["steps"]
    total_ms = sum(v["ms"] for v in by_kind.values())
    grid_em = params.get("emission") == "grid"
    fps = (FLOPS_PER_STEP_POL if params.get("stokes", 1) == 4
           else FLOPS_PER_STEP_GRID if grid_em else FLOPS_PER_STEP)
    traces = [k for k in by_kind if k in fps]
    dom = max(by_kind, key=lambda k: by_kind[k]["ms"])
    meas = ctx.art_measure_alu_peaks()
    out = {}
    for k in traces:
        d = by_kind[k]
        if d["ms"] <= 0:
            continue
        achieved = d["steps"] * fps[k] / (d["ms"] / 1000.0) / 1e12
        mp = meas["fp64_tflops"] if k == "trace_fp64" else meas["fp32_tflops"]
        rec = {"bound": "alu", "kernel": k, "achieved": achieved, "peak": mp, "unit": "TFLOP/s",
               "frac": achieved / mp if mp > 0 else None, "traffic": None,
               "peak_source": "measured: art_measure_alu_peaks (FMA chains on every SM, this GPU)",
               "peak_derived": PEAK_TFLOPS[k], "peak_derived_source": PEAK_SOURCE[k],
               "frac_of_derived": achieved / PEAK_TFLOPS[k],
               "flops_per_step": fps[k], "launches": d["launches"], "steps": d["steps"],
               "share_of_step": d["ms"] / total_ms}
        if grid_em:
            # every RK4 step samples the grid once
            gbs = d["steps"] * GRID_BYTES_PER_SAMPLE / (d["ms"] / 1000.0) / 1e9
            rec["grid_lookup"] = {
                "bytes_per_sample": GRID_BYTES_PER_SAMPLE, "samples": d["steps"],
                "achieved_GBps": gbs, "hbm_peak_GBps": peaks["hbm_gbs"],
                "frac_of_hbm": gbs / peaks["hbm_gbs"], "hbm_peak_source": peaks["source"],
                "note": "algorithmic bytes (8 cells x 32 B per sample) over the kernel time; most "
                        "are served from L1/L2 (neighbouring samples share cells)"}
        out[k] = rec
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                   "share": round(v["ms"] / total_ms, 4)} for k, v in by_kind.items()}
    main_k = dom if dom in out else (max(out, key=lambda k: out[k]["share_of_step"]) if out else None)
    return (out.get(main_k) if main_k else None), out, kernels


def _fe(metrics):
    return metrics.get("FE")


def time_to_mse(args, params, ctx, lctx, learned, img, mask, flush, dev):
    """Wall time to an image with the paper's MSE <= 1e-3 against a full trace of the final grid
    (Eq. msedef), per path: on the calibration seed (the workload itself) the fastest
    (R_rel, R_abs) of a log grid meeting the target, then that setting's time and MSE on held-out
    seeds (new snapshots of the grid model; analytic workloads are deterministic and have none)."""
    import numpy as np
    import torch
    from paper_2103_07417_gb300 import art
    grid_em = params.get("emission") == "grid"
    R0r, R0a = params["R_rel"], params["R_abs"]
    # The settings: the paper's tolerances scaled down and up, on the workload's base grid and on
    # bases 4x and 16x finer at the same final grid.  On the turbulent synthetic snapshot the
    # estimator under-flags small-scale structure (the paper's power-law ratio of ~0.27, Sec. 3.2):
    # at 16385^2 over 1000 M no tolerance brings a 257^2 base below an MSE of ~2e-3, while finer
    # bases reach 1e-3.  If no adaptive setting meets the target, the full trace is the answer.
    L0, n00 = params["levels"], params["n0x"]
    settings = []
    for k, (frs, fas) in ((0, ((0.1, 1.0, 10.0), (0.01, 1.0))), (2, ((0.1, 1.0, 10.0), (0.01, 1.0))),
                          (4, ((1.0, 10.0, 100.0), (1.0,)))):
        if L0 - k < 1:
            continue
        nb = (n00 - 1) * 2 ** k + 1
        settings += [dict(n0x=nb, n0y=nb, levels=L0 - k, R_rel=R0r * f1, R_abs=R0a * f2)
                     for f1 in frs for f2 in fas]
    full_setting = dict(n0x=n00, n0y=n00, levels=L0, R_rel=-1.0, R_abs=-1.0)
    truth_prec = "fp64" if args.fp64_truth else "mixed_exact"

    def truth_of(cx):
        tj = art.make_job(**{**params, "precision": truth_prec, "R_rel": -1.0, "R_abs": -1.0,
                             "crit_band": 0.0, "proposal": 0})
        t = torch.empty_like(img)
        cx.art_render(tj, t, mask, stats=False)
        return t

    variants = [("fp64", ctx, {"precision": "fp64", "crit_band": 0.0}),
                ("mixed_df", ctx, {"precision": "mixed_df"}),
                ("mixed_exact", ctx, {"precision": "mixed_exact"})]
    if lctx is not None and learned is not None:
        lb = learned["best"]
        lover = {"proposal": 1, "proposal_p": lb["threshold"], "proposal_depth": lb["depth"],
                 "crit_band": lb["crit_band"]}
        variants.append(("mixed_df+learned", lctx, {"precision": "mixed_df", **lover}))
        variants.append(("mixed_exact+learned", lctx, {"precision": "mixed_exact", **lover}))
    out = {"target_mse": 1e-3,
           "truth": f"full {truth_prec} trace of the final grid (R = -1): "
                    + ("FP64 rays" if args.fp64_truth else
                       "FP32 rays with the FP64 hand-overs of the exact mode and an FP64 base "
                       "level; measured against the full FP64 trace: paper MSE 4.7e-9 (16385^2), "
                       "1.9e-8 (8193^2)"),
           "settings": settings + ["full trace if none meets the target"],
           "calibration": "the workload itself (snapshot seed 0 for grid models)", "paths": {}}
    truth = truth_of(ctx)
    ltruth = truth if lctx is None else None
    sweeps = {}
    for name, cx, over in variants:
        if cx is not ctx and ltruth is None:
            ltruth = truth_of(cx)
        tr = truth if cx is ctx else ltruth
        rec, sweep = None, []
        for setting in settings + [None]:
            if setting is None:
                if rec is not None:
                    break
                setting = full_setting
            vj = art.make_job(**{**params, **over, **setting})
            vst = cx.art_render(vj, img, mask, stats=True)
            met = cx.art_metrics(tr[0], img[0], mask)
            ok = met["MSE"] <= 1e-3
            tv = _timed_ctx(cx, vj, img, mask, flush, 3 if setting is not full_setting else 1) \
                if ok else None
            sweep.append({**setting, "mse": met["MSE"], "IF": met["IF"], "FE": met["FE"],
                          "seconds": tv, "rays": vst["rays_traced"]})
            if ok and (rec is None or tv < rec["seconds"]):
                rec = {"seconds": tv, **setting, "mse": met["MSE"], "rays": vst["rays_traced"]}
        mses = [x["mse"] for x in sweep]
        out["paths"][name] = {"calibration": rec,
                              "bracketed": bool(min(mses) <= 1e-3 < max(mses)),
                              "sweep": sweep}
        sweeps[name] = rec
    del truth, ltruth
    # held-out seeds: the calibrated setting of every path on new snapshots
    if grid_em and args.heldout > 0:
        held = {name: [] for name, _, _ in variants}
        for seed in range(1, 1 + args.heldout):
            snap = W.grmhd_snapshot(seed=seed)
            ctx.load_grid(snap)
            if lctx is not None:
                lctx.load_grid(snap)
            truth = truth_of(ctx)
            for name, cx, over in variants:
                rec = sweeps[name]
                if rec is None:
                    continue
                vj = art.make_job(**{**params, **over, **{k: rec[k] for k in
                                                           ("n0x", "n0y", "levels", "R_rel", "R_abs")}})
                cx.art_render(vj, img, mask, stats=False)
                met = cx.art_metrics(truth[0], img[0], mask)
                tv = _timed_ctx(cx, vj, img, mask, flush, 3 if rec["R_rel"] >= 0 else 1)
                held[name].append({"seed": seed, "seconds": tv, "mse": met["MSE"]})
            del truth
        snap0 = W.grmhd_snapshot(seed=0)
        ctx.load_grid(snap0)
        if lctx is not None:
            lctx.load_grid(snap0)
        for name, h in held.items():
            if h:
                out["paths"][name]["heldout"] = {
                    "seeds": [x["seed"] for x in h], "mean_seconds": float(np.mean([x["seconds"] for x in h])),
                    "max_mse": float(max(x["mse"] for x in h)), "runs": h}
    base = out["paths"]["fp64"].get("heldout", {}).get("mean_seconds") or \
        (out["paths"]["fp64"]["calibration"] or {}).get("seconds")
    for name in out["paths"]:
        t = out["paths"][name].get("heldout", {}).get("mean_seconds") or \
            (out["paths"][name]["calibration"] or {}).get("seconds")
        out["paths"][name]["speedup_vs_fp64"] = (base / t) if (base and t) else None
    return out


def contours(args, ctx, flush):
    """The paper's tolerance study (Sec. 4.1) on the 8193^2 grid workload: IF, FE and MSE against
    the full trace over a log grid of (R_rel, R_abs), on the exact-decision mixed path."""
    import torch
    from paper_2103_07417_gb300 import art
    params = W.grmhd_8193(precision="mixed_exact")
    ctx.load_grid(W.grmhd_snapshot(seed=0))
    job = art.make_job(**params)
    nx, ny = art.art_image_size(job)
    img = torch.empty((1, ny, nx), dtype=torch.float64, device="cuda")
    mask = torch.empty((ny, nx), dtype=torch.uint8, device="cuda")
    tj = art.make_job(**{**params, "R_rel": -1.0, "R_abs": -1.0})
    truth = torch.empty_like(img)
    ctx.art_render(tj, truth, mask, stats=False)
    rows = []
    for rr in (1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1):
        for ra in (1e-3, 3e-3, 1e-2, 2.5e-2, 1e-1, 3e-1, 1.0):
            j = art.make_job(**{**params, "R_rel": rr, "R_abs": ra})
            st = ctx.art_render(j, img, mask, stats=True)
            met = ctx.art_metrics(truth[0], img[0], mask)
            rows.append({"R_rel": rr, "R_abs": ra, "IF": met["IF"], "FE": met["FE"],
                         "MSE": met["MSE"], "rays": st["rays_traced"]})
    print(json.dumps({"contours": "grmhd_8193", "precision": "mixed_exact",
                      "truth": "full trace (mixed_exact, R = -1)", "rows": rows}), flush=True)


# Angular size of GM/c^2 of the M87*-mass hole the synthetic models are scaled to (length unit
# 9.6e14 cm at 16.8 Mpc), to express baselines in G-lambda as the paper does.
THETA_M_RAD = 9.6e14 / (16.8 * 3.0857e24)


def visibility_spectra(ctx, flush):
    """Sec. 4.3 on the 8193^2 grid workload: the image is rendered with the field of view and
    pixel count doubled (same resolution), adaptively (exact decisions) and fully traced, then
    tapered by a Gaussian of FWHM FOV/4 (the original FOV) and transformed; |V| and the residual
    |dV| (adaptive minus full) along the u and v axes, out to 1000 G-lambda."""
    import numpy as np
    import torch
    from paper_2103_07417_gb300 import art
    base = W.grmhd_8193(precision="mixed_exact")
    ctx.load_grid(W.grmhd_snapshot(seed=0))
    p2 = W.doubled_fov(base)
    job = art.make_job(**p2)
    nx, ny = art.art_image_size(job)
    img = torch.empty((1, ny, nx), dtype=torch.float64, device="cuda")
    mask = torch.empty((ny, nx), dtype=torch.uint8, device="cuda")
    st = ctx.art_render(job, img, mask, stats=True)
    full = torch.empty_like(img)
    ctx.art_render(art.make_job(**{**p2, "R_rel": -1.0, "R_abs": -1.0}), full, mask, stats=False)
    dx = p2["fov"] / (nx - 1)
    m = 1
    while m < nx:
        m *= 2
    fwhm = base["fov"] / 4.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    v = ctx.art_visibilities(img[0], dx, fwhm, m)
    torch.cuda.synchronize()
    t_vis = time.perf_counter() - t0
    vu, vv = v[0, : m // 2].abs().cpu().numpy(), v[: m // 2, 0].abs().cpu().numpy()
    del v
    torch.cuda.empty_cache()
    dv = ctx.art_visibilities(img[0], dx, fwhm, m, ref=full[0])
    du, dvv = dv[0, : m // 2].abs().cpu().numpy(), dv[: m // 2, 0].abs().cpu().numpy()
    del dv, img, full, mask
    torch.cuda.empty_cache()
    u = np.arange(m // 2) / (m * dx)                       # cycles per M
    glam = u / THETA_M_RAD / 1e9
    keep = (glam > 0) & (glam <= 1000.0)
    idx = np.unique(np.geomspace(1, keep.sum(), 48).astype(int))
    sel = np.nonzero(keep)[0][idx - 1]
    v0 = float(vu[0])
    # the residual against the visibility amplitude, on the baselines up to 1000 G-lambda (the
    # amplitude has nulls where any residual exceeds it: quoted as quantiles)
    ru = du[keep] / np.maximum(vu[keep], 1e-300)
    rv = dvv[keep] / np.maximum(vv[keep], 1e-300)
    return {"workload": "grmhd_8193 with FOV and pixels doubled (320 M, 16385^2), mixed_exact; "
                        "residual against the full trace (mixed_exact, R = -1)",
            "fft": f"{m}x{m} FP64", "seconds_per_transform": t_vis, "taper_fwhm_M": fwhm,
            "rays": st["rays_traced"], "V0": v0,
            "baseline_Glambda": glam[sel].tolist(),
            "amp_u": (vu[sel] / v0).tolist(), "amp_v": (vv[sel] / v0).tolist(),
            "resid_u": (du[sel] / v0).tolist(), "resid_v": (dvv[sel] / v0).tolist(),
            "resid_over_amp_u_quantiles_50_90": np.quantile(ru, [0.5, 0.9]).tolist(),
            "resid_over_amp_v_quantiles_50_90": np.quantile(rv, [0.5, 0.9]).tolist(),
            "resid_rms_over_amp_rms": float(np.sqrt(np.sum(du[keep] ** 2 + dvv[keep] ** 2) /
                                                    np.sum(vu[keep] ** 2 + vv[keep] ** 2)))}


def axis_sampling(ctx, flush):
    """Adaptive sampling along a third axis (Sec. 6 proposal): the 2049^2 disk workload's
    geometry, unpolarized, 513^2 images at 17 frequencies from 86 to 690 GHz (3 base frequencies,
    3 axis levels, R_rel3 = R_abs3 = 1e-3), against 17 independent adaptive renders."""
    import numpy as np
    import torch
    from paper_2103_07417_gb300 import art
    F, L3, R3 = 17, 3, 1e-3
    nus = 86e9 * 2.0 ** (3.0 * np.arange(F) / (F - 1))
    params = [W.kerr_disk_2049(n0x=129, n0y=129, levels=2, stokes=1, precision="mixed_df",
                               nu_hz=float(nu)) for nu in nus]
    jobs = [art.make_job(**p) for p in params]
    nx, ny = art.art_image_size(jobs[0])
    imgs = [torch.empty((1, ny, nx), dtype=torch.float64, device="cuda") for _ in range(F)]
    ref = [torch.empty_like(t) for t in imgs]
    ctx.art_render_axis(jobs, L3, R3, R3, imgs)      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ctx.art_render_axis(jobs, L3, R3, R3, imgs)
    torch.cuda.synchronize()
    t_axis = time.perf_counter() - t0
    rays_axis = sum(x["rays_traced"] for x in st)
    t0 = time.perf_counter()
    rays_all = 0
    for j, r in zip(jobs, ref):
        rays_all += ctx.art_render(j, r, None, stats=True)["rays_traced"]
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    num = sum(float(((a - b).double() ** 2).sum()) for a, b in zip(imgs, ref))
    den = sum(float((b.double() ** 2).sum()) for b in ref)
    return {"workload": "kerr_disk_2049 geometry, unpolarized, 129^2 -> 513^2 per frequency; 17 "
                        "frequencies 86-690 GHz (3 base, 3 axis levels, R3 = 1e-3), mixed_df",
            "rays_axis": rays_axis, "rays_independent": rays_all,
            "ray_fraction": rays_axis / rays_all, "seconds_axis": t_axis,
            "seconds_independent": t_all, "mse_vs_independent": num / den,
            "rays_per_sample": [x["rays_traced"] for x in st]}


def main():
    args = parse()
    desc, fn = W.BENCH_WORKLOADS[args.workload]
    params = fn(precision=args.precision)
    band_default = params.get("crit_band", 0.0)
    if args.precision == "mixed_exact":
        # exact decisions trace the band's photon-ring rays in FP32 and double-float with the base
        # level and still need their stencils' FP64 values at their own level: the render is
        # faster without the band (the variant with it is reported in paths)
        params["crit_band"] = 0.0
    if args.impl == "reference":
        return run_reference(args, params, desc)

    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = measured_peaks()

    from paper_2103_07417_gb300 import art
    ctx = art.Context(local)
    stream = ctx.stream
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if args.contours:
        contours(args, ctx, flush)
        ctx.close()
        return
    snap = None
    if params.get("emission") == "grid":
        # the seeded snapshot, resident on the device before timing (151 MB of FP32)
        snap = W.grmhd_snapshot(seed=0)
        ctx.load_grid(snap)
    job = art.make_job(**params)
    nx, ny = art.art_image_size(job)
    planes = art.art_planes(job)
    img = torch.empty((planes, ny, nx), dtype=torch.float64, device=dev)
    mask = torch.empty((ny, nx), dtype=torch.uint8, device=dev)

    stats = None
    if args.cnn:
        ctx.art_cnn_load(W.cnn_init(0))
        cnn_measure(ctx, 1025, reps=1)
        print(json.dumps({"cnn": 1025}))
        ctx.close()
        return
    if args.batch_only:
        if snap is None:
            snap = W.grmhd_snapshot(seed=0)
            ctx.load_grid(snap)
        bjobs = [art.make_job(**p) for p in W.grmhd_batch(seed=0, n=256)]
        bimgs, bmasks, _ = ctx.render_batch(bjobs)
        bst = ctx.art_render_batch(bjobs, bimgs, bmasks)
        print(json.dumps({"batch": len(bjobs), "rays": sum(b["rays_traced"] for b in bst),
                          "steps": bst[0]["steps"]}))
        ctx.close()
        return
    if args.single:
        # one warm-up render, then one render with the library's launch profiler on: per launch
        # its kind, level, CUDA-event ms and, for trace launches, rays, steps and longest ray
        ctx.art_render(job, img, mask, stats=True)
        ctx.art_profile(True)
        st = ctx.art_render(job, img, mask, stats=True)
        recs = ctx.art_profile_read()
        ctx.art_profile(False)
        launches = [{k: (round(v, 4) if k == "ms" else v) for k, v in r.items()}
                    for r in recs if r["kind"] != "other"]
        print(json.dumps({"single": args.workload, "precision": args.precision, **st,
                          "launches": launches}))
        ctx.close()
        return
    # the library's autotuner picks the FP32 kernel-form thresholds for this workload (outside
    # the timed region; every setting renders the same image)
    tune = None
    if not args.no_tune:
        (tq, tp, tb64, tb32, tq64), tms = ctx.art_autotune(job, img, mask, reps=3)
        tune = {"quad_rays": tq, "pair_rays": tp, "blocks64": tb64, "blocks32": tb32,
                "quad64_rays": tq64,
                "median_ms": tms,
                "default": list(art.TUNE_DEFAULT)}
    for _ in range(max(args.warmup, 1)):
        stats = ctx.art_render(job, img, mask, stats=True)
    rays = stats["rays_traced"]
    steps_per_render = stats["steps"]

    def timed(k, precision_job):
        evs = []
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.art_render(precision_job, img, mask, stats=False)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / 1000.0

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_dev = timed(args.steps, job)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_dev = max_over_ranks(t_dev, dist, dev)
    value = whole_job_value(rays, args.steps, world, t_dev)
    clocks = clk.summary()

    # per-kernel timing of one render with CUDA events on the library's stream
    ctx.art_profile(True)
    ctx.art_render(job, img, mask, stats=False)
    recs = ctx.art_profile_read()
    ctx.art_profile(False)
    roofline, roofline_all, kernels = _roofline(ctx, recs, params, peaks)

    # the other precision paths on the same workload, for comparison
    paths = {}
    for prec in ("fp64", "mixed_df", "mixed_exact", "mixed"):
        if prec == args.precision:
            continue
        jobp = art.make_job(**{**params, "precision": prec})
        stp = ctx.art_render(jobp, img, mask, stats=True)
        kp = 3
        tp = timed(kp, jobp)
        paths[prec] = {"rays_per_s": stp["rays_traced"] * kp / tp,
                       "geodesic_steps_per_s": stp["steps"] * kp / tp,
                       "ms_per_step": 1000 * tp / kp, "rays_high_precision": stp["rays_fp64"],
                       "rays_exact": stp["rays_exact"]}
        if prec == "mixed_df":
            ctx.art_profile(True)
            ctx.art_render(jobp, img, mask, stats=False)
            r2 = ctx.art_profile_read()
            ctx.art_profile(False)
            paths[prec]["roofline"], _, paths[prec]["kernels"] = _roofline(ctx, r2, params, peaks)
    if params.get("crit_band", 0.0) > 0.0:
        # the same precision without the near-critical band speculation (same image)
        jnb = art.make_job(**{**params, "crit_band": 0.0})
        stp = ctx.art_render(jnb, img, mask, stats=True)
        tp = timed(3, jnb)
        paths[args.precision + "_no_band"] = {
            "rays_per_s": stp["rays_traced"] * 3 / tp,
            "geodesic_steps_per_s": stp["steps"] * 3 / tp, "ms_per_step": 1000 * tp / 3,
            "rays_high_precision": stp["rays_fp64"]}
    elif band_default > 0.0:
        # the same precision with the workload's near-critical band (same image)
        jb = art.make_job(**{**params, "crit_band": band_default})
        stp = ctx.art_render(jb, img, mask, stats=True)
        tp = timed(3, jb)
        paths[args.precision + "_with_band"] = {
            "rays_per_s": stp["rays_traced"] * 3 / tp,
            "geodesic_steps_per_s": stp["steps"] * 3 / tp, "ms_per_step": 1000 * tp / 3,
            "rays_high_precision": stp["rays_fp64"], "crit_band": band_default}
    # the same render replayed from a CUDA graph (one capture of the whole level loop)
    if not params.get("proposal", 0):
        ctx.art_graph_render(job, img, mask)
        kp = 3
        evs = []
        for _ in range(kp):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.art_graph_render(job, img, mask)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        tg = sum(a.elapsed_time(b) for a, b in evs) / 1000.0
        paths[args.precision + "_graph"] = {"rays_per_s": rays * kp / tg,
                                            "geodesic_steps_per_s": steps_per_render * kp / tg,
                                            "ms_per_step": 1000 * tg / kp,
                                            "rays_high_precision": stats["rays_fp64"]}
    paths[args.precision] = {"rays_per_s": value / world,
                             "geodesic_steps_per_s": steps_per_render * args.steps / t_dev,
                             "ms_per_step": 1000 * t_dev / args.steps,
                             "rays_high_precision": stats["rays_fp64"],
                             "rays_exact": stats["rays_exact"],
                             "border_points": stats["border_points"]}

    # accuracy of the measured path (and of the other mixed path) against the FP64 render
    acc = None
    if args.precision != "fp64":
        ref = torch.empty_like(img)
        rmask = torch.empty_like(mask)
        rst = ctx.art_render(art.make_job(**{**params, "precision": "fp64"}), ref, rmask, stats=True)
        ctx.art_render(job, img, mask, stats=False)
        acc = {args.precision: accuracy(params, img, mask, ref, rmask, rst["norm"], ctx)}
        for other in ("mixed_df", "mixed_exact"):
            if other != args.precision:
                ctx.art_render(art.make_job(**{**params, "precision": other}), img, mask, stats=False)
                acc[other] = accuracy(params, img, mask, ref, rmask, rst["norm"], None)
        del ref, rmask
        ctx.art_render(job, img, mask, stats=False)

    # end to end through the public C-ABI with host buffers (D2H of image + mask inside)
    himg = torch.empty((planes, ny, nx), dtype=torch.float64).pin_memory().numpy()
    hmask = torch.empty((ny, nx), dtype=torch.uint8).pin_memory().numpy()
    ctx.art_render_host(job, himg, hmask)
    ke = 5
    hgrid = None
    if snap is not None:
        # a new snapshot per frame: its upload from pinned host memory is inside the timed loop
        hgrid = torch.from_numpy(snap["data"]).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        if hgrid is not None:
            ctx.art_load_grid(hgrid, snap["n1"], snap["n2"], snap["n3"], snap["logr_min"],
                              snap["logr_max"])
        ctx.art_render_host(job, himg, hmask)
    te = time.perf_counter() - t0
    e2e = {"value": rays * ke / te, "unit": "rays/s",
           "h2d_bytes_per_step": int(ctypes_sizeof_job()) + (int(hgrid.nbytes) if hgrid is not None else 0),
           "d2h_bytes_per_step": int(himg.nbytes + hmask.nbytes)}
    del himg, hmask
    if snap is not None:
        ctx.load_grid(snap)

    # the batched form (256 images of random spin, inclination, FOV, grid and depth, one pass per
    # level for all of them) on the same GPU
    batched = None
    if not args.no_batch:
        if snap is None:   # the batch renders the grid emission model: load its snapshot
            ctx.load_grid(W.grmhd_snapshot(seed=0))
        bparams = W.grmhd_batch(seed=0, n=256)
        bjobs = [art.make_job(**p) for p in bparams]
        bimgs, bmasks = [], []
        for bj in bjobs:
            bnx, bny = art.art_image_size(bj)
            bimgs.append(torch.empty((art.art_planes(bj), bny, bnx), dtype=torch.float64, device=dev))
            bmasks.append(torch.empty((bny, bnx), dtype=torch.uint8, device=dev))
        bst = ctx.art_render_batch(bjobs, bimgs, bmasks, stats=True)
        brays = sum(x["rays_traced"] for x in bst)
        bpix = sum(int(m.numel()) for m in bmasks)

        def tbatch(jobs, graph=False):
            evs = []
            for _ in range(3):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if graph:
                    ctx.art_graph_render_batch(jobs, bimgs, bmasks)
                else:
                    ctx.art_render_batch(jobs, bimgs, bmasks, stats=False)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            return sum(a.elapsed_time(b) for a, b in evs) / 1000.0 / len(evs)

        tb = tbatch(bjobs)
        ctx.art_graph_render_batch(bjobs, bimgs, bmasks)
        tg = tbatch(bjobs, graph=True)
        batched = {"workload": "256 images (mixed-parameter batch): a~U[-0.94,0.94], i~U[10,170] deg, "
                               "FOV log-U[40,400] M, 65^2..513^2 over 2-6 levels, emission from "
                               "the GRMHD-like snapshot (288x128x128 grid), subrings n=0,1,2, "
                               "mixed_df",
                   "rays_per_s": brays / tb, "images_per_s": len(bjobs) / tb,
                   "ms_per_batch": 1000 * tb, "ms_per_batch_graph": 1000 * tg,
                   "rays": brays, "pixels": bpix,
                   "geodesic_steps_per_s": bst[0]["steps"] / tb,
                   "rays_speculative": bst[0]["rays_speculative"],
                   "rays_spec_used": bst[0]["rays_spec_used"]}
        ctx.art_profile(True)
        ctx.art_render_batch(bjobs, bimgs, bmasks, stats=False)
        brecs = ctx.art_profile_read()
        ctx.art_profile(False)
        batched["launches"] = [{"kind": r["kind"], "level": r["level"], "ms": round(r["ms"], 4),
                                "steps": r["steps"]} for r in brecs]
        # per-image error against the FP64 batch, per subring plane, for the batched mixed_df
        # render and for exact decisions (each image through the single-image level loop)
        rjobs = [art.make_job(**{**p, "precision": "fp64"}) for p in bparams]
        rimgs, rmasks, rst = ctx.render_batch(rjobs)

        def per_image(imgs_, masks_):
            per, flips, dmax = [], 0, 0.0
            for p, a, b, ma, mb, s in zip(bparams, imgs_, rimgs, rmasks, masks_, rst):
                m0 = float(b.sum(0).double().mean())
                n = a[0].numel()
                per.append([float(((a[c] - b[c]).double() ** 2).sum()) / (n * m0 * m0)
                            for c in range(a.shape[0])])
                if not torch.equal(ma, mb):
                    fl = int((ma != mb).sum())
                    flips += fl
            per = np.array(per)
            return {"against": "the FP64 batch", "planes": [f"I_n{c}" for c in range(per.shape[1])],
                    "image_bj_median": np.median(per, 0).tolist(), "image_bj_max": per.max(0).tolist(),
                    "images_above_1e-5": int((per.max(1) > 1e-5).sum()), "mask_flips": flips}
        batched["accuracy"] = per_image(bimgs, bmasks)
        xjobs = [art.make_job(**{**p, "precision": "mixed_exact"}) for p in bparams]
        ctx.art_render_batch(xjobs, bimgs, bmasks, stats=False)  # warm-up (sub-context scratch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.art_render_batch(xjobs, bimgs, bmasks, stats=False)
        torch.cuda.synchronize()
        tx = time.perf_counter() - t0
        batched["exact"] = {"ms_per_batch": 1000 * tx,
                            "note": "mixed_exact, the 256 images rendered concurrently on the "
                                    "library's 32 sub-contexts (streams of their own)",
                            "accuracy": per_image(bimgs, bmasks)}
        del rimgs, rmasks
        del bimgs, bmasks

    # the learned path: train the block-proposal network on seeded plain renders (the library's
    # own tensor-core forward/backward and Adam), then render the workload with it
    learned = None
    lctx = None
    if not args.no_learned:
        from paper_2103_07417_gb300 import learn
        t0 = time.perf_counter()
        lctx, hist, tr_info = learn.trained_context(
            seed=0, n_jobs=args.learn_jobs, epochs=args.learn_epochs, device=local,
            snapshot=snap if snap is not None else W.grmhd_snapshot(seed=0), info=True)
        t_train = time.perf_counter() - t0
        best, best_nb = None, None
        band0 = params.get("crit_band", 0.0)
        for band in sorted({0.0, band0}):
            for depth in (1, 2, 3):
                for thr in (0.2, 0.3, 0.5, 0.7):
                    lj = art.make_job(**{**params, "proposal": 1, "proposal_p": thr,
                                         "proposal_depth": depth, "crit_band": band})
                    lst = lctx.art_render(lj, img, mask, stats=True)
                    tl = _timed_ctx(lctx, lj, img, mask, flush, 3)
                    cand = dict(depth=depth, threshold=thr, crit_band=band, ms_per_step=1000 * tl,
                                rays_per_s=lst["rays_traced"] / tl,
                                rays_speculative=lst["rays_speculative"],
                                rays_spec_used=lst["rays_spec_used"])
                    if best is None or cand["ms_per_step"] < best["ms_per_step"]:
                        best = cand
                    if band == 0.0 and (best_nb is None or cand["ms_per_step"] < best_nb["ms_per_step"]):
                        best_nb = cand
        plain_nb = paths.get(args.precision + "_no_band", paths[args.precision])["ms_per_step"]
        learned = {"training": {"jobs": args.learn_jobs, "epochs": args.learn_epochs,
                                "seconds": t_train, **tr_info,
                                "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]},
                   "precision": args.precision,
                   "best": best, "best_without_band": best_nb,
                   "gain_vs_plain": (1000 * t_dev / args.steps) / best["ms_per_step"],
                   "gain_vs_plain_both_without_band": plain_nb / best_nb["ms_per_step"],
                   "note": "same image and mask as the plain render (the exact criterion decides "
                           "every point); lookahead depth, threshold and band chosen among "
                           "{1,2,3} x {0.2,0.3,0.5,0.7} x {0, default} by timing"}

    # the proposal network's tensor-core kernels alone: forward (4 implicit-GEMM convolutions +
    # head) and forward + backward on a 2049 x 2049 lattice, host-timed (each call synchronises)
    cnn = None
    if lctx is not None:
        nlat = 2049
        t_fw, t_fb = cnn_measure(lctx, nlat)
        fl = cnn_flops(nlat, nlat)
        peak = peaks["bf16_tflops"]
        cnn = {"lattice": f"{nlat}x{nlat}", "forward_ms": 1000 * t_fw,
               "forward_backward_ms": 1000 * t_fb,
               "roofline": {"bound": "tensor", "achieved": fl / t_fw / 1e12, "peak": peak,
                            "unit": "TFLOP/s", "frac": fl / t_fw / 1e12 / peak,
                            "peak_source": peaks["source"] + ": cuBLAS bf16 dense GEMM, burst",
                            "flops_per_forward": fl}}

    axis = None
    if world == 1 and not args.no_vis:
        axis = axis_sampling(ctx, flush)
        if snap is not None:
            ctx.load_grid(snap)

    visib = None
    if not args.no_vis and world == 1:
        visib = visibility_spectra(ctx, flush)
        if snap is not None:
            ctx.load_grid(snap)

    tmse = None
    if not args.no_mse and not args.gpus > 1:
        tmse = time_to_mse(args, params, ctx, lctx, learned, img, mask, flush, dev)
    if lctx is not None:
        lctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(params, snap)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000 * t_dev / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[args.precision],
                "data": "synthetic",
                "config": {"workload": desc, "name": args.workload, "image": f"{nx}x{ny}",
                           "precision": args.precision, "rays_per_step": rays, "tune": tune,
                           "crit_band": params.get("crit_band", 0.0),
                           "adaptive_ray_fraction": rays / (nx * ny),
                           "l2": "flushed (512 MB write) before every step, outside the timed "
                                 "region", "parallelism": f"replicas x{world}"},
                "geodesic_steps_per_s": steps_per_render * args.steps * world / t_dev,
                "paths": paths, "batched": batched, "learned": learned, "cnn": cnn,
                "time_to_mse": tmse, "accuracy": acc, "roofline": roofline,
                "visibilities": visib, "axis_sampling": axis,
                "roofline_kernels": roofline_all, "kernels": kernels, "peaks": peaks,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(stats["kernel_launches"]) * args.steps}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def _timed_ctx(c, job, img, mask, flush, k):
    """Median seconds of k renders of `job` on context c (CUDA events on its stream, L2 flushed
    before each)."""
    import torch
    ts = []
    for _ in range(k):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(c.stream)
        c.art_render(job, img, mask, stats=False)
        e1.record(c.stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1000.0)
    return float(statistics.median(ts))


def cnn_flops(H: int, W: int) -> float:
    """Algorithmic FLOPs of one forward pass of the proposal network on an H x W lattice (2 per
    multiply-add): 3x3 convolutions 3 -> 32 at H x W, 32 -> 32 at H x W, H/2 x W/2 and H/4 x W/4,
    and the 32 -> 1 head."""
    o = lambda n: (n - 1) // 2 + 1
    H2, W2, H4, W4 = o(H), o(W), o(o(H)), o(o(W))
    return 2.0 * (H * W * 32 * 27 + H * W * 32 * 288 + H2 * W2 * 32 * 288 + H4 * W4 * 32 * 288
                  + H4 * W4 * 32)


def cnn_measure(ctx, n: int, reps: int = 5):
    """Forward and forward+backward times of the proposal network on a seeded n x n lattice."""
    import numpy as np
    import torch
    rng = np.random.default_rng(0)
    feat = torch.from_numpy(np.stack([rng.normal(0, 1, (n, n)), rng.uniform(0, 2, (n, n)),
                                      rng.integers(0, 3, (n, n)).astype(float)], -1)
                            .astype(np.float32)).cuda()
    H4 = ((n - 1) // 2) // 2 + 1
    tgt = torch.from_numpy((rng.uniform(size=(H4, H4)) < 0.3).astype(np.float32)).cuda()
    ctx.art_cnn_forward(feat)
    ctx.art_cnn_grad(feat, tgt)
    fw, fb = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        ctx.art_cnn_forward(feat)      # synchronises
        fw.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        ctx.art_cnn_grad(feat, tgt)
        fb.append(time.perf_counter() - t0)
    return statistics.median(fw), statistics.median(fb)


def ctypes_sizeof_job():
    import ctypes

    from paper_2103_07417_gb300 import art
    return ctypes.sizeof(art.Job)


if __name__ == "__main__":
    main()
