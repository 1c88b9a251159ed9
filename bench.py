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
# update arithmetic for 6 variables (81), the new point's radius (15), the Keplerian emissivity
# (44), the polar-turn test (11) and the transfer segment (11); the FP32 pass of the mixed path
# adds the swept-angle accumulation (28).
# The double-float re-trace counts the same 550 algorithmic flops per step (each carried out as
# a double-float operation of several FP32 instructions).
FLOPS_PER_STEP = {"trace_fp64": 550, "trace_fp32": 578, "trace_df": 550}
# Polarized synchrotron steps, counted from the kernel's formulas (+-10 %): the geodesic (495),
# parallel transport of the polarization covector at the 4 RK4 stages plus its update (1332), the
# synchrotron coefficients in the fluid frame (590) and the exact Stokes segment (590).
FLOPS_PER_STEP_POL = {"trace_fp64": 3007, "trace_fp32": 3035, "trace_df": 3007}
# Fluid-grid (GRMHD-like snapshot) steps, unpolarized: the geodesic and transfer as above (506)
# plus the grid emission instead of the analytic one: angles and cell coordinates (22), the
# trilinear interpolation of 8 fields from 8 cells (147), the Jacobian to Cartesian components and
# u, B (46), Kerr-Schild metric pieces (18), u^t from the normalisation (28), b^mu and b^2 (41),
# the two-temperature plasma state (29) and the thermal-synchrotron j_I, alpha_I (164).
FLOPS_PER_STEP_GRID = {"trace_fp64": 999, "trace_fp32": 1027, "trace_df": 999}
# Algorithmic bytes of one grid sample: 8 cells x 8 FP32 fields (before any cache reuse).
GRID_BYTES_PER_SAMPLE = 256
# Peaks for "alu"-bound kernels: FP32 = 152 SMs x 128 lanes x 2 flops x 2.07 GHz; FP64 = the
# GB300's nominal dense FP64 rate.
PEAK_TFLOPS = {"trace_fp32": 152 * 128 * 2 * 2.07e9 / 1e12, "trace_fp64": 1.25,
               "trace_df": 152 * 128 * 2 * 2.07e9 / 1e12}
PEAK_SOURCE = {"trace_fp32": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
               "trace_df": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (FP32 pipes)",
               "trace_fp64": "nominal GB300 dense FP64"}
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture of the
# second of two renders (`bench.py --single [--workload grmhd_8193]` under
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:trace_kernel`), averaged over
# that render's FP32-pass launches (5 for the 2049^2 polarized render, 6 for the 8193^2 grid
# render).  Reset to None whenever the trace kernels change.
TRAFFIC_PER_LAUNCH = {("kerr_disk_2049", "trace_fp32"): 437558.0,
                      ("grmhd_8193", "trace_fp32"): 90996130.0}
HBM_PEAK_GBPS = 6779.0  # measured STREAM-style copy bandwidth of a GB300, GB/s
DTYPE = {"mixed": "f32+f64", "mixed_df": "f32+df32x2", "fp64": "f64", "fp32": "f32"}
METRIC = "rays/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kerr_disk_2049", choices=sorted(W.BENCH_WORKLOADS))
    ap.add_argument("--precision", default="mixed_df", choices=["mixed", "mixed_df", "fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-render measurement")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default kernel-form thresholds (skip the autotuner)")
    ap.add_argument("--no-mse", action="store_true",
                    help="skip the time-to-0.1%%-MSE sweep (needs a full FP64 trace as truth)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training the block-proposal network and the learned path")
    ap.add_argument("--single", action="store_true",
                    help="one warm-up and one render, nothing else (for profiler captures)")
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


def cpu_baseline(params: dict, snap=None):
    """The FP64 oracle on the host cores.  Unpolarized analytic workloads: one full adaptive
    render.  Polarized and grid ones: the whole base level of the workload."""
    import oracle as O
    job = O.make_job(grid=snap, **params)
    if _sampled_on_cpu(params):
        pix = _base_pixels(params)
        t0 = time.perf_counter()
        _, info = O.trace_pixels(job, pix)
        dt = time.perf_counter() - t0
        rays, steps = pix.size, int(info["steps"].sum())
        note = f"the {params['n0x']}x{params['n0y']} base level of the workload ({rays} rays)"
    else:
        t0 = time.perf_counter()
        img, mask, st = O.render(job, None)
        dt = time.perf_counter() - t0
        rays, steps = int(st["rays_traced"]), int(st["steps"])
        note = "one full adaptive render of the workload"
    cores = O.get_threads()
    # one core: every 16th base-level ray (a bounded sample of a few seconds)
    pix1 = _base_pixels(params)[::16]
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        O.trace_pixels(job, pix1)
        dt1 = time.perf_counter() - t0
    finally:
        O.set_threads(cores)
    return {"value": rays / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": note + " by the FP64 oracle (OpenMP over rays, all host cores)",
            "seconds": dt, "rays": rays, "steps_per_s": steps / dt,
            "single_core": {"value": pix1.size / dt1, "unit": "rays/s", "cores": 1,
                            "sample": f"every 16th base-level ray ({pix1.size} rays)",
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


def accuracy(ctx, params: dict, img, mask):
    """The render against the FP64 path on the same workload, per plane (Stokes parameter, or
    subring n for unpolarized subring images): the BJ error sum (dI)^2 / (N mean(I)^2) of the
    whole adaptive image against the FP64 adaptive render, the part of it on points whose mask
    differs (the criterion decided them differently because its inputs differ by rounding; one
    render traced the point, the other interpolated it), and the per-ray error over every traced
    ray against the FP64 trace of the same ray."""
    import torch
    from paper_2103_07417_gb300 import art
    if params.get("precision") == "fp64":
        return None
    job64 = art.make_job(**{**params, "precision": "fp64"})
    ref, rmask, _ = ctx.render(job64)
    planes = img.shape[0]
    m0 = float(ref[0].double().mean())
    n = img[0].numel()
    d2 = (img - ref).double() ** 2
    flip = mask != rmask
    whole = [float(d2[c].sum()) / (n * m0 * m0) for c in range(planes)]
    on_flips = [float(d2[c][flip].sum()) / (n * m0 * m0) for c in range(planes)]
    pix = torch.nonzero(mask.reshape(-1) == art.MASK_TRACED).reshape(-1).to(torch.int32)
    out = torch.empty((pix.numel(), planes), dtype=torch.float64, device=img.device)
    ctx.art_trace_pixels(job64, pix, out)
    got = img.reshape(planes, -1)[:, pix.long()].T
    mr = float(out[:, 0].mean())
    per_ray = [float(((got[:, c] - out[:, c]) ** 2).sum()) / (pix.numel() * mr * mr)
               for c in range(planes)]
    if params.get("stokes", 1) == 4:
        names = [f"{'IQUV'[c % 4]}" + (f"_n{c // 4}" if params.get("subrings", 0) else "")
                 for c in range(planes)]
    else:
        names = [f"I_n{c}" if params.get("subrings", 0) else "I" for c in range(planes)]
    del ref, rmask, d2, out, got
    return {"against": "the FP64 path on the same workload (equal to the FP64 oracle to 1e-6)",
            "planes": names, "image_bj": whole, "image_bj_on_mask_flips": on_flips,
            "mask_flips": int(flip.sum()), "traced_rays": int(pix.numel()),
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


def main():
    args = parse()
    desc, fn = W.BENCH_WORKLOADS[args.workload]
    params = fn(precision=args.precision)
    if args.impl == "reference":
        return run_reference(args, params, desc)

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

    from paper_2103_07417_gb300 import art
    ctx = art.Context(local)
    stream = ctx.stream
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
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

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
        ctx.art_render(job, img, mask, stats=True)
        st = ctx.art_render(job, img, mask, stats=True)
        print(json.dumps({"single": args.workload, "precision": args.precision, **st}))
        ctx.close()
        return
    # the library's autotuner picks the FP32 kernel-form thresholds for this workload (outside
    # the timed region; every setting renders the same image)
    tune = None
    if not args.no_tune:
        (tq, tp), tms = ctx.art_autotune(job, img, mask, reps=3)
        tune = {"quad_rays": tq, "pair_rays": tp, "median_ms": tms,
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
    by_kind = {}
    for r in recs:
        d = by_kind.setdefault(r["kind"], {"launches": 0, "ms": 0.0, "steps": 0})
        d["launches"] += 1
        d["ms"] += r["ms"]
        d["steps"] += r["steps"]
    dom = max(by_kind, key=lambda k: by_kind[k]["ms"])
    total_ms = sum(v["ms"] for v in by_kind.values())
    roofline = None
    grid_em = params.get("emission") == "grid"
    fps = (FLOPS_PER_STEP_POL if params.get("stokes", 1) == 4
           else FLOPS_PER_STEP_GRID if grid_em else FLOPS_PER_STEP)
    if dom in fps:
        d = by_kind[dom]
        achieved = d["steps"] * fps[dom] / (d["ms"] / 1000.0) / 1e12
        peak = PEAK_TFLOPS[dom]
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": TRAFFIC_PER_LAUNCH.get((args.workload, dom)),
                    "traffic_unit": "bytes per launch (ncu, cold cache)",
                    "peak_source": PEAK_SOURCE[dom],
                    "launches": d["launches"], "steps": d["steps"],
                    "share_of_step": d["ms"] / total_ms}
        # the same against this GPU's measured fused multiply-add throughput (own microbenchmark)
        meas = ctx.art_measure_alu_peaks()
        mp = meas["fp64_tflops"] if dom == "trace_fp64" else meas["fp32_tflops"]
        roofline["peak_measured"] = {**meas, "frac": achieved / mp if mp > 0 else None,
                                     "source": "art_measure_alu_peaks: FMA chains on every SM"}
        if grid_em:
            # every RK4 step samples the grid once (the start point of a ray once more)
            gbs = d["steps"] * GRID_BYTES_PER_SAMPLE / (d["ms"] / 1000.0) / 1e9
            roofline["grid_lookup"] = {
                "bytes_per_sample": GRID_BYTES_PER_SAMPLE, "samples": d["steps"],
                "achieved_GBps": gbs, "hbm_peak_GBps": HBM_PEAK_GBPS, "frac_of_hbm": gbs / HBM_PEAK_GBPS,
                "note": "algorithmic bytes (8 cells x 32 B per sample) over the kernel time; most "
                        "are served from L1/L2 (neighbouring samples share cells), so DRAM "
                        "traffic is far lower"}
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                   "share": round(v["ms"] / total_ms, 4)} for k, v in by_kind.items()}

    # the other precision paths on the same workload, for comparison
    paths = {}
    for prec in ("fp64", "mixed", "mixed_df"):
        if prec == args.precision:
            continue
        jobp = art.make_job(**{**params, "precision": prec})
        stp = ctx.art_render(jobp, img, mask, stats=True)
        kp = max(3, args.steps // 5)
        tp = timed(kp, jobp)
        paths[prec] = {"rays_per_s": stp["rays_traced"] * kp / tp,
                       "geodesic_steps_per_s": stp["steps"] * kp / tp,
                       "ms_per_step": 1000 * tp / kp, "rays_high_precision": stp["rays_fp64"]}
    if params.get("crit_band", 0.0) > 0.0:
        # the same precision without the near-critical band speculation (same image)
        jnb = art.make_job(**{**params, "crit_band": 0.0})
        stp = ctx.art_render(jnb, img, mask, stats=True)
        kp = max(3, args.steps // 5)
        tp = timed(kp, jnb)
        paths[args.precision + "_no_band"] = {
            "rays_per_s": stp["rays_traced"] * kp / tp,
            "geodesic_steps_per_s": stp["steps"] * kp / tp, "ms_per_step": 1000 * tp / kp,
            "rays_high_precision": stp["rays_fp64"]}
    # the same render replayed from a CUDA graph (one capture of the whole level loop)
    if not params.get("proposal", 0):
        ctx.art_graph_render(job, img, mask)
        kp = max(3, args.steps // 5)
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
    ctx.art_render(job, img, mask, stats=False)
    acc = accuracy(ctx, params, img, mask)
    paths[args.precision] = {"rays_per_s": value / world,
                             "geodesic_steps_per_s": steps_per_render * args.steps / t_dev,
                             "ms_per_step": 1000 * t_dev / args.steps,
                             "rays_high_precision": stats["rays_fp64"]}

    # end to end through the public C-ABI with host buffers (D2H of image + mask inside)
    import numpy as np
    himg = torch.empty((planes, ny, nx), dtype=torch.float64).pin_memory().numpy()
    hmask = torch.empty((ny, nx), dtype=torch.uint8).pin_memory().numpy()
    ctx.art_render_host(job, himg, hmask)
    ke = max(3, args.steps // 3)
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
        evs = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.art_render_batch(bjobs, bimgs, bmasks, stats=False)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        tb = sum(a.elapsed_time(b) for a, b in evs) / 1000.0 / len(evs)
        # the same batch replayed from a CUDA graph (captured on the first call)
        ctx.art_graph_render_batch(bjobs, bimgs, bmasks)
        evs = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.art_graph_render_batch(bjobs, bimgs, bmasks)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        tg = sum(a.elapsed_time(b) for a, b in evs) / 1000.0 / len(evs)
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
        # per-launch split of one batched render (CUDA events on the library's stream)
        ctx.art_profile(True)
        ctx.art_render_batch(bjobs, bimgs, bmasks, stats=False)
        brecs = ctx.art_profile_read()
        ctx.art_profile(False)
        batched["launches"] = [{"kind": r["kind"], "level": r["level"], "ms": round(r["ms"], 4),
                                "steps": r["steps"]} for r in brecs]
        # per-image error against the FP64 batch, per subring plane
        rjobs = [art.make_job(**{**p, "precision": "fp64"}) for p in bparams]
        rimgs, rmasks, _ = ctx.render_batch(rjobs)
        per = []
        flips = 0
        for a, b, ma, mb in zip(bimgs, rimgs, bmasks, rmasks):
            m0 = float(b.sum(0).double().mean())
            n = a[0].numel()
            per.append([float(((a[c] - b[c]).double() ** 2).sum()) / (n * m0 * m0)
                        for c in range(a.shape[0])])
            flips += int((ma != mb).sum())
        per = np.array(per)
        batched["accuracy"] = {
            "against": "the FP64 batch", "planes": [f"I_n{c}" for c in range(per.shape[1])],
            "image_bj_median": np.median(per, 0).tolist(), "image_bj_max": per.max(0).tolist(),
            "images_above_1e-5": int((per.sum(1) > 1e-5).sum()), "mask_flips": flips}
        del rimgs, rmasks
        del bimgs, bmasks

    # the learned path: train the block-proposal network on seeded plain renders (the library's
    # own tensor-core forward/backward and Adam), then render the workload with it
    learned = None
    lctx = None
    if not args.no_learned:
        from paper_2103_07417_gb300 import learn
        t0 = time.perf_counter()
        lctx, hist = learn.trained_context(seed=0, n_jobs=96, epochs=12, device=local,
                                           snapshot=snap if snap is not None else W.grmhd_snapshot(seed=0))
        t_train = time.perf_counter() - t0
        best, best_nb = None, None
        band0 = params.get("crit_band", 0.0)
        for band in sorted({0.0, band0}):
            for depth in (2, 3):
                for thr in (0.2, 0.3, 0.5, 0.7):
                    lj = art.make_job(**{**params, "proposal": 1, "proposal_p": thr,
                                         "proposal_depth": depth, "crit_band": band})
                    lst = lctx.art_render(lj, img, mask, stats=True)
                    tl = _timed_ctx(lctx, lj, img, mask, flush, 5)
                    cand = dict(depth=depth, threshold=thr, crit_band=band, ms_per_step=1000 * tl,
                                rays_per_s=lst["rays_traced"] / tl,
                                rays_speculative=lst["rays_speculative"],
                                rays_spec_used=lst["rays_spec_used"])
                    if best is None or cand["ms_per_step"] < best["ms_per_step"]:
                        best = cand
                    if band == 0.0 and (best_nb is None or cand["ms_per_step"] < best_nb["ms_per_step"]):
                        best_nb = cand
        plain_nb = paths.get(args.precision + "_no_band", paths[args.precision])["ms_per_step"]
        learned = {"training": {"jobs": 96, "epochs": 12, "seconds": t_train,
                                "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]},
                   "best": best, "best_without_band": best_nb,
                   "gain_vs_plain": (1000 * t_dev / args.steps) / best["ms_per_step"],
                   "gain_vs_plain_both_without_band": plain_nb / best_nb["ms_per_step"],
                   "note": "same image and mask as the plain render (the exact criterion decides "
                           "every point); lookahead depth, threshold and band chosen among "
                           "{2,3} x {0.2,0.3,0.5,0.7} x {0, default} by timing"}

    # the proposal network's tensor-core kernels alone: forward (4 implicit-GEMM convolutions +
    # head) and forward + backward on a 2049 x 2049 lattice, host-timed (each call synchronises)
    cnn = None
    if lctx is not None:
        nlat = 2049
        t_fw, t_fb = cnn_measure(lctx, nlat)
        fl = cnn_flops(nlat, nlat)
        peak = 1941.4  # measured cuBLAS BF16 dense GEMM rate of a GB300 (burst), TFLOP/s
        cnn = {"lattice": f"{nlat}x{nlat}", "forward_ms": 1000 * t_fw,
               "forward_backward_ms": 1000 * t_fb,
               "roofline": {"bound": "tensor", "achieved": fl / t_fw / 1e12, "peak": peak,
                            "unit": "TFLOP/s", "frac": fl / t_fw / 1e12 / peak,
                            "peak_source": "measured cuBLAS bf16 dense GEMM, burst",
                            "flops_per_forward": fl}}

    # time to a 0.1 %-MSE image (paper MSE vs the full FP64 trace) for each path: the fastest
    # tolerance R = R_rel = R_abs meeting it
    time_to_mse = None
    if not args.no_mse and not args.gpus > 1:
        if nx * ny <= (1 << 23):
            tjob = art.make_job(**{**params, "precision": "fp64", "R_rel": -1.0, "R_abs": -1.0})
            truth = torch.empty_like(img)
            ctx.art_render(tjob, truth, mask, stats=False)
            rlist = (3e-3, 1e-3, 3e-4, 1e-4) if params.get("emission") != "grid" else (0.1, 0.025, 1e-2, 3e-3)
            time_to_mse = {"target_mse": 1e-3, "truth": "full FP64 trace of the final grid",
                           "sweep_R": list(rlist), "paths": {}}
            variants = [("fp64", ctx, {"precision": "fp64", "crit_band": 0.0}),
                        ("mixed_df_no_band", ctx, {"precision": "mixed_df", "crit_band": 0.0}),
                        ("mixed_df", ctx, {"precision": "mixed_df"})]
            if lctx is not None:
                variants.append(("mixed_df+learned", lctx,
                                 {"precision": "mixed_df", "proposal": 1,
                                  "proposal_p": learned["best"]["threshold"],
                                  "proposal_depth": learned["best"]["depth"],
                                  "crit_band": learned["best"]["crit_band"]}))
            for name, cx, over in variants:
                rec, sweep = None, []
                for R in rlist:
                    rr = {"R_abs": R} if params.get("emission") == "grid" else {"R_abs": R, "R_rel": R}
                    vj = art.make_job(**{**params, **over, **rr})
                    vst = cx.art_render(vj, img, mask, stats=True)
                    met = cx.art_metrics(truth[0], img[0], mask)
                    tv = _timed_ctx(cx, vj, img, mask, flush, 3)
                    sweep.append({"R": R, "mse": met["MSE"], "IF": met["IF"], "seconds": tv,
                                  "rays": vst["rays_traced"]})
                    if met["MSE"] <= 1e-3 and (rec is None or tv < rec["seconds"]):
                        rec = {"seconds": tv, "R": R, "mse": met["MSE"]}
                time_to_mse["paths"][name] = {"best": rec, "sweep": sweep}
            del truth
        else:
            time_to_mse = {"skipped": "final grid above 2^23 points: the FP64 truth trace is too "
                                      "long for the default run"}
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
                           "adaptive_ray_fraction": rays / (nx * ny),
                           "l2": "flushed (512 MB write) before every step, outside the timed "
                                 "region", "parallelism": f"replicas x{world}"},
                "geodesic_steps_per_s": steps_per_render * args.steps * world / t_dev,
                "paths": paths, "batched": batched, "learned": learned, "cnn": cnn,
                "time_to_mse": time_to_mse, "accuracy": acc, "roofline": roofline,
                "kernels": kernels,
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
