"""Training and use of the learned block proposal through the C-ABI (art_cnn_*).

The network (see include/art.h) is trained on masks of the plain method: each finished render of
a seeded job yields, for every level L with L + 2 <= N, the features of the level-L lattice and
the block labels "the exact criterion traced a point of a level >= L + 2 here" (art_cnn_sample).
Training runs on the GPU through the library's own tensor-core forward and backward passes and
its Adam step (art_cnn_train_step).  Argument marshalling only; no arithmetic of the method here.
"""
from __future__ import annotations

import numpy as np

from . import art
from . import workloads as W


def training_jobs(seed: int, n: int) -> list:
    """n seeded jobs mixing the three emission models at small sizes (final 129^2 .. 513^2 over
    3..5 levels), random spin, inclination and field of view: the configuration-3 recipe,
    alternating the grid snapshot, the polarized synchrotron disk and the analytic
    Keplerian emissivity."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        a = float(rng.uniform(-0.94, 0.94))
        k = int(rng.integers(7, 10))
        N = int(rng.integers(3, 6))
        n0 = (1 << (k - N)) + 1
        incl = float(rng.uniform(10.0, 170.0))
        fov = float(np.exp(rng.uniform(np.log(30.0), np.log(200.0))))
        common = dict(a=a, incl_deg=incl, fov=fov, n0x=n0, n0y=n0, levels=N, precision="mixed_df")
        kind = i % 3
        if kind == 0:
            p = W.grmhd_8193(**common)
        elif kind == 1:
            p = W.kerr_disk_2049(**common, stokes=1, r_in=W.r_isco(a))
        else:
            p = W.kerr_analytic_2049(**common)
        out.append(p)
    return out


def collect(ctx, jobs) -> list:
    """(features, targets) device tensors of every level with a target, from plain renders.
    The context must hold a network (so renders record the per-pixel diagnostics) and, for grid
    jobs, the snapshot."""
    samples = []
    for p in jobs:
        job = art.make_job(**{**p, "proposal": 0})
        img, mask, _ = ctx.render(job)
        for L in range(0, p["levels"] - 1):
            samples.append(ctx.art_cnn_sample(job, img[0], mask, L))
    return samples


def train(ctx, samples, epochs: int = 12, lr: float = 3e-3, seed: int = 0) -> list:
    """Adam over the samples in seeded random order; returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        tot = 0.0
        for i in rng.permutation(len(samples)):
            f, t = samples[i]
            tot += ctx.art_cnn_train_step(f, t, lr)
        hist.append(tot / max(len(samples), 1))
    return hist


def block_scores(ctx, samples, thr: float) -> dict:
    """Recall and precision of the blocks the network proposes at threshold thr."""
    tp = fp = fn = 0
    for f, t in samples:
        p = ctx.art_cnn_forward(f)
        pred = (p > thr).cpu().numpy()
        tru = t.cpu().numpy() > 0.5
        tp += int((pred & tru).sum())
        fp += int((pred & ~tru).sum())
        fn += int((~pred & tru).sum())
    return dict(recall=tp / max(tp + fn, 1), precision=tp / max(tp + fp, 1), positives=tp + fn)


def trained_context(seed: int = 0, n_jobs: int = 96, epochs: int = 12, device: int = 0,
                    snapshot=None, info: bool = False):
    """A context with the snapshot loaded and a network trained from W.cnn_init(seed) on
    n_jobs seeded plain renders; returns (ctx, loss history[, dict of sample count and the
    seconds spent rendering and training])."""
    import time
    ctx = art.Context(device)
    ctx.load_grid(snapshot if snapshot is not None else W.grmhd_snapshot(seed=0))
    ctx.art_cnn_load(W.cnn_init(seed))
    t0 = time.perf_counter()
    samples = collect(ctx, training_jobs(seed, n_jobs))
    t1 = time.perf_counter()
    hist = train(ctx, samples, epochs=epochs, seed=seed)
    t2 = time.perf_counter()
    if info:
        return ctx, hist, {"samples": len(samples), "render_seconds": t1 - t0,
                           "train_seconds": t2 - t1}
    return ctx, hist
