"""TEST INFRASTRUCTURE ONLY: CPU oracle of adaptive sampling along a third axis (frequency or
time).

Sec. 6 of the paper proposes extending the adaptive scheme to sample the time and frequency
domains selectively.  Reading used here: the samples of the axis (frequencies, movie frames) form a
one-dimensional grid that is refined exactly as a line of the image is in Sec. 3.2.  With F0 base
samples and N3 levels there are F = 2^N3 (F0 - 1) + 1 samples; the images at the base samples
(indices that are multiples of 2^N3) are rendered by the ordinary adaptive scheme; then, for
k = 1..N3, every pixel of every new sample f (an odd multiple of s = 2^(N3 - k)) is decided with the
one-dimensional estimator of Sec. 3.2 (the category 2/3 form of Eqs. epabs and eprel, Appendix A):

    S_in  = I(f - s) + I(f + s),   second difference along the axis
    d     = I(f - 3s) - I(f - s) - I(f + s) + I(f + 3s)
            (one-sided where one outer sample is missing: 2 (I_out - 2 I_in,near + I_in,far);
             none: the estimate is infinite),
    eps_abs = |d| / (8 I_bar),  eps_rel = |d| / (4 |S_in| / 2) = |d| / (2 |S_in|),
    trace iff eps_abs > R_abs3 and eps_rel > R_rel3 (strict), NaN traces;
    otherwise the pixel's value at f is S_in / 2 in every plane,

on plane 0 (I), reading only samples of level k - 1.  I_bar is the mean over the base samples of
their I_bar_int (the interpolated mean intensity of each base image's first pass), fixed for all
levels like I_bar_int in Sec. 3.2.

With a truth cube (the axis logic alone) every pixel of a new sample is decided along the axis.
With jobs (`render_axis_jobs`) the axis is combined with the spatial scheme: a new sample's image
is refined in x and y as in Sec. 3.2, and every point that scheme would trace is traced only if the
axis estimate also asks for it; otherwise it receives the axis interpolant (mask AXIS = 3).  A
point is then traced only where neither interpolant is good enough.  Pinned by
tests/test_oracle_axis.py.
"""
from __future__ import annotations

import numpy as np

MASK_TRACED, MASK_INTERP, MASK_AXIS = 1, 2, 3


def axis_decide(lo3, lo1, hi1, hi3, norm, R_rel, R_abs):
    """Decisions, interpolants and estimates for arrays of axis neighbours (NaN = missing outer
    sample).  Returns (trace bool array, interpolant array, eps_abs, eps_rel)."""
    lo3, lo1, hi1, hi3 = (np.asarray(v, dtype=np.float64) for v in (lo3, lo1, hi1, hi3))
    has_lo, has_hi = ~np.isnan(lo3), ~np.isnan(hi3)
    both = ((lo3 - lo1) - hi1) + hi3
    one_lo = 2.0 * ((lo3 - 2.0 * lo1) + hi1)
    one_hi = 2.0 * ((hi3 - 2.0 * hi1) + lo1)
    d = np.where(has_lo & has_hi, both, np.where(has_lo, one_lo, np.where(has_hi, one_hi, np.nan)))
    none = ~has_lo & ~has_hi
    s_in = lo1 + hi1
    num = np.abs(d) / 8.0
    den = np.abs(s_in) / 2.0
    with np.errstate(divide="ignore", invalid="ignore"):
        ea = np.where(none, np.inf, num / norm)
        er = np.where(none, np.inf, np.where(den == 0.0, np.where(num == 0.0, 0.0, np.inf), num / den))
    trace = (ea > R_abs) & (er > R_rel)
    trace |= np.isnan(ea) | np.isnan(er) | np.isnan(s_in)
    return trace, 0.5 * s_in, ea, er


def render_axis(n_samples, levels3, R_rel3, R_abs3, truth=None, base_render=None,
                trace_pixels=None):
    """The cube (F, planes, ny, nx), the axis mask (F, ny, nx) and per-sample traced counts.

    truth: (F, planes, ny, nx) -- base samples copy it, traced pixels read it.  Otherwise
    base_render(f) -> (image (planes, ny, nx), I_bar_int) and trace_pixels(f, pix) ->
    values (n, planes) supply the images and traces."""
    F = n_samples
    S = 1 << levels3
    if (F - 1) % S:
        raise ValueError("F must be 2^levels3 (F0 - 1) + 1")
    cube, norms, counts = [None] * F, [], [0] * F
    amask = None
    for f in range(0, F, S):
        if truth is not None:
            img = np.array(truth[f], dtype=np.float64)
            from oracle import ibar_int
            norms.append(ibar_int(img[0], 1))
        else:
            img, nb = base_render(f)
            norms.append(nb)
        cube[f] = img
    planes, ny, nx = cube[0].shape
    amask = np.zeros((F, ny, nx), np.uint8)
    for f in range(0, F, S):
        amask[f] = MASK_TRACED
        counts[f] = ny * nx
    norm = float(np.mean(norms))
    for k in range(1, levels3 + 1):
        s = 1 << (levels3 - k)
        for f in range(s, F, 2 * s):
            lo1, hi1 = cube[f - s][0], cube[f + s][0]
            nan = np.full((ny, nx), np.nan)
            lo3 = cube[f - 3 * s][0] if f - 3 * s >= 0 else nan
            hi3 = cube[f + 3 * s][0] if f + 3 * s < F else nan
            tr, _, _, _ = axis_decide(lo3, lo1, hi1, hi3, norm, R_rel3, R_abs3)
            img = 0.5 * (cube[f - s] + cube[f + s])
            pix = np.flatnonzero(tr.ravel())
            if pix.size:
                if truth is not None:
                    vals = np.asarray(truth[f], dtype=np.float64).reshape(planes, -1)[:, pix].T
                else:
                    vals = trace_pixels(f, pix)
                flat = img.reshape(planes, -1)
                flat[:, pix] = vals.T
            cube[f] = img
            amask[f] = np.where(tr, MASK_TRACED, MASK_INTERP)
            counts[f] = int(pix.size)
    return np.stack(cube), amask, counts, norm


def render_axis_jobs(ojobs, levels3, R_rel3, R_abs3):
    """The combined scheme with the oracle's tracer: ojobs[f] the oracle job of sample f (all with
    the same pixel grid).  Returns (cube (F, planes, ny, nx), mask (F, ny, nx), rays traced per
    sample, I_bar)."""
    import oracle as O
    F = len(ojobs)
    S = 1 << levels3
    if (F - 1) % S:
        raise ValueError("F must be 2^levels3 (F0 - 1) + 1")
    cube, masks, counts, norms = [None] * F, [None] * F, [0] * F, []
    for f in range(0, F, S):
        img, m, st = O.render(ojobs[f], None)
        img = img if img.ndim == 3 else img[None]
        cube[f], masks[f], counts[f] = img, m, st["rays_traced"]
        norms.append(st["ibar"])
    norm = float(np.mean(norms))
    planes, ny, nx = cube[0].shape
    for k in range(1, levels3 + 1):
        s = 1 << (levels3 - k)
        for f in range(s, F, 2 * s):
            job = ojobs[f]
            nan = np.full(ny * nx, np.nan)
            lo1, hi1 = cube[f - s][0].ravel(), cube[f + s][0].ravel()
            lo3 = cube[f - 3 * s][0].ravel() if f - 3 * s >= 0 else nan
            hi3 = cube[f + 3 * s][0].ravel() if f + 3 * s < F else nan
            axis_tr, _, _, _ = axis_decide(lo3, lo1, hi1, hi3, norm, R_rel3, R_abs3)
            axis_val = 0.5 * (cube[f - s] + cube[f + s])
            img = np.full((planes, ny, nx), np.nan)
            mask = np.zeros((ny, nx), np.uint8)
            N = job.levels
            S0 = 1 << N

            def settle(cand):
                """Trace the candidates the axis also asks for; axis-interpolate the rest."""
                keep = cand[axis_tr[cand]]
                rest = cand[~axis_tr[cand]]
                flat = img.reshape(planes, -1)
                if keep.size:
                    vals, _ = O.trace_pixels(job, keep.astype(np.int64))
                    flat[:, keep] = vals.T
                    mask.ravel()[keep] = MASK_TRACED
                flat[:, rest] = axis_val.reshape(planes, -1)[:, rest]
                mask.ravel()[rest] = MASK_AXIS
                return int(keep.size)

            jj, ii = np.mgrid[0:ny:S0, 0:nx:S0]
            n_tr = settle((jj * nx + ii).ravel())
            crit = img[job.criterion_plane]
            lvl_norm = O.ibar_int(crit, S0)
            for level in range(1, N + 1):
                full = img if planes > 1 else img[0]
                out, m2, _, _ = O.refine_level(job, full, mask, level, lvl_norm)
                out = out if out.ndim == 3 else out[None]
                sl = 1 << (N - level)
                newpts = np.zeros((ny, nx), bool)
                newpts[::sl, ::sl] = True
                newpts[::2 * sl, ::2 * sl] = False
                cand = np.flatnonzero((newpts & (m2 == MASK_TRACED)).ravel())
                interp = newpts & (m2 == MASK_INTERP)
                img[:, interp] = out[:, interp]
                mask[interp] = MASK_INTERP
                n_tr += settle(cand)
            cube[f], masks[f], counts[f] = img, mask, n_tr
    return np.stack(cube), np.stack(masks), counts, norm
