"""Pins of the oracle's adaptive-refinement logic (Sec. 3.2, Eqs. epabs/eprel, Appendix A/B).

Each test checks the oracle against something other than itself: the paper's printed power-law
ratios, closed forms on polynomial images, a library bilinear interpolator, numpy's trapezoid
rule, or brute force.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _job(**kw):
    return O.make_job(**W.job(**kw))


def _paper_values():
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        return json.load(f)


# ------------------------------------------------------------------------------------------
# grid
# ------------------------------------------------------------------------------------------

def test_image_size_matches_paper_examples():
    """Sec. 3.2: n = 2^N (n0-1) + 1; the paper's 65 -> 1025 and 65 -> 4097 examples."""
    for case in _paper_values()["image_sizes"]:
        job = _job(n0x=case["n0"], n0y=case["n0"], levels=case["levels"])
        assert O.image_size(job) == (case["n"], case["n"]), case


def test_level_plan_visits_every_pixel_once():
    """Brute force: base points plus the new points of every level tile the final grid."""
    job = _job(n0x=5, n0y=4, levels=3, R_abs=-1.0, R_rel=-1.0)
    nx, ny = O.image_size(job)
    truth = np.arange(nx * ny, dtype=np.float64).reshape(ny, nx) + 1.0
    img, mask, st = O.render(job, truth)
    assert (mask == O.MASK_TRACED).all()
    assert st["rays_traced"] == nx * ny
    expect = [5 * 4]
    prev = (5, 4)
    for _ in range(3):
        cur = (2 * prev[0] - 1, 2 * prev[1] - 1)
        expect.append(cur[0] * cur[1] - prev[0] * prev[1])
        prev = cur
    assert st["rays_per_level"] == expect


# ------------------------------------------------------------------------------------------
# I_bar_int
# ------------------------------------------------------------------------------------------

def test_ibar_int_is_trapezoid_mean():
    """I_bar_int = mean of the bilinear interpolant = 2-D trapezoid rule / area."""
    rng = np.random.default_rng(3)
    for nx0, ny0 in [(9, 9), (17, 5), (2, 2)]:
        base = rng.uniform(0.1, 2.0, size=(ny0, nx0))
        stride = 4
        nx, ny = (nx0 - 1) * stride + 1, (ny0 - 1) * stride + 1
        img = np.full((ny, nx), np.nan)
        img[::stride, ::stride] = base
        got = O.ibar_int(img, stride)
        ref = np.trapezoid(np.trapezoid(base, axis=1), axis=0) / ((nx0 - 1) * (ny0 - 1))
        assert got == pytest.approx(ref, rel=1e-14)
    img = np.full((9, 9), 3.25)
    assert O.ibar_int(img, 4) == 3.25


# ------------------------------------------------------------------------------------------
# estimator closed forms
# ------------------------------------------------------------------------------------------

def _level_setup(truth, levels, level):
    """Image holding the truth on the level-(level-1) lattice and NaN elsewhere."""
    ny, nx = truth.shape
    sprev = 1 << (levels - level + 1)
    img = np.full_like(truth, np.nan)
    img[::sprev, ::sprev] = truth[::sprev, ::sprev]
    mask = np.zeros(truth.shape, np.uint8)
    mask[::sprev, ::sprev] = O.MASK_TRACED
    return img, mask


def test_planes_give_zero_estimate_and_exact_interpolation():
    """A plane is reproduced exactly by linear interpolation and its second differences vanish,
    so every estimate is 0 and nothing is traced (Appendix A) -- except the four corner cell
    centres of each level, whose anti-diagonal has no outer point at all (edge reading)."""
    job = _job(n0x=9, n0y=7, levels=3, R_abs=1e-12, R_rel=1e-12)
    nx, ny = O.image_size(job)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    truth = 2.0 + 0.25 * x - 0.125 * y  # dyadic coefficients: exact in binary
    img, mask, st = O.render(job, truth)
    assert st["rays_traced"] == 9 * 7 + 4 * 3
    np.testing.assert_array_equal(img, truth)
    for level in (1, 2, 3):
        im, m = _level_setup(truth, 3, level)
        _, _, ea, er = O.refine_level(job, im, m, level, 1.0)
        new = np.isfinite(ea)
        assert new.sum() > 0
        assert np.all(ea[new] == 0.0) and np.all(er[new] == 0.0)
        assert np.isinf(ea).sum() == 4


@pytest.mark.parametrize("edge_mode", ["onesided", "trace"])
def test_quadratic_estimate_is_twice_true_residual(edge_mode):
    """On I = x^2 + y^2 (pixel units) the printed estimators (second derivative written as
    (I8 - I4 - I1 + I5)/(4 dx^2), Appendix A) give exactly twice the true linear-interpolation
    residual, for every category and also where the one-sided edge rule applies."""
    levels, level = 3, 2
    job = _job(n0x=9, n0y=9, levels=levels, R_abs=np.inf, R_rel=np.inf, edge_mode=edge_mode)
    nx, ny = O.image_size(job)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    truth = x * x + y * y
    im, m = _level_setup(truth, levels, level)
    out, m2, ea, er = O.refine_level(job, im, m, level, 1.0)
    new = ~np.isnan(ea) & (m2 == O.MASK_INTERP)
    s = 1 << (levels - level)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    cat4 = new & ((ii // s) % 2 == 1) & ((jj // s) % 2 == 1)
    cat23 = new & ~cat4
    resid = np.abs(out - truth)
    # category 4: corners at distance sqrt(2) s -> residual 2 s^2 ; categories 2/3: s^2
    np.testing.assert_array_equal(resid[cat4], 2.0 * s * s)
    np.testing.assert_array_equal(resid[cat23], 1.0 * s * s)
    finite = new & np.isfinite(ea)
    np.testing.assert_array_equal(ea[finite], 2.0 * resid[finite])
    assert finite.sum() > 0.8 * (~np.isnan(ea)).sum()
    if edge_mode == "trace":
        assert (m2[~np.isnan(ea)] == O.MASK_TRACED).sum() > 4  # edge points forced to trace


@pytest.mark.parametrize("coef", [(0.0, 0.0, 0.0, 0.75, -0.5), (0.125, -0.375, 0.25, 1.5, 0.25),
                                  (-0.25, 0.5, 0.0, -2.0, 1.0)])
def test_nearest_estimate_is_gradient_times_distance(coef):
    """Nearest scheme, Appendix A.1: the residual of a nearest-neighbour copy is extremised by
    |grad I| dx with dx the distance to the nearest sample, and the gradient comes from central
    differences along the two diagonals through the corners (1-4 and 2-3).  On any quadratic
    I = c2x x^2 + cxy x y + c2y y^2 + c1x x + c1y y the central differences are exact, so at
    every cell centre (category 4) eps_abs * norm = |grad I(x)| * sqrt(2) s, and at every edge
    midpoint (categories 2/3) it is |dI/dx| s (or |dI/dy| s) along the pair; eps_rel divides the
    same numerator by |I_1| (the lower-left corner, resp. the lower/left neighbour), and the
    interpolant is I_1.  A swapped diagonal pairing, a wrong divisor or another corner as the
    nearest neighbour changes these values for a gradient that is not along an axis."""
    c2x, cxy, c2y, c1x, c1y = coef
    levels, level = 3, 2
    norm = 1.75
    job = _job(n0x=9, n0y=7, levels=levels, R_abs=np.inf, R_rel=np.inf, interp="nearest")
    nx, ny = O.image_size(job)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    truth = 3.0 + c2x * x * x + cxy * x * y + c2y * y * y + c1x * x + c1y * y
    gx = 2 * c2x * x + cxy * y + c1x
    gy = cxy * x + 2 * c2y * y + c1y
    im, m = _level_setup(truth, levels, level)
    out, m2, ea, er = O.refine_level(job, im, m, level, norm)
    s = 1 << (levels - level)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    new = ~np.isnan(ea)
    oi, oj = (ii // s) % 2 == 1, (jj // s) % 2 == 1
    cat4 = new & oi & oj
    cat3 = new & oi & ~oj   # between a left/right pair
    cat2 = new & ~oi & oj   # between a pair below/above
    assert cat4.sum() > 0 and cat3.sum() > 0 and cat2.sum() > 0
    num4 = np.hypot(gx, gy) * np.sqrt(2.0) * s
    np.testing.assert_allclose(ea[cat4] * norm, num4[cat4], rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(ea[cat3] * norm, np.abs(gx[cat3]) * s, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(ea[cat2] * norm, np.abs(gy[cat2]) * s, rtol=1e-13, atol=1e-12)
    # I_1 of a centre is its lower-left corner (i - s, j - s); of a midpoint the lower/left one
    i1 = np.full_like(truth, np.nan)
    i1[s:, s:][cat4[s:, s:]] = truth[:-s, :-s][cat4[s:, s:]]
    i1[:, s:][cat3[:, s:]] = truth[:, :-s][cat3[:, s:]]
    i1[s:, :][cat2[s:, :]] = truth[:-s, :][cat2[s:, :]]
    for sel, numv in ((cat4, num4), (cat3, np.abs(gx) * s), (cat2, np.abs(gy) * s)):
        with np.errstate(divide="ignore"):
            ref = numv[sel] / np.abs(i1[sel])
        np.testing.assert_allclose(er[sel], ref, rtol=1e-13, atol=1e-12)
        np.testing.assert_array_equal(out[sel], i1[sel])


def test_tie_and_zero_denominator_rules():
    """Strict '>' (Sec. 3.2): an estimate equal to the tolerance interpolates.  S_in = 0 with a
    zero numerator gives eps_rel = 0; with a non-zero numerator eps_rel = inf."""
    levels = 1
    nx = 9
    truth = np.zeros((1, nx))
    truth[0, ::2] = [0.0, 0.0, 0.0, 4.0, 0.0]      # level-0 samples at x = 0, 2, 4, 6, 8
    job = _job(n0x=5, n0y=1, levels=levels, R_abs=0.5, R_rel=0.0)
    im, m = _level_setup(truth, levels, 1)
    out, m2, ea, er = O.refine_level(job, im, m, 1, 1.0)
    # point x=1: inner (0, 0), outer one-sided (x=-1 missing, x=3 -> 0): num 0 -> interp
    assert ea[0, 1] == 0.0 and er[0, 1] == 0.0 and m2[0, 1] == O.MASK_INTERP
    # point x=3: inner (0, 4), outer (0 at x=0? no: x=0 and x=6) -> |0 + 0 - 0 - 4|/8 = 0.5 == R
    assert ea[0, 3] == 0.5 and m2[0, 3] == O.MASK_INTERP
    # point x=5: inner (4, 0), outer (x=2 -> 0, x=8 -> 0): 0.5 as well
    assert ea[0, 5] == 0.5
    job2 = _job(n0x=5, n0y=1, levels=levels, R_abs=0.49, R_rel=0.0)
    _, m3, _, _ = O.refine_level(job2, im, m, 1, 1.0)
    assert m3[0, 3] == O.MASK_TRACED
    # S_in = 0, numerator != 0 -> eps_rel = inf
    truth2 = np.zeros((1, nx))
    truth2[0, ::2] = [3.0, 1.0, -1.0, 5.0, 0.0]
    im2, mm = _level_setup(truth2, levels, 1)
    _, _, ea2, er2 = O.refine_level(job, im2, mm, 1, 1.0)
    assert np.isinf(er2[0, 3])  # inner pair (1, -1) sums to 0


def test_nan_input_is_traced():
    job = _job(n0x=9, n0y=9, levels=1, R_abs=1e9, R_rel=1e9)
    truth = np.ones((17, 17))
    im, m = _level_setup(truth, 1, 1)
    im[8, 8] = np.nan
    _, m2, _, _ = O.refine_level(job, im, m, 1, 1.0)
    assert m2[7, 7] == O.MASK_TRACED and m2[8, 7] == O.MASK_TRACED
    assert m2[5, 5] == O.MASK_TRACED  # outer diagonal point is the NaN
    assert m2[11, 3] == O.MASK_INTERP


# ------------------------------------------------------------------------------------------
# limits of the decision rule
# ------------------------------------------------------------------------------------------

def test_always_trace_limit_reproduces_truth():
    """R -> -inf: every point is traced and the image equals the full trace bit for bit."""
    job = _job(n0x=9, n0y=6, levels=3, R_abs=-np.inf, R_rel=-np.inf)
    nx, ny = O.image_size(job)
    truth = W.ring_image(5, nx, ny)
    img, mask, st = O.render(job, truth)
    np.testing.assert_array_equal(img, truth)
    assert st["rays_traced"] == nx * ny


def test_never_trace_limit_is_bilinear_upsampling():
    """R -> +inf: recursive midpoint interpolation equals the bilinear interpolant of the base
    grid (scipy's RegularGridInterpolator) -- Sec. 4.1's 'initial sampling' limit."""
    from scipy.interpolate import RegularGridInterpolator

    job = _job(n0x=7, n0y=5, levels=3, R_abs=np.inf, R_rel=np.inf)
    nx, ny = O.image_size(job)
    truth = W.smooth_image(11, nx, ny)
    img, mask, st = O.render(job, truth)
    s0 = 8
    base = truth[::s0, ::s0]
    f = RegularGridInterpolator((np.arange(0, ny, s0), np.arange(0, nx, s0)), base)
    yy, xx = np.mgrid[0:ny, 0:nx]
    ref = f(np.stack([yy.ravel(), xx.ravel()], axis=1)).reshape(ny, nx)
    np.testing.assert_allclose(img, ref, rtol=1e-13, atol=1e-15)
    assert st["rays_traced"] == 7 * 5
    interp_frac = O.metrics(truth, img, mask)["IF"]
    assert interp_frac == pytest.approx(1 - 35 / (nx * ny))


def test_adaptive_traced_points_equal_truth_and_interpolants_are_means():
    """Brute force on a small image: traced points carry the truth; every interpolated point
    equals the mean of its 2 or 4 level-(k-1) neighbours."""
    levels = 3
    job = _job(n0x=5, n0y=5, levels=levels, R_abs=1e-3, R_rel=1e-3)
    nx, ny = O.image_size(job)
    truth = W.ring_image(2, nx, ny)
    img, mask, st = O.render(job, truth)
    tr = mask == O.MASK_TRACED
    np.testing.assert_array_equal(img[tr], truth[tr])
    assert 0 < st["rays_traced"] < nx * ny
    for level in range(1, levels + 1):
        s = 1 << (levels - level)
        for j in range(0, ny, s):
            for i in range(0, nx, s):
                oi, oj = (i // s) % 2, (j // s) % 2
                if (oi, oj) == (0, 0) or mask[j, i] != O.MASK_INTERP:
                    continue
                if oi and oj:
                    ref = (img[j - s, i - s] + img[j + s, i - s] + img[j - s, i + s]
                           + img[j + s, i + s]) / 4
                elif oi:
                    ref = (img[j, i - s] + img[j, i + s]) / 2
                else:
                    ref = (img[j - s, i] + img[j + s, i]) / 2
                assert img[j, i] == pytest.approx(ref, rel=1e-15)


# ------------------------------------------------------------------------------------------
# power-law (turbulent) fields: the paper's printed ensemble ratios (Sec. 3.2, Appendix B)
# ------------------------------------------------------------------------------------------

def _powerlaw_row(beta, n, seed):
    return W.fbm(seed, n, hurst=(beta - 2.0) / 2.0)


@pytest.mark.parametrize("beta", [2.5, 3.0])
def test_powerlaw_ratio_linear(beta):
    """1-D linear scheme: <eps_hat^2>^1/2 / <eps^2>^1/2 = 2^(b/2-4) sqrt((1+2^(b-1)-3^(b-2)) /
    (1-2^(b-4))), 0.27 at beta = 2.5 (Sec. 3.2).  This pins the category-2/3 divisor 8."""
    pv = _paper_values()["powerlaw"]
    n = 1 << 19
    truth = _powerlaw_row(beta, n, seed=7)[None, :]
    job = _job(n0x=n // 2 + 1, n0y=1, levels=1, R_abs=np.inf, R_rel=np.inf)
    im, m = _level_setup(truth, 1, 1)
    out, _, ea, _ = O.refine_level(job, im, m, 1, 1.0)
    sl = slice(5, truth.shape[1] - 5, 2)
    est = ea[0, sl]
    err = (out - truth)[0, sl]
    ratio = np.sqrt(np.mean(est ** 2) / np.mean(err ** 2))
    formula = 2 ** (beta / 2 - 4) * np.sqrt((1 + 2 ** (beta - 1) - 3 ** (beta - 2))
                                            / (1 - 2 ** (beta - 4)))
    assert ratio == pytest.approx(formula, rel=0.02)
    if beta == 2.5:
        assert ratio == pytest.approx(pv["linear_ratio_beta_2.5"], abs=0.01)


def test_powerlaw_ratio_nearest_and_linear_vs_nearest():
    """1-D nearest scheme: ratio 2^(b/2-2) = 0.59 at beta 2.5 (Sec. 3.2); and the true linear /
    nearest residual ratio sqrt(1 - 2^(b-4)) = 0.80 (Appendix B)."""
    pv = _paper_values()["powerlaw"]
    beta, n = 2.5, 1 << 19
    truth = _powerlaw_row(beta, n, seed=8)[None, :]
    jn = _job(n0x=n // 2 + 1, n0y=1, levels=1, R_abs=np.inf, R_rel=np.inf, interp="nearest")
    jl = _job(n0x=n // 2 + 1, n0y=1, levels=1, R_abs=np.inf, R_rel=np.inf, interp="linear")
    im, m = _level_setup(truth, 1, 1)
    outn, _, ean, _ = O.refine_level(jn, im, m, 1, 1.0)
    outl, _, _, _ = O.refine_level(jl, im, m, 1, 1.0)
    sl = slice(5, truth.shape[1] - 5, 2)
    errn = (outn - truth)[0, sl]
    errl = (outl - truth)[0, sl]
    ratio = np.sqrt(np.mean(ean[0, sl] ** 2) / np.mean(errn ** 2))
    assert ratio == pytest.approx(2 ** (beta / 2 - 2), rel=0.02)
    assert ratio == pytest.approx(pv["nearest_ratio_beta_2.5"], abs=0.01)
    lin_vs_nn = np.sqrt(np.mean(errl ** 2) / np.mean(errn ** 2))
    assert lin_vs_nn == pytest.approx(np.sqrt(1 - 2 ** (beta - 4)), rel=0.02)
    assert lin_vs_nn == pytest.approx(pv["linear_over_nearest_beta_2.5"], abs=0.01)


# ------------------------------------------------------------------------------------------
# metrics (Eqs. interpdef, fluxdef, msedef)
# ------------------------------------------------------------------------------------------

def test_metrics_small_example():
    truth = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    img = truth.copy()
    img[1, 1] = 6.0
    mask = np.full(truth.shape, O.MASK_TRACED, np.uint8)
    mask[1, 1] = O.MASK_INTERP
    mt = O.metrics(truth, img, mask)
    assert mt["IF"] == pytest.approx(1 / 6)
    assert mt["MSE"] == pytest.approx(1.0 / np.sum(truth ** 2))
    F = np.trapezoid(np.trapezoid(truth, axis=1))
    Fh = np.trapezoid(np.trapezoid(img, axis=1))
    assert mt["FE"] == pytest.approx(abs(F - Fh) / F)
    assert mt["MSE_mean"] == pytest.approx(1.0 / (6 * np.mean(truth) ** 2))


# ------------------------------------------------------------------------------------------
# polarized criterion (Sec. 6: "replacing I by Q, U, V")
# ------------------------------------------------------------------------------------------

def _pol_job(criterion, **kw):
    return O.make_job(**W.job(stokes=4, emission="synch_disk", criterion=criterion, **kw))


def test_stokes_any_reduces_to_the_intensity_criterion_without_polarization():
    """Q = U = V = 0: the any-Stokes mask and interpolants equal those of the I criterion."""
    rng = np.random.default_rng(7)
    levels, level = 3, 2
    kw = dict(n0x=9, n0y=7, levels=levels, R_abs=0.02, R_rel=0.01)
    nx, ny = O.image_size(_pol_job("I", **kw))
    truth = np.zeros((4, ny, nx))
    truth[0] = W.smooth_image(3, nx, ny, noise=0.05)
    im, m = _level_setup(truth[0], levels, level)
    img = np.zeros_like(truth)
    img[0] = im
    a, ma, ea, _ = O.refine_level(_pol_job("I", **kw), img, m, level, 1.0)
    b, mb, eb, _ = O.refine_level(_pol_job("stokes_any", **kw), img, m, level, 1.0)
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(np.nan_to_num(a, nan=-1), np.nan_to_num(b, nan=-1))
    assert (ma == O.MASK_TRACED).sum() > 0 and (ma == O.MASK_INTERP).sum() > 0
    assert rng is not None


def test_stokes_any_traces_where_q_curves_and_i_is_flat():
    """I a constant plateau (zero estimates: the I criterion traces nothing), Q = x^2 + y^2
    (pixel units): the Q estimates are the closed forms of the quadratic test, eps_abs * norm =
    2 x (true residual) = 4 s^2 at cell centres and 2 s^2 at edge midpoints, and eps_rel is that
    over I's interpolant.  With R_abs between the two, the any-Stokes criterion traces exactly the
    cell centres (and the corner cells without any outer point), and the I criterion only those
    corners."""
    levels, level = 3, 2
    s = 1 << (levels - level)
    c0 = 8.0
    kw = dict(n0x=9, n0y=9, levels=levels, R_abs=3.0 * s * s, R_rel=0.5 * s * s / c0)
    nx, ny = O.image_size(_pol_job("I", **kw))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    truth = np.zeros((4, ny, nx))
    truth[0] = c0
    truth[1] = x * x + y * y
    im = np.full_like(truth, np.nan)
    sp = 2 * s
    im[:, ::sp, ::sp] = truth[:, ::sp, ::sp]
    m = np.zeros((ny, nx), np.uint8)
    m[::sp, ::sp] = O.MASK_TRACED
    _, mi, ea, _ = O.refine_level(_pol_job("I", **kw), im, m, level, 1.0)
    _, mq, _, _ = O.refine_level(_pol_job("stokes_any", **kw), im, m, level, 1.0)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    new = ~np.isnan(ea)
    cat4 = new & ((ii // s) % 2 == 1) & ((jj // s) % 2 == 1)
    corner = new & np.isinf(ea)
    assert corner.sum() == 4
    np.testing.assert_array_equal(mi[new] == O.MASK_TRACED, corner[new])
    np.testing.assert_array_equal(mq[new] == O.MASK_TRACED, (cat4 | corner)[new])
