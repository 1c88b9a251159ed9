"""Pins of the third-axis oracle (adaptive sampling in frequency or time, Sec. 6 proposal, with
the one-dimensional estimator of Sec. 3.2 / Appendix A along the axis)."""
import numpy as np
import pytest

from oracle import axis as A
from paper_2103_07417_gb300 import workloads as W


def _cube(fun, F=17, ny=5, nx=6):
    f = np.arange(F, dtype=np.float64)[:, None, None, None]
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return fun(f, y[None, None], x[None, None]) * np.ones((F, 1, ny, nx))


def test_linear_in_the_axis_is_never_traced_and_interpolated_exactly():
    """A cube linear along the axis: every second difference vanishes, so nothing beyond the
    base samples is traced and the interpolants are exact (dyadic values: exact in binary)."""
    c = _cube(lambda f, y, x: 1.0 + 0.25 * f + 0.125 * x)
    cube, m, counts, _ = A.render_axis(17, 3, 1e-12, 1e-12, truth=c)
    np.testing.assert_array_equal(cube, c)
    assert counts == [30, 0, 0, 0, 0, 0, 0, 0, 30, 0, 0, 0, 0, 0, 0, 0, 30]


def test_quadratic_estimate_is_twice_the_true_residual():
    """I = f^2 along the axis: the printed 1-D estimator gives 2 x the true linear residual
    (s^2 at spacing s): eps_abs * I_bar = 2 s^2 (Appendix A's factor of two), also one-sided."""
    F, L = 17, 3
    c = _cube(lambda f, y, x: f * f + 0.0 * x, F=F)
    norm = 1.0
    for k in range(1, L + 1):
        s = 1 << (L - k)
        for f in range(s, F, 2 * s):
            nan = np.full(1, np.nan)
            lo3 = c[f - 3 * s, 0, 0, :1] if f - 3 * s >= 0 else nan
            hi3 = c[f + 3 * s, 0, 0, :1] if f + 3 * s < F else nan
            tr, interp, ea, er = A.axis_decide(lo3, c[f - s, 0, 0, :1], c[f + s, 0, 0, :1], hi3,
                                               norm, 0.0, 0.0)
            assert interp[0] - f * f == s * s          # true residual
            assert ea[0] * norm == 2.0 * s * s         # estimate


def test_limits_reproduce_the_truth_and_linear_interpolation():
    rng = np.random.default_rng(3)
    c = rng.uniform(0.5, 2.0, size=(9, 2, 4, 5))
    cube, m, counts, _ = A.render_axis(9, 2, -1.0, -1.0, truth=c)
    np.testing.assert_array_equal(cube, c)
    assert (m == A.MASK_TRACED).all()
    cube, m, counts, _ = A.render_axis(9, 2, np.inf, np.inf, truth=c)
    f = np.arange(9)
    for j in range(9):
        lo, hi = (j // 4) * 4, min((j // 4) * 4 + 4, 8)
        w = (j - lo) / 4.0 if hi > lo else 0.0
        np.testing.assert_allclose(cube[j], (1 - w) * c[lo] + w * c[hi], rtol=1e-15)
    assert counts[1:4] == [0, 0, 0]


def test_missing_outer_samples_take_the_one_sided_rule():
    """With 3 samples and one level the new sample has no outer sample on either side: its
    estimate is infinite (traced for any finite tolerance); with 5 samples each new sample has
    one outer sample (one-sided second difference)."""
    c = _cube(lambda f, y, x: f ** 3 + 0.0 * x, F=5)
    _, m, counts, _ = A.render_axis(3, 1, 1e300, 1e300, truth=c[::2])
    assert counts[1] == 30
    lo3, lo1, hi1, hi3 = np.nan, 0.0, 8.0, 64.0   # f = 1 of 0..4 at s = 1: outer sample f = 4
    tr, interp, ea, er = A.axis_decide([np.nan], [0.0], [8.0], [64.0], 1.0, 0.0, 0.0)
    assert ea[0] == 2.0 * abs((64.0 - 2 * 8.0) + 0.0) / 8.0


def test_combined_scheme_reduces_to_the_spatial_render_when_the_axis_always_asks():
    """With R3 = -1 the axis estimate asks for every point, so each new sample is exactly the
    plain adaptive render of its own job (traced points equal the truth, interpolants the stated
    means); base samples are plain renders too."""
    import oracle as O
    params = [W.schwarzschild_129(n0x=5, n0y=5, levels=2, R_rel=1e-2, R_abs=1e-3,
                                  step_frac=0.05 + 0.01 * f) for f in range(5)]
    ojobs = [O.make_job(**p) for p in params]
    cube, mask, counts, _ = A.render_axis_jobs(ojobs, 2, -1.0, -1.0)
    for f in range(5):
        ref, rmask, st = O.render(ojobs[f], None)
        np.testing.assert_array_equal(cube[f, 0], ref)
        np.testing.assert_array_equal(mask[f], rmask)
        assert counts[f] == st["rays_traced"]


def test_combined_scheme_interpolates_along_the_axis_when_it_is_linear():
    """Jobs whose images are exactly linear in the sample index (a truth-like synthetic check
    through the same code path is not available for traced jobs): with R3 = +inf the axis never
    asks, so every point the spatial scheme would trace at a new sample takes the axis mean."""
    import oracle as O
    params = [W.schwarzschild_129(n0x=5, n0y=5, levels=1, R_rel=-1.0, R_abs=-1.0,
                                  step_frac=0.05 + 0.01 * f) for f in range(3)]
    ojobs = [O.make_job(**p) for p in params]
    cube, mask, counts, _ = A.render_axis_jobs(ojobs, 1, np.inf, np.inf)
    np.testing.assert_array_equal(cube[1], 0.5 * (cube[0] + cube[2]))
    assert (mask[1] == A.MASK_AXIS).all() and counts[1] == 0
