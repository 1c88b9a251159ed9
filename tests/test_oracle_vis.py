"""Pins of the visibility oracle (Sec. 4.3): the transform of a tapered image against closed
forms and exact identities of the discrete sum."""
import numpy as np
import pytest

from oracle import vis as V


def _gauss(n, dx, sigma, amp=1.0, x0=0.0, y0=0.0):
    X = (np.arange(n) - 0.5 * (n - 1)) * dx
    return amp * np.exp(-((X[None, :] - x0) ** 2 + (X[:, None] - y0) ** 2) / (2 * sigma ** 2))


@pytest.mark.parametrize("fwhm", [0.0, 30.0])
def test_gaussian_has_gaussian_visibilities(fwhm):
    """A well-sampled Gaussian blob of width sigma (sum ~ integral): V = 2 pi s^2 A
    exp(-2 pi^2 s^2 q^2) with 1/s^2 = 1/sigma^2 + 1/sigma_T^2, sigma_T = fwhm / (2 sqrt(2 ln 2))
    (the taper multiplies two Gaussians).  Pins the 2 pi in the exponent, dx^2, the centring and
    the taper's FWHM convention."""
    n, dx, sigma, amp, m = 129, 0.5, 4.0, 1.7, 256
    img = _gauss(n, dx, sigma, amp)
    got = V.visibilities(img, dx, fwhm, m)
    s2 = sigma ** 2
    if fwhm > 0:
        st = fwhm / (2 * np.sqrt(2 * np.log(2)))
        s2 = 1.0 / (1.0 / sigma ** 2 + 1.0 / st ** 2)
    u = V.frequencies(m, dx)
    q2 = u[None, :] ** 2 + u[:, None] ** 2
    ref = 2 * np.pi * s2 * amp * np.exp(-2 * np.pi ** 2 * s2 * q2)
    assert np.abs(got - ref).max() <= 1e-9 * ref.max()


def test_point_source_is_a_phase_ramp():
    """One pixel of value A at (x0, y0) from the centre: V = A dx^2 exp(-2 pi i (u X0 + v Y0)),
    exactly, for an image with an even and an odd side."""
    nx, ny, dx, m = 20, 13, 0.7, 64
    img = np.zeros((ny, nx))
    xi, yi, A = 14, 3, 2.5
    img[yi, xi] = A
    X0, Y0 = (xi - 0.5 * (nx - 1)) * dx, (yi - 0.5 * (ny - 1)) * dx
    u = V.frequencies(m, dx)
    ref = A * dx * dx * np.exp(-2j * np.pi * (u[None, :] * X0 + u[:, None] * Y0))
    np.testing.assert_allclose(V.visibilities(img, dx, 0.0, m), ref, rtol=0, atol=1e-13)


def test_real_image_is_hermitian_and_parseval_holds():
    """Real input: V(-k) = conj V(k) (k != -m/2 rows/columns wrap onto themselves);
    Parseval for the m x m DFT of the zero-padded image: sum |V|^2 = m^2 dx^4 sum (T A)^2."""
    rng = np.random.default_rng(4)
    nx, ny, dx, m, fwhm = 37, 29, 0.3, 64, 5.0
    img = rng.normal(size=(ny, nx))
    v = V.visibilities(img, dx, fwhm, m)
    neg = (-np.arange(m)) % m
    np.testing.assert_allclose(v[np.ix_(neg, neg)], np.conj(v), atol=1e-12)
    ta = img * V.taper(nx, ny, dx, fwhm)
    assert np.sum(np.abs(v) ** 2) == pytest.approx(m * m * dx ** 4 * np.sum(ta ** 2), rel=1e-12)


def test_residual_is_the_difference_and_rows_select():
    rng = np.random.default_rng(5)
    a, b = rng.uniform(size=(17, 17)), rng.uniform(size=(17, 17))
    full = V.visibilities(a, 0.5, 3.0, 32, ref=b)
    np.testing.assert_allclose(full, V.visibilities(a, 0.5, 3.0, 32) - V.visibilities(b, 0.5, 3.0, 32),
                               atol=1e-13)
    np.testing.assert_allclose(V.visibilities(a, 0.5, 3.0, 32, ref=b, rows=[0, 5, 31]),
                               full[[0, 5, 31]], atol=1e-13)
