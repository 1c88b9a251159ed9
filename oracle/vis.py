"""TEST INFRASTRUCTURE ONLY: CPU oracle of the visibility-domain analysis (Sec. 4.3).

The visibilities of an image are its 2-D Fourier transform, the quantity an interferometer
baseline (u, v) samples.  Before transforming, the paper doubles the field of view (and the pixel
count) and applies a Gaussian taper of full width at half maximum FOV/4 to suppress the spurious
high-frequency power of the image's edges; visibility errors are the transform of the residual
image (adaptive minus full resolution).  This module writes that transform out as a plain
discrete Fourier sum, with the same conventions as the library's art_visibilities:

    V(u, v) = dx^2 sum_{x,y} T(x, y) A(x, y) exp(-2 pi i (u X + v Y)),
    X = (x - (nx - 1)/2) dx, Y = (y - (ny - 1)/2) dx,
    T = exp(-4 ln 2 (X^2 + Y^2) / fwhm^2)   (none for fwhm <= 0),
    A = img (or img - ref),
    u = k_u / (m dx), v = k_v / (m dx), k in [-m/2, m/2) stored at k mod m.

The sum is evaluated as two matrix products with explicit exponential matrices (FP64 complex):
no FFT, so it shares nothing with the library's butterflies.  Pinned by tests/test_oracle_vis.py
against the closed-form transform of a Gaussian (with and without taper), a point source's phase
ramp, Hermitian symmetry and Parseval's theorem.
"""
from __future__ import annotations

import numpy as np


def frequencies(m: int, dx: float) -> np.ndarray:
    """u of every FFT index k (k mod m storage): signed index / (m dx)."""
    k = np.arange(m)
    return np.where(k < m // 2, k, k - m) / (m * dx)


def taper(nx: int, ny: int, dx: float, fwhm: float) -> np.ndarray:
    """The Gaussian taper T on the image's pixels (ones when fwhm <= 0)."""
    if not fwhm > 0:
        return np.ones((ny, nx))
    X = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    Y = (np.arange(ny) - 0.5 * (ny - 1)) * dx
    r2 = Y[:, None] ** 2 + X[None, :] ** 2
    return np.exp(-4.0 * np.log(2.0) * r2 / (fwhm * fwhm))


def visibilities(img, dx: float, fwhm: float, m: int, ref=None, rows=None) -> np.ndarray:
    """V on the m x m grid (row k_v, column k_u); `rows` (optional) selects k_v rows only."""
    a = np.asarray(img, dtype=np.float64)
    if ref is not None:
        a = a - np.asarray(ref, dtype=np.float64)
    ny, nx = a.shape
    X = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    Y = (np.arange(ny) - 0.5 * (ny - 1)) * dx
    u = frequencies(m, dx)
    v = u if rows is None else u[np.asarray(rows)]
    Fx = np.exp(-2j * np.pi * np.outer(u, X))      # (m, nx)
    Fy = np.exp(-2j * np.pi * np.outer(v, Y))      # (rows, ny)
    return (Fy @ (a * taper(nx, ny, dx, fwhm)) @ Fx.T) * dx * dx
