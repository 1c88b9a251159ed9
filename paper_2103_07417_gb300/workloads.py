"""Seeded synthetic workloads: job parameter sets and input generators.

This module holds inputs only -- parameter dictionaries and seeded random fields -- and none of
the adaptive-ray-tracing arithmetic.  Both the CUDA library's binding and the CPU oracle take
their inputs from here; each side maps the symbolic option names to its own enums.

The configurations stand in for the paper's GRMHD snapshots and semi-analytic models, which are
not available: the analytic emission models below have the shapes and scales of the paper's
semi-analytic tests (Sec. 4.1: spin 0 and 0.94, inclinations 17 and 60 degrees, fields of view
30-45 M, 65^2 to 4097^2 images, tolerances 1e-3).
"""
from __future__ import annotations

import numpy as np

# Options shared by both sides by NAME (each side owns its enum values).
EMISSION = ("cfg0", "synch_disk", "blob")
FLOW = ("kepler", "static")
ABS_NORM = ("ibar_int", "peak")
INTERP = ("linear", "nearest")
EDGE = ("onesided", "trace")
PRECISION = ("fp64", "mixed", "fp32")

BASE = dict(a=0.0, r_obs=1000.0, incl_deg=60.0, fov=40.0, n0x=33, n0y=33, levels=2,
            R_rel=0.01, R_abs=1e-4, abs_norm="ibar_int", interp="linear", edge_mode="onesided",
            emission="cfg0", flow="kepler", stokes=1, subrings=0, precision="fp64",
            max_steps=100000, step_frac=0.05, h_min=1e-4, horizon_eps=0.01, escape_frac=1.01,
            disk_w=0.3, blob_sigma=1.0, ne0=0.0, thetae0=0.0, b0=0.0, nu_hz=230e9,
            ne_slope=-1.1, te_slope=-0.84, r_in=0.0, length_cm=9.6e14, bz_ratio=1.0)


def job(**over) -> dict:
    d = dict(BASE)
    d.update(over)
    return d


def cfg0(**over) -> dict:
    """Schwarzschild, inclination 60 deg, r_obs 1000 M, FOV 40 M, j = r^-2 exp(-z^2/(2(0.3r)^2)),
    Keplerian, no absorption, FP64 RK4 with h = 0.05 r, 33^2 -> 129^2 over 2 levels,
    R_rel = 0.01, R_abs = 1e-4 of the peak."""
    return job(**{**dict(a=0.0, incl_deg=60.0, fov=40.0, n0x=33, n0y=33, levels=2, R_rel=0.01,
                         R_abs=1e-4, abs_norm="peak", emission="cfg0", disk_w=0.3), **over})


def cfg0_large(**over) -> dict:
    """The cfg0 emission model on the 129^2 -> 2049^2 (4 levels) grid, paper tolerances
    R_rel = R_abs = 1e-3 of I_bar_int (Sec. 4.1, semi-analytic models)."""
    return cfg0(**{**dict(n0x=129, n0y=129, levels=4, R_rel=1e-3, R_abs=1e-3,
                          abs_norm="ibar_int"), **over})


def smooth_image(seed: int, nx: int, ny: int, n_bumps: int = 12, noise: float = 0.0) -> np.ndarray:
    """A positive image made of random Gaussian bumps plus optional white noise (seeded)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    img = np.full((ny, nx), 0.05)
    for _ in range(n_bumps):
        cx, cy = rng.uniform(0, nx - 1), rng.uniform(0, max(ny - 1, 1))
        sx, sy = rng.uniform(0.02, 0.2) * nx, rng.uniform(0.02, 0.2) * max(ny, 2)
        img += rng.uniform(0.1, 1.0) * np.exp(-0.5 * (((x - cx) / sx) ** 2 + ((y - cy) / sy) ** 2))
    if noise > 0:
        img += noise * rng.standard_normal((ny, nx))
    return img


def ring_image(seed: int, nx: int, ny: int) -> np.ndarray:
    """A thin bright ring on a diffuse background, the structure adaptive tracing targets."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cx, cy = (nx - 1) * rng.uniform(0.4, 0.6), (ny - 1) * rng.uniform(0.4, 0.6)
    rr = np.hypot(x - cx, y - cy)
    r0, w = 0.3 * min(nx, ny), rng.uniform(0.005, 0.02) * min(nx, ny)
    return 0.02 + np.exp(-0.5 * ((rr - r0) / w) ** 2) + 0.1 * np.exp(-rr / (0.3 * nx))


def fbm(seed: int, n: int, hurst: float) -> np.ndarray:
    """Fractional Brownian motion of n+1 samples with structure function D(k) = |k|^(2 hurst),
    by exact circulant embedding of fractional Gaussian noise (Davies & Harte 1987)."""
    rng = np.random.default_rng(seed)
    k = np.arange(n + 1, dtype=np.float64)
    h2 = 2.0 * hurst
    gam = 0.5 * (np.abs(k + 1) ** h2 - 2 * np.abs(k) ** h2 + np.abs(k - 1) ** h2)
    c = np.concatenate([gam, gam[-2:0:-1]])
    lam = np.fft.fft(c).real
    lam = np.clip(lam, 0.0, None)
    m = c.size
    z = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    w = np.fft.fft(np.sqrt(lam / m) * z)
    fgn = w.real[:n]
    return np.concatenate([[0.0], np.cumsum(fgn)])


def r_isco(a: float) -> float:
    """Prograde innermost stable circular orbit (Bardeen, Press & Teukolsky 1972)."""
    z1 = 1 + (1 - a * a) ** (1 / 3) * ((1 + a) ** (1 / 3) + (1 - a) ** (1 / 3))
    z2 = (3 * a * a + z1 * z1) ** 0.5
    return 3 + z2 - ((3 - z1) * (3 + z1 + 2 * z2)) ** 0.5 * (1 if a >= 0 else -1)


def cfg1(**over) -> dict:
    """Kerr a = 0.94, inclination 17 deg, FOV 40 M; thermal-synchrotron thin disk
    (n_e ~ r^-1.1, T_e ~ r^-0.84, toroidal : vertical field = 1 : 1, |B| ~ r^-0.97, Gaussian
    vertical profile of width 0.1 r, Keplerian, inner edge at the ISCO) at 230 GHz for an M87*-mass
    hole (GM/c^2 = 9.6e14 cm), normalised to n_e = 1e5 cm^-3, Theta_e = 20, |B| = 5 G at r = 5 M
    (optical and Faraday depths of order unity through the disk); polarized IQUV transfer with
    Faraday rotation and conversion; 129^2 -> 2049^2 over 4 levels, R_rel = R_abs = 1e-3."""
    return job(**{**dict(a=0.94, incl_deg=17.0, fov=40.0, n0x=129, n0y=129, levels=4,
                         R_rel=1e-3, R_abs=1e-3, abs_norm="ibar_int", emission="synch_disk",
                         stokes=4, disk_w=0.1, ne0=1e5 * 5 ** 1.1, thetae0=20.0 * 5 ** 0.84,
                         b0=5.0 * 5 ** 0.97, nu_hz=230e9, ne_slope=-1.1, te_slope=-0.84,
                         r_in=r_isco(0.94), length_cm=9.6e14, bz_ratio=1.0,
                         precision="mixed_df"), **over})


def cfg1_analytic(**over) -> dict:
    """The Kerr geometry of the 128^2 -> 2048^2 configuration (a = 0.94, inclination 17 deg,
    FOV 40 M, base 129^2, 4 levels to 2049^2, R_rel = R_abs = 1e-3 of I_bar_int) with the
    analytic emissivity j = r^-2 exp(-z^2/(2 (0.3 r)^2)) of a Keplerian flow, mixed precision."""
    return job(**{**dict(a=0.94, incl_deg=17.0, fov=40.0, n0x=129, n0y=129, levels=4,
                         R_rel=1e-3, R_abs=1e-3, abs_norm="ibar_int", emission="cfg0",
                         disk_w=0.3, precision="mixed"), **over})


BENCH_WORKLOADS = {
    "cfg1": ("adaptive polarized render 129^2 -> 2049^2 (4 levels), Kerr a=0.94, i=17 deg, FOV 40 M, "
             "r_obs 1000 M, RK4 h=0.05r; thermal-synchrotron thin disk (n_e~r^-1.1, T_e~r^-0.84, "
             "toroidal:vertical B = 1:1) at 230 GHz, Stokes IQUV with Faraday rotation/conversion; "
             "R_rel=R_abs=1e-3", cfg1),
    "cfg1_analytic": ("adaptive render 129^2 -> 2049^2 (4 levels), Kerr a=0.94, i=17 deg, "
                      "FOV 40 M, r_obs 1000 M, RK4 h=0.05r, analytic Keplerian emissivity "
                      "r^-2 exp(-z^2/(2(0.3r)^2)), R_rel=R_abs=1e-3", cfg1_analytic),
    "cfg0": ("adaptive render 33^2 -> 129^2 (2 levels), Schwarzschild, i=60 deg, FOV 40 M, "
             "R_rel=0.01, R_abs=1e-4 of peak", cfg0),
}


def cfg3(seed: int = 0, n: int = 256, **over) -> list:
    """A batch of n images: spin a ~ U[-0.94, 0.94], inclination ~ U[10, 170] deg, FOV log-uniform
    in [40, 400] M, final grid 2^k + 1 with k ~ U{6..9} (65^2 .. 513^2) reached over N ~ U{2..6}
    levels (base grid at least 5 points), the thermal-synchrotron disk model of config 1 (inner
    edge at each spin's ISCO) traced unpolarized with subrings n = 0, 1, 2; mixed precision."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a = float(rng.uniform(-0.94, 0.94))
        k = int(rng.integers(6, 10))
        N = int(rng.integers(2, 7))
        N = min(N, k - 2)
        n0 = (1 << (k - N)) + 1
        p = cfg1(a=a, incl_deg=float(rng.uniform(10.0, 170.0)),
                 fov=float(np.exp(rng.uniform(np.log(40.0), np.log(400.0)))),
                 n0x=n0, n0y=n0, levels=N, r_in=r_isco(a), stokes=1, subrings=3)
        p.update(over)
        out.append(p)
    return out
