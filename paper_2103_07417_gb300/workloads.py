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
EMISSION = ("analytic", "synch_disk", "grid", "blob")
FLOW = ("kepler", "static")
ABS_NORM = ("ibar_int", "peak")
INTERP = ("linear", "nearest")
EDGE = ("onesided", "trace")
PRECISION = ("fp64", "mixed", "fp32")

BASE = dict(a=0.0, r_obs=1000.0, incl_deg=60.0, fov=40.0, n0x=33, n0y=33, levels=2,
            R_rel=0.01, R_abs=1e-4, abs_norm="ibar_int", interp="linear", edge_mode="onesided",
            emission="analytic", flow="kepler", stokes=1, subrings=0, precision="fp64",
            max_steps=100000, step_frac=0.05, h_min=1e-4, horizon_eps=0.01, escape_frac=1.01,
            disk_w=0.3, blob_sigma=1.0, ne0=0.0, thetae0=0.0, b0=0.0, nu_hz=230e9,
            ne_slope=-1.1, te_slope=-0.84, r_in=0.0, length_cm=9.6e14, bz_ratio=1.0,
            gamma_ad=13.0 / 9.0, m_unit=3e26, r_high=20.0, r_low=1.0, sigma_cut=1.0,
            proposal=0, proposal_depth=2, proposal_p=0.5, crit_band=0.0)


def job(**over) -> dict:
    d = dict(BASE)
    d.update(over)
    return d


# Half-width of the near-critical band traced with the base level (a scheduling choice that leaves
# images unchanged; 0.02 covered every re-traced ray of the 2049^2 and 8193^2 workloads).
CRIT_BAND = 0.03


def schwarzschild_129(**over) -> dict:
    """Schwarzschild, inclination 60 deg, r_obs 1000 M, FOV 40 M, j = r^-2 exp(-z^2/(2(0.3r)^2)),
    Keplerian, no absorption, FP64 RK4 with h = 0.05 r, 33^2 -> 129^2 over 2 levels,
    R_rel = 0.01, R_abs = 1e-4 of the peak."""
    return job(**{**dict(a=0.0, incl_deg=60.0, fov=40.0, n0x=33, n0y=33, levels=2, R_rel=0.01,
                         R_abs=1e-4, abs_norm="peak", emission="analytic", disk_w=0.3), **over})


def schwarzschild_large(**over) -> dict:
    """The schwarzschild_129 emission model on the 129^2 -> 2049^2 (4 levels) grid, paper tolerances
    R_rel = R_abs = 1e-3 of I_bar_int (Sec. 4.1, semi-analytic models)."""
    return schwarzschild_129(**{**dict(n0x=129, n0y=129, levels=4, R_rel=1e-3, R_abs=1e-3,
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


def kerr_disk_2049(**over) -> dict:
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
                         precision="mixed_df", crit_band=CRIT_BAND), **over})


def kerr_analytic_2049(**over) -> dict:
    """The Kerr geometry of the 128^2 -> 2048^2 configuration (a = 0.94, inclination 17 deg,
    FOV 40 M, base 129^2, 4 levels to 2049^2, R_rel = R_abs = 1e-3 of I_bar_int) with the
    analytic emissivity j = r^-2 exp(-z^2/(2 (0.3 r)^2)) of a Keplerian flow, mixed precision."""
    return job(**{**dict(a=0.94, incl_deg=17.0, fov=40.0, n0x=129, n0y=129, levels=4,
                         R_rel=1e-3, R_abs=1e-3, abs_norm="ibar_int", emission="analytic",
                         disk_w=0.3, precision="mixed", crit_band=CRIT_BAND), **over})


def grmhd_8193(**over) -> dict:
    """The seeded GRMHD-like snapshot (grmhd_snapshot(0): Fishbone-Moncrief torus, a = 0.94,
    288 x 128 x 128 cells over ln r in [ln 1.2, ln 1000]) seen at inclination 163 deg with a
    160 M field of view, 257^2 -> 8193^2 over 5 levels, at 230 GHz with R_high = 20, R_low = 1,
    a magnetisation cut at sigma = 1 (Sec. 4.2 and 5), mass unit 3e26 g for an M87*-mass hole, and
    the tolerances the paper chose for its GRMHD images, R_rel = 1e-3, R_abs = 0.025 (Sec. 4.1).
    Unpolarized transfer with thermal-synchrotron emission and absorption; the snapshot itself
    is passed separately (grid=)."""
    return job(**{**dict(a=0.94, incl_deg=163.0, fov=160.0, n0x=257, n0y=257, levels=5,
                         R_rel=1e-3, R_abs=0.025, abs_norm="ibar_int", emission="grid",
                         stokes=1, nu_hz=230e9, length_cm=9.6e14, gamma_ad=13.0 / 9.0,
                         m_unit=3e26, r_high=20.0, r_low=1.0, sigma_cut=1.0,
                         precision="mixed_df", crit_band=CRIT_BAND), **over})


def doubled_fov(params: dict) -> dict:
    """The same job with its field of view and pixel count doubled at the same resolution (the
    visibility analysis of Sec. 4.3): fov x 2 and a base grid of 2 n0 - 1 points per axis."""
    return {**params, "fov": 2.0 * params["fov"], "n0x": 2 * params["n0x"] - 1,
            "n0y": 2 * params["n0y"] - 1}


def grmhd_16385(**over) -> dict:
    """Evaluation workload of the learned block proposal: the GRMHD-like snapshot and its emission seen
    with a 1000 M field of view, 257^2 -> 16385^2 over 6 levels (the photon ring and the torus
    cover a small part of the image; most blocks of the finer levels are never refined)."""
    return grmhd_8193(**{**dict(fov=1000.0, levels=6), **over})


BENCH_WORKLOADS = {
    "kerr_disk_2049": (
        "adaptive polarized render 129^2 -> 2049^2 (4 levels), Kerr a=0.94, i=17 deg, FOV 40 M, "
        "r_obs 1000 M, RK4 h=0.05r; thermal-synchrotron thin disk (n_e~r^-1.1, T_e~r^-0.84, "
        "toroidal:vertical B = 1:1) at 230 GHz, Stokes IQUV with Faraday rotation/conversion; "
        "R_rel=R_abs=1e-3", kerr_disk_2049),
    "kerr_analytic_2049": (
        "adaptive render 129^2 -> 2049^2 (4 levels), Kerr a=0.94, i=17 deg, FOV 40 M, "
        "r_obs 1000 M, RK4 h=0.05r, analytic Keplerian emissivity r^-2 exp(-z^2/(2(0.3r)^2)), "
        "R_rel=R_abs=1e-3", kerr_analytic_2049),
    "grmhd_8193": (
        "adaptive render 257^2 -> 8193^2 (5 levels) of a seeded GRMHD-like snapshot "
        "(Fishbone-Moncrief torus a=0.94 + lognormal k^-11/3 turbulence, 288x128x128 FP32 "
        "cells over ln r in [ln 1.2, ln 1000]), i=163 deg, FOV 160 M, r_obs 1000 M, RK4 "
        "h=0.05r, thermal synchrotron at 230 GHz with R_high=20, sigma cut 1; "
        "R_rel=1e-3, R_abs=0.025", grmhd_8193),
    "grmhd_16385": (
        "learned-proposal evaluation render 257^2 -> 16385^2 (6 levels) of the GRMHD-like "
        "snapshot and emission, i=163 deg, FOV 1000 M, r_obs 1000 M, RK4 h=0.05r; "
        "R_rel=1e-3, R_abs=0.025", grmhd_16385),
    "schwarzschild_129": (
        "adaptive render 33^2 -> 129^2 (2 levels), Schwarzschild, i=60 deg, FOV 40 M, "
        "R_rel=0.01, R_abs=1e-4 of peak", schwarzschild_129),
}


def grmhd_batch(seed: int = 0, n: int = 256, **over) -> list:
    """A batch of n images: spin a ~ U[-0.94, 0.94], inclination ~ U[10, 170] deg, FOV log-uniform
    in [40, 400] M, final grid 2^k + 1 with k ~ U{6..9} (65^2 .. 513^2) reached over N ~ U{2..6}
    levels (base grid at least 5 points), the grid emission model (the seeded snapshot
    grmhd_snapshot(0), shared by every image whatever its spin) traced unpolarized with subrings
    n = 0, 1, 2; FP32 with the double-float re-trace."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a = float(rng.uniform(-0.94, 0.94))
        k = int(rng.integers(6, 10))
        N = int(rng.integers(2, 7))
        N = min(N, k - 2)
        n0 = (1 << (k - N)) + 1
        p = grmhd_8193(a=a, incl_deg=float(rng.uniform(10.0, 170.0)),
                 fov=float(np.exp(rng.uniform(np.log(40.0), np.log(400.0)))),
                 n0x=n0, n0y=n0, levels=N, stokes=1, subrings=3)
        p.update(over)
        out.append(p)
    return out


# ---------------------------------------------------------------------------------------------
# A seeded, GRMHD-like snapshot on a spherical Kerr-Schild grid
# ---------------------------------------------------------------------------------------------

GRID_FIELDS = ("rho", "uu", "U1", "U2", "U3", "B1", "B2", "B3")


def _bl_metric(a, r, th):
    s2, c2 = np.sin(th) ** 2, np.cos(th) ** 2
    Sig = r * r + a * a * c2
    gtt = -(1 - 2 * r / Sig)
    gtp = -2 * a * r * s2 / Sig
    gpp = (r * r + a * a + 2 * a * a * r * s2 / Sig) * s2
    return gtt, gtp, gpp


def _bl_geom(a, r, th):
    """Boyer-Lindquist Sigma, Delta, A = (r^2+a^2)^2 - a^2 Delta sin^2 theta."""
    Sig = r * r + a * a * np.cos(th) ** 2
    Delta = r * r - 2 * r + a * a
    A = (r * r + a * a) ** 2 - a * a * Delta * np.sin(th) ** 2
    return Sig, Delta, A


def fm_ell(a: float, r_max: float) -> float:
    """u^t u_phi of the prograde circular geodesic at r_max in the equatorial plane: the
    Fishbone-Moncrief constant that puts the pressure maximum of the torus at r_max."""
    gtt, gtp, gpp = _bl_metric(a, np.array(r_max), np.array(np.pi / 2))
    Om = 1.0 / (r_max ** 1.5 + a)
    ut = 1.0 / np.sqrt(-(gtt + 2 * Om * gtp + Om * Om * gpp))
    return float(ut * ut * (gtp + Om * gpp))


def fm_lnh(a: float, ell: float, r, th):
    """ln h + const of the Fishbone & Moncrief (1976) torus, u^t u_phi = ell.

    With the zero-angular-momentum observers' lapse e^nu = sqrt(Sigma Delta / A), e^psi =
    sqrt(g_phiphi), omega = 2 a r / A and the fluid's velocity v relative to them (Lorentz factor
    G), u^t u_phi = ell gives G^2 = (1 + s)/2 with s = sqrt(1 + 4 ell^2 e^(2 nu - 2 psi)); the
    Euler equation d ln h = u^t d u_t + u^phi d u_phi then integrates to
    ln h = 1/2 ln((1 + s) A / (Sigma Delta)) - s/2 - ell omega + const."""
    Sig, Delta, A = _bl_geom(a, r, th)
    X = Sig * Sig * Delta / (A * A * np.sin(th) ** 2)
    s = np.sqrt(1 + 4 * ell * ell * X)
    return 0.5 * np.log((1 + s) * A / (Sig * Delta)) - 0.5 * s - ell * 2 * a * r / A


def fm_velocity(a: float, ell: float, r, th):
    """(u^t, u^phi) of the Fishbone-Moncrief torus flow (u^r = u^theta = 0)."""
    Sig, Delta, A = _bl_geom(a, r, th)
    X = Sig * Sig * Delta / (A * A * np.sin(th) ** 2)
    s = np.sqrt(1 + 4 * ell * ell * X)
    G2 = 0.5 * (1 + s)
    v = np.sqrt(1 - 1 / G2) * np.sign(ell)
    enu = np.sqrt(Sig * Delta / A)
    epsi = np.sqrt(A / Sig) * np.sin(th)
    ut = np.sqrt(G2) / enu
    Om = 2 * a * r / A + v * enu / epsi
    return ut, ut * Om


def _ks_frame(a, r, th, ph):
    """Outgoing Kerr-Schild Cartesian position, F, L and the Jacobian d(x,y,z)/d(r,theta,phi)."""
    e = np.exp(1j * ph)
    xy = (r - 1j * a) * np.sin(th) * e
    x, y, z = xy.real, xy.imag, r * np.cos(th)
    F = 2 * r ** 3 / (r ** 4 + a * a * z * z)
    L = np.stack([(r * x - a * y) / (r * r + a * a), (r * y + a * x) / (r * r + a * a), z / r], -1)
    dr = np.sin(th) * e
    dth = (r - 1j * a) * np.cos(th) * e
    dph = 1j * xy
    Jm = np.stack([np.stack([dr.real, dth.real, dph.real], -1),
                   np.stack([dr.imag, dth.imag, dph.imag], -1),
                   np.stack([np.cos(th), -r * np.sin(th), np.zeros_like(r)], -1)], -2)
    return F, L, Jm


def grmhd_snapshot(seed: int = 0, n1: int = 288, n2: int = 128, n3: int = 128, a: float = 0.94,
                   r_in: float = 6.0, r_max: float = 12.0, sigma: float = 0.3, beta_max: float = 10.0,
                   gamma: float = 13.0 / 9.0, logr_min: float = np.log(1.2),
                   logr_max: float = np.log(1000.0)) -> dict:
    """A Fishbone-Moncrief torus with a lognormal turbulent density, on the grid x1 = ln r
    (n1 cells in [logr_min, logr_max]), theta (n2 cells in [0, pi]), phi (n3 cells in [0, 2 pi))
    of Kerr-Schild spherical coordinates, cell-centred.

    Torus: u^t u_phi = ell with ell from the circular geodesic at r_max, enthalpy h from
    fm_lnh normalised to h = 1 at (r_in, pi/2); polytrope rho ~ ((h - 1)(gamma - 1)/gamma)^(1/(gamma-1))
    scaled to rho_max = 1, internal energy u = rho (h - 1)/gamma.  Density and internal energy are
    multiplied by exp(sigma G - sigma^2/2), G a unit-variance Gaussian random field with
    P(k) ~ k^-11/3 on the index grid (seeded FFT).  Field: B^r = -d_theta A_phi / sqrt(-g),
    B^theta = d_r A_phi / sqrt(-g), sqrt(-g) = Sigma sin(theta), A_phi = max(rho/rho_max - 0.2, 0),
    scaled to gas/magnetic pressure beta_max at the density maximum.  Outside the torus a floor
    rho = 1e-4 r^-1.5, u = 1e-6 r^-2.5 moving with the zero-angular-momentum observers.
    Velocities are the contravariant u^r, u^theta, u^phi (u^r = u^theta = 0: the same in
    Boyer-Lindquist and Kerr-Schild coordinates).  Returns float32 (n3, n2, n1, 8) in the order
    of GRID_FIELDS plus the grid description."""
    rng = np.random.default_rng(seed)
    x1 = logr_min + (np.arange(n1) + 0.5) * (logr_max - logr_min) / n1
    th = (np.arange(n2) + 0.5) * np.pi / n2
    r = np.exp(x1)
    R, TH = np.meshgrid(r, th, indexing="ij")          # (n1, n2)
    Sig, Delta, A_ = _bl_geom(a, R, TH)
    ok = Delta > 0
    ell = fm_ell(a, r_max)
    with np.errstate(invalid="ignore", divide="ignore"):
        lnh = fm_lnh(a, ell, R, TH) - fm_lnh(a, ell, np.array(r_in), np.array(np.pi / 2))
        h = np.where(ok & (R >= r_in), np.exp(np.where(ok, lnh, 0.0)), 0.0)
        ut_t, uph_t = fm_velocity(a, ell, R, TH)
    inside = h > 1.0
    hm1 = np.where(inside, h - 1.0, 0.0)
    rho_t = (hm1 * (gamma - 1) / gamma) ** (1 / (gamma - 1))
    rho_t /= rho_t.max()
    uu_t = rho_t * hm1 / gamma
    rho = np.maximum(rho_t, 1e-4 * R ** -1.5)
    uu = np.maximum(uu_t, 1e-6 * R ** -2.5)
    gtt, gtp, gpp = _bl_metric(a, R, TH)
    uph_z = np.where(ok, np.sqrt(np.clip(A_ / (Sig * np.where(ok, Delta, 1.0)), 0.0, None)), 0.0) \
        * (-gtp / gpp)
    ut = np.where(inside, ut_t, 0.0)
    uph = np.where(inside, uph_t, uph_z)
    Aphi = np.maximum(rho_t - 0.2, 0.0)
    dAr = np.gradient(Aphi, r, axis=0)
    dAth = np.gradient(Aphi, th, axis=1)
    B1 = -dAth / (Sig * np.sin(TH))
    B2 = dAr / (Sig * np.sin(TH))
    # plasma beta at the density maximum (u^r = u^theta = 0 there: b^t = 0 in Boyer-Lindquist
    # form, b^2 = (g_rr B1^2 + g_thth B2^2)/(u^t)^2 ... evaluated with the Kerr-Schild relation below)
    imax = np.unravel_index(np.argmax(rho_t), rho_t.shape)
    b2 = _b2_ks(a, R[imax], TH[imax], ut[imax], uph[imax], B1[imax], B2[imax])
    pmax = (gamma - 1) * uu[imax]
    scale = np.sqrt(2 * pmax / beta_max / b2) if b2 > 0 else 0.0
    B1 *= scale
    B2 *= scale
    k1 = np.fft.fftfreq(n1)[:, None, None]
    k2 = np.fft.fftfreq(n2)[None, :, None]
    k3 = np.fft.rfftfreq(n3)[None, None, :]
    kk = np.sqrt(k1 ** 2 + k2 ** 2 + k3 ** 2)
    amp = np.where(kk > 0, np.where(kk > 0, kk, 1.0) ** (-11.0 / 6.0), 0.0)
    noise = rng.standard_normal(amp.shape) + 1j * rng.standard_normal(amp.shape)
    G = np.fft.irfftn(noise * amp, s=(n1, n2, n3), axes=(0, 1, 2))
    G = (G - G.mean()) / G.std()
    pert = np.exp(sigma * G - 0.5 * sigma * sigma)
    out = np.zeros((n3, n2, n1, 8), np.float32)

    def put(idx, field2d, p=None):
        f = np.broadcast_to(field2d[:, :, None], (n1, n2, n3)) if p is None else field2d[:, :, None] * p
        out[..., idx] = np.transpose(f, (2, 1, 0))

    put(0, rho, pert)
    put(1, uu, pert)
    put(4, uph)
    put(5, B1)
    put(6, B2)
    return dict(data=np.ascontiguousarray(out), n1=n1, n2=n2, n3=n3, logr_min=float(logr_min),
                logr_max=float(logr_max), a=a, gamma=gamma)


def _b2_ks(a, r, th, ut, uph, B1, B2):
    """b^2 = b^mu b_mu from B^i and u^mu (u^r = u^theta = 0) with the Kerr-Schild metric:
    b^t = B^i u^mu g_{i mu}, b^i = (B^i + b^t u^i)/u^t (Gammie, McKinney & Toth 2003)."""
    F, L, Jm = _ks_frame(a, np.array(r), np.array(th), np.array(0.0))
    uc = Jm[:, 2] * uph
    Bc = Jm @ np.array([B1, B2, 0.0])
    g = np.eye(4)
    g[0, 0] = -1.0
    l = np.concatenate([[1.0], -L])
    g = g + F * np.outer(l, l)
    u = np.concatenate([[ut], uc])
    Bv = np.concatenate([[0.0], Bc])
    bt = Bv @ g @ u
    b = (Bv + bt * u) / ut
    b[0] = bt
    return float(b @ g @ b)


# ---------------------------------------------------------------------------------------------
# Learned proposal: the seeded starting weights of the block-proposal network
# ---------------------------------------------------------------------------------------------

CNN_CH = 32
CNN_SHAPES = [("W1", (CNN_CH, 3, 3, 3)), ("b1", (CNN_CH,)), ("W2", (CNN_CH, 3, 3, CNN_CH)),
              ("b2", (CNN_CH,)), ("W3", (CNN_CH, 3, 3, CNN_CH)), ("b3", (CNN_CH,)),
              ("W4", (CNN_CH, 3, 3, CNN_CH)), ("b4", (CNN_CH,)), ("wh", (CNN_CH,)), ("bh", (1,))]


def cnn_init(seed: int) -> np.ndarray:
    """Flat FP32 parameter vector in the documented order (conv weights [out][ky][kx][in]):
    He-normal conv weights (std sqrt(2 / fan_in)), zero biases, head weights N(0, 1/32), head
    bias 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in CNN_SHAPES:
        if name.startswith("W"):
            fan_in = shp[1] * shp[2] * shp[3]
            parts.append(rng.standard_normal(shp) * np.sqrt(2.0 / fan_in))
        elif name == "wh":
            parts.append(rng.standard_normal(shp) / np.sqrt(CNN_CH))
        else:
            parts.append(np.zeros(shp))
    return np.concatenate([q.ravel() for q in parts]).astype(np.float32)
