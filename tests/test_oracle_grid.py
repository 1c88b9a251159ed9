"""Pins of the oracle's fluid-grid emission model (the GRMHD-like snapshot path).

The paper images GRMHD snapshots through ipole (Sec. 4.2, 5: R_high electron temperatures, a
magnetisation cut); the lookup and fluid reconstruction are the oracle's own.  They are pinned
here to exact properties: trilinear interpolation reproduces multilinear data, the clamped and
periodic axes, the four-velocity normalisation and b.u = 0, the zero-angular-momentum observers'
closed-form u^t inside and outside the ergosphere, the Lorentz invariant B^2 - E^2 of an
ideal-MHD flow in flat space, the limits of the two-temperature prescription, the sigma cut,
and Kirchhoff saturation of an optically thick isothermal medium.  The snapshot generator's
Fishbone-Moncrief torus is pinned to its own Euler equation."""
import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W

MP, ME, C, H, KB = 1.67262192369e-24, 9.1093837015e-28, 2.99792458e10, 6.62607015e-27, 1.380649e-16


def _grid(data, logr_min, logr_max):
    n3, n2, n1, _ = data.shape
    return dict(data=np.ascontiguousarray(data, np.float32), n1=n1, n2=n2, n3=n3,
                logr_min=logr_min, logr_max=logr_max)


def _cart(a, r, th, ph):
    xy = (r - 1j * a) * np.sin(th) * np.exp(1j * ph)
    return np.stack([np.zeros_like(r), xy.real, xy.imag, r * np.cos(th)], -1)


def _cell_coords(n1, n2, n3, lo, hi):
    x1 = lo + (np.arange(n1) + 0.5) * (hi - lo) / n1
    th = (np.arange(n2) + 0.5) * np.pi / n2
    ph = (np.arange(n3) + 0.5) * 2 * np.pi / n3
    return x1, th, ph


def _metric(a, x, M=1.0):
    rho2 = (x[1:] ** 2).sum()
    b = rho2 - a * a
    r = np.sqrt(0.5 * (b + np.sqrt(b * b + 4 * a * a * x[3] ** 2)))
    F = 2 * M * r ** 3 / (r ** 4 + a * a * x[3] ** 2)
    l = np.array([1.0, -(r * x[1] - a * x[2]) / (r * r + a * a), -(r * x[2] + a * x[1]) / (r * r + a * a),
                  -x[3] / r])
    return np.diag([-1.0, 1, 1, 1]) + F * np.outer(l, l)


def test_trilinear_reproduces_multilinear_data():
    """Data multilinear in the cell indices (i, j) and constant in k is reproduced exactly at
    interior points; the phi axis is checked with a field that depends on k only."""
    n1, n2, n3 = 12, 10, 8
    lo, hi = np.log(2.0), np.log(50.0)
    i, j, k = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    f_rho = 1.0 + 0.5 * i + 0.25 * j + 0.125 * i * j
    data = np.zeros((n3, n2, n1, 8))
    data[..., 0] = np.transpose(f_rho, (2, 1, 0))
    data[..., 1] = np.transpose(3.0 + k, (2, 1, 0))
    job = O.make_job(grid=_grid(data, lo, hi), a=0.5, emission="grid")
    rng = np.random.default_rng(0)
    f1 = rng.uniform(0.0, n1 - 1, 50)
    f2 = rng.uniform(0.0, n2 - 1, 50)
    f3 = rng.uniform(0.0, n3 - 1, 50)
    r = np.exp(lo + (f1 + 0.5) * (hi - lo) / n1)
    th = (f2 + 0.5) * np.pi / n2
    ph = (f3 + 0.5) * 2 * np.pi / n3
    out = O.grid_fluid(job, _cart(0.5, r, th, ph))
    np.testing.assert_allclose(out["prim"][:, 0], 1 + 0.5 * f1 + 0.25 * f2 + 0.125 * f1 * f2,
                               rtol=1e-10)
    np.testing.assert_allclose(out["prim"][:, 1], 3.0 + f3, rtol=1e-10)


def test_periodic_phi_and_clamped_theta_and_radius():
    n1, n2, n3 = 6, 6, 8
    lo, hi = np.log(3.0), np.log(30.0)
    data = np.zeros((n3, n2, n1, 8))
    k = np.arange(n3)[:, None, None]
    j = np.arange(n2)[None, :, None]
    data[..., 0] = 10.0 + k + 0 * j
    data[..., 1] = 1.0 + j + 0 * k
    job = O.make_job(grid=_grid(data, lo, hi), a=0.0, emission="grid")
    dph = 2 * np.pi / n3
    r = np.full(4, 8.0)
    th = np.array([1.0, 1.0, 1.0, 1.0])
    # phi = 0 lies half-way between the last cell (k = 7) and the first (k = 0)
    ph = np.array([0.0, 0.25 * dph, 2 * np.pi - 0.25 * dph, 0.5 * dph])
    out = O.grid_fluid(job, _cart(0.0, r, th, ph))
    np.testing.assert_allclose(out["prim"][:, 0], [13.5, 0.75 * 10 + 0.25 * 17, 0.25 * 10 + 0.75 * 17, 10.0],
                               rtol=1e-12)
    # theta inside the first / last half cell takes the edge cell's value
    th = np.array([0.01, np.pi / n2 * 0.5, np.pi - 0.01])
    out = O.grid_fluid(job, _cart(0.0, np.full(3, 8.0), th, np.full(3, 0.5 * dph)))
    np.testing.assert_allclose(out["prim"][:, 1], [1.0, 1.0, float(n2)], rtol=1e-12)
    # outside the radial range: nothing, inside the outer half cell: the edge value
    out = O.grid_fluid(job, _cart(0.0, np.array([2.9, 31.0, 29.9]), np.full(3, 1.0), np.full(3, 0.5 * dph)))
    assert np.all(out["prim"][:2] == 0.0)
    assert out["prim"][2, 0] == pytest.approx(10.0)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.94])
def test_zamo_four_velocity_inside_and_outside_ergosphere(a):
    """A grid holding the zero-angular-momentum observers' u^phi = omega u^t (u^r = u^theta = 0):
    at cell centres the recovered u^t equals sqrt(A/(Sigma Delta)) (Bardeen, Press & Teukolsky
    1972), also inside the ergosphere where g_tt > 0; u.u = -1 throughout."""
    n1, n2, n3 = 40, 16, 4
    lo, hi = np.log(1.02 * (1 + np.sqrt(1 - a * a))), np.log(40.0)
    x1, th, ph = _cell_coords(n1, n2, n3, lo, hi)
    r = np.exp(x1)
    R, TH = np.meshgrid(r, th, indexing="ij")
    Sig, Delta, A = W._bl_geom(a, R, TH)
    ok = Delta > 0
    ut = np.sqrt(np.where(ok, A / (Sig * np.where(ok, Delta, 1)), 1.0))
    uph = np.where(ok, 2 * a * R / A * ut, 0.0)
    data = np.zeros((n3, n2, n1, 8))
    data[..., 0] = 1.0
    data[..., 1] = 1.0
    data[..., 4] = np.transpose(np.broadcast_to(uph[:, :, None], (n1, n2, n3)), (2, 1, 0))
    job = O.make_job(grid=_grid(data, lo, hi), a=a, emission="grid")
    gtt_all = W._bl_metric(a, R, TH)[0]
    ii, jj = np.nonzero(ok & (gtt_all <= 0))
    sel = np.random.default_rng(1).choice(len(ii), 40, replace=False)
    ie, je = np.nonzero(ok & (gtt_all > 0))          # every cell inside the ergosphere
    ii, jj = np.concatenate([ii[sel], ie]), np.concatenate([jj[sel], je])
    kk = np.random.default_rng(2).integers(0, n3, len(ii))
    pts = _cart(a, r[ii], th[jj], ph[kk])
    out = O.grid_fluid(job, pts)
    uph32 = data[kk, jj, ii, 4].astype(np.float32).astype(np.float64)
    # expected u^t from the Boyer-Lindquist normalisation with the stored (FP32) u^phi
    gtt, gtp, gpp = W._bl_metric(a, r[ii], th[jj])
    qa, qb, qc = gtt, 2 * gtp * uph32, gpp * uph32 ** 2 + 1
    root = (-qb - np.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
    np.testing.assert_allclose(out["u"][:, 0], root, rtol=1e-9)
    np.testing.assert_allclose(out["u"][:, 0], ut[ii, jj], rtol=2e-6)
    if a > 0:
        assert np.any(gtt > 0), "the sample should reach inside the ergosphere"
    for p, u in zip(pts, out["u"]):
        assert u @ _metric(a, p) @ u == pytest.approx(-1.0, abs=1e-11)


def test_ideal_mhd_field_invariant_flat_space():
    """Flat space (M = 0), uniform spherical-component velocity and field: b.u = 0, u^t = gamma,
    and b^2 equals the invariant B^2 - E^2 = B^2/gamma^2 + (v.B)^2 of the lab fields with
    E = -v x B (the comoving frame has no electric field)."""
    n1, n2, n3 = 8, 8, 8
    lo, hi = np.log(2.0), np.log(20.0)
    data = np.zeros((n3, n2, n1, 8))
    data[..., 0] = 1.0
    data[..., 1] = 1.0
    data[..., 2:5] = [0.3, -0.02, 0.05]
    data[..., 5:8] = [0.7, 0.1, -0.04]
    job = O.make_job(grid=_grid(data, lo, hi), a=0.0, mass=0.0, emission="grid", sigma_cut=1e9)
    rng = np.random.default_rng(3)
    r, th, ph = rng.uniform(3, 15, 20), rng.uniform(0.3, 2.8, 20), rng.uniform(0, 6.2, 20)
    out = O.grid_fluid(job, _cart(0.0, r, th, ph))
    e_r = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    e_t = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], -1)
    e_p = np.stack([-np.sin(ph), np.cos(ph), 0 * ph], -1)
    f32 = lambda v: float(np.float32(v))
    ucar = f32(0.3) * e_r + f32(-0.02) * r[:, None] * e_t + f32(0.05) * (r * np.sin(th))[:, None] * e_p
    Bcar = f32(0.7) * e_r + f32(0.1) * r[:, None] * e_t + f32(-0.04) * (r * np.sin(th))[:, None] * e_p
    gam = np.sqrt(1 + (ucar ** 2).sum(-1))
    v = ucar / gam[:, None]
    np.testing.assert_allclose(out["u"][:, 0], gam, rtol=1e-12)
    np.testing.assert_allclose(out["u"][:, 1:], ucar, rtol=1e-12, atol=1e-14)
    eta = np.diag([-1.0, 1, 1, 1])
    b, u = out["b"], out["u"]
    bu = np.einsum("ni,ij,nj->n", b, eta, u)
    np.testing.assert_allclose(bu, 0.0, atol=1e-12)
    b2 = np.einsum("ni,ij,nj->n", b, eta, b)
    inv = (Bcar ** 2).sum(-1) / gam ** 2 + (v * Bcar).sum(-1) ** 2
    np.testing.assert_allclose(b2, inv, rtol=1e-12)
    np.testing.assert_allclose(out["plasma"][:, 3], b2, rtol=1e-12)   # sigma = b^2/rho, rho = 1


def test_snapshot_normalisation_and_orthogonality():
    """On the seeded torus snapshot: u.u = -1 and b.u = 0 at every sample (Kerr, a = 0.94)."""
    g = W.grmhd_snapshot(seed=0, n1=48, n2=32, n3=16)
    job = O.make_job(grid=g, **W.grmhd_8193())
    rng = np.random.default_rng(4)
    r = np.exp(rng.uniform(np.log(1.5), np.log(60), 200))
    th = rng.uniform(0.05, np.pi - 0.05, 200)
    ph = rng.uniform(0, 2 * np.pi, 200)
    pts = _cart(0.94, r, th, ph)
    out = O.grid_fluid(job, pts)
    for p, u, b in zip(pts, out["u"], out["b"]):
        g4 = _metric(0.94, p)
        assert u @ g4 @ u == pytest.approx(-1.0, abs=1e-10)
        assert abs(b @ g4 @ u) <= 1e-10 * max(1.0, np.sqrt(abs(b @ g4 @ b)) * u[0])
    assert out["emits"].sum() > 10


def _uniform_grid(rho, ug, B1, m_unit=1e27, a=0.0, **kw):
    n1, n2, n3 = 8, 8, 8
    data = np.zeros((n3, n2, n1, 8))
    data[..., 0], data[..., 1], data[..., 5] = rho, ug, B1
    g = _grid(data, np.log(2.0), np.log(40.0))
    return O.make_job(grid=g, a=a, emission="grid", m_unit=m_unit, **kw)


def test_two_temperature_limits_and_sigma_cut():
    """T_i/T_e -> R_low at low plasma beta, -> R_high at high beta, their mean at beta = 1;
    sigma above the cut removes the emission, at the cut it stays."""
    gam = 13.0 / 9.0
    x = _cart(0.0, np.array([6.0]), np.array([1.2]), np.array([0.3]))
    r = 6.0
    # B^r = B1 in flat space (mass 0) gives b^2 = B1^2 for a static fluid
    for ug, B1, trat in [(1e-9, 1.0, 1.0), (1.0, 1e-9, 20.0)]:
        job = _uniform_grid(1.0, ug, B1, mass=0.0, sigma_cut=1e9)
        out = O.grid_fluid(job, x)
        th_e = out["plasma"][0, 1]
        assert th_e == pytest.approx(MP / ME * (gam - 1) * ug / (1 + trat), rel=1e-6)
    # beta = 1: (gamma - 1) u = b^2/2
    B1 = 0.5
    ug = 0.5 * B1 ** 2 / (gam - 1)
    job = _uniform_grid(1.0, ug, B1, mass=0.0, sigma_cut=1e9)
    out = O.grid_fluid(job, x)
    assert out["plasma"][0, 1] == pytest.approx(MP / ME * (gam - 1) * ug / (1 + 10.5), rel=1e-6)
    # sigma cut (b^2/rho = 0.25 here)
    assert O.grid_fluid(_uniform_grid(1.0, ug, B1, mass=0.0, sigma_cut=0.2499), x)["emits"][0] == False
    assert O.grid_fluid(_uniform_grid(1.0, ug, B1, mass=0.0, sigma_cut=0.2501), x)["emits"][0] == True
    del r


def test_optically_thick_isothermal_medium_saturates_at_planck():
    """A static, uniform, optically thick medium filling space around a flat-space camera: every
    ray's intensity is B_nu(T_e) at the observing frequency (Kirchhoff), whatever the field
    direction along the ray."""
    gam = 13.0 / 9.0
    ug, B1 = 2e-3, 0.02
    job = _uniform_grid(1.0, ug, B1, m_unit=1e33, mass=0.0, sigma_cut=1e9, r_obs=30.0,
                        fov=20.0, n0x=4, n0y=4, levels=0, incl_deg=60.0, max_steps=4000)
    x = _cart(0.0, np.array([10.0]), np.array([1.0]), np.array([1.0]))
    f = O.grid_fluid(job, x)
    assert f["emits"][0]
    th_e = f["plasma"][0, 1]
    nu = 230e9
    planck = 2 * H * nu ** 3 / C ** 2 / np.expm1(H * nu / (th_e * ME * C * C))
    img = O.render(job)[0]
    np.testing.assert_allclose(img.ravel(), planck, rtol=1e-6)
    # and a small optical depth gives much less than B_nu
    job2 = _uniform_grid(1.0, ug, B1, m_unit=1e20, mass=0.0, sigma_cut=1e9, r_obs=30.0,
                         fov=20.0, n0x=4, n0y=4, levels=0, incl_deg=60.0, max_steps=4000)
    assert O.render(job2)[0].max() < 1e-3 * planck
    del gam


def test_fishbone_moncrief_enthalpy_satisfies_euler_equation():
    """d ln h = u^t d u_t + u^phi d u_phi for the torus flow u^t u_phi = ell (finite differences
    in r and theta at several points), the pressure maximum sits at r_max on the equator, and the
    flow is normalised."""
    a, rmax = 0.94, 12.0
    ell = W.fm_ell(a, rmax)

    def cov(r, th):
        ut, uph = W.fm_velocity(a, ell, np.array(r), np.array(th))
        gtt, gtp, gpp = W._bl_metric(a, np.array(r), np.array(th))
        return ut, uph, gtt * ut + gtp * uph, gtp * ut + gpp * uph, gtt, gtp, gpp

    d = 1e-5
    for r, th in [(8.0, 1.3), (12.0, np.pi / 2), (17.0, 1.9), (25.0, 1.1)]:
        ut, uph, u_t, u_ph, gtt, gtp, gpp = cov(r, th)
        assert gtt * ut * ut + 2 * gtp * ut * uph + gpp * uph * uph == pytest.approx(-1, abs=1e-12)
        assert ut * u_ph == pytest.approx(ell, rel=1e-12)
        for dr, dth in [(d, 0.0), (0.0, d)]:
            lnh = lambda s: float(W.fm_lnh(a, ell, np.array(r + s * dr), np.array(th + s * dth)))
            dlnh = (lnh(1) - lnh(-1)) / 2
            p, m = cov(r + dr, th + dth), cov(r - dr, th - dth)
            rhs = ut * (p[2] - m[2]) / 2 + uph * (p[3] - m[3]) / 2
            assert dlnh == pytest.approx(rhs, rel=1e-6, abs=1e-12)
    eq = lambda r: float(W.fm_lnh(a, ell, np.array(r), np.array(np.pi / 2)))
    assert (eq(rmax + d) - eq(rmax - d)) / (2 * d) == pytest.approx(0.0, abs=1e-9)
