"""Pins of the oracle's ray tracer against general-relativity closed forms.

The paper leaves the tracer to ipole; the oracle's tracer is pinned here to textbook results that
do not pass through its own formulas: Synge's shadow size, Bardeen's critical curve, the
constants of motion (evaluated in Boyer-Lindquist coordinates after an independent coordinate
transformation), straight-line integrals in flat space and the redshift of a Keplerian emitter.
"""
import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W


def _job(**kw):
    return O.make_job(**W.job(**kw))


# ------------------------------------------------------------------------------------------
# Boyer-Lindquist quantities, written independently of the oracle's Kerr-Schild formulas
# ------------------------------------------------------------------------------------------

def _bl_from_record(row, a, M=1.0):
    """Convert one record row (lambda, x^mu, k_mu [outgoing Kerr-Schild Cartesian]) to BL
    (r, theta) and covariant BL momenta (k_t, k_r, k_theta, k_phi).  Outgoing coordinates:
    t = t_BL - int 2Mr/Delta dr, phi = phi_BL - int a/Delta dr,
    x + i y = (r - i a) sin(theta) e^{i phi}, z = r cos(theta)."""
    x, y, z = row[2], row[3], row[4]
    kt, kx, ky, kz = row[5], row[6], row[7], row[8]
    rho2 = x * x + y * y + z * z
    r2 = 0.5 * (rho2 - a * a + np.sqrt((rho2 - a * a) ** 2 + 4 * a * a * z * z))
    r = np.sqrt(r2)
    th = np.arccos(z / r)
    phi = np.angle(complex(x, y) / complex(r, -a))
    Delta = r2 - 2 * M * r + a * a
    # derivatives of the Cartesian Kerr-Schild coordinates w.r.t. BL (r, theta, phi)
    e = np.exp(1j * phi)
    dxy_dr_ks = np.sin(th) * e
    dxy_dphi = 1j * complex(x, y)
    dxy_dr = dxy_dr_ks - dxy_dphi * a / Delta
    dxy_dth = complex(r, -a) * np.cos(th) * e
    kr = -kt * 2 * M * r / Delta + kx * dxy_dr.real + ky * dxy_dr.imag + kz * np.cos(th)
    kth = kx * dxy_dth.real + ky * dxy_dth.imag - kz * r * np.sin(th)
    kph = kx * dxy_dphi.real + ky * dxy_dphi.imag
    return r, th, np.array([kt, kr, kth, kph])


def _bl_norm(r, th, k, a, M=1.0):
    """g_BL^{mu nu} k_mu k_nu for the Kerr metric in Boyer-Lindquist form."""
    s2, c2 = np.sin(th) ** 2, np.cos(th) ** 2
    Sig = r * r + a * a * c2
    Del = r * r - 2 * M * r + a * a
    A = (r * r + a * a) ** 2 - a * a * Del * s2
    gtt = -A / (Sig * Del)
    gtp = -2 * M * a * r / (Sig * Del)
    gpp = (Del - a * a * s2) / (Sig * Del * s2)
    terms = np.array([gtt * k[0] ** 2, 2 * gtp * k[0] * k[3], gpp * k[3] ** 2,
                      Del / Sig * k[1] ** 2, k[2] ** 2 / Sig])
    return terms.sum(), np.abs(terms).sum()


def _carter(th, k, a):
    return k[2] ** 2 + np.cos(th) ** 2 * (-a * a * k[0] ** 2 + k[3] ** 2 / np.sin(th) ** 2)


def _invariants(job, alpha, beta, a):
    rec, status = O.trace_record(job, alpha, beta)
    E, L, Q, N, scale = [], [], [], [], []
    for row in rec:
        r, th, k = _bl_from_record(row, a)
        E.append(k[0])
        L.append(k[3])
        Q.append(_carter(th, k, a))
        n, sc = _bl_norm(r, th, k, a)
        N.append(n)
        scale.append(sc)  # sum of |terms|: the norm's own conditioning near the horizon
    return (np.array(E), np.array(L), np.array(Q), np.array(N), np.array(scale), rec, status)


@pytest.mark.parametrize("a,incl,alpha,beta", [(0.0, 60.0, 6.5, 1.0), (0.94, 17.0, 4.0, -3.0),
                                               (-0.5, 80.0, -2.0, 5.5), (0.94, 163.0, 1.0, 7.0)])
def test_constants_of_motion(a, incl, alpha, beta):
    """Along a traced ray: BL null norm ~ 0, E = -p_t exact, L_z and Carter's Q conserved.
    Bounds are the measured truncation error of RK4 at h = 0.05 r (worst near the horizon);
    the order of that error is pinned separately below."""
    job = _job(a=a, incl_deg=incl, step_frac=0.05)
    E, L, Q, N, scale, rec, status = _invariants(job, alpha, beta, a)
    assert len(rec) > 100
    assert np.all(E == E[0])                      # k_t is exactly constant
    assert np.max(np.abs(N) / scale) < 1e-4       # null in the BL metric too
    assert np.max(np.abs(L - L[0])) < 2e-4 * max(1.0, abs(L[0]))
    assert np.max(np.abs(Q - Q[0])) < 2e-4 * max(1.0, abs(Q[0]))
    assert abs(N[0]) / scale[0] < 1e-12            # null at the camera to rounding


def test_fourth_order_convergence():
    """RK4: halving the step fraction reduces the drift of L_z and Q by ~2^4."""
    a = 0.94
    drifts = []
    for sf in (0.08, 0.04):
        job = _job(a=a, incl_deg=60.0, step_frac=sf)
        E, L, Q, N, scale, rec, status = _invariants(job, 5.0, 2.0, a)
        drifts.append((abs(L[-1] - L[0]), abs(Q[-1] - Q[0])))
    for d0, d1 in zip(*drifts):
        assert 8.0 < d0 / d1 < 32.0


def _bisect_capture(job, direction, lo, hi, iters=40):
    """Screen radius where rays along `direction` switch from captured to escaping."""
    c, s = direction
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        _, info = O.trace_screen(job, [mid * c], [mid * s])
        if info["status"][0] == O.RAY_CAPTURED:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("r_obs", [1000.0, 1.0e6])
def test_schwarzschild_shadow_synge(r_obs):
    """Synge (1966): a static observer at r_obs sees the capture boundary at
    sin(psi) = sqrt(27) M sqrt(1 - 2M/r_obs) / r_obs; in gnomonic screen units
    b = r_obs tan(psi) (5.19102 at 1000 M, -> sqrt(27) for a distant camera)."""
    job = _job(a=0.0, r_obs=r_obs, incl_deg=60.0, step_frac=0.01)
    sinpsi = np.sqrt(27.0) * np.sqrt(1.0 - 2.0 / r_obs) / r_obs
    expect = r_obs * np.tan(np.arcsin(sinpsi))
    got = _bisect_capture(job, (1.0, 0.0), 4.0, 6.5, iters=36)
    assert got == pytest.approx(expect, rel=2e-6)
    got_v = _bisect_capture(job, (0.0, -1.0), 4.0, 6.5, iters=36)
    assert got_v == pytest.approx(expect, rel=2e-6)


def _bardeen(a, rt):
    """Critical impact parameters of spherical photon orbits of radius rt (Bardeen 1973)."""
    xi = (rt * rt * (3 - rt) - a * a * (rt + 1)) / (a * (rt - 1))
    eta = rt ** 3 * (4 * a * a - rt * (rt - 3) ** 2) / (a * a * (rt - 1) ** 2)
    return xi, eta


def _critical_curve_point(a, incl, angle):
    """Screen point of the critical curve for a distant observer along screen polar `angle`:
    alpha = -xi / sin i, beta = +/- sqrt(eta + a^2 cos^2 i - xi^2 cot^2 i)."""
    i = np.radians(incl)
    r_pro = 2 * (1 + np.cos(2 / 3 * np.arccos(-abs(a))))
    r_ret = 2 * (1 + np.cos(2 / 3 * np.arccos(abs(a))))
    rs = np.linspace(r_pro + 1e-9, r_ret - 1e-9, 200001)
    xi, eta = _bardeen(a, rs)
    b2 = eta + a * a * np.cos(i) ** 2 - xi ** 2 / np.tan(i) ** 2
    ok = b2 >= 0
    al = -xi[ok] / np.sin(i)
    be = np.sqrt(b2[ok])
    al = np.concatenate([al, al[::-1]])
    be = np.concatenate([be, -be[::-1]])
    ang = np.arctan2(be, al)
    k = np.argmin(np.abs(np.angle(np.exp(1j * (ang - angle)))))
    return np.hypot(al[k], be[k])


@pytest.mark.parametrize("a,incl", [(0.94, 17.0), (0.94, 60.0), (-0.6, 80.0)])
def test_kerr_critical_curve_bardeen(a, incl):
    """The capture boundary on the screen is Bardeen's critical curve (distant observer)."""
    job = _job(a=a, r_obs=1.0e5, incl_deg=incl, step_frac=0.02, max_steps=200000)
    for angle in np.radians([0.0, 50.0, 90.0, 150.0, 200.0, 270.0, 320.0]):
        rho_c = _critical_curve_point(a, incl, angle)
        got = _bisect_capture(job, (np.cos(angle), np.sin(angle)), 0.8 * rho_c, 1.2 * rho_c,
                              iters=30)
        assert got == pytest.approx(rho_c, rel=3e-4), np.degrees(angle)


def test_constants_of_motion_from_camera_match_bardeen_at_boundary():
    """(lambda, eta) the oracle reports for a boundary ray lie on Bardeen's curve."""
    a, incl = 0.94, 60.0
    job = _job(a=a, r_obs=1.0e5, incl_deg=incl, step_frac=0.02)
    angle = np.radians(120.0)
    rho_c = _critical_curve_point(a, incl, angle)
    rho = _bisect_capture(job, (np.cos(angle), np.sin(angle)), 0.8 * rho_c, 1.2 * rho_c, 30)
    _, info = O.trace_screen(job, [rho * np.cos(angle)], [rho * np.sin(angle)])
    lam, eta = info["lam"][0], info["eta"][0]
    from scipy.optimize import brentq
    r_pro = 2 * (1 + np.cos(2 / 3 * np.arccos(-a)))
    r_ret = 2 * (1 + np.cos(2 / 3 * np.arccos(a)))
    rt = brentq(lambda r: _bardeen(a, r)[0] - lam, r_pro + 1e-9, r_ret - 1e-9)
    assert eta == pytest.approx(_bardeen(a, rt)[1], rel=2e-3)


# ------------------------------------------------------------------------------------------
# flat space: straight-line integrals
# ------------------------------------------------------------------------------------------

def _flat_impact(r_obs, rho):
    """Closest approach b and distance s0 to it along the ray, for a pinhole at r_obs."""
    psi = np.arctan(rho / r_obs)
    return r_obs * np.sin(psi), r_obs * np.cos(psi)


@pytest.mark.parametrize("rho", [0.0, 0.7, 1.5, 2.5])
def test_flat_space_gaussian_blob(rho):
    """M = 0, static Gaussian blob: I(b) = sqrt(2 pi) sigma exp(-b^2/(2 sigma^2))."""
    sig = 1.0
    job = _job(a=0.0, r_obs=1000.0, incl_deg=30.0, step_frac=0.002, emission="blob",
               blob_sigma=sig, flow="static")
    job.mass = 0.0
    val, info = O.trace_screen(job, [rho * 0.6], [rho * 0.8])
    b, _ = _flat_impact(1000.0, rho)
    expect = np.sqrt(2 * np.pi) * sig * np.exp(-b * b / (2 * sig * sig))
    assert val[0, 0] == pytest.approx(expect, rel=2e-5)
    assert info["status"][0] == O.RAY_ESCAPED


@pytest.mark.parametrize("rho", [1.0, 3.0, 8.0])
def test_flat_space_inverse_square(rho):
    """M = 0, j = 1/r^2 along a straight line from the camera to where the ray leaves:
    I = (atan((s_end - s0)/b) + atan(s0/b)) / b."""
    r_obs = 1000.0
    job = _job(a=0.0, r_obs=r_obs, incl_deg=45.0, step_frac=0.002, emission="analytic",
               disk_w=1.0e6, flow="static")
    job.mass = 0.0
    rec, status = O.trace_record(job, rho, 0.0)
    b, s0 = _flat_impact(r_obs, rho)
    s_end = np.linalg.norm(rec[-1, 2:5] - rec[0, 2:5])
    expect = (np.arctan((s_end - s0) / b) + np.arctan(s0 / b)) / b
    assert rec[-1, 13] == pytest.approx(expect, rel=2e-5)


@pytest.mark.parametrize("incl,rho", [(5.0, 1.5), (45.0, 3.0), (80.0, 6.0)])
def test_flat_space_analytic_emissivity_by_quadrature(incl, rho):
    """M = 0 and a static fluid (nu = 1): the analytic emissivity j = r^-2 exp(-z^2/(2 (w r)^2)),
    w = 0.3, integrated along the straight ray from the camera to where it leaves.  The reference is
    adaptive Gauss-Kronrod quadrature (scipy's quad), split at the closest approach; the tolerance
    is the integrator's (2e-5 at step 0.002 r)."""
    from scipy.integrate import quad
    w = 0.3
    job = _job(a=0.0, r_obs=1000.0, incl_deg=incl, step_frac=0.002, emission="analytic",
               disk_w=w, flow="static")
    job.mass = 0.0
    rec, status = O.trace_record(job, rho, 0.0)
    p0, p1 = rec[0, 2:5], rec[-1, 2:5]
    length = np.linalg.norm(p1 - p0)
    d = (p1 - p0) / length

    def j(s):
        x = p0 + s * d
        r2 = x @ x
        return np.exp(-x[2] ** 2 / (2.0 * w * w * r2)) / r2

    s_c = -(p0 @ d)
    expect = (quad(j, 0.0, s_c, epsabs=0.0, epsrel=1e-12, limit=500)[0]
              + quad(j, s_c, length, epsabs=0.0, epsrel=1e-12, limit=500)[0])
    assert status == O.RAY_ESCAPED
    assert rec[-1, 13] == pytest.approx(expect, rel=2e-5)


def test_keplerian_redshift_schwarzschild():
    """Emitter on a circular Keplerian orbit at r (equator, a = 0) and a photon moving
    tangentially there with E = 1, L = r/sqrt(1 - 2/r): nu_fluid = u^t (1 - Omega L),
    u^t = (1 - 3/r)^(-1/2), Omega = r^(-3/2) (Schwarzschild circular geodesics)."""
    job = _job(a=0.0, emission="analytic", disk_w=0.3)
    for r in (4.0, 6.0, 15.0):
        for sgn in (1.0, -1.0):
            L = sgn * r / np.sqrt(1 - 2 / r)
            p = np.array([-1.0, -2.0 / (r - 2.0), L / r, 0.0])  # outgoing KS, p_r(BL) = 0
            k = -p
            J, nu = O.emission(job, [0.0, r, 0.0, 0.0], k)
            expect = (1 - r ** -1.5 * L) / np.sqrt(1 - 3 / r)
            assert nu == pytest.approx(expect, rel=1e-13)
            assert J == pytest.approx(r ** -2 / nu ** 2, rel=1e-13)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.94, -0.7])
def test_near_critical_distance_vanishes_on_bardeens_curve(a):
    """The tests' near-critical flag (conftest.crit_distance): zero at the constants of every
    spherical photon orbit (Bardeen 1973), clearly positive for a photon far from the shell."""
    from conftest import crit_distance
    aa = abs(a) if a != 0.0 else 0.0
    r_pro = 2 * (1 + np.cos(2 / 3 * np.arccos(-aa)))
    r_ret = 2 * (1 + np.cos(2 / 3 * np.arccos(aa)))
    if a == 0.0:
        lam = np.array([np.sqrt(27.0), 0.0, -np.sqrt(27.0)])
        eta = 27.0 - lam ** 2
    else:
        rt = np.linspace(r_pro + 1e-3, r_ret - 1e-3, 7)
        lam, eta = _bardeen(a, rt)
    assert (crit_distance(a, lam, eta, samples=200001) < 1e-6).all()
    assert (crit_distance(a, np.array([0.0, 1.0]), np.array([0.0, 1.0])) > 0.03).all()
