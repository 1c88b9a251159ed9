"""Pins of the oracle's polarized transfer: Bessel functions, the constant-coefficient segment
solver, the thermal-synchrotron coefficients, parallel transport and the Stokes conventions.

The paper only states that the method carries over to Q, U, V (Sec. 6); the transfer itself is
ipole's.  These tests pin the oracle's own transfer to library routines (scipy's Bessel K and
matrix exponential), to the exact thermal average of the single-electron synchrotron functions,
to the textbook rotation-measure constant, and to conserved quantities of parallel transport."""
import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W

special = pytest.importorskip("scipy.special")
integrate = pytest.importorskip("scipy.integrate")
linalg = pytest.importorskip("scipy.linalg")

E_CGS, ME, C = 4.80320471e-10, 9.1093837015e-28, 2.99792458e10


def _job(**kw):
    return O.make_job(**W.job(**kw))


@pytest.mark.parametrize("n", [0, 1, 2])
def test_bessel_k_matches_scipy(n):
    for x in (0.005, 0.05, 0.3, 1.0, 4.0, 30.0):
        assert O.bessel_k(n, x) == pytest.approx(special.kv(n, x), rel=1e-12)


def _kmat(K7):
    aI, aQ, aU, aV, rQ, rU, rV = K7
    return np.array([[aI, aQ, aU, aV], [aQ, aI, rV, -rU], [aU, -rV, aI, rQ], [aV, rU, -rQ, aI]])


def test_segment_matches_matrix_exponential():
    rng = np.random.default_rng(1)
    for _ in range(20):
        aI = rng.uniform(0, 3)
        pol = rng.uniform(-1, 1, 3)
        pol *= rng.uniform(0, aI) / max(np.linalg.norm(pol), 1e-12)
        K7 = [aI, *pol, *rng.uniform(-20, 20, 3)]
        J4 = rng.uniform(-1, 1, 4)
        J4[0] = abs(J4[0]) + np.linalg.norm(J4[1:])
        h = rng.uniform(0.01, 3.0)
        E, X = O.segment(K7, J4, h)
        A = np.zeros((5, 5))
        A[:4, :4] = -_kmat(K7) * h
        A[:4, 4] = J4 * h
        R = linalg.expm(A)
        np.testing.assert_allclose(E, R[:4, :4], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(X, R[:4, 4], rtol=1e-10, atol=1e-12)


def test_segment_closed_forms():
    """Pure rho_V rotates (Q, U) by rho_V h; pure rho_Q exchanges U and V; pure alpha_I decays
    as exp(-alpha h) with the source J (1 - exp(-alpha h))/alpha (thick limit: J/alpha)."""
    h = 0.7
    E, X = O.segment([0, 0, 0, 0, 0, 0, 2.0], [0, 0, 0, 0], h)
    c, s = np.cos(2.0 * h), np.sin(2.0 * h)
    np.testing.assert_allclose(E, [[1, 0, 0, 0], [0, c, -s, 0], [0, s, c, 0], [0, 0, 0, 1]],
                               atol=1e-14)
    E, X = O.segment([0, 0, 0, 0, 1.5, 0, 0], [0, 0, 0, 0], h)
    c, s = np.cos(1.5 * h), np.sin(1.5 * h)
    np.testing.assert_allclose(E, [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, c, -s], [0, 0, s, c]],
                               atol=1e-14)
    E, X = O.segment([0.8, 0, 0, 0, 0, 0, 0], [2.0, 0, 0, 0], h)
    np.testing.assert_allclose(np.diag(E), np.exp(-0.8 * h), rtol=1e-14)
    assert X[0] == pytest.approx(2.0 * -np.expm1(-0.8 * h) / 0.8, rel=1e-14)
    E, X = O.segment([50.0, 0, 0, 0, 0, 0, 0], [3.0, 0, 0, 0], 10.0)
    assert X[0] == pytest.approx(3.0 / 50.0, rel=1e-12)


def _exact_thermal(ne, Th, B, nu, thb):
    """Thermal (Maxwell-Juettner) average of the single-electron synchrotron emissivities,
    j = (1/4pi) int N(gamma) sqrt3 e^3 B sin(theta)/(m c^2) F(nu/nu_cr) dgamma with
    F(x) = x int_x^inf K_5/3, G(x) = x K_2/3(x), nu_cr = 3/2 gamma^2 nu_B sin(theta)
    (Rybicki & Lightman 1979, Eqs. 6.17, 6.31)."""
    nuB = E_CGS * B / (2 * np.pi * ME * C)
    s = np.sin(thb)
    K2 = special.kv(2, 1 / Th)

    def F(x):
        return x * integrate.quad(lambda t: special.kv(5 / 3, t), x, np.inf, limit=200)[0]

    def G(x):
        return x * special.kv(2 / 3, x)

    def integrand(g, fn):
        N = ne * g * g * np.sqrt(1 - 1 / g ** 2) * np.exp(-g / Th) / (Th * K2)
        return N * np.sqrt(3) * E_CGS ** 3 * B * s / (ME * C * C) * fn(nu / (1.5 * g * g * nuB * s)) / (4 * np.pi)

    pts = [Th, 3 * Th, 10 * Th]
    jI = integrate.quad(lambda g: integrand(g, F), 1.0, 60 * Th, limit=400, points=pts)[0]
    jQ = integrate.quad(lambda g: integrand(g, G), 1.0, 60 * Th, limit=400, points=pts)[0]
    return jI, jQ


@pytest.mark.parametrize("Th", [3.0, 10.0, 30.0])
def test_synchrotron_fits_against_exact_thermal_average(Th):
    """The fitted j_I (Leung et al. 2011) within 6 % and j_Q (Pandya et al. 2016) within 15 % of
    the exact thermal average; Kirchhoff: j/alpha = B_nu(T) exactly."""
    B, thb = 5.0, 1.0
    nuB = E_CGS * B / (2 * np.pi * ME * C)
    for X in (1.0, 10.0, 100.0, 1000.0):
        nu = X * 2 / 9 * nuB * Th * Th * np.sin(thb)
        co = O.synch_coeffs(1e5, Th, B, nu, thb)
        jI, jQ = _exact_thermal(1e5, Th, B, nu, thb)
        assert co[0] / jI == pytest.approx(1.0, abs=0.06)
        assert co[1] / jQ == pytest.approx(1.0, abs=0.15)
        assert 0 < co[1] < co[0]
        hp, kB = 6.62607015e-27, 1.380649e-16
        T = Th * ME * C * C / kB
        Bnu = 2 * hp * nu ** 3 / C ** 2 / np.expm1(hp * nu / (kB * T))
        assert co[0] / co[3] == pytest.approx(Bnu, rel=1e-12)
        assert co[1] / co[4] == pytest.approx(Bnu, rel=1e-12)


def test_faraday_rotation_matches_rotation_measure():
    """Cold-plasma limit: the EVPA turns by RM lambda^2 with RM = 0.812 rad m^-2 per
    (n_e / cm^-3)(B_par / microgauss)(L / pc) (textbook rotation measure); the thermal factor
    K0/K2 multiplies it."""
    ne, B, Th, nu = 1.0, 1e-6, 0.02, 1.4e9
    co = O.synch_coeffs(ne, Th, B, nu, 0.0)
    pc = 3.0857e18
    lam_m = C / nu / 100.0
    evpa_turn = 0.5 * co[6] * pc
    factor = special.kv(0, 1 / Th) / special.kv(2, 1 / Th)
    assert evpa_turn == pytest.approx(0.812 * lam_m ** 2 * factor, rel=2e-3)
    assert co[5] == 0.0 and O.synch_coeffs(ne, Th, B, nu, 1.0)[5] > 0  # conversion ~ sin^2
    assert O.synch_coeffs(ne, Th, B, nu, np.pi)[6] == pytest.approx(-co[6], rel=1e-12)


# ------------------------------------------------------------------------------------------
# transport along a traced ray
# ------------------------------------------------------------------------------------------

def _ks_to_bl(row, a, M=1.0):
    x, y, z = row[2], row[3], row[4]
    rho2 = x * x + y * y + z * z
    r2 = 0.5 * (rho2 - a * a + np.sqrt((rho2 - a * a) ** 2 + 4 * a * a * z * z))
    r = np.sqrt(r2)
    th = np.arccos(z / r)
    phi = np.angle(complex(x, y) / complex(r, -a))
    Delta = r2 - 2 * M * r + a * a
    e = np.exp(1j * phi)
    dphi = 1j * complex(x, y)
    dr = np.sin(th) * e - dphi * a / Delta
    dth = complex(r, -a) * np.cos(th) * e

    def lower(v):  # Kerr-Schild Cartesian covector -> BL covector
        vt, vx, vy, vz = v
        return np.array([vt, -vt * 2 * M * r / Delta + vx * dr.real + vy * dr.imag + vz * np.cos(th),
                         vx * dth.real + vy * dth.imag - vz * r * np.sin(th),
                         vx * dphi.real + vy * dphi.imag])

    s2, c2 = np.sin(th) ** 2, np.cos(th) ** 2
    Sig = r * r + a * a * c2
    A = (r * r + a * a) ** 2 - a * a * Delta * s2
    gi = np.zeros((4, 4))
    gi[0, 0] = -A / (Sig * Delta)
    gi[0, 3] = gi[3, 0] = -2 * M * a * r / (Sig * Delta)
    gi[3, 3] = (Delta - a * a * s2) / (Sig * Delta * s2)
    gi[1, 1] = Delta / Sig
    gi[2, 2] = 1 / Sig
    k = gi @ lower(row[5:9])
    f = gi @ lower(row[9:13])
    return r, th, k, f, gi


def _walker_penrose(r, th, k, f, a):
    """kappa = (A - i B)(r - i a cos(theta)) (Walker & Penrose 1970; Chandrasekhar 1983)."""
    st, ct = np.sin(th), np.cos(th)
    A = (k[0] * f[1] - k[1] * f[0]) + a * st * st * (k[1] * f[3] - k[3] * f[1])
    B = ((r * r + a * a) * (k[3] * f[2] - k[2] * f[3]) - a * (k[0] * f[2] - k[2] * f[0])) * st
    return complex(A, -B) * complex(r, -a * ct)


def _wp_drift(a, incl, alpha, beta, step_frac):
    job = _job(a=a, incl_deg=incl, stokes=4, emission="synch_disk", ne0=0.0, step_frac=step_frac)
    rec, status = O.trace_record(job, alpha, beta)
    kap = []
    for row in rec[:-2]:
        r, th, k, f, gi = _ks_to_bl(row, a)
        if r >= 2.5:
            kap.append(_walker_penrose(r, th, k, f, a))
    kap = np.array(kap)
    return np.max(np.abs(kap - kap[0])) / abs(kap[0])


@pytest.mark.parametrize("a,incl,alpha,beta", [(0.94, 17.0, 4.5, -2.0), (-0.5, 70.0, -3.0, 5.5)])
def test_parallel_transport_invariants(a, incl, alpha, beta):
    """Along a polarized ray: f.k = 0, f.f = 1 and the Walker-Penrose constant are conserved
    to the RK4 truncation error at h = 0.05 r (measured bound), which falls at 4th order."""
    job = _job(a=a, incl_deg=incl, stokes=4, emission="synch_disk", ne0=0.0)
    rec, status = O.trace_record(job, alpha, beta)
    assert len(rec) > 100
    d05, d025 = _wp_drift(a, incl, alpha, beta, 0.05), _wp_drift(a, incl, alpha, beta, 0.025)
    assert d05 < 5e-4 and (d025 < 1e-9 or d05 / d025 > 8.0)
    fk, ff, kap = [], [], []
    for row in rec[:-2]:
        r, th, k, f, gi = _ks_to_bl(row, a)
        if r < 2.5:  # Boyer-Lindquist components are ill-conditioned near the horizon
            continue
        g = np.linalg.inv(gi)
        fk.append(f @ g @ k / (np.abs(f) @ np.abs(g) @ np.abs(k)))
        ff.append(f @ g @ f)
        kap.append(_walker_penrose(r, th, k, f, a))
    fk, ff, kap = np.array(fk), np.array(ff), np.array(kap)
    assert np.max(np.abs(fk)) < 1e-5
    assert np.max(np.abs(ff - 1.0)) < 1e-5
    assert np.max(np.abs(kap - kap[0])) < 5e-4 * abs(kap[0])
    assert abs(kap[0]) > 1e-3


def test_stokes_convention_toroidal_field_face_on():
    """A face-on, optically thin, Faraday-free disk with a purely toroidal field emits with the
    E-vector radial on the sky: Q < 0 on the horizontal axis, Q > 0 on the vertical axis, U > 0 in
    the north-east quadrant (up, left) and U < 0 in the north-west one (IAU: angle from north
    through east, east = left on the screen)."""
    p = W.kerr_disk_2049(a=0.0, incl_deg=1.0, bz_ratio=0.0, ne0=1e3, r_in=6.0)
    job = O.make_job(**p)
    al = np.array([8.0, 0.0, -6.0, 6.0])
    be = np.array([0.0, 8.0, 6.0, 6.0])
    out, _ = O.trace_screen(job, al, be)
    I, Q, U, V = out.T
    assert (I > 0).all()
    assert Q[0] < -0.3 * I[0] and abs(U[0]) < 0.05 * abs(Q[0])
    assert Q[1] > 0.3 * I[1]
    assert U[2] > 0.3 * I[2] and U[3] < -0.3 * I[3]
    assert (np.sqrt(Q ** 2 + U ** 2 + V ** 2) <= I).all()


def test_polarized_image_is_physical():
    """|Q, U, V| <= I on every ray of a polarized disk image (a Mueller-matrix invariant), V present
    (Faraday conversion), and the I plane of the polarized trace close to the unpolarized one."""
    p = W.kerr_disk_2049(n0x=9, n0y=9, levels=1, fov=30.0)
    job = O.make_job(**p)
    nx, ny = O.image_size(job)
    pix = np.arange(nx * ny)
    out, info = O.trace_pixels(job, pix)
    I, Q, U, V = out.T
    assert I.max() > 0
    assert (np.sqrt(Q ** 2 + U ** 2 + V ** 2) <= I * (1 + 1e-12) + 1e-300).all()
    assert np.abs(V).max() > 1e-6 * I.max()
    unpol, _ = O.trace_pixels(O.make_job(**{**p, "stokes": 1}), pix)
    bright = I > 0.05 * I.max()
    assert np.median(np.abs(unpol[bright, 0] / I[bright] - 1)) < 0.2
