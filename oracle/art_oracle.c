/*
 * art_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, FP64 CPU implementation of adaptive ray tracing of Kerr black-hole images,
 * written to check the CUDA library against.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load it; the CUDA library never calls it and shares
 * no source with it.
 *
 * What it follows (Gelles et al. 2021, arXiv:2103.07417):
 *   - Sec. 3.2: base grid n0x x n0y, N levels of recursive subdivision, final size
 *     n = 2^N (n0 - 1) + 1; the four point categories; trace iff eps_abs > R_abs AND
 *     eps_rel > R_rel, else interpolate.
 *   - Eqs. (epabs), (eprel) and Appendix A: the estimated errors for the linear and the
 *     nearest-neighbour schemes, with I_bar_int the interpolated mean of the first pass.
 *   - Eqs. (interpdef), (fluxdef), (msedef): interpolation fraction, flux error, MSE.
 * The paper delegates the ray tracer itself to ipole; the tracer here is a textbook one:
 *   - Kerr metric in Cartesian Kerr-Schild form g = eta + f l l (Kerr 1963; Kerr & Schild 1965),
 *     null geodesics from the Hamiltonian H = 1/2 g^{mu nu} k_mu k_nu.  The partial derivatives
 *     of H are taken by the complex-step method (Squire & Trapp 1998) from H written once, so no
 *     hand-derived derivative enters the oracle.
 *   - Classical RK4 in the affine parameter with h = step_frac * r.
 *   - Covariant transfer d(I/nu^3)/dlambda = j/nu^2 - (nu alpha)(I/nu^3) integrated per step with
 *     the trapezoid-averaged coefficients and the exact constant-coefficient solution.
 * Readings where the paper is silent (edge handling, the 1-D divisors of categories 2/3, the
 * normalisation I_bar_int, tie breaking, camera, emission) are those listed in the design notes;
 * each function below says which one it implements.
 */
#include "art_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static int g_threads = 0;
void orc_set_threads(int n) { g_threads = n; }
int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Grid (Sec. 3.2)                                                                             */
/* ------------------------------------------------------------------------------------------ */

/* n = 2^N (n0 - 1) + 1 per axis (Sec. 3.2). */
int orc_image_size(const orc_job* job, int* nx, int* ny)
{
    if (job->n0x < 2 || job->n0y < 1 || job->levels < 0 || job->levels > 14) return -1;
    *nx = (1 << job->levels) * (job->n0x - 1) + 1;
    *ny = (1 << job->levels) * (job->n0y - 1) + 1;
    return 0;
}

int orc_planes(const orc_job* job)
{
    int st = job->stokes == 4 ? 4 : 1;
    return st * (job->subrings > 0 ? job->subrings : 1);
}

/* Screen coordinates: points span the field of view inclusively, equal spacing on both axes,
 * centred on the optical axis. */
static void screen_of_pixel(const orc_job* job, int nx, int ny, int i, int j, double* al,
                            double* be)
{
    double d = job->fov / (double)(nx - 1);
    *al = (i - 0.5 * (nx - 1)) * d;
    *be = (j - 0.5 * (ny - 1)) * d;
}

/* ------------------------------------------------------------------------------------------ */
/* Kerr-Schild geometry                                                                        */
/* ------------------------------------------------------------------------------------------ */

/* Kerr-Schild radius r from (x, y, z): (x^2+y^2)/(r^2+a^2) + z^2/r^2 = 1. */
static cplx ks_radius(double a, cplx x, cplx y, cplx z)
{
    cplx rho2 = x * x + y * y + z * z;
    cplx b = rho2 - a * a;
    cplx r2 = 0.5 * (b + csqrt(b * b + 4.0 * a * a * z * z));
    return csqrt(r2);
}

/* The Hamiltonian H = 1/2 g^{mu nu} k_mu k_nu of the Kerr metric in OUTGOING Cartesian
 * Kerr-Schild coordinates, g^{mu nu} = eta^{mu nu} - f l^mu l^nu with f = 2 M r^3/(r^4 + a^2 z^2)
 * and l_mu = (1, -(r x - a y)/(r^2+a^2), -(r y + a x)/(r^2+a^2), -z/r) -- the time reverse of the
 * ingoing form with the spin reversed (Kerr & Schild 1965).  Rays traced backward from the camera
 * are past-directed; in these coordinates they stay regular across the (past) horizon, whereas in
 * ingoing coordinates their covariant momentum diverges like 1/(r - r_+).  The coordinates satisfy
 * x + i y = (r - i a) sin(theta) e^{i phi}, z = r cos(theta).
 * Written in complex arithmetic so that the complex-step method can differentiate it. */
static cplx hamiltonian(double a, double M, const cplx* x, const cplx* k)
{
    cplx r = ks_radius(a, x[1], x[2], x[3]);
    cplx r2 = r * r;
    cplx f = 2.0 * M * r * r2 / (r2 * r2 + a * a * x[3] * x[3]);
    cplx lx = -(r * x[1] - a * x[2]) / (r2 + a * a);
    cplx ly = -(r * x[2] + a * x[1]) / (r2 + a * a);
    cplx lz = -x[3] / r;
    cplx lk = -k[0] + lx * k[1] + ly * k[2] + lz * k[3]; /* l^mu k_mu, l^t = -1 */
    cplx eta = -k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3];
    return 0.5 * (eta - f * lk * lk);
}

/* Right-hand side of Hamilton's equations, y = (x^mu, k_mu):
 * dx^mu/dlambda = dH/dk_mu, dk_mu/dlambda = -dH/dx^mu, by complex steps of size 1e-20. */
static void geodesic_rhs(double a, double M, const double* y, double* dy)
{
    const double hstep = 1e-20;
    cplx x[4], k[4];
    for (int m = 0; m < 4; ++m) { x[m] = y[m]; k[m] = y[4 + m]; }
    for (int m = 0; m < 4; ++m) {
        cplx save = k[m];
        k[m] = save + I * hstep;
        dy[m] = cimag(hamiltonian(a, M, x, k)) / hstep;
        k[m] = save;
    }
    for (int m = 0; m < 4; ++m) {
        cplx save = x[m];
        x[m] = save + I * hstep;
        dy[4 + m] = -cimag(hamiltonian(a, M, x, k)) / hstep;
        x[m] = save;
    }
}

/* Covariant metric g_{mu nu} = eta_{mu nu} + f l_mu l_nu, outgoing form (real arguments). */
static void metric_cov(double a, double M, const double* x, double g[4][4])
{
    double r = creal(ks_radius(a, x[1], x[2], x[3]));
    double r2 = r * r;
    double f = 2.0 * M * r * r2 / (r2 * r2 + a * a * x[3] * x[3]);
    double l[4] = {1.0, -(r * x[1] - a * x[2]) / (r2 + a * a), -(r * x[2] + a * x[1]) / (r2 + a * a),
                   -x[3] / r};
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            g[m][n] = ((m == n) ? (m == 0 ? -1.0 : 1.0) : 0.0) + f * l[m] * l[n];
}

static double dot_g(double g[4][4], const double* u, const double* v)
{
    double s = 0;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n) s += g[m][n] * u[m] * v[n];
    return s;
}

static double horizon_radius(double a, double M)
{
    double d = M * M - a * a;
    return d > 0 ? M + sqrt(d) : M;
}

/* ------------------------------------------------------------------------------------------ */
/* Camera: static observer at (r_obs, theta_o, phi = 0), tetrad by Gram-Schmidt, pinhole.      */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    double x0[4];
    double e0[4], e1[4], e2[4], e3[4]; /* u, outward, screen-up, screen-right (contravariant) */
    double g[4][4];
} camera;

static void camera_setup(const orc_job* job, camera* c)
{
    double th = job->incl_deg * M_PI / 180.0, a = job->a, ro = job->r_obs;
    c->x0[0] = 0.0;
    c->x0[1] = sqrt(ro * ro + a * a) * sin(th);
    c->x0[2] = 0.0;
    c->x0[3] = ro * cos(th);
    metric_cov(a, job->mass, c->x0, c->g);
    double ut = 1.0 / sqrt(-c->g[0][0]);
    double u[4] = {ut, 0, 0, 0};
    double v1[4] = {0, sin(th), 0, cos(th)};  /* outward */
    double v2[4] = {0, -cos(th), 0, sin(th)}; /* toward the spin axis on the screen */
    double v3[4] = {0, 0, 1, 0};              /* screen right */
    double* src[3] = {v1, v2, v3};
    double* dst[3] = {c->e1, c->e2, c->e3};
    memcpy(c->e0, u, sizeof u);
    for (int q = 0; q < 3; ++q) {
        double w[4];
        memcpy(w, src[q], sizeof w);
        double pu = dot_g(c->g, u, src[q]);
        for (int m = 0; m < 4; ++m) w[m] += pu * u[m];
        for (int p = 0; p < q; ++p) {
            double pe = dot_g(c->g, dst[p], src[q]);
            for (int m = 0; m < 4; ++m) w[m] -= pe * dst[p][m];
        }
        double nn = sqrt(dot_g(c->g, w, w));
        for (int m = 0; m < 4; ++m) dst[q][m] = w[m] / nn;
    }
}

/* Backward wave covector of the pixel at screen (alpha, beta):  the photon arrives from the
 * sky direction n = (-e1 + (alpha/r_obs) e3 + (beta/r_obs) e2)/|.|, its momentum is
 * p = e0 - n (camera-frame frequency 1) and the traced vector is k = -p, lowered with g. */
static void camera_ray(const orc_job* job, const camera* c, double al, double be, double* y)
{
    double ro = job->r_obs;
    double s = 1.0 / sqrt(1.0 + (al * al + be * be) / (ro * ro));
    double kup[4];
    for (int m = 0; m < 4; ++m)
        kup[m] = -c->e0[m] + s * (-c->e1[m] + (al / ro) * c->e3[m] + (be / ro) * c->e2[m]);
    for (int m = 0; m < 4; ++m) {
        y[m] = c->x0[m];
        double kl = 0;
        for (int n = 0; n < 4; ++n) kl += c->g[m][n] * kup[n];
        y[4 + m] = kl;
    }
}

/* Constants of motion of the traced covector: lambda = L_z/E, eta = Q/E^2 with
 * E = k_t, L_z = -(x k_y - y k_x) (for p = -k), p_theta from the Kerr-Schild spherical
 * angles, Q = p_theta^2 + cos^2(theta) (-a^2 E^2 + L_z^2 / sin^2(theta)) (Carter 1968). */
static void constants_of_motion(double a, const double* y, double* lam, double* eta)
{
    double r = creal(ks_radius(a, y[1], y[2], y[3]));
    double E = y[4];
    double L = -(y[1] * y[6] - y[2] * y[5]);
    double ct = y[3] / r, st2 = 1.0 - ct * ct, st = sqrt(st2);
    double pth = -((y[1] * y[5] + y[2] * y[6]) * ct / st - r * st * y[7]);
    double Q = pth * pth + ct * ct * (-a * a * E * E + L * L / st2);
    *lam = L / E;
    *eta = Q / (E * E);
}

/* ------------------------------------------------------------------------------------------ */
/* Emission models                                                                             */
/* ------------------------------------------------------------------------------------------ */

/* Fluid four-velocity (Kerr-Schild Cartesian, contravariant).  Keplerian: Omega =
 * sqrt(M)/(r^{3/2} + a sqrt(M)) at Boyer-Lindquist (r, theta), u = u^t (1, -Omega y, Omega x, 0),
 * u^t from g_tt + 2 Omega g_tphi + Omega^2 g_phiphi (Boyer-Lindquist) = -1/(u^t)^2.
 * Static: u = (1/sqrt(-g_tt), 0, 0, 0).  Returns 0 where no timelike velocity exists. */
static int fluid_velocity(const orc_job* job, const double* x, double r, double* u)
{
    double a = job->a, M = job->mass;
    if (job->flow == ORC_FLOW_STATIC || M == 0.0) {
        double g[4][4];
        metric_cov(a, M, x, g);
        if (g[0][0] >= 0) return 0;
        u[0] = 1.0 / sqrt(-g[0][0]);
        u[1] = u[2] = u[3] = 0.0;
        return 1;
    }
    double ct = x[3] / r, st2 = 1.0 - ct * ct;
    double Sig = r * r + a * a * ct * ct;
    double gtt = -(1.0 - 2.0 * M * r / Sig);
    double gtp = -2.0 * M * a * r * st2 / Sig;
    double gpp = (r * r + a * a + 2.0 * M * a * a * r * st2 / Sig) * st2;
    double Om = sqrt(M) / (r * sqrt(r) + a * sqrt(M));
    double nrm = -(gtt + 2.0 * Om * gtp + Om * Om * gpp);
    if (!(nrm > 0)) return 0;
    double ut = 1.0 / sqrt(nrm);
    u[0] = ut;
    u[1] = -Om * x[2] * ut;
    u[2] = Om * x[1] * ut;
    u[3] = 0.0;
    return 1;
}

/* Kerr-Schild spherical angles of a Cartesian point: theta = acos(z/r) and phi from
 * x + i y = (r - i a) sin(theta) e^{i phi}, i.e. phi = atan2(y, x) + atan2(a, r), in [0, 2 pi). */
static void ks_angles(double a, const double* x, double r, double* th, double* ph)
{
    double ct = x[3] / r;
    if (ct > 1) ct = 1;
    if (ct < -1) ct = -1;
    *th = acos(ct);
    double p = atan2(x[2], x[1]) + atan2(a, r);
    if (p < 0) p += 2.0 * M_PI;
    if (p >= 2.0 * M_PI) p -= 2.0 * M_PI;
    *ph = p;
}

/* Trilinear interpolation of the eight cell-centred FP32 primitives at (ln r, theta, phi).
 * Reading of the fluid-grid lookup: the coordinate of each axis in cell units is
 * f = (coordinate - start)/spacing - 1/2; ln r and theta clamp f to [0, n - 1] (the outer half
 * cells take the edge value), phi is periodic.  Points with ln r outside [glogr_min, glogr_max]
 * are outside the fluid and return 0. */
static int grid_prims(const orc_job* job, double r, double th, double ph, double* P)
{
    double x1 = log(r);
    if (!(x1 >= job->glogr_min && x1 <= job->glogr_max)) return 0;
    int n[3] = {job->gn1, job->gn2, job->gn3};
    double f[3] = {(x1 - job->glogr_min) / ((job->glogr_max - job->glogr_min) / n[0]) - 0.5,
                   th / (M_PI / n[1]) - 0.5, ph / (2.0 * M_PI / n[2]) - 0.5};
    int lo[3], hi[3];
    double w[3];
    for (int d = 0; d < 2; ++d) {
        double fd = f[d];
        if (fd < 0) fd = 0;
        if (fd > n[d] - 1) fd = n[d] - 1;
        int i = (int)floor(fd);
        if (i > n[d] - 2) i = n[d] - 2;
        if (i < 0) i = 0;
        lo[d] = i;
        hi[d] = n[d] > 1 ? i + 1 : i;
        w[d] = n[d] > 1 ? fd - i : 0.0;
    }
    {
        double fl = floor(f[2]);
        int i = (int)fl;
        w[2] = f[2] - fl;
        lo[2] = ((i % n[2]) + n[2]) % n[2];
        hi[2] = (lo[2] + 1) % n[2];
    }
    for (int q = 0; q < 8; ++q) P[q] = 0.0;
    for (int c = 0; c < 8; ++c) {
        int ii = (c & 1) ? hi[0] : lo[0], jj = (c & 2) ? hi[1] : lo[1], kk = (c & 4) ? hi[2] : lo[2];
        double wt = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) *
                    ((c & 4) ? w[2] : 1.0 - w[2]);
        const float* cell = job->grid + (((size_t)kk * n[1] + jj) * n[0] + ii) * 8;
        for (int q = 0; q < 8; ++q) P[q] += wt * (double)cell[q];
    }
    return 1;
}

/* Fluid state from the grid at a Cartesian point x (r its Kerr-Schild radius):
 *   u^i, B^i: the interpolated spherical components mapped to Cartesian ones by the Jacobian of
 *     x + i y = (r - i a) sin(theta) e^{i phi}, z = r cos(theta);
 *   u^t: the positive root of g_{mu nu} u^mu u^nu = -1.  With q = 1 + g_ij u^i u^j and
 *     p = g_ti u^i the equation is g_tt (u^t)^2 + 2 p u^t + q = 0, whose root continuous across
 *     the ergosurface (g_tt = 0) is u^t = q / (sqrt(p^2 - g_tt q) - p);
 *   b^mu from the ideal-MHD relations b^t = g_{i mu} B^i u^mu, b^i = (B^i + b^t u^i)/u^t
 *     (Gammie, McKinney & Toth 2003);
 *   electron temperature from the two-temperature prescription of Moscibrodzka, Falcke &
 *     Shiokawa (2016): T_i/T_e = (R_high beta^2 + R_low)/(1 + beta^2) with the plasma
 *     beta = (gamma - 1) u / (b^2/2), Theta_e = (m_p/m_e)(gamma - 1) u / (rho (1 + T_i/T_e));
 *   n_e = rho m_unit / (L^3 (m_p + m_e)), |B| = sqrt(b^2) c sqrt(4 pi m_unit / L^3) gauss.
 * plasma4 = {n_e, Theta_e, |B|, sigma = b^2/rho}.  Returns 1 where the point emits: inside the
 * radial range of the grid, a timelike u, rho > 0, u > 0, b^2 > 0 and sigma <= sigma_cut
 * (the magnetisation cut: more strongly magnetised fluid does not emit). */
int orc_grid_fluid(const orc_job* job, const double* x, double* P, double* u, double* b,
                   double* pl)
{
    const double mp = 1.67262192369e-24, me = 9.1093837015e-28, c = 2.99792458e10;
    double a = job->a, M = job->mass;
    double r = creal(ks_radius(a, x[1], x[2], x[3]));
    double th, ph;
    for (int q = 0; q < 8; ++q) P[q] = 0.0;
    for (int m = 0; m < 4; ++m) u[m] = b[m] = 0.0;
    for (int m = 0; m < 4; ++m) pl[m] = 0.0;
    if (!job->grid) return 0;
    ks_angles(a, x, r, &th, &ph);
    if (!grid_prims(job, r, th, ph, P)) return 0;
    double st = sin(th), ct = cos(th), cp = cos(ph), sp = sin(ph);
    double Jm[3][3] = {{st * cp, ct * (r * cp + a * sp), -x[2]},
                       {st * sp, ct * (r * sp - a * cp), x[1]},
                       {ct, -r * st, 0.0}};
    double uc[4] = {0, 0, 0, 0}, Bc[4] = {0, 0, 0, 0};
    for (int i = 0; i < 3; ++i)
        for (int m = 0; m < 3; ++m) {
            uc[1 + i] += Jm[i][m] * P[2 + m];
            Bc[1 + i] += Jm[i][m] * P[5 + m];
        }
    double g[4][4];
    metric_cov(a, M, x, g);
    double q = 1.0, p = 0.0;
    for (int i = 1; i < 4; ++i) {
        p += g[0][i] * uc[i];
        for (int j = 1; j < 4; ++j) q += g[i][j] * uc[i] * uc[j];
    }
    double D = p * p - g[0][0] * q;
    if (!(D >= 0)) return 0;
    double den = sqrt(D) - p;
    if (!(den > 0)) return 0;
    uc[0] = q / den;
    double bt = 0.0;
    for (int i = 1; i < 4; ++i)
        for (int m = 0; m < 4; ++m) bt += g[i][m] * Bc[i] * uc[m];
    b[0] = bt;
    for (int i = 1; i < 4; ++i) b[i] = (Bc[i] + bt * uc[i]) / uc[0];
    for (int m = 0; m < 4; ++m) u[m] = uc[m];
    double b2 = dot_g(g, b, b);
    double rho = P[0], ug = P[1];
    double L3 = job->length_cm * job->length_cm * job->length_cm;
    double sigma = rho > 0 ? b2 / rho : 0.0;
    double pg = (job->gamma_ad - 1.0) * ug, pm = 0.5 * b2;
    double trat = (job->r_high * pg * pg + job->r_low * pm * pm) / (pg * pg + pm * pm);
    pl[0] = rho * job->m_unit / (L3 * (mp + me));
    pl[1] = (mp / me) * (job->gamma_ad - 1.0) * ug / (rho * (1.0 + trat));
    pl[2] = sqrt(b2 > 0 ? b2 : 0.0) * c * sqrt(4.0 * M_PI * job->m_unit / L3);
    pl[3] = sigma;
    if (!(rho > 0) || !(ug > 0) || !(b2 > 0)) return 0;
    if (sigma > job->sigma_cut) return 0;
    return 1;
}

/* Invariant emission J = j_nu / nu^2 and absorption A = nu alpha_nu at one point (unpolarized
 * models), with nu = k_mu u^mu the fluid-frame frequency in units of the camera frequency. */
static void emission_unpol(const orc_job* job, const double* y, double* J, double* A,
                           double* nu_out)
{
    double a = job->a;
    double r = creal(ks_radius(a, y[1], y[2], y[3]));
    *J = 0.0;
    *A = 0.0;
    if (nu_out) *nu_out = 0.0;
    double rstop = (1.0 + job->horizon_eps) * horizon_radius(a, job->mass);
    if (job->mass > 0 && r < rstop) return;
    double jnu;
    if (job->emission == ORC_EMIT_BLOB) {
        double s2 = job->blob_sigma * job->blob_sigma;
        double d2 = y[1] * y[1] + y[2] * y[2] + y[3] * y[3];
        jnu = exp(-d2 / (2.0 * s2));
    } else { /* ORC_EMIT_ANALYTIC: j = r^-2 exp(-z^2 / (2 (w r)^2)), z = r cos(theta) */
        double ct = y[3] / r;
        double w = job->disk_w;
        jnu = exp(-ct * ct / (2.0 * w * w)) / (r * r);
    }
    double u[4];
    if (!fluid_velocity(job, y, r, u)) return;
    double nu = y[4] * u[0] + y[5] * u[1] + y[6] * u[2] + y[7] * u[3];
    if (nu_out) *nu_out = nu;
    if (!(nu > 0)) return;
    *J = jnu / (nu * nu);
}

int orc_emission(const orc_job* job, const double* x, const double* k, double* jnu, double* nu)
{
    double y[8], A;
    for (int m = 0; m < 4; ++m) { y[m] = x[m]; y[4 + m] = k[m]; }
    emission_unpol(job, y, jnu, &A, nu);
    return 0;
}


/* ------------------------------------------------------------------------------------------ */
/* Polarized transfer: parallel transport, thermal synchrotron, constant-coefficient segments  */
/* ------------------------------------------------------------------------------------------ */

static void metric_cov_c(double a, double M, const cplx* x, cplx g[4][4])
{
    cplx r = ks_radius(a, x[1], x[2], x[3]);
    cplx r2 = r * r;
    cplx f = 2.0 * M * r * r2 / (r2 * r2 + a * a * x[3] * x[3]);
    cplx l[4] = {1.0, -(r * x[1] - a * x[2]) / (r2 + a * a), -(r * x[2] + a * x[1]) / (r2 + a * a),
                 -x[3] / r};
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            g[m][n] = ((m == n) ? (m == 0 ? -1.0 : 1.0) : 0.0) + f * l[m] * l[n];
}

/* Inverse of a 4x4 matrix by Gauss-Jordan elimination with partial pivoting. */
static void inv4(double A[4][4], double B[4][4])
{
    double W[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) W[i][j] = j < 4 ? A[i][j] : (j - 4 == i ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int i = c + 1; i < 4; ++i)
            if (fabs(W[i][c]) > fabs(W[p][c])) p = i;
        for (int j = 0; j < 8; ++j) { double t = W[c][j]; W[c][j] = W[p][j]; W[p][j] = t; }
        double d = W[c][c];
        for (int j = 0; j < 8; ++j) W[c][j] /= d;
        for (int i = 0; i < 4; ++i)
            if (i != c) {
                double m = W[i][c];
                for (int j = 0; j < 8; ++j) W[i][j] -= m * W[c][j];
            }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) B[i][j] = W[i][j + 4];
}

static void raise4(double gi[4][4], const double* v, double* w)
{
    for (int m = 0; m < 4; ++m) {
        w[m] = 0;
        for (int n = 0; n < 4; ++n) w[m] += gi[m][n] * v[n];
    }
}

/* Parallel transport of a covector along the geodesic:
 * df_mu/dlambda = Gamma^alpha_{mu beta} k^beta f_alpha
 *               = 1/2 f^alpha k^beta (d_mu g_{alpha beta} + d_beta g_{alpha mu} - d_alpha g_{mu beta}),
 * with k^beta = dx^beta/dlambda; metric derivatives by complex steps. */
static void transport_rhs(double a, double M, const double* x, const double* kup, const double* f,
                          double* df)
{
    const double hstep = 1e-20;
    double g[4][4], gi[4][4], dg[4][4][4], fup[4];
    metric_cov(a, M, x, g);
    inv4(g, gi);
    raise4(gi, f, fup);
    memset(dg, 0, sizeof dg);
    for (int sdx = 1; sdx < 4; ++sdx) {
        cplx xc[4], gc[4][4];
        for (int m = 0; m < 4; ++m) xc[m] = x[m];
        xc[sdx] += I * hstep;
        metric_cov_c(a, M, xc, gc);
        for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n) dg[sdx][m][n] = cimag(gc[m][n]) / hstep;
    }
    for (int mu = 0; mu < 4; ++mu) {
        double acc = 0;
        for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be)
                acc += fup[al] * kup[be] * (dg[mu][al][be] + dg[be][al][mu] - dg[al][mu][be]);
        df[mu] = 0.5 * acc;
    }
}

/* Modified Bessel function of the second kind from its integral representation
 * K_n(x) = int_0^inf exp(-x cosh t) cosh(n t) dt (Abramowitz & Stegun 9.6.24), by the trapezoid
 * rule, which converges exponentially for this analytic, double-exponentially decaying integrand. */
double orc_bessel_k(int n, double x)
{
    double T = acosh(1.0 + 60.0 / x) + 1.0, h = 1.0 / 64.0;
    int m = (int)(T / h) + 1;
    double s = 0.5 * exp(-x);
    for (int i = 1; i <= m; ++i) {
        double t = i * h;
        s += exp(-x * cosh(t)) * cosh(n * t);
    }
    return s * h;
}

/* Thermal synchrotron coefficients in the frame whose Q axis is the emission's E-vector (normal
 * to the projected field), cgs units, at frequency nu, for electron density ne, dimensionless
 * temperature Th = kT/(m c^2), field B and angle theta_b between the wave vector and the field:
 *   j_I: Leung, Gammie & Noble (2011): n sqrt2 pi e^2 nu_s / (3 K_2(1/Th) c)
 *        (X^1/2 + 2^(11/12) X^1/6)^2 exp(-X^1/3), X = nu/nu_s, nu_s = (2/9) nu_B Th^2 sin theta,
 *        nu_B = e B / (2 pi m c);
 *   j_Q: the same with 2^(11/12) multiplied by (7 Th^0.96 + 35)/(10 Th^0.96 + 75)
 *        (Pandya et al. 2016);
 *   j_V = 0 (no intrinsic circular emission; V arises by Faraday conversion);
 *   alpha_S = j_S / B_nu(T) (Kirchhoff);
 *   rho_V = e^3 n B cos theta / (pi m^2 c^2 nu^2) K_0(1/Th)/K_2(1/Th),
 *   rho_Q = e^4 n B^2 sin^2 theta / (4 pi^2 m^3 c^3 nu^3) (K_1(1/Th)/K_2(1/Th) + 6 Th)
 *        (high-frequency thermal rotativities, e.g. Shcherbakov 2008; their cold-plasma limit is
 *        the textbook rotation measure).
 * out7 = {j_I, j_Q, j_V, alpha_I, alpha_Q, rho_Q, rho_V}. */
int orc_synch_coeffs(double ne, double Th, double B, double nu, double thb, double* out)
{
    const double e = 4.80320471e-10, me = 9.1093837015e-28, c = 2.99792458e10;
    const double hp = 6.62607015e-27;
    for (int i = 0; i < 7; ++i) out[i] = 0.0;
    if (!(ne > 0) || !(Th > 0) || !(B > 0) || !(nu > 0)) return 0;
    double sn = sin(thb), cs = cos(thb);
    double K0 = orc_bessel_k(0, 1.0 / Th), K1 = orc_bessel_k(1, 1.0 / Th), K2 = orc_bessel_k(2, 1.0 / Th);
    double nuB = e * B / (2.0 * M_PI * me * c);
    double Bnu = 2.0 * hp * nu * nu * nu / (c * c) / expm1(hp * nu / (Th * me * c * c));
    if (fabs(sn) > 1e-12) {
        double nus = 2.0 / 9.0 * nuB * Th * Th * fabs(sn);
        double X = nu / nus;
        double pre = ne * sqrt(2.0) * M_PI * e * e * nus / (3.0 * K2 * c) * exp(-cbrt(X));
        double t96 = pow(Th, 24.0 / 25.0);
        double q = (7.0 * t96 + 35.0) / (10.0 * t96 + 75.0);
        double xa = sqrt(X), xb = pow(X, 1.0 / 6.0), k = pow(2.0, 11.0 / 12.0);
        out[0] = pre * (xa + k * xb) * (xa + k * xb);
        out[1] = pre * (xa + q * k * xb) * (xa + q * k * xb);
    }
    out[3] = out[0] / Bnu;
    out[4] = out[1] / Bnu;
    out[5] = e * e * e * e * ne * B * B * sn * sn / (4.0 * M_PI * M_PI * me * me * me * c * c * c * nu * nu * nu) *
             (K1 / K2 + 6.0 * Th);
    out[6] = e * e * e * ne * B * cs / (M_PI * me * me * c * c * nu * nu) * (K0 / K2);
    return 0;
}

/* Exact solution over a segment of length h with constant coefficients of
 * dS/ds = J - K S, K = [[aI,aQ,aU,aV],[aQ,aI,rV,-rU],[aU,-rV,aI,rQ],[aV,rU,-rQ,aI]]
 * (Landi Degl'Innocenti & Landi Degl'Innocenti 1985 sign convention), K7 = {aI,aQ,aU,aV,rQ,rU,rV}:
 * S(h) = E S(0) + X with E = exp(-K h), X = int_0^h exp(-K s) ds J, read off the exponential of
 * the 5x5 augmented matrix [[-K h, J h], [0, 0]], computed by scaling and squaring with a
 * Taylor series (Moler & Van Loan 2003). */
void orc_segment(const double* K7, const double* J4, double h, double* E16, double* X4)
{
    double aI = K7[0], aQ = K7[1], aU = K7[2], aV = K7[3], rQ = K7[4], rU = K7[5], rV = K7[6];
    double K[4][4] = {{aI, aQ, aU, aV}, {aQ, aI, rV, -rU}, {aU, -rV, aI, rQ}, {aV, rU, -rQ, aI}};
    double A[5][5];
    memset(A, 0, sizeof A);
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) A[i][j] = -K[i][j] * h;
        A[i][4] = J4[i] * h;
    }
    double nrm = 0;
    for (int i = 0; i < 5; ++i) {
        double rs = 0;
        for (int j = 0; j < 5; ++j) rs += fabs(A[i][j]);
        if (rs > nrm) nrm = rs;
    }
    int sq = 0;
    while (nrm > 0.125) { nrm *= 0.5; ++sq; }
    double scale = ldexp(1.0, -sq);
    double T[5][5], R[5][5], P[5][5];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            A[i][j] *= scale;
            T[i][j] = (i == j) ? 1.0 : 0.0;
            R[i][j] = T[i][j];
        }
    for (int k = 1; k <= 24; ++k) {
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double v = 0;
                for (int m = 0; m < 5; ++m) v += T[i][m] * A[m][j];
                P[i][j] = v / k;
            }
        memcpy(T, P, sizeof T);
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) R[i][j] += T[i][j];
    }
    for (int q = 0; q < sq; ++q) {
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double v = 0;
                for (int m = 0; m < 5; ++m) v += R[i][m] * R[m][j];
                P[i][j] = v;
            }
        memcpy(R, P, sizeof R);
    }
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) E16[4 * i + j] = R[i][j];
        X4[i] = R[i][4];
    }
}

/* Polarized emission at one point of the ray, in code units and in the polarization basis
 * (e_N, e_E) carried by the transported covector f:  J4 = L j_S / nu^2 and
 * K7 = L nu {alpha_I, alpha_Q, alpha_U, alpha_V, rho_Q, rho_U, rho_V}, with nu = k.u the fluid-frame
 * frequency ratio and L = GM/c^2 in cm.  e_N is f projected normal to the fluid velocity u and
 * to the propagation direction d = p/nu - u (p = -k); e_E = d x e_N in the fluid frame (at the
 * camera: north = screen up, east = screen left, the IAU convention); the emission's E-vector
 * d x b is at angle chi from e_N, so (Q, U) = P (cos 2 chi, sin 2 chi).
 * Disk model: n_e = ne0 r^ne_slope exp(-cos^2(theta)/(2 w^2)), Th_e = thetae0 r^te_slope,
 * |B| = b0 r^((ne_slope + te_slope)/2), direction (e_phi + q e_z)/sqrt(1 + q^2) in the fluid
 * frame with q = bz_ratio (toroidal : vertical = 1 : q), Keplerian flow; zero inside r_in.
 * Grid model: u, b, n_e, Theta_e and |B| from orc_grid_fluid. */
static void emission_pol(const orc_job* job, const double* y, const double* fcov, double* J4,
                         double* K7)
{
    double a = job->a, M = job->mass;
    for (int i = 0; i < 4; ++i) J4[i] = 0;
    for (int i = 0; i < 7; ++i) K7[i] = 0;
    double r = creal(ks_radius(a, y[1], y[2], y[3]));
    double rstop = (1.0 + job->horizon_eps) * horizon_radius(a, M);
    if (r < rstop || r < job->r_in) return;
    double u[4], b[4], ne, Th, Bm;
    double g[4][4], gi[4][4];
    metric_cov(a, M, y, g);
    if (job->emission == ORC_EMIT_GRID) {
        /* fluid grid: u, b and the plasma from the lookup; b made a unit vector */
        double P[8], pl[4];
        if (!orc_grid_fluid(job, y, P, u, b, pl)) return;
        ne = pl[0];
        Th = pl[1];
        Bm = pl[2];
        double bb = sqrt(dot_g(g, b, b));
        for (int m = 0; m < 4; ++m) b[m] /= bb;
    } else {
        if (!fluid_velocity(job, y, r, u)) return;
        double ct = y[3] / r;
        ne = job->ne0 * pow(r, job->ne_slope) * exp(-ct * ct / (2.0 * job->disk_w * job->disk_w));
        Th = job->thetae0 * pow(r, job->te_slope);
        Bm = job->b0 * pow(r, 0.5 * (job->ne_slope + job->te_slope));
        if (!(ne > 0)) return;
        /* field direction: toroidal and vertical unit vectors of the fluid frame */
        double vphi[4] = {0, -y[2], y[1], 0}, vz[4] = {0, 0, 0, 1}, ephi[4], ez[4];
        double pu = dot_g(g, u, vphi);
        for (int m = 0; m < 4; ++m) ephi[m] = vphi[m] + pu * u[m];
        double nph = sqrt(dot_g(g, ephi, ephi));
        for (int m = 0; m < 4; ++m) ephi[m] /= nph;
        double pz = dot_g(g, u, vz), pe = dot_g(g, ephi, vz);
        for (int m = 0; m < 4; ++m) ez[m] = vz[m] + pz * u[m] - pe * ephi[m];
        double nz = sqrt(dot_g(g, ez, ez));
        double bn = 1.0 / sqrt(1.0 + job->bz_ratio * job->bz_ratio);
        for (int m = 0; m < 4; ++m) {
            ez[m] /= nz;
            b[m] = (ephi[m] + job->bz_ratio * ez[m]) * bn;
        }
    }
    inv4(g, gi);
    double kup[4], p[4], fup[4] = {0, 0, 0, 0};
    raise4(gi, y + 4, kup);
    if (fcov) raise4(gi, fcov, fup);
    double nu = 0;
    for (int m = 0; m < 4; ++m) nu += y[4 + m] * u[m];
    if (!(nu > 0)) return;
    double d[4];
    for (int m = 0; m < 4; ++m) {
        p[m] = -kup[m];
        d[m] = p[m] / nu - u[m];
    }
    /* the propagation direction is a unit vector of the fluid frame; the integrated k is null only
     * to the RK4 truncation error, so normalise it */
    double dn = sqrt(dot_g(g, d, d));
    for (int m = 0; m < 4; ++m) d[m] /= dn;
    double cthb = dot_g(g, d, b);
    if (cthb > 1) cthb = 1;
    if (cthb < -1) cthb = -1;
    double thb = acos(cthb);
    if (!fcov) { /* unpolarized: total intensity only */
        double co[7];
        orc_synch_coeffs(ne, Th, Bm, job->nu_hz * nu, thb, co);
        J4[0] = job->length_cm * co[0] / (nu * nu);
        K7[0] = job->length_cm * nu * co[3];
        return;
    }
    /* basis: e_N from f, e_E = d x e_N; E-vector of the emission: d x b */
    double eN[4], fu = dot_g(g, fup, u), fd = dot_g(g, fup, d);
    for (int m = 0; m < 4; ++m) eN[m] = fup[m] + fu * u[m] - fd * d[m];
    double nN = sqrt(dot_g(g, eN, eN));
    for (int m = 0; m < 4; ++m) eN[m] /= nN;
    double eEc[4], eE[4], evc[4], ev[4];
    for (int m = 0; m < 4; ++m) { eEc[m] = 0; evc[m] = 0; }
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            for (int q = 0; q < 4; ++q)
                for (int w = 0; w < 4; ++w) {
                    if (m == n || m == q || m == w || n == q || n == w || q == w) continue;
                    /* sign of the permutation (m n q w) of (0 1 2 3) */
                    int pidx[4] = {m, n, q, w}, sg = 1;
                    for (int i = 0; i < 4; ++i)
                        for (int j = i + 1; j < 4; ++j)
                            if (pidx[i] > pidx[j]) sg = -sg;
                    eEc[m] -= sg * u[n] * d[q] * eN[w];
                    evc[m] -= sg * u[n] * d[q] * b[w];
                }
    raise4(gi, eEc, eE);
    raise4(gi, evc, ev);
    double nv = sqrt(dot_g(g, ev, ev));
    double c1 = 0, s1 = 0;
    if (nv > 0) {
        c1 = dot_g(g, ev, eN) / nv;
        s1 = dot_g(g, ev, eE) / nv;
    }
    double c2 = c1 * c1 - s1 * s1, s2 = 2.0 * c1 * s1;
    double co[7];
    orc_synch_coeffs(ne, Th, Bm, job->nu_hz * nu, thb, co);
    double L = job->length_cm;
    J4[0] = L * co[0] / (nu * nu);
    J4[1] = L * co[1] * c2 / (nu * nu);
    J4[2] = L * co[1] * s2 / (nu * nu);
    J4[3] = L * co[2] / (nu * nu);
    K7[0] = L * nu * co[3];
    K7[1] = L * nu * co[4] * c2;
    K7[2] = L * nu * co[4] * s2;
    K7[3] = 0.0;
    K7[4] = L * nu * co[5] * c2;
    K7[5] = L * nu * co[5] * s2;
    K7[6] = L * nu * co[6];
}

/* ------------------------------------------------------------------------------------------ */
/* Ray tracer                                                                                  */
/* ------------------------------------------------------------------------------------------ */

/* Right-hand side of the ray ODE: y = (x^mu, k_mu[, f_mu]) with n = 8 (geodesic) or 12 (geodesic
 * plus the parallel-transported polarization covector). */
static void ray_rhs(double a, double M, int n, const double* y, double* dy)
{
    geodesic_rhs(a, M, y, dy);
    if (n == 12) transport_rhs(a, M, y, dy, y + 8, dy + 8);
}

static void rk4_step(double a, double M, int n, double h, const double* y, double* yn)
{
    double k1[12], k2[12], k3[12], k4[12], t[12];
    ray_rhs(a, M, n, y, k1);
    for (int m = 0; m < n; ++m) t[m] = y[m] + 0.5 * h * k1[m];
    ray_rhs(a, M, n, t, k2);
    for (int m = 0; m < n; ++m) t[m] = y[m] + 0.5 * h * k2[m];
    ray_rhs(a, M, n, t, k3);
    for (int m = 0; m < n; ++m) t[m] = y[m] + h * k3[m];
    ray_rhs(a, M, n, t, k4);
    for (int m = 0; m < n; ++m) yn[m] = y[m] + h / 6.0 * (k1[m] + 2.0 * k2[m] + 2.0 * k3[m] + k4[m]);
}

/* (1 - exp(-x))/x, continuous at 0. */
static double phi1(double x) { return x > 1e-8 ? -expm1(-x) / x : 1.0 - 0.5 * x; }

/* Sign of d(theta)/d(lambda) along the traced ray, from the covariant theta momentum in the
 * Kerr-Schild spherical angles: k_theta sin(theta) = (x k_x + y k_y) z/r - (r - z^2/r) k_z.
 * Values within 1e-9 r of zero return 0 (no decision), so radial rays count no turning points.
 * Turning points of theta after the ray's first crossing of the equatorial plane separate its
 * passes through that plane: the subring index n of an emission point is the number of them
 * between it and the camera. */
static int polar_sign(const double* y, double r)
{
    double q = (y[1] * y[5] + y[2] * y[6]) * y[3] / r - (r - y[3] * y[3] / r) * y[7];
    double tol = 1e-9 * r;
    return q > tol ? 1 : (q < -tol ? -1 : 0);
}

/* Camera polarization reference: the screen's up vector e2 made normal to the pixel's line of
 * sight n = s (-e1 + (alpha/r_obs) e3 + (beta/r_obs) e2), normalised and lowered. */
static void camera_polbasis(const orc_job* job, const camera* c, double al, double be, double* fcov)
{
    double ro = job->r_obs;
    double s = 1.0 / sqrt(1.0 + (al * al + be * be) / (ro * ro));
    double en = s * be / ro, f[4];
    for (int m = 0; m < 4; ++m) {
        double n = s * (-c->e1[m] + (al / ro) * c->e3[m] + (be / ro) * c->e2[m]);
        f[m] = c->e2[m] - en * n;
    }
    double nn = sqrt(dot_g((double(*)[4])c->g, f, f));
    for (int m = 0; m < 4; ++m) f[m] /= nn;
    for (int m = 0; m < 4; ++m) {
        fcov[m] = 0;
        for (int n = 0; n < 4; ++n) fcov[m] += c->g[m][n] * f[n];
    }
}

/* Emission (J4) and absorption/rotation (K7) coefficients at one point, code units. */
static void coefficients(const orc_job* job, const double* y, int pol, double* J4, double* K7)
{
    if (job->emission == ORC_EMIT_SYNCH_DISK || job->emission == ORC_EMIT_GRID) {
        emission_pol(job, y, pol ? y + 8 : NULL, J4, K7);
        return;
    }
    for (int i = 0; i < 4; ++i) J4[i] = 0;
    for (int i = 0; i < 7; ++i) K7[i] = 0;
    emission_unpol(job, y, &J4[0], &K7[0], NULL);
}

/* Exported for tests: transport derivative and point coefficients of a 12-component state. */
void orc_transport_rhs(const orc_job* job, const double* y, double* df)
{
    double dy[8];
    geodesic_rhs(job->a, job->mass, y, dy);
    transport_rhs(job->a, job->mass, y, dy, y + 8, df);
}

void orc_coefficients(const orc_job* job, const double* y, int pol, double* J4, double* K7)
{
    coefficients(job, y, pol, J4, K7);
}

/* Trace one ray backward from the camera.  out[] receives the planes of this ray (Stokes inside
 * subring index).  Per RK4 step, the coefficients at both ends are averaged and the segment is
 * solved exactly; contributions are carried to the camera by the accumulated propagator. */
static void trace_one(const orc_job* job, const camera* cam, double al, double be, double* out,
                      orc_rayinfo* info, double* rec, int maxrec, int* nrec)
{
    double a = job->a, M = job->mass;
    const int pol = job->stokes == 4;
    const int n = pol ? 12 : 8;
    const int nst = pol ? 4 : 1;
    int planes = orc_planes(job);
    double y[12], yn[12];
    memset(y, 0, sizeof y);
    camera_ray(job, cam, al, be, y);
    if (pol) camera_polbasis(job, cam, al, be, y + 8);
    for (int p = 0; p < planes; ++p) out[p] = 0.0;
    double rin = M > 0 ? (1.0 + job->horizon_eps) * horizon_radius(a, M) : 0.0;
    double rout = job->escape_frac * job->r_obs;
    double r = creal(ks_radius(a, y[1], y[2], y[3]));
    double J0[4], K0[7], J1[4], K1[7];
    coefficients(job, y, pol, J0, K0);
    double T = 1.0, lam_aff = 0.0, Iacc = 0.0;
    double P[16];
    for (int i = 0; i < 16; ++i) P[i] = (i % 5 == 0) ? 1.0 : 0.0;
    double min_r = r;
    int nturn = 0, steps = 0, status = ORC_RAY_CAP, crossed = 0;
    int theta_sign = polar_sign(y, r);
    if (rec && maxrec > 0) {
        memset(rec, 0, sizeof(double) * 14);
        for (int m = 0; m < n; ++m) rec[1 + m] = y[m];
        *nrec = 1;
    }
    while (steps < job->max_steps) {
        double h = job->step_frac * r;
        if (h < job->h_min) h = job->h_min;
        rk4_step(a, M, n, h, y, yn);
        ++steps;
        lam_aff += h;
        int finite = 1;
        for (int m = 0; m < n; ++m) finite &= isfinite(yn[m]);
        if (!finite) { status = ORC_RAY_NAN; break; }
        double rn = creal(ks_radius(a, yn[1], yn[2], yn[3]));
        coefficients(job, yn, pol, J1, K1);
        /* subring index of this segment: polar turning points before the segment starts,
         * counted from the first crossing of the equatorial plane on (a turning point on the
         * camera side of the first crossing does not end a half-orbit) */
        int seg_turn = nturn;
        if (y[3] * yn[3] < 0) crossed = 1;
        int sg = polar_sign(yn, rn);
        if (sg != 0) {
            if (crossed && theta_sign != 0 && sg != theta_sign) ++nturn;
            theta_sign = sg;
        }
        int plane0 = 0;
        if (job->subrings > 0) plane0 = nst * (seg_turn < job->subrings ? seg_turn : job->subrings - 1);
        if (!pol) {
            /* trapezoid-averaged coefficients, exact constant-coefficient segment */
            double Jb = 0.5 * (J0[0] + J1[0]), Ab = 0.5 * (K0[0] + K1[0]);
            double dtau = Ab * h;
            double dI = T * Jb * h * phi1(dtau);
            Iacc += dI;
            out[plane0] += dI;
            T *= exp(-dtau);
        } else {
            double Jb[4], Kb[7], E[16], X[4];
            for (int i = 0; i < 4; ++i) Jb[i] = 0.5 * (J0[i] + J1[i]);
            for (int i = 0; i < 7; ++i) Kb[i] = 0.5 * (K0[i] + K1[i]);
            int active = 0;
            for (int i = 0; i < 4; ++i) active |= (Jb[i] != 0.0);
            for (int i = 0; i < 7; ++i) active |= (Kb[i] != 0.0);
            if (active) {
                orc_segment(Kb, Jb, h, E, X);
                double Pn[16];
                for (int i = 0; i < 4; ++i) {
                    double c = 0;
                    for (int j = 0; j < 4; ++j) c += P[4 * i + j] * X[j];
                    out[plane0 + i] += c;
                    if (i == 0) Iacc += c;
                    for (int j = 0; j < 4; ++j) {
                        double v = 0;
                        for (int m = 0; m < 4; ++m) v += P[4 * i + m] * E[4 * m + j];
                        Pn[4 * i + j] = v;
                    }
                }
                memcpy(P, Pn, sizeof P);
            }
        }
        memcpy(y, yn, sizeof y);
        memcpy(J0, J1, sizeof J0);
        memcpy(K0, K1, sizeof K0);
        r = rn;
        if (r < min_r) min_r = r;
        if (rec && *nrec < maxrec) {
            double* row = rec + 14 * (*nrec);
            memset(row, 0, sizeof(double) * 14);
            row[0] = lam_aff;
            for (int m = 0; m < n; ++m) row[1 + m] = y[m];
            row[13] = Iacc;
            ++(*nrec);
        }
        if (r < rin) { status = ORC_RAY_CAPTURED; break; }
        if (r > rout) { status = ORC_RAY_ESCAPED; break; }
    }
    if (info) {
        info->status = status;
        info->steps = steps;
        info->nturn = nturn;
        info->min_r = min_r;
        double y0[8];
        camera_ray(job, cam, al, be, y0);
        constants_of_motion(a, y0, &info->lam, &info->eta);
    }
}

int orc_trace_screen(const orc_job* job, int n, const double* alpha, const double* beta,
                     double* out, orc_rayinfo* info)
{
    if (job->stokes != 1 && job->stokes != 4) return -2;
    camera cam;
    camera_setup(job, &cam);
    int planes = orc_planes(job);
#pragma omp parallel for schedule(dynamic, 8) num_threads(orc_get_threads())
    for (int q = 0; q < n; ++q)
        trace_one(job, &cam, alpha[q], beta[q], out + (size_t)q * planes, info ? info + q : NULL,
                  NULL, 0, NULL);
    return 0;
}

int orc_trace_pixels(const orc_job* job, int n, const int64_t* pix, double* out,
                     orc_rayinfo* info)
{
    int nx, ny;
    if (orc_image_size(job, &nx, &ny)) return -1;
    double* al = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* be = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int q = 0; q < n; ++q)
        screen_of_pixel(job, nx, ny, (int)(pix[q] % nx), (int)(pix[q] / nx), &al[q], &be[q]);
    int rc = orc_trace_screen(job, n, al, be, out, info);
    free(al);
    free(be);
    return rc;
}

int orc_trace_record(const orc_job* job, double alpha, double beta, int maxrec, double* rec,
                     int* nrec)
{
    camera cam;
    camera_setup(job, &cam);
    double out[64];
    orc_rayinfo info;
    *nrec = 0;
    if (orc_planes(job) > 64) return -2;
    trace_one(job, &cam, alpha, beta, out, &info, rec, maxrec, nrec);
    return info.status;
}

/* ------------------------------------------------------------------------------------------ */
/* Adaptive refinement (Sec. 3.2, Appendix A)                                                  */
/* ------------------------------------------------------------------------------------------ */

/* I_bar_int: mean over the field of view of the bilinear interpolant of the base samples
 * (sub-lattice of stride `stride`), i.e. trapezoid weights 1/2 on the edges, 1 inside. */
double orc_ibar_int(const double* img, int nx, int ny, int stride)
{
    int n0x = (nx - 1) / stride + 1, n0y = (ny - 1) / stride + 1;
    double s = 0, w = 0;
    for (int jj = 0; jj < n0y; ++jj) {
        double wy = (n0y > 1 && (jj == 0 || jj == n0y - 1)) ? 0.5 : 1.0;
        for (int ii = 0; ii < n0x; ++ii) {
            double wx = (n0x > 1 && (ii == 0 || ii == n0x - 1)) ? 0.5 : 1.0;
            s += wx * wy * img[(size_t)jj * stride * nx + (size_t)ii * stride];
            w += wx * wy;
        }
    }
    return s / w;
}

/* Category of the point (i, j) on the level with stride s (Sec. 3.2): 1 = computed at the
 * previous level, 2 = between a pair above/below, 3 = between a pair left/right, 4 = centre. */
static int category(int i, int j, int s)
{
    int oi = (i / s) & 1, oj = (j / s) & 1;
    if (!oi && !oj) return 1;
    if (!oi && oj) return 2;
    if (oi && !oj) return 3;
    return 4;
}

/* The sum of the two central second differences along one line through the point, with inner
 * neighbours at -/+ d and outer ones at -/+ 3d (Appendix A): I(-3) - I(-1) - I(+1) + I(+3).
 * Where one outer point lies outside the image the one available second difference is doubled;
 * where none is available, *ok = 0.  `get` reads the image with bounds. */
static double second_diff_sum(const double* img, int nx, int ny, int i, int j, int di, int dj,
                              int* ok)
{
    int im = i - di, jm = j - dj, ip = i + di, jp = j + dj;
    int iom = i - 3 * di, jom = j - 3 * dj, iop = i + 3 * di, jop = j + 3 * dj;
    int has_m = iom >= 0 && iom < nx && jom >= 0 && jom < ny;
    int has_p = iop >= 0 && iop < nx && jop >= 0 && jop < ny;
    double Im = img[(size_t)jm * nx + im], Ip = img[(size_t)jp * nx + ip];
    if (has_m && has_p) return img[(size_t)jom * nx + iom] - Im - Ip + img[(size_t)jop * nx + iop];
    if (has_m) return 2.0 * (img[(size_t)jom * nx + iom] - 2.0 * Im + Ip);
    if (has_p) return 2.0 * (img[(size_t)jop * nx + iop] - 2.0 * Ip + Im);
    *ok = 0;
    return 0.0;
}

/* Estimated errors and interpolant of one new point (Eqs. epabs, eprel; Appendix A).
 * Linear, category 4: eps_abs = |S_out - S_in| / (16 norm), eps_rel = |S_out - S_in|/(4 |S_in|),
 *   interpolant S_in / 4.
 * Linear, categories 2/3 (the 1-D simplification): eps_abs = |S_out - S_in| / (8 norm),
 *   eps_rel = |S_out - S_in| / (4 |S_in|), interpolant S_in / 2.
 * Nearest, category 4: sqrt(((I4-I1)/2)^2 + ((I3-I2)/2)^2) over norm and over |I1|,
 *   interpolant I1;  categories 2/3: |I2 - I1|/2 over norm and over |I1|, interpolant I1.
 * Returns 1 when the point must be traced. */
static int estimate_point_nd(const orc_job* job, const double* img, int nx, int ny, int i, int j,
                             int s, double norm, double* interp, double* ea, double* er,
                             double* num_out, double* den_out)
{
    int cat = category(i, j, s);
    int ok = 1;
    double num, sin_, i1;
    if (cat == 4) {
        /* 1 = (-,-), 4 = (+,+) on one diagonal; 2 = (-,+), 3 = (+,-) on the other. */
        double I1 = img[(size_t)(j - s) * nx + (i - s)], I4 = img[(size_t)(j + s) * nx + (i + s)];
        double I2 = img[(size_t)(j + s) * nx + (i - s)], I3 = img[(size_t)(j - s) * nx + (i + s)];
        sin_ = I1 + I2 + I3 + I4;
        i1 = I1;
        if (job->interp == ORC_INTERP_NEAREST) {
            num = sqrt(0.25 * (I4 - I1) * (I4 - I1) + 0.25 * (I3 - I2) * (I3 - I2));
            *interp = I1;
        } else {
            double dA = second_diff_sum(img, nx, ny, i, j, s, s, &ok);
            double dB = second_diff_sum(img, nx, ny, i, j, s, -s, &ok);
            num = fabs(dA + dB) / 16.0;
            *interp = 0.25 * sin_;
        }
    } else {
        int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
        double I1 = img[(size_t)(j - dj) * nx + (i - di)], I2 = img[(size_t)(j + dj) * nx + (i + di)];
        sin_ = I1 + I2;
        i1 = I1;
        if (job->interp == ORC_INTERP_NEAREST) {
            num = fabs(I2 - I1) / 2.0;
            *interp = I1;
        } else {
            double d = second_diff_sum(img, nx, ny, i, j, di, dj, &ok);
            num = fabs(d) / 8.0;
            *interp = 0.5 * sin_;
        }
    }
    /* no second difference available on some line: the estimate is +inf, so the point is
     * traced for every finite tolerance (and still interpolated in the R = +inf limit) */
    if (!ok && job->interp == ORC_INTERP_LINEAR) {
        *ea = INFINITY;
        *er = INFINITY;
        *num_out = INFINITY;
        *den_out = 0.0;
        return (*ea > job->R_abs) && (*er > job->R_rel);
    }
    /* eps_abs = num / norm; eps_rel = num / |interpolant| (linear: (S_out-S_in)/(4 S_in)) */
    double den = (job->interp == ORC_INTERP_NEAREST) ? fabs(i1)
                 : (cat == 4 ? fabs(sin_) / 4.0 : fabs(sin_) / 2.0);
    *num_out = num;
    *den_out = den;
    *ea = num / norm;
    if (den == 0.0) *er = (num == 0.0) ? 0.0 : INFINITY;
    else *er = num / den;
    if (isnan(*ea) || isnan(*er) || isnan(*interp)) return 1;
    return (*ea > job->R_abs) && (*er > job->R_rel);
}

static int estimate_point(const orc_job* job, const double* img, int nx, int ny, int i, int j,
                          int s, double norm, double* interp, double* ea, double* er)
{
    double num, den;
    return estimate_point_nd(job, img, nx, ny, i, j, s, norm, interp, ea, er, &num, &den);
}

/* The polarized variant of the criterion (Sec. 6: "replacing I by Q, U, V"): the estimate of
 * plane `plane` (Q, U or V) at the point from the same stencil and divisors as I's, eps_abs over
 * the same normalisation, eps_rel over I's denominator |S_in(I)|/4 (centre) or /2 (midpoint), or
 * |I_1| (nearest) -- Q, U and V themselves may vanish or change sign.  Returns 1 when that plane
 * asks for the point to be traced. */
static int plane_triggers(const orc_job* job, const double* img, const double* plane, int nx,
                          int ny, int i, int j, int s, double norm)
{
    double ic, eac, erc, numc, denc, iI, eaI, erI, numI, denI;
    estimate_point_nd(job, plane, nx, ny, i, j, s, norm, &ic, &eac, &erc, &numc, &denc);
    estimate_point_nd(job, img, nx, ny, i, j, s, norm, &iI, &eaI, &erI, &numI, &denI);
    if (isinf(numc)) return (INFINITY > job->R_abs) && (INFINITY > job->R_rel);
    double er = (denI == 0.0) ? (numc == 0.0 ? 0.0 : INFINITY) : numc / denI;
    if (isnan(eac) || isnan(er)) return 1;
    return (eac > job->R_abs) && (er > job->R_rel);
}

/* One refinement level (Sec. 3.2): every new point of level `level` reads only points of the
 * previous level; it is marked ORC_MASK_TRACED (to be traced by the caller) or receives its
 * interpolant and ORC_MASK_INTERP.  est_abs / est_rel (nullable) receive the estimates. */
int orc_refine_level(const orc_job* job, double* img, uint8_t* mask, int nx, int ny, int level,
                     double norm, double* est_abs, double* est_rel)
{
    if (level < 1 || level > job->levels) return -1;
    const int planes = orc_planes(job);
    const size_t npix = (size_t)nx * ny;
    int s = 1 << (job->levels - level);
    for (int j = 0; j < ny; j += s)
        for (int i = 0; i < nx; i += s) {
            int cat = category(i, j, s);
            if (cat == 1) continue;
            double interp, ea, er;
            const double* dimg = img + (size_t)job->criterion_plane * npix;
            int tr = estimate_point(job, dimg, nx, ny, i, j, s, norm, &interp, &ea, &er);
            if (!tr && job->criterion == ORC_CRIT_STOKES_ANY && job->stokes == 4)
                for (int c = 1; c < 4 && !tr; ++c)
                    tr = plane_triggers(job, img, img + c * npix, nx, ny, i, j, s, norm);
            if (job->edge_mode == ORC_EDGE_TRACE) {
                int di = (cat == 2) ? 0 : s, dj = (cat == 3) ? 0 : s;
                if (i - 3 * di < 0 || i + 3 * di >= nx || j - 3 * dj < 0 || j + 3 * dj >= ny) tr = 1;
            }
            size_t p = (size_t)j * nx + i;
            if (est_abs) est_abs[p] = ea;
            if (est_rel) est_rel[p] = er;
            if (tr) {
                mask[p] = ORC_MASK_TRACED;
                continue;
            }
            mask[p] = ORC_MASK_INTERP;
            (void)interp;
            /* every plane (I and Stokes Q, U, V; subrings) takes the same interpolation weights */
            for (int c = 0; c < planes; ++c) {
                const double* pl = img + c * npix;
                double v;
                if (job->interp == ORC_INTERP_NEAREST) {
                    v = (cat == 4) ? pl[(size_t)(j - s) * nx + (i - s)]
                                   : pl[(size_t)(j - (cat == 2 ? s : 0)) * nx + (i - (cat == 3 ? s : 0))];
                } else if (cat == 4) {
                    v = 0.25 * (pl[(size_t)(j - s) * nx + (i - s)] + pl[(size_t)(j + s) * nx + (i - s)] +
                                pl[(size_t)(j - s) * nx + (i + s)] + pl[(size_t)(j + s) * nx + (i + s)]);
                } else {
                    int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
                    v = 0.5 * (pl[(size_t)(j - dj) * nx + (i - di)] + pl[(size_t)(j + dj) * nx + (i + di)]);
                }
                img[c * npix + p] = v;
            }
        }
    return 0;
}

/* The whole adaptive scheme (Sec. 3.2).  `truth` (nullable, nx*ny) replaces the ray tracer by
 * a lookup, so the refinement logic can be checked on analytic images. */
int orc_render(const orc_job* job, const double* truth, double* img, uint8_t* mask,
               orc_stats* stats_out)
{
    int nx, ny;
    if (orc_image_size(job, &nx, &ny)) return -1;
    if (job->stokes != 1 && job->stokes != 4) return -2;
    const int planes = orc_planes(job);
    size_t npix = (size_t)nx * ny;
    memset(mask, 0, npix);
    for (size_t p = 0; p < npix * planes; ++p) img[p] = 0.0;
    int64_t* list = malloc(sizeof(int64_t) * npix);
    double* vals = malloc(sizeof(double) * npix * planes);
    orc_rayinfo* info = malloc(sizeof(orc_rayinfo) * npix);
    orc_stats st;
    memset(&st, 0, sizeof st);
    int S0 = 1 << job->levels, rc = 0;
    for (int level = 0; level <= job->levels && rc == 0; ++level) {
        int s = 1 << (job->levels - level);
        int64_t n = 0;
        if (level == 0) {
            for (int j = 0; j < ny; j += S0)
                for (int i = 0; i < nx; i += S0) list[n++] = (int64_t)j * nx + i;
        } else {
            orc_refine_level(job, img, mask, nx, ny, level, st.ibar, NULL, NULL);
            for (int j = 0; j < ny; j += s)
                for (int i = 0; i < nx; i += s) {
                    size_t p = (size_t)j * nx + i;
                    if (category(i, j, s) != 1 && mask[p] == ORC_MASK_TRACED) list[n++] = (int64_t)p;
                }
        }
        if (truth) {
            for (int64_t q = 0; q < n; ++q)
                for (int c = 0; c < planes; ++c) vals[q * planes + c] = truth[c * npix + list[q]];
        } else {
            rc = orc_trace_pixels(job, (int)n, list, vals, info);
            for (int64_t q = 0; q < n && rc == 0; ++q) st.steps += info[q].steps;
        }
        for (int64_t q = 0; q < n; ++q) {
            for (int c = 0; c < planes; ++c) img[c * npix + list[q]] = vals[q * planes + c];
            mask[list[q]] = ORC_MASK_TRACED;
        }
        st.rays_traced += n;
        if (level < 16) st.rays_per_level[level] = n;
        if (level == 0) {
            if (job->abs_norm == ORC_NORM_PEAK) {
                st.ibar = -INFINITY;
                for (int64_t q = 0; q < n; ++q)
                    st.ibar = fmax(st.ibar, vals[q * planes + job->criterion_plane]);
            } else {
                st.ibar = orc_ibar_int(img + (size_t)job->criterion_plane * npix, nx, ny, S0);
            }
        }
    }
    free(list);
    free(vals);
    free(info);
    if (stats_out) *stats_out = st;
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Image metrics (Eqs. interpdef, fluxdef, msedef)                                             */
/* ------------------------------------------------------------------------------------------ */

/* out[0] = interpolation fraction, out[1] = flux error |F - F_hat| / |F| with F the trapezoid
 * integral over the nodal grid, out[2] = MSE = sum |I - I_hat|^2 / sum |I|^2,
 * out[3] = sum |I - I_hat|^2 / (N mean(I)^2). */
void orc_metrics(const double* truth, const double* img, const uint8_t* mask, int nx, int ny,
                 double* out)
{
    double ninterp = 0, F = 0, Fh = 0, se = 0, s2 = 0, sm = 0;
    for (int j = 0; j < ny; ++j) {
        double wy = (ny > 1 && (j == 0 || j == ny - 1)) ? 0.5 : 1.0;
        for (int i = 0; i < nx; ++i) {
            double wx = (nx > 1 && (i == 0 || i == nx - 1)) ? 0.5 : 1.0;
            size_t p = (size_t)j * nx + i;
            if (mask && mask[p] == ORC_MASK_INTERP) ninterp += 1;
            F += wx * wy * truth[p];
            Fh += wx * wy * img[p];
            double d = truth[p] - img[p];
            se += d * d;
            s2 += truth[p] * truth[p];
            sm += truth[p];
        }
    }
    double N = (double)nx * ny;
    double mean = sm / N;
    out[0] = ninterp / N;
    out[1] = fabs(F - Fh) / fabs(F);
    out[2] = se / s2;
    out[3] = se / (N * mean * mean);
}
