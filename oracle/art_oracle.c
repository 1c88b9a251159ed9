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
    } else { /* ORC_EMIT_CFG0: j = r^-2 exp(-z^2 / (2 (w r)^2)), z = r cos(theta) */
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
/* Ray tracer                                                                                  */
/* ------------------------------------------------------------------------------------------ */

static void rk4_step(double a, double M, double h, const double* y, double* yn)
{
    double k1[8], k2[8], k3[8], k4[8], t[8];
    geodesic_rhs(a, M, y, k1);
    for (int m = 0; m < 8; ++m) t[m] = y[m] + 0.5 * h * k1[m];
    geodesic_rhs(a, M, t, k2);
    for (int m = 0; m < 8; ++m) t[m] = y[m] + 0.5 * h * k2[m];
    geodesic_rhs(a, M, t, k3);
    for (int m = 0; m < 8; ++m) t[m] = y[m] + h * k3[m];
    geodesic_rhs(a, M, t, k4);
    for (int m = 0; m < 8; ++m) yn[m] = y[m] + h / 6.0 * (k1[m] + 2.0 * k2[m] + 2.0 * k3[m] + k4[m]);
}

/* (1 - exp(-x))/x, continuous at 0. */
static double phi1(double x) { return x > 1e-8 ? -expm1(-x) / x : 1.0 - 0.5 * x; }

/* Sign of d(theta)/d(lambda) along the traced ray, from the covariant theta momentum in the
 * Kerr-Schild spherical angles: k_theta sin(theta) = (x k_x + y k_y) z/r - (r - z^2/r) k_z.
 * Values within 1e-9 r of zero return 0 (no decision), so radial rays count no turning points.
 * Turning points of theta separate the passes of the ray through the equatorial plane: the
 * subring index n of an emission point is the number of them between it and the camera. */
static int polar_sign(const double* y, double r)
{
    double q = (y[1] * y[5] + y[2] * y[6]) * y[3] / r - (r - y[3] * y[3] / r) * y[7];
    double tol = 1e-9 * r;
    return q > tol ? 1 : (q < -tol ? -1 : 0);
}

/* Trace one ray backward from the camera.  out[] receives the planes of this ray. */
static void trace_one(const orc_job* job, const camera* cam, double al, double be, double* out,
                      orc_rayinfo* info, double* rec, int maxrec, int* nrec)
{
    double a = job->a, M = job->mass;
    int planes = orc_planes(job);
    double y[8], yn[8];
    camera_ray(job, cam, al, be, y);
    for (int p = 0; p < planes; ++p) out[p] = 0.0;
    double rin = M > 0 ? (1.0 + job->horizon_eps) * horizon_radius(a, M) : 0.0;
    double rout = job->escape_frac * job->r_obs;
    double r = creal(ks_radius(a, y[1], y[2], y[3]));
    double J0, A0, J1, A1;
    emission_unpol(job, y, &J0, &A0, NULL);
    double Iacc = 0.0, T = 1.0, lam_aff = 0.0;
    double min_r = r;
    int nturn = 0, steps = 0, status = ORC_RAY_CAP;
    int theta_sign = polar_sign(y, r);
    if (rec && maxrec > 0) {
        rec[0] = 0.0;
        for (int m = 0; m < 8; ++m) rec[1 + m] = y[m];
        rec[9] = 0.0;
        *nrec = 1;
    }
    while (steps < job->max_steps) {
        double h = job->step_frac * r;
        if (h < job->h_min) h = job->h_min;
        rk4_step(a, M, h, y, yn);
        ++steps;
        lam_aff += h;
        int finite = 1;
        for (int m = 0; m < 8; ++m) finite &= isfinite(yn[m]);
        if (!finite) { status = ORC_RAY_NAN; break; }
        double rn = creal(ks_radius(a, yn[1], yn[2], yn[3]));
        emission_unpol(job, yn, &J1, &A1, NULL);
        /* subring index of this segment: polar turning points before the segment starts */
        int seg_turn = nturn;
        int sg = polar_sign(yn, rn);
        if (sg != 0) {
            if (theta_sign != 0 && sg != theta_sign) ++nturn;
            theta_sign = sg;
        }
        /* trapezoid-averaged coefficients, exact constant-coefficient segment */
        double Jb = 0.5 * (J0 + J1), Ab = 0.5 * (A0 + A1);
        double dtau = Ab * h;
        double dI = T * Jb * h * phi1(dtau);
        Iacc += dI;
        if (job->subrings > 0) out[seg_turn < job->subrings ? seg_turn : job->subrings - 1] += dI;
        T *= exp(-dtau);
        memcpy(y, yn, sizeof y);
        J0 = J1;
        A0 = A1;
        r = rn;
        if (r < min_r) min_r = r;
        if (rec && *nrec < maxrec) {
            double* row = rec + 10 * (*nrec);
            row[0] = lam_aff;
            for (int m = 0; m < 8; ++m) row[1 + m] = y[m];
            row[9] = Iacc;
            ++(*nrec);
        }
        if (r < rin) { status = ORC_RAY_CAPTURED; break; }
        if (r > rout) { status = ORC_RAY_ESCAPED; break; }
    }
    if (job->subrings <= 0) out[0] = Iacc;
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
    if (job->stokes != 1) return -2;
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
static int estimate_point(const orc_job* job, const double* img, int nx, int ny, int i, int j,
                          int s, double norm, double* interp, double* ea, double* er)
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
        return (*ea > job->R_abs) && (*er > job->R_rel);
    }
    /* eps_abs = num / norm; eps_rel = num / |interpolant| (linear: (S_out-S_in)/(4 S_in)) */
    double den = (job->interp == ORC_INTERP_NEAREST) ? fabs(i1)
                 : (cat == 4 ? fabs(sin_) / 4.0 : fabs(sin_) / 2.0);
    *ea = num / norm;
    if (den == 0.0) *er = (num == 0.0) ? 0.0 : INFINITY;
    else *er = num / den;
    if (isnan(*ea) || isnan(*er) || isnan(*interp)) return 1;
    return (*ea > job->R_abs) && (*er > job->R_rel);
}

/* One refinement level (Sec. 3.2): every new point of level `level` reads only points of the
 * previous level; it is marked ORC_MASK_TRACED (to be traced by the caller) or receives its
 * interpolant and ORC_MASK_INTERP.  est_abs / est_rel (nullable) receive the estimates. */
int orc_refine_level(const orc_job* job, double* img, uint8_t* mask, int nx, int ny, int level,
                     double norm, double* est_abs, double* est_rel)
{
    if (level < 1 || level > job->levels) return -1;
    int s = 1 << (job->levels - level);
    for (int j = 0; j < ny; j += s)
        for (int i = 0; i < nx; i += s) {
            if (category(i, j, s) == 1) continue;
            double interp, ea, er;
            int tr = estimate_point(job, img, nx, ny, i, j, s, norm, &interp, &ea, &er);
            if (job->edge_mode == ORC_EDGE_TRACE) {
                int cat = category(i, j, s);
                int di = (cat == 2) ? 0 : s, dj = (cat == 3) ? 0 : s;
                if (i - 3 * di < 0 || i + 3 * di >= nx || j - 3 * dj < 0 || j + 3 * dj >= ny) tr = 1;
            }
            size_t p = (size_t)j * nx + i;
            if (est_abs) est_abs[p] = ea;
            if (est_rel) est_rel[p] = er;
            if (tr) {
                mask[p] = ORC_MASK_TRACED;
            } else {
                mask[p] = ORC_MASK_INTERP;
                img[p] = interp;
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
    if (job->stokes != 1 || job->subrings > 0) return -2;
    size_t npix = (size_t)nx * ny;
    memset(mask, 0, npix);
    for (size_t p = 0; p < npix; ++p) img[p] = 0.0;
    int64_t* list = malloc(sizeof(int64_t) * npix);
    double* vals = malloc(sizeof(double) * npix);
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
            for (int64_t q = 0; q < n; ++q) vals[q] = truth[list[q]];
        } else {
            rc = orc_trace_pixels(job, (int)n, list, vals, info);
            for (int64_t q = 0; q < n && rc == 0; ++q) st.steps += info[q].steps;
        }
        for (int64_t q = 0; q < n; ++q) {
            img[list[q]] = vals[q];
            mask[list[q]] = ORC_MASK_TRACED;
        }
        st.rays_traced += n;
        if (level < 16) st.rays_per_level[level] = n;
        if (level == 0) {
            if (job->abs_norm == ORC_NORM_PEAK) {
                st.ibar = -INFINITY;
                for (int64_t q = 0; q < n; ++q) st.ibar = fmax(st.ibar, vals[q]);
            } else {
                st.ibar = orc_ibar_int(img, nx, ny, S0);
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
