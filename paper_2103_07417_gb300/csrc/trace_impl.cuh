// trace_impl.cuh -- the fused ray tracer shared by the single-image and the batched kernels:
// camera ray set-up, RK4 null geodesic integration in outgoing Kerr-Schild coordinates and the
// covariant transfer step, with the whole ray state in registers.  The kernels built on it (trace.cu,
// trace_batch.cu) are persistent grids (SM count x resident blocks) that drain a device-side queue;
// each lane refills itself with the next ray as soon as its own ray terminates, so rays of very
// different path length (photon-ring rays take many more steps, Sec. 4.2) do not idle a warp.
//
// Transfer per RK4 step of length h (the intensity function I(x) of Sec. 3): the invariant
// emissivity J = j_nu/nu^2 is evaluated at the step's end point and averaged with the start
// point (trapezoid); absorption A likewise; the segment adds T J h (1 - e^{-A h})/(A h) and
// multiplies the transmission T by e^{-A h} (rays are traced from the camera outward, so T is
// the transmission between the camera and the segment).  Polarized rays solve the Stokes segment
// exactly (synch.cuh) with the parallel-transported basis.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "dfloat.cuh"
#include "internal.cuh"
#include "grid.cuh"
#include "synch.cuh"

namespace art {

// Arithmetic of the parts of a step outside the geodesic (radius for step size and stopping,
// emission, transfer, turn counting): the geodesic type itself, except for double-float
// geodesics, whose ray needs the extra precision only in its orbit.
template <class R>
struct Aux {
    using Q = R;
};
template <>
struct Aux<df> {
    using Q = float;
};

template <class Q, class R>
__device__ __forceinline__ RayState<Q> to_q(const RayState<R>& s)
{
    return RayState<Q>{Q(s.x), Q(s.y), Q(s.z), Q(s.kx), Q(s.ky), Q(s.kz)};
}

// --------------------------------------------------------------------------------------------
// camera
// --------------------------------------------------------------------------------------------

__device__ inline void ks_metric_cov(double a, const double x[3], double g[4][4])
{
    double r = ks_radius<double>(x[0], x[1], x[2], a * a);
    double r2 = r * r;
    double f = 2.0 * r2 * r / (r2 * r2 + a * a * x[2] * x[2]);
    double l[4] = {1.0, -(r * x[0] - a * x[1]) / (r2 + a * a), -(r * x[1] + a * x[0]) / (r2 + a * a),
                   -x[2] / r};
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n) g[m][n] = (m == n ? (m == 0 ? -1.0 : 1.0) : 0.0) + f * l[m] * l[n];
}

// Static observer at (r_obs, theta_o, phi = 0): x = sqrt(r^2 + a^2) sin(th), y = 0, z = r cos(th).
// Orthonormal tetrad by Gram-Schmidt in g from u = d_t / sqrt(-g_tt) and the coordinate vectors
// (sin th, 0, cos th) [outward], (-cos th, 0, sin th) [screen up, toward the spin axis],
// (0, 1, 0) [screen right]; stored lowered.
__device__ inline void camera_compute(double a, double r_obs, double incl_deg, Camera* cam)
{
    double th = incl_deg * 3.14159265358979323846 / 180.0;
    double sn, cs;
    sincos(th, &sn, &cs);
    double x0[3] = {sqrt(r_obs * r_obs + a * a) * sn, 0.0, r_obs * cs};
    double g[4][4];
    ks_metric_cov(a, x0, g);
    double e[4][4] = {{1.0 / sqrt(-g[0][0]), 0, 0, 0},
                      {0, sn, 0, cs},
                      {0, -cs, 0, sn},
                      {0, 0, 1, 0}};
    auto dot = [&](const double* u, const double* v) {
        double s = 0;
        for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n) s += g[m][n] * u[m] * v[n];
        return s;
    };
    for (int q = 1; q < 4; ++q) {
        double w[4], v[4];
        for (int m = 0; m < 4; ++m) v[m] = w[m] = e[q][m];
        double pu = dot(e[0], v);
        for (int m = 0; m < 4; ++m) w[m] += pu * e[0][m];
        for (int p = 1; p < q; ++p) {
            double pe = dot(e[p], v);
            for (int m = 0; m < 4; ++m) w[m] -= pe * e[p][m];
        }
        double nn = sqrt(dot(w, w));
        for (int m = 0; m < 4; ++m) e[q][m] = w[m] / nn;
    }
    for (int m = 0; m < 3; ++m) cam->x0[m] = x0[m];
    for (int q = 0; q < 4; ++q)
        for (int m = 0; m < 4; ++m) {
            double s = 0;
            for (int n = 0; n < 4; ++n) s += g[m][n] * e[q][n];
            cam->E[q][m] = s;
        }
}

// --------------------------------------------------------------------------------------------
// tracing
// --------------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long warp_fetch(unsigned long long* counter)
{
    unsigned m = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    return base + __popc(m & ((1u << lane) - 1u));
}

constexpr int MAXPL = 16;        // planes per ray: 4 Stokes x 4 subrings
constexpr int RAY_REROUTE = 16;  // internal status: handed to the high-precision pass

template <class R>
struct Tracer {
    using Q = typename Aux<R>::Q;
    RayState<R> s;
    R kt;
    Q r, T, sweep;
    Q J0[4], K0[7];   // coefficients at the start of the current step
    Q f[4];           // polarized rays: parallel-transported reference covector
    Q P[16];          // polarized rays: accumulated Stokes propagator (camera <- here)
    Q acc[MAXPL];     // accumulated planes
    float min_r;
    int steps, nturn, tsign, status, crossed;
    int32_t pix, img;
    int64_t slot;  // queue position
};

template <class R>
__device__ __forceinline__ R phi1(R x)
{
    return x > R(1e-8) ? -expm1(-x) / x : R(1) - R(0.5) * x;
}

// Emission models as a compile-time choice of the trace kernels: the analytic models (selected at
// run time by the job) or the fluid grid, whose lookup is kept out of the other kernels' code.
enum EmitKernel { EM_ANALYTIC = 0, EM_GRID = 1 };

// Emission/absorption/rotation coefficients at a point (J4, K7 as in synch.cuh).
template <class Q, bool POL, int EM>
__device__ __forceinline__ void coefficients(const RayState<Q>& q, Q r, Q kt, const Q* f,
                                             const DevJob& J, const SynchConst& S, Q* J4, Q* K7)
{
    if (EM == EM_GRID) {
        emission_grid<Q>(q, r, kt, POL ? f : nullptr, J, S, J4, K7);
        return;
    }
    if (J.emission == ART_EMIT_SYNCH_DISK) {
        emission_synch<Q>(q, r, kt, POL ? f : nullptr, J, S, J4, K7);
        return;
    }
    for (int i = 1; i < 4; ++i) J4[i] = Q(0);
    for (int i = 0; i < 7; ++i) K7[i] = Q(0);
    J4[0] = emission_cfg0<Q>(q, r, kt, J);
}

template <class R, bool POL, int EM>
__device__ __forceinline__ void ray_init(Tracer<R>& t, const DevJob& J, const SynchConst& S,
                                         const Camera& cam, int32_t pix)
{
    using Q = typename Aux<R>::Q;
    int i = pix % J.nx, j = pix / J.nx;
    double al = (i - 0.5 * (J.nx - 1)) * J.pix;
    double be = (j - 0.5 * (J.ny - 1)) * J.pix;
    double ro = J.r_obs;
    double sc = 1.0 / sqrt(1.0 + (al * al + be * be) / (ro * ro));
    double k[4];
    for (int m = 0; m < 4; ++m)
        k[m] = -cam.E[0][m] + sc * (-cam.E[1][m] + (al / ro) * cam.E[3][m] + (be / ro) * cam.E[2][m]);
    t.s.x = R(cam.x0[0]);
    t.s.y = R(cam.x0[1]);
    t.s.z = R(cam.x0[2]);
    t.kt = R(k[0]);
    t.s.kx = R(k[1]);
    t.s.ky = R(k[2]);
    t.s.kz = R(k[3]);
    if (POL) {
        // screen-up vector made normal to the line of sight n: e2 - (e2.n) n, e2.n = sc be/ro
        double c = sc * be / ro, nrm = 1.0 / sqrt(1.0 - c * c);
        for (int m = 0; m < 4; ++m) {
            double n = sc * (-cam.E[1][m] + (al / ro) * cam.E[3][m] + (be / ro) * cam.E[2][m]);
            t.f[m] = Q((cam.E[2][m] - c * n) * nrm);
        }
        for (int m = 0; m < 16; ++m) t.P[m] = (m % 5 == 0) ? Q(1) : Q(0);
    }
    RayState<Q> q = to_q<Q>(t.s);
    t.r = ks_radius<Q>(q.x, q.y, q.z, Q(J.a2));
    coefficients<Q, POL, EM>(q, t.r, Q(t.kt), t.f, J, S, t.J0, t.K0);
    t.T = Q(1);
    for (int p = 0; p < MAXPL; ++p) t.acc[p] = Q(0);
    t.min_r = float(t.r);
    t.sweep = Q(0);
    t.steps = 0;
    t.nturn = 0;
    t.crossed = 0;
    t.tsign = polar_sign<Q>(q, t.r);
    t.status = ART_RAY_CAP;
    t.pix = pix;
}

// One RK4 step plus the transfer segment; returns true when the ray has terminated.  SWEEP
// accumulates the angle swept by the position vector (used to route rays in mixed precision);
// POL carries the polarization covector through the RK4 stages and solves the Stokes segment.
template <class R, bool SWEEP, bool POL, int EM>
__device__ __forceinline__ bool ray_step(Tracer<R>& t, const DevJob& J, const SynchConst& S)
{
    using Q = typename Aux<R>::Q;
    const R a = R(J.a), a2 = R(J.a2);
    const Q aq = Q(J.a), a2q = Q(J.a2);
    Q hq = Q(J.step_frac) * t.r;
    if (hq < Q(J.h_min)) hq = Q(J.h_min);
    const R h = R(hq);
    const R hh = R(0.5) * h;
    const Q hhq = Q(0.5) * hq;
    RayState<R> k1, k2, k3, k4, y;
    Q d1[4], d2[4], d3[4], d4[4], fy[4];
    geodesic_rhs<R>(t.s, t.kt, a, a2, k1);
    if (POL) transport_rhs<Q>(to_q<Q>(t.s), Q(t.kt), t.f, aq, a2q, d1);
    y.x = t.s.x + hh * k1.x; y.y = t.s.y + hh * k1.y; y.z = t.s.z + hh * k1.z;
    y.kx = t.s.kx + hh * k1.kx; y.ky = t.s.ky + hh * k1.ky; y.kz = t.s.kz + hh * k1.kz;
    geodesic_rhs<R>(y, t.kt, a, a2, k2);
    if (POL) {
        for (int m = 0; m < 4; ++m) fy[m] = t.f[m] + hhq * d1[m];
        transport_rhs<Q>(to_q<Q>(y), Q(t.kt), fy, aq, a2q, d2);
    }
    y.x = t.s.x + hh * k2.x; y.y = t.s.y + hh * k2.y; y.z = t.s.z + hh * k2.z;
    y.kx = t.s.kx + hh * k2.kx; y.ky = t.s.ky + hh * k2.ky; y.kz = t.s.kz + hh * k2.kz;
    geodesic_rhs<R>(y, t.kt, a, a2, k3);
    if (POL) {
        for (int m = 0; m < 4; ++m) fy[m] = t.f[m] + hhq * d2[m];
        transport_rhs<Q>(to_q<Q>(y), Q(t.kt), fy, aq, a2q, d3);
    }
    y.x = t.s.x + h * k3.x; y.y = t.s.y + h * k3.y; y.z = t.s.z + h * k3.z;
    y.kx = t.s.kx + h * k3.kx; y.ky = t.s.ky + h * k3.ky; y.kz = t.s.kz + h * k3.kz;
    geodesic_rhs<R>(y, t.kt, a, a2, k4);
    if (POL) {
        for (int m = 0; m < 4; ++m) fy[m] = t.f[m] + hq * d3[m];
        transport_rhs<Q>(to_q<Q>(y), Q(t.kt), fy, aq, a2q, d4);
    }
    const R h6 = h / R(6);
    const Q ox = Q(t.s.x), oy = Q(t.s.y), oz = Q(t.s.z);
    t.s.x += h6 * (k1.x + R(2) * k2.x + R(2) * k3.x + k4.x);
    t.s.y += h6 * (k1.y + R(2) * k2.y + R(2) * k3.y + k4.y);
    t.s.z += h6 * (k1.z + R(2) * k2.z + R(2) * k3.z + k4.z);
    t.s.kx += h6 * (k1.kx + R(2) * k2.kx + R(2) * k3.kx + k4.kx);
    t.s.ky += h6 * (k1.ky + R(2) * k2.ky + R(2) * k3.ky + k4.ky);
    t.s.kz += h6 * (k1.kz + R(2) * k2.kz + R(2) * k3.kz + k4.kz);
    if (POL) {
        const Q h6q = hq / Q(6);
        for (int m = 0; m < 4; ++m) t.f[m] += h6q * (d1[m] + Q(2) * d2[m] + Q(2) * d3[m] + d4[m]);
    }
    ++t.steps;
    if (!(isfinite(t.s.x) && isfinite(t.s.y) && isfinite(t.s.z) && isfinite(t.s.kx) &&
          isfinite(t.s.ky) && isfinite(t.s.kz))) {
        t.status = ART_RAY_NAN;
        return true;
    }
    const RayState<Q> q = to_q<Q>(t.s);
    if (SWEEP) {
        // |x_old x x_new| / (|x_old| |x_new|): the sine of the angle the position vector turns
        Q cx = oy * q.z - oz * q.y, cy = oz * q.x - ox * q.z, cz = ox * q.y - oy * q.x;
        Q n2 = (ox * ox + oy * oy + oz * oz) * (q.x * q.x + q.y * q.y + q.z * q.z);
        t.sweep += sqrt((cx * cx + cy * cy + cz * cz) / n2);
        // a near-critical ray is re-traced at high precision anyway: stop it as soon as it is
        // known to be one (these orbiting rays are also the longest of the FP32 pass)
        if (t.sweep >= Q(J.fp64_sweep)) {
            t.status = RAY_REROUTE;
            return true;
        }
    }
    Q rn = ks_radius<Q>(q.x, q.y, q.z, a2q);
    Q J1[4], K1[7];
    coefficients<Q, POL, EM>(q, rn, Q(t.kt), t.f, J, S, J1, K1);
    // subring index: polar turning points counted from the first equatorial crossing on
    int seg = t.nturn;
    if (oz * q.z < Q(0)) t.crossed = 1;
    int sg = polar_sign<Q>(q, rn);
    if (sg != 0) {
        if (t.crossed && t.tsign != 0 && sg != t.tsign) ++t.nturn;
        t.tsign = sg;
    }
    const int sub = J.subrings > 0 ? (seg < J.subrings ? seg : J.subrings - 1) : 0;
    if (POL) {
        Q Jb[4], Kb[7];
        bool active = false;
        for (int i = 0; i < 4; ++i) {
            Jb[i] = Q(0.5) * (t.J0[i] + J1[i]);
            active |= Jb[i] != Q(0);
        }
        for (int i = 0; i < 7; ++i) {
            Kb[i] = Q(0.5) * (t.K0[i] + K1[i]);
            active |= Kb[i] != Q(0);
        }
        if (active) {
            Q add[4] = {Q(0), Q(0), Q(0), Q(0)};
            segment_pol<Q>(Kb, Jb, hq, t.P, add);
#pragma unroll
            for (int c = 0; c < MAXPL; ++c)
                if ((c >> 2) == sub) t.acc[c] += add[c & 3];
        }
    } else {
        Q Jb = Q(0.5) * (t.J0[0] + J1[0]), Ab = Q(0.5) * (t.K0[0] + K1[0]);
        Q dtau = Ab * hq;
        Q dI = t.T * Jb * hq * phi1<Q>(dtau);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c == sub) t.acc[c] += dI;
        if (Ab != Q(0)) t.T *= exp(-dtau);
    }
    for (int i = 0; i < 4; ++i) t.J0[i] = J1[i];
    for (int i = 0; i < 7; ++i) t.K0[i] = K1[i];
    t.r = rn;
    if (float(rn) < t.min_r) t.min_r = float(rn);
    if (rn < Q(J.r_in_stop)) { t.status = ART_RAY_CAPTURED; return true; }
    if (rn > Q(J.r_out_stop)) { t.status = ART_RAY_ESCAPED; return true; }
    if (t.steps >= J.max_steps) { t.status = ART_RAY_CAP; return true; }
    return false;
}

}  // namespace art
