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
#include <type_traits>

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

// A job constant in the geodesic's arithmetic R (double-float: the float copy and its low part).
template <class R>
__device__ __forceinline__ R jr(double d, float f, float) { return jq<R>(d, f); }
template <>
__device__ __forceinline__ df jr<df>(double, float f, float lo) { return df(f, lo); }

// The synchrotron constants of the arithmetic Q: the double originals or their float copy.
template <class Q>
__device__ __forceinline__ const SynchConstT<Q>& synch_of(const SynchConst& d, const SynchConstF& f);
template <>
__device__ __forceinline__ const SynchConst& synch_of<double>(const SynchConst& d, const SynchConstF&)
{
    return d;
}
template <>
__device__ __forceinline__ const SynchConstF& synch_of<float>(const SynchConst&, const SynchConstF& f)
{
    return f;
}

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
constexpr int RAY_GOING = -1;    // internal status: the ray continues

// A ray's state is kept in two parts, so that the geodesic and the transfer can run on different
// warps (trace_kernels.cuh): the geodesic part (position, momentum, transported covector, step
// count, swept angle) and the transfer part (coefficients at the current point, accumulated
// propagator and planes, turn counting).  The one-thread kernels hold both in one thread.
template <class R>
struct GeoState {
    using Q = typename Aux<R>::Q;
    RayState<R> s;
    RayState<R> k1;  // the geodesic right-hand side at s (CarryRhs kernels)
    R kt;
    Q r, sweep;
    Q f[4];  // polarized rays: parallel-transported reference covector
    int steps;
};

// Where the polarization covector's transport runs: with the geodesic, except for double-float
// geodesics, whose step is the longer half; there the geodesic half records the intermediate RK4
// states and the transfer half transports the covector along them.
template <class R, bool POL>
struct XportOnGeo {
    static constexpr bool value = !(std::is_same<R, df>::value && POL);
};
constexpr int NSTG = 18;  // the intermediate RK4 states of one step: 3 x (x y z kx ky kz)

template <class Q>
struct XferState {
    Q f[4];          // covector, when the transfer half transports it
    RayState<Q> y0;  // start of the current step, for that transport
    Q J0[4], K0[7];  // coefficients at the start of the current step
    Q P[16];         // polarized rays: accumulated Stokes propagator (camera <- here)
    Q acc[MAXPL];    // accumulated planes
    Q T, oz;         // transmission (unpolarized); z of the current point
    float min_r;
    int nturn, tsign, crossed;
    int edge;  // a sample lay near a discontinuity of the emission model (coefficients())
};

// The end point of a geodesic step as the transfer part needs it.
template <class Q>
struct StepPoint {
    RayState<Q> q;
    Q kt, r, h;
    Q f[4];
    Q ks[5];  // CarryRhs kernels: 1/r, F, Lx, Ly, Lz at the point (geodesic_rhs)
};

template <class R>
struct Tracer {
    using Q = typename Aux<R>::Q;
    GeoState<R> g;
    XferState<Q> x;
    int status;
    int32_t pix, img;
    int64_t slot;  // queue position
};

// A float that is zero or normal (a radius) in the arithmetic Q (FP64: widened on the integer
// units, grid.cuh).
template <class Q>
__device__ __forceinline__ Q from_float(float v)
{
    if constexpr (std::is_same<Q, double>::value)
        return widen(v);
    else
        return Q(v);
}

// Emission models as a compile-time choice of the trace kernels: the analytic models (selected at
// run time by the job) or the fluid grid, whose lookup is kept out of the other kernels' code.
enum EmitKernel { EM_ANALYTIC = 0, EM_GRID = 1 };

// Kernels whose step runs its four RK4 stages as one rolled loop (the double-float and the
// polarized analytic-emission kernels: see geo_step) hold the geodesic right-hand side once in
// their code.  The others evaluate the right-hand side at the end point of each step, where it is
// both the next step's first stage and the source of the end point's radius (no separate solve of
// the radius quadratic).
template <class R, bool POL, int EM>
struct CarryRhs {
    static constexpr bool value = !((POL && EM == EM_ANALYTIC) || std::is_same<R, df>::value);
};

// Emission/absorption/rotation coefficients at a point (J4, K7 as in synch.cuh).
// edge: set to 1 when the point lies within the FP32 pass's tolerance of a discontinuity of the
// emission model (left unchanged otherwise).  KS: the point carries its Kerr-Schild pieces
// (StepPoint::ks, from the geodesic's right-hand side there), which the grid model then reuses.
template <class Q, bool POL, int EM, bool KS>
__device__ __forceinline__ void coefficients(const StepPoint<Q>& pt, const DevJob& J,
                                             const SynchConstT<Q>& S, Q* J4, Q* K7, int& edge)
{
    const RayState<Q>& q = pt.q;
    const Q r = pt.r, kt = pt.kt;
    const Q* f = pt.f;
    if (EM == EM_GRID) {
        emission_grid<Q>(q, r, kt, POL ? f : nullptr, KS ? pt.ks : nullptr, J, S, J4, K7, &edge);
        return;
    }
    if (J.emission == ART_EMIT_SYNCH_DISK) {
        emission_synch<Q>(q, r, kt, POL ? f : nullptr, J, S, J4, K7, &edge);
        return;
    }
    for (int i = 1; i < 4; ++i) J4[i] = Q(0);
    for (int i = 0; i < 7; ++i) K7[i] = Q(0);
    J4[0] = emission_analytic<Q>(q, r, kt, J);
}

// Geodesic part of a ray's start: camera ray of pixel pix; fills the start point for the transfer
// part's initialisation.
template <class R, bool POL, int EM>
__device__ __forceinline__ void geo_init(GeoState<R>& g, const DevJob& J, const Camera& cam,
                                         int32_t pix, StepPoint<typename Aux<R>::Q>& pt)
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
    g.s.x = R(cam.x0[0]);
    g.s.y = R(cam.x0[1]);
    g.s.z = R(cam.x0[2]);
    g.kt = R(k[0]);
    g.s.kx = R(k[1]);
    g.s.ky = R(k[2]);
    g.s.kz = R(k[3]);
    if (POL) {
        // screen-up vector made normal to the line of sight n: e2 - (e2.n) n, e2.n = sc be/ro
        double c = sc * be / ro, nrm = 1.0 / sqrt(1.0 - c * c);
        for (int m = 0; m < 4; ++m) {
            double n = sc * (-cam.E[1][m] + (al / ro) * cam.E[3][m] + (be / ro) * cam.E[2][m]);
            g.f[m] = Q((cam.E[2][m] - c * n) * nrm);
        }
    }
    pt.q = to_q<Q>(g.s);
    if constexpr (CarryRhs<R, POL, EM>::value) {
        R kr[5];
        g.r = Q(geodesic_rhs<R>(g.s, g.kt, jr<R>(J.a, J.f_a, J.f_a_lo),
                                jr<R>(J.a2, J.f_a2, J.f_a2_lo), g.k1, kr));
        for (int m = 0; m < 5; ++m) pt.ks[m] = Q(kr[m]);
    } else
        g.r = ks_radius<Q>(pt.q.x, pt.q.y, pt.q.z, jq<Q>(J.a2, J.f_a2));
    g.sweep = Q(0);
    g.steps = 0;
    pt.kt = Q(g.kt);
    pt.r = g.r;
    pt.h = Q(0);
    if (POL)
        for (int m = 0; m < 4; ++m) pt.f[m] = g.f[m];
}

// Transfer part of a ray's start, given the coefficients J1, K1 at the camera point: identity
// propagator, empty planes, turn counting from there.
template <class Q, bool POL>
__device__ __forceinline__ void xfer_init_with(XferState<Q>& x, const StepPoint<Q>& pt,
                                               const Q* J1, const Q* K1, int e1)
{
    x.edge = e1;
    for (int i = 0; i < 4; ++i) x.J0[i] = J1[i];
    for (int i = 0; i < 7; ++i) x.K0[i] = K1[i];
    if (POL)
        for (int m = 0; m < 16; ++m) x.P[m] = (m % 5 == 0) ? Q(1) : Q(0);
    x.T = Q(1);
    for (int p = 0; p < MAXPL; ++p) x.acc[p] = Q(0);
    x.min_r = float(pt.r);
    x.nturn = 0;
    x.crossed = 0;
    x.tsign = polar_sign<Q>(pt.q, pt.r);
    x.oz = pt.q.z;
    if (POL)
        for (int m = 0; m < 4; ++m) x.f[m] = pt.f[m];
    x.y0 = pt.q;
}

// Transfer part of a ray's start: coefficients at the camera point, identity propagator.
template <class Q, bool POL, int EM, bool KS>
__device__ __forceinline__ void xfer_init(XferState<Q>& x, const StepPoint<Q>& pt, const DevJob& J,
                                          const SynchConstT<Q>& S)
{
    Q J1[4], K1[7];
    int e1 = 0;
    coefficients<Q, POL, EM, KS>(pt, J, S, J1, K1, e1);
    xfer_init_with<Q, POL>(x, pt, J1, K1, e1);
}

template <class R, bool POL, int EM>
__device__ __forceinline__ void ray_init(Tracer<R>& t, const DevJob& J,
                                         const SynchConstT<typename Aux<R>::Q>& S,
                                         const Camera& cam, int32_t pix)
{
    StepPoint<typename Aux<R>::Q> pt;
    geo_init<R, POL, EM>(t.g, J, cam, pix, pt);
    xfer_init<typename Aux<R>::Q, POL, EM, CarryRhs<R, POL, EM>::value>(t.x, pt, J, S);
    t.status = ART_RAY_CAP;
    t.pix = pix;
}

// y = s + c k (the state of an intermediate RK4 stage)
template <class R>
__device__ __forceinline__ void rk4_offset(const RayState<R>& s, R c, const RayState<R>& k,
                                           RayState<R>& y)
{
    y.x = fmad(c, k.x, s.x);
    y.y = fmad(c, k.y, s.y);
    y.z = fmad(c, k.z, s.z);
    y.kx = fmad(c, k.kx, s.kx);
    y.ky = fmad(c, k.ky, s.ky);
    y.kz = fmad(c, k.kz, s.kz);
}

// Geodesic part of one step: RK4 of (x, k) (and of the covector f for polarized rays), the
// non-finite and swept-angle tests, the end point's radius and the stopping tests.  Returns
// RAY_GOING, or the ray's final status: ART_RAY_NAN and RAY_REROUTE end the ray before the
// segment, the other statuses after it.  SWEEP accumulates the angle swept by the position vector
// (used to route rays in mixed precision).
// Stage states are stored at stg[(3 stage + component) * sstride] when the transport runs on the
// transfer half.
template <class R, bool SWEEP, bool POL, int EM>
__device__ __forceinline__ int geo_step(GeoState<R>& t, const DevJob& J,
                                        StepPoint<typename Aux<R>::Q>& pt,
                                        typename Aux<R>::Q* stg, int sstride)
{
    using Q = typename Aux<R>::Q;
    const R a = jr<R>(J.a, J.f_a, J.f_a_lo), a2 = jr<R>(J.a2, J.f_a2, J.f_a2_lo);
    const Q aq = jq<Q>(J.a, J.f_a), a2q = jq<Q>(J.a2, J.f_a2);
    const Q hmin = jq<Q>(J.h_min, J.f_h_min);
    Q hq = jq<Q>(J.step_frac, J.f_step_frac) * t.r;
    if (hq < hmin) hq = hmin;
    const R h = R(hq);
    const R hh = scale2(h, 0.5f);
    const Q hhq = Q(0.5) * hq;
    // ks = k1 + 2 k2 + 2 k3 + k4 (summed in that order) and likewise ds for the polarization.
    // The double-float and the polarized analytic-emission kernels run the four stages as one
    // rolled loop, so the geodesic (and transport) right-hand sides appear once in their code: the
    // trace kernels are latency-bound with few warps per SM, and their fully unrolled step no
    // longer fits the instruction cache (measured: the double-float pass of the polarized disk
    // 2.3x faster).  The other kernels keep the unrolled stages, which measured faster for them.
    constexpr bool ROLLED = (POL && EM == EM_ANALYTIC) || std::is_same<R, df>::value;
    constexpr bool XP = XportOnGeo<R, POL>::value;
    RayState<R> ks;
    Q ds[4];
    if (!XP) {
        // geodesic only, recording the stage states; rolled for the same reason
        RayState<R> k, y = t.s;
#pragma unroll(ROLLED ? 1 : 4)
        for (int st = 0; st < 4; ++st) {
            geodesic_rhs<R>(y, t.kt, a, a2, k);
            if (st == 0) {
                ks = k;
            } else if (st < 3) {
                ks.x = twice_plus(k.x, ks.x); ks.y = twice_plus(k.y, ks.y);
                ks.z = twice_plus(k.z, ks.z); ks.kx = twice_plus(k.kx, ks.kx);
                ks.ky = twice_plus(k.ky, ks.ky); ks.kz = twice_plus(k.kz, ks.kz);
            } else {
                ks.x = ks.x + k.x; ks.y = ks.y + k.y; ks.z = ks.z + k.z;
                ks.kx = ks.kx + k.kx; ks.ky = ks.ky + k.ky; ks.kz = ks.kz + k.kz;
                break;
            }
            rk4_offset(t.s, st < 2 ? hh : h, k, y);
            const RayState<Q> yq = to_q<Q>(y);
            Q* o = stg + 6 * st * sstride;
            o[0] = yq.x;
            o[sstride] = yq.y;
            o[2 * sstride] = yq.z;
            o[3 * sstride] = yq.kx;
            o[4 * sstride] = yq.ky;
            o[5 * sstride] = yq.kz;
        }
    } else if (ROLLED) {
        RayState<R> k, y = t.s;
        Q d[4], fy[4];
        for (int m = 0; m < 4; ++m) fy[m] = t.f[m];
#pragma unroll 1
        for (int st = 0; st < 4; ++st) {
            geodesic_rhs<R>(y, t.kt, a, a2, k);
            if (POL) transport_rhs<Q>(to_q<Q>(y), Q(t.kt), fy, aq, a2q, d);
            if (st == 0) {
                ks = k;
                if (POL)
                    for (int m = 0; m < 4; ++m) ds[m] = d[m];
            } else if (st < 3) {
                ks.x = twice_plus(k.x, ks.x); ks.y = twice_plus(k.y, ks.y);
                ks.z = twice_plus(k.z, ks.z); ks.kx = twice_plus(k.kx, ks.kx);
                ks.ky = twice_plus(k.ky, ks.ky); ks.kz = twice_plus(k.kz, ks.kz);
                if (POL)
                    for (int m = 0; m < 4; ++m) ds[m] = fmad(Q(2), d[m], ds[m]);
            } else {
                ks.x = ks.x + k.x; ks.y = ks.y + k.y; ks.z = ks.z + k.z;
                ks.kx = ks.kx + k.kx; ks.ky = ks.ky + k.ky; ks.kz = ks.kz + k.kz;
                if (POL)
                    for (int m = 0; m < 4; ++m) ds[m] = ds[m] + d[m];
                break;
            }
            const R c = st < 2 ? hh : h;  // offset of the next stage
            const Q cq = st < 2 ? hhq : hq;
            rk4_offset(t.s, c, k, y);
            if (POL)
                for (int m = 0; m < 4; ++m) fy[m] = fmad(cq, d[m], t.f[m]);
        }
    } else {
        RayState<R> k1, k2, k3, k4, y;
        Q d1[4], d2[4], d3[4], d4[4], fy[4];
        if constexpr (CarryRhs<R, POL, EM>::value)
            k1 = t.k1;  // evaluated at the end of the previous step (or by geo_init)
        else
            geodesic_rhs<R>(t.s, t.kt, a, a2, k1);
        if (POL) transport_rhs<Q>(to_q<Q>(t.s), Q(t.kt), t.f, aq, a2q, d1);
        rk4_offset(t.s, hh, k1, y);
        geodesic_rhs<R>(y, t.kt, a, a2, k2);
        if (POL) {
            for (int m = 0; m < 4; ++m) fy[m] = fmad(hhq, d1[m], t.f[m]);
            transport_rhs<Q>(to_q<Q>(y), Q(t.kt), fy, aq, a2q, d2);
        }
        rk4_offset(t.s, hh, k2, y);
        geodesic_rhs<R>(y, t.kt, a, a2, k3);
        if (POL) {
            for (int m = 0; m < 4; ++m) fy[m] = fmad(hhq, d2[m], t.f[m]);
            transport_rhs<Q>(to_q<Q>(y), Q(t.kt), fy, aq, a2q, d3);
        }
        rk4_offset(t.s, h, k3, y);
        geodesic_rhs<R>(y, t.kt, a, a2, k4);
        if (POL) {
            for (int m = 0; m < 4; ++m) fy[m] = fmad(hq, d3[m], t.f[m]);
            transport_rhs<Q>(to_q<Q>(y), Q(t.kt), fy, aq, a2q, d4);
        }
        ks.x = twice_plus(k3.x, twice_plus(k2.x, k1.x)) + k4.x;
        ks.y = twice_plus(k3.y, twice_plus(k2.y, k1.y)) + k4.y;
        ks.z = twice_plus(k3.z, twice_plus(k2.z, k1.z)) + k4.z;
        ks.kx = twice_plus(k3.kx, twice_plus(k2.kx, k1.kx)) + k4.kx;
        ks.ky = twice_plus(k3.ky, twice_plus(k2.ky, k1.ky)) + k4.ky;
        ks.kz = twice_plus(k3.kz, twice_plus(k2.kz, k1.kz)) + k4.kz;
        if (POL)
            for (int m = 0; m < 4; ++m)
                ds[m] = fmad(Q(2), d3[m], fmad(Q(2), d2[m], d1[m])) + d4[m];
    }
    R h6;
    if constexpr (std::is_same<R, double>::value)
        h6 = h * R(1.0 / 6.0);  // a multiply in place of the FP64 division
    else
        h6 = h / R(6);
    const Q ox = Q(t.s.x), oy = Q(t.s.y), oz = Q(t.s.z);
    t.s.x = fmad(h6, ks.x, t.s.x);
    t.s.y = fmad(h6, ks.y, t.s.y);
    t.s.z = fmad(h6, ks.z, t.s.z);
    t.s.kx = fmad(h6, ks.kx, t.s.kx);
    t.s.ky = fmad(h6, ks.ky, t.s.ky);
    t.s.kz = fmad(h6, ks.kz, t.s.kz);
    if (POL && XP) {
        const Q h6q = hq / Q(6);
        for (int m = 0; m < 4; ++m) t.f[m] = fmad(h6q, ds[m], t.f[m]);
    }
    ++t.steps;
    if (!(isfinite(t.s.x) && isfinite(t.s.y) && isfinite(t.s.z) && isfinite(t.s.kx) &&
          isfinite(t.s.ky) && isfinite(t.s.kz)))
        return ART_RAY_NAN;
    const RayState<Q> q = to_q<Q>(t.s);
    if (SWEEP) {
        // |x_old x x_new| / (|x_old| |x_new|): the sine of the angle the position vector turns
        Q cx = fmad(oy, q.z, -(oz * q.y)), cy = fmad(oz, q.x, -(ox * q.z));
        Q cz = fmad(ox, q.y, -(oy * q.x));
        Q n2 = fmad(oz, oz, fmad(oy, oy, ox * ox)) * fmad(q.z, q.z, fmad(q.y, q.y, q.x * q.x));
        t.sweep += sqrt(fmad(cz, cz, fmad(cy, cy, cx * cx)) / n2);
        // a near-critical ray is re-traced at high precision anyway: stop it as soon as it is
        // known to be one (these orbiting rays are also the longest of the FP32 pass)
        if (t.sweep >= jq<Q>(J.fp64_sweep, J.f_fp64_sweep)) return RAY_REROUTE;
    }
    Q rn;
    if constexpr (CarryRhs<R, POL, EM>::value) {
        R kr[5];
        rn = Q(geodesic_rhs<R>(t.s, t.kt, a, a2, t.k1, kr));
        for (int m = 0; m < 5; ++m) pt.ks[m] = Q(kr[m]);
    } else
        rn = ks_radius<Q>(q.x, q.y, q.z, a2q);
    t.r = rn;
    pt.q = q;
    pt.kt = Q(t.kt);
    pt.r = rn;
    pt.h = hq;
    if (POL && XP)
        for (int m = 0; m < 4; ++m) pt.f[m] = t.f[m];
    if (rn < jq<Q>(J.r_in_stop, J.f_r_in_stop)) return ART_RAY_CAPTURED;
    if (rn > jq<Q>(J.r_out_stop, J.f_r_out_stop)) return ART_RAY_ESCAPED;
    if (t.steps >= J.max_steps) return ART_RAY_CAP;
    return RAY_GOING;
}

// Transfer part of one step ending at pt, given the coefficients J1, K1 there: the subring index
// (polar turning points counted from the first equatorial crossing on) and the segment (trapezoid
// in J and A, or the exact Stokes segment of the averaged coefficients).
template <class Q, bool POL>
__device__ __forceinline__ void xfer_apply(XferState<Q>& t, const StepPoint<Q>& pt, const Q* J1,
                                           const Q* K1, const DevJob& J, int e1)
{
    t.edge |= e1;
    const RayState<Q>& q = pt.q;
    const Q rn = pt.r, hq = pt.h;
    int seg = t.nturn;
    if (t.oz * q.z < Q(0)) t.crossed = 1;
    int sg = polar_sign<Q>(q, rn);
    // subring planes: a turn counted differently in another precision moves emission between
    // planes; the mixed modes hand such rays on (FP32 -> double-float -> FP64)
    if (J.subrings > 0 && polar_marginal<Q>(q, rn)) t.edge = 1;
    if (sg != 0) {
        if (t.crossed && t.tsign != 0 && sg != t.tsign) ++t.nturn;
        t.tsign = sg;
    }
    t.oz = q.z;
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
        // slab of constant coefficients: dI = T J h (1 - e^-dtau)/dtau, T <- T e^-dtau, both from
        // one expm1 (e^-dtau = 1 + expm1(-dtau), accurate where 1 - e^-dtau would cancel)
        Q ph = Q(1) - Q(0.5) * dtau, em1 = Q(0);
        if (dtau > Q(1e-8)) {
            em1 = expm1(-dtau);
            ph = -em1 / dtau;
        } else if (Ab != Q(0)) {
            em1 = -dtau * ph;
        }
        Q dI = t.T * Jb * hq * ph;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c == sub) t.acc[c] += dI;
        if (Ab != Q(0)) t.T = fmad(t.T, em1, t.T);
    }
    for (int i = 0; i < 4; ++i) t.J0[i] = J1[i];
    for (int i = 0; i < 7; ++i) t.K0[i] = K1[i];
    // the smallest radius as a float: compared in Q, converted only when it changes (a float
    // rounds monotonically, so the result is the smallest float(r))
    if (rn < from_float<Q>(t.min_r)) t.min_r = float(rn);
}

// Transfer part of one step ending at pt: the coefficients there, then xfer_apply.
template <class Q, bool POL, int EM, bool KS>
__device__ __forceinline__ void xfer_step(XferState<Q>& t, const StepPoint<Q>& pt, const DevJob& J,
                                          const SynchConstT<Q>& S)
{
    Q J1[4], K1[7];
    int e1 = 0;
    coefficients<Q, POL, EM, KS>(pt, J, S, J1, K1, e1);
    xfer_apply<Q, POL>(t, pt, J1, K1, J, e1);
}

// The covector's RK4 step on the transfer half, along the stage states recorded by the geodesic
// half (stg as in geo_step); leaves the transported covector in pt.f and the step's end point as
// the next start.
template <class Q>
__device__ __forceinline__ void xfer_transport(XferState<Q>& x, StepPoint<Q>& pt, const Q* stg,
                                               int sstride, const DevJob& J)
{
    const Q aq = jq<Q>(J.a, J.f_a), a2q = jq<Q>(J.a2, J.f_a2), hq = pt.h, hhq = Q(0.5) * hq;
    Q d[4], ds[4], fy[4];
    RayState<Q> y = x.y0;
#pragma unroll 1
    for (int st = 0; st < 4; ++st) {
        transport_rhs<Q>(y, pt.kt, st == 0 ? x.f : fy, aq, a2q, d);
        if (st == 0) {
            for (int m = 0; m < 4; ++m) ds[m] = d[m];
        } else if (st < 3) {
            for (int m = 0; m < 4; ++m) ds[m] = fmad(Q(2), d[m], ds[m]);
        } else {
            for (int m = 0; m < 4; ++m) ds[m] = ds[m] + d[m];
            break;
        }
        const Q cq = st < 2 ? hhq : hq;
        for (int m = 0; m < 4; ++m) fy[m] = fmad(cq, d[m], x.f[m]);
        const Q* o = stg + 6 * st * sstride;
        y.x = o[0];
        y.y = o[sstride];
        y.z = o[2 * sstride];
        y.kx = o[3 * sstride];
        y.ky = o[4 * sstride];
        y.kz = o[5 * sstride];
    }
    const Q h6q = hq / Q(6);
    for (int m = 0; m < 4; ++m) {
        x.f[m] = fmad(h6q, ds[m], x.f[m]);
        pt.f[m] = x.f[m];
    }
    x.y0 = pt.q;
}

// One RK4 step plus the transfer segment in one thread; returns true when the ray has terminated.
template <class R, bool SWEEP, bool POL, int EM>
__device__ __forceinline__ bool ray_step(Tracer<R>& t, const DevJob& J,
                                         const SynchConstT<typename Aux<R>::Q>& S)
{
    using Q = typename Aux<R>::Q;
    StepPoint<Q> pt;
    Q stg[XportOnGeo<R, POL>::value ? 1 : NSTG];
    const int st = geo_step<R, SWEEP, POL, EM>(t.g, J, pt, stg, 1);
    if (st == ART_RAY_NAN || st == RAY_REROUTE) {
        t.status = st;
        return true;
    }
    if (!XportOnGeo<R, POL>::value) xfer_transport<Q>(t.x, pt, stg, 1, J);
    xfer_step<Q, POL, EM, CarryRhs<R, POL, EM>::value>(t.x, pt, J, S);
    if (st == RAY_GOING) return false;
    t.status = st;
    return true;
}

}  // namespace art
