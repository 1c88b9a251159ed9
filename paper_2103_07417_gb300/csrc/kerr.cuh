// kerr.cuh -- device geometry of the ray tracer: Kerr metric in outgoing Cartesian Kerr-Schild
// coordinates, Hamilton's equations for null geodesics, the static camera and the emission models.
//
// Metric (Kerr & Schild 1965, outgoing form): g^{mu nu} = eta^{mu nu} - f l^mu l^nu with
//   f = 2 r^3 / (r^4 + a^2 z^2),  l_mu = (1, -L_x, -L_y, -L_z),
//   L = ((r x - a y)/(r^2 + a^2), (r y + a x)/(r^2 + a^2), z/r),
//   r^4 - (x^2 + y^2 + z^2 - a^2) r^2 - a^2 z^2 = 0,   x + i y = (r - i a) sin(th) e^{i phi}.
// Rays are traced backward from the camera (past-directed); these coordinates keep them regular
// through the past horizon.  H = 1/2 g^{mu nu} k_mu k_nu does not depend on t, so k_t is exact
// and t is not integrated; the state is (x, y, z, k_x, k_y, k_z).
//
// The partial derivatives below are derived by hand from H (the CPU oracle takes them by complex
// steps instead).  With Lam = L.k, lk = l^mu k_mu = -k_t - Lam and
//   dr/dx_i = (x r, y r, z (r^2 + a^2)/r) / Sigma,   Sigma = r^2 + a^2 z^2 / r^2,
//   df/dx_i = B dr/dx_i - delta_iz 2 f a^2 z / Q,     B = (f/r)(3 - 4 r^4/Q),  Q = r^4 + a^2 z^2,
//   dLam/dx_i = A dr/dx_i + T_i,  A = (x k_x + y k_y - 2 r (L_x k_x + L_y k_y))/(r^2+a^2) - k_z z/r^2,
//   T = ((r k_x + a k_y)/(r^2+a^2), (r k_y - a k_x)/(r^2+a^2), k_z/r),
// Hamilton's equations read
//   dx_i/dlambda = k_i + f lk L_i,
//   dk_i/dlambda = (B lk^2/2 - f lk A) dr/dx_i - f lk T_i - delta_iz f a^2 z lk^2 / Q.
#pragma once
#include <cmath>
#include <cstdint>
#include <type_traits>

#if defined(__CUDACC__)
#define ART_HD __host__ __device__ __forceinline__
#else
#define ART_HD inline
#endif

namespace art {

#if !defined(__CUDACC__)
inline double rsqrt(double v) { return 1.0 / sqrt(v); }
inline float rsqrt(float v) { return 1.0f / sqrt(v); }
#endif

// Fused multiply-add a b + c, written out.  The trace kernels are compiled without automatic
// contraction, so that a step rounds the same way in every kernel that inlines it (the one-thread
// and the warp-pair forms give bit-identical rays); the fused operations are the ones written with
// fmad.  For double-float values it is a b + c in that arithmetic.
template <class R>
ART_HD R fmad(R a, R b, R c)
{
    return a * b + c;
}
template <>
ART_HD float fmad<float>(float a, float b, float c)
{
    return fmaf(a, b, c);
}
template <>
ART_HD double fmad<double>(double a, double b, double c)
{
    return fma(a, b, c);
}

// x c for a power of two c: exact in every arithmetic (a double-float scales both parts, which
// keeps them normalised, instead of a full double-float product).
template <class R>
ART_HD R scale2(R x, float c)
{
    return x * R(c);
}

#ifdef __CUDA_ARCH__
// FP64 on the device: the product with 2^k as integer arithmetic on the exponent field (GB300 issues
// an FP64 instruction per scheduler every 64 cycles, an integer one every cycle).  Equal to the
// product for every finite normal x whose product is normal; zeros, infinities and NaNs keep their
// exponent (only the sign follows c).  Subnormal inputs (not met by the tracer's values) would
// stay unscaled.
template <>
ART_HD double scale2<double>(double x, float c)
{
    const int cb = __float_as_int(c);
    const int k = ((cb >> 23) & 0xff) - 127;  // c = +-2^k, a compile-time constant at every use
    const int hi = __double2hiint(x);
    const int e = hi & 0x7ff00000;
    const int hs = (e != 0 && e != 0x7ff00000) ? hi + k * (1 << 20) : hi;
    return __hiloint2double(hs ^ (cb & (int)0x80000000), __double2loint(x));
}
#endif

// 2 x + c: one fused multiply-add (for double-float: the exact scaling above and one addition).
template <class R>
ART_HD R twice_plus(R x, R c)
{
    return fmad(R(2), x, c);
}

// Job parameters as the kernels see them (POD, passed by value).
struct DevJob {
    double a, a2, r_obs, pix, step_frac, h_min, r_in_stop, r_out_stop, inv_2w2;
    double R_abs, R_rel, fp64_sweep;
    int32_t nx, ny, levels, emission, flow, stokes, subrings, planes, max_steps;
    int32_t interp, edge_mode, abs_norm, precision, criterion, cplane;
    // float copies of the constants the per-step code reads, for the FP32 and double-float kernels
    // (a conversion from double runs on GB300's FP64 pipe, one warp instruction per 64 cycles on a
    // scheduler), with the low parts of a and a^2 for double-float geodesics
    float f_a, f_a2, f_a_lo, f_a2_lo, f_step_frac, f_h_min, f_r_in_stop, f_r_out_stop;
    float f_fp64_sweep, f_inv_2w2;
};

// A job constant in arithmetic T: the double itself, or its float copy.
template <class T>
ART_HD T jq(double d, float) { return T(d); }
template <>
ART_HD float jq<float>(double, float f) { return f; }

// Static camera: position and the covariant (lowered) tetrad E0 (observer), E1 (outward),
// E2 (screen up), E3 (screen right), so that k_mu = -E0 + s (-E1 + (al/r_obs) E3 + (be/r_obs) E2).
struct Camera {
    double x0[3];
    double E[4][4];  // E[a][mu]
};

template <class R>
struct RayState {
    R x, y, z, kx, ky, kz;
};

template <class R>
ART_HD R ks_radius(R x, R y, R z, R a2)
{
    R z2 = z * z;
    R b = (fmad(y, y, x * x) + z2) - a2;
    R r2 = scale2(b + sqrt(fmad(b, b, scale2(a2, 4.f) * z2)), 0.5f);
    return sqrt(r2);
}

// Hamilton's equations (see the header comment); returns r of the evaluation point.  ks
// (nullable) receives the Kerr-Schild pieces of the point the emission models use: 1/r,
// F = 2 r^3 / (r^4 + a^2 z^2) and L = (Lx, Ly, Lz).
template <class R>
ART_HD R geodesic_rhs(const RayState<R>& s, R kt, R a, R a2, RayState<R>& d, R* ks = nullptr)
{
    const R x = s.x, y = s.y, z = s.z, kx = s.kx, ky = s.ky, kz = s.kz;
    R z2 = z * z;
    R a2z2 = a2 * z2;
    R b = (fmad(y, y, x * x) + z2) - a2;
    R r2 = scale2(b + sqrt(fmad(b, b, scale2(a2z2, 4.f))), 0.5f);
    R r4 = r2 * r2;
    const R Qd = r4 + a2z2, ra2 = r2 + a2;
    R ir, r, iP;  // 1/r, r and 1/P with P = Q (r^2 + a^2)
    if constexpr (std::is_same<R, double>::value) {
        // all three from one reciprocal square root X = 1/(r P) (no division): 1/r = X P,
        // r = r^2 / r, 1/P = X r.  r^2 P^2 ~ r^14 stays finite for r <= 1e8 (the job's bound).
        const R P = Qd * ra2;
        const R X = rsqrt(r2 * P * P);
        ir = X * P;
        r = r2 * ir;
        iP = X * r;
    } else {
        // r^14 would leave the single-precision range: a reciprocal square root and a reciprocal
        ir = rsqrt(r2);
        r = r2 * ir;
        iP = R(1) / (Qd * ra2);
    }
    // 1/Q and 1/(r^2 + a^2) from the one reciprocal of their product
    R iQ = ra2 * iP;
    R u = r * iQ;
    R rs = r2 * u;            // r^3 / Q = r / Sigma, Sigma = r^2 + a^2 z^2 / r^2 = Q / r^2
    R f = scale2(rs, 2.f);    // 2 r^3 / Q
    R ira2 = Qd * iP;
    R Lx = fmad(r, x, -(a * y)) * ira2;
    R Ly = fmad(r, y, a * x) * ira2;
    R Lz = z * ir;
    R Lkxy = fmad(Ly, ky, Lx * kx);
    R lk = -kt - fmad(Lz, kz, Lkxy);
    // grad r = (x r / Sigma, y r / Sigma, z (r^2 + a^2) / (r Sigma))
    R drx = x * rs, dry = y * rs, drz = (z * ra2) * u;
    R B = f * ir * fmad(scale2(r4, -4.f), iQ, R(3));
    R Tz = kz * ir;
    R A = fmad(fmad(scale2(r, -2.f), Lkxy, fmad(y, ky, x * kx)), ira2, -(Lz * Tz));
    R flk = f * lk;
    R C = fmad(scale2(B, 0.5f) * lk, lk, -(flk * A));
    R Tx = fmad(r, kx, a * ky) * ira2;
    R Ty = fmad(r, ky, -(a * kx)) * ira2;
    d.kx = fmad(C, drx, -(flk * Tx));
    d.ky = fmad(C, dry, -(flk * Ty));
    d.kz = fmad(-(flk * lk), (a2 * z) * iQ, fmad(C, drz, -(flk * Tz)));
    d.x = fmad(flk, Lx, kx);
    d.y = fmad(flk, Ly, ky);
    d.z = fmad(flk, Lz, kz);
    if (ks) {
        ks[0] = ir;
        ks[1] = f;
        ks[2] = Lx;
        ks[3] = Ly;
        ks[4] = Lz;
    }
    return r;
}

// Invariant emissivity J = j_nu / nu^2 of the analytic model j = r^-2 exp(-z^2 / (2 (w r)^2))
// (z = r cos(theta)) for a fluid that is Keplerian (Omega = 1/(r^{3/2} + a) at Boyer-Lindquist
// (r, theta), zero where no timelike such orbit exists) or static; nu = k_mu u^mu.
template <class R>
ART_HD R emission_analytic(const RayState<R>& s, R r, R kt, const DevJob& J)
{
    if (r < jq<R>(J.r_in_stop, J.f_r_in_stop)) return R(0);
    R ct = s.z / r;
    R ct2 = ct * ct;
    R r2 = r * r;
    R jnu = exp(-ct2 * jq<R>(J.inv_2w2, J.f_inv_2w2)) / r2;
    R a = jq<R>(J.a, J.f_a), a2 = jq<R>(J.a2, J.f_a2);
    R nu;
    if (J.flow == 0) {
        R st2 = R(1) - ct2;
        R iSig = R(1) / (r2 + a2 * ct2);
        R gtt = -(R(1) - R(2) * r * iSig);
        R gtp = -R(2) * a * r * st2 * iSig;
        R gpp = fmad(R(2) * a2 * r * st2, iSig, r2 + a2) * st2;
        R Om = R(1) / fmad(r, sqrt(r), a);
        R nrm = -fmad(Om * Om, gpp, fmad(R(2) * Om, gtp, gtt));
        if (!(nrm > R(0))) return R(0);
        R ut = R(1) / sqrt(nrm);
        nu = ut * fmad(Om, fmad(s.x, s.ky, -(s.y * s.kx)), kt);
    } else {
        R z2 = s.z * s.z;
        R f = R(2) * r2 * r / fmad(r2, r2, a2 * z2);
        if (!(f < R(1))) return R(0);
        nu = kt / sqrt(R(1) - f);
    }
    if (!(nu > R(0))) return R(0);
    return jnu / (nu * nu);
}

// Sign of d(theta)/d(lambda) from k_theta sin(theta) = (x k_x + y k_y) z/r - (r - z^2/r) k_z,
// 0 inside a dead band of 1e-9 r (1e-5 r in FP32) so radial rays count no turns.
template <class R>
ART_HD R polar_q(const RayState<R>& s, R r)
{
    return fmad(s.y, s.ky, s.x * s.kx) * s.z / r - (r - s.z * s.z / r) * s.kz;
}

template <class R>
ART_HD int polar_sign(const RayState<R>& s, R r)
{
    R q = polar_q<R>(s, r);
    R tol = R(sizeof(R) == 4 ? 1e-5 : 1e-9) * r;  // dead band above the rounding noise
    return q > tol ? 1 : (q < -tol ? -1 : 0);
}

// A sample whose turning-point quantity lies between the FP64 and the FP32 dead bands (x 10):
// the two precisions may count that turn differently, which moves emission between subrings.
template <class R>
ART_HD bool polar_marginal(const RayState<R>& s, R r)
{
    const R q = polar_q<R>(s, r);
    return fabs(q) < R(1e-4) * r && fabs(q) > R(1e-9) * r;
}

}  // namespace art
