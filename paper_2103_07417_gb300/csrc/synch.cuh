// synch.cuh -- polarized transfer on the device: thermal-synchrotron thin disk, parallel transport
// of the polarization reference covector, and the exact constant-coefficient Stokes segment.
//
// Stokes transfer d S/ds = J - K S with K = [[aI,aQ,aU,aV],[aQ,aI,rV,-rU],[aU,-rV,aI,rQ],
// [aV,rU,-rQ,aI]] (Landi Degl'Innocenti & Landi Degl'Innocenti 1985 conventions), in invariant
// code units: J = L j_nu / nu^2, K = L nu {alpha, rho}, nu = k.u the fluid-frame frequency ratio,
// L = GM/c^2 in cm.  The polarization basis at every point is the parallel-transported covector
// f projected into the fluid frame (e_N) and e_E = d x e_N (d the propagation direction), which at
// the camera is north = screen up, east = screen left (IAU).
//
// Synchrotron coefficients (frame with Q along the emission's E-vector, normal to the field):
// j_I from Leung, Gammie & Noble (2011); j_Q the same form with the X^(1/6) coefficient scaled by
// (7 Th^0.96 + 35)/(10 Th^0.96 + 75) (Pandya et al. 2016); j_V = 0; Kirchhoff absorption;
// rho_V ~ n B cos(theta) K0/K2 / nu^2 and rho_Q ~ n B^2 sin^2(theta) (K1/K2 + 6 Th) / nu^3 (the
// high-frequency thermal rotativities).  K_0 and K_1 are the polynomial approximations of
// Abramowitz & Stegun 9.8.1-9.8.8, K_2 = K_0 + 2 K_1 / x.
//
// The segment solution uses the eigenstructure of the polarized part K' = K - aI 1: its
// eigenvalues are +-L1, +-i L2 with L1^2, L2^2 = +-(a^2 - r^2)/2 + sqrt(((a^2 - r^2)/2)^2 + (a.r)^2)
// (a = (aQ,aU,aV), r = (rQ,rU,rV)), so by Cayley-Hamilton
//   exp(-K' s) = C0 1 + C1 K' + C2 K'^2 + C3 K'^3,  D = L1^2 + L2^2,
//   C0 = (L2^2 cosh L1 s + L1^2 cos L2 s)/D,  C1 = -(L2^2 sinh(L1 s)/L1 + L1^2 sin(L2 s)/L2)/D,
//   C2 = (cosh L1 s - cos L2 s)/D,            C3 = -(sinh(L1 s)/L1 - sin(L2 s)/L2)/D,
// and the source integral int_0^h exp(-K s) ds J is the same combination with each function of s
// replaced by its integral against exp(-aI s) (closed forms through (1 - e^{-z})/z, real and
// complex).  Small arguments use the limits of these expressions.
#pragma once
#include <cstdint>

#include "kerr.cuh"
#include "fmath64.cuh"

namespace art {

// Constants of the synchrotron models, precomputed on the host in double (keeps FP32 in range);
// the FP32 and double-float kernels read a float copy (SynchConstF) made on the host, so that no
// per-step conversion from double runs on the FP64 pipe.
template <class T>
struct SynchConstT {
    T ne0, th0, b0, ne_s, te_s, b_s, inv_2w2, r_in, bz, bnorm;
    T LCj;    // L sqrt2 pi e^2 / (3 c)
    T CB;     // e / (2 pi m c)   [nu_B per gauss]
    T nu_obs; // observed frequency [Hz]
    T xB;     // h nu_obs / (m c^2)
    T invKB;  // c^2 / (2 h nu_obs^3)
    T LCV;    // L e^3 / (pi m^2 c^2 nu_obs^2)
    T LCQ;    // L e^4 / (4 pi^2 m^3 c^3 nu_obs^3)
    // fluid grid (ART_EMIT_GRID): cells of 8 FP32 primitives as two float4
    // {rho, u, u^r, u^theta}, {u^phi, B^r, B^theta, B^phi}, cell (k, j, i) at float4 index
    // 2 ((k n2 + j) n1 + i); cell centres at ln r = x1_min + (i + 1/2)/inv_dx1, theta = (j + 1/2)
    // pi/n2, phi = (k + 1/2) 2 pi/n3
    const float4* grid;
    int32_t g_n1, g_n2, g_n3, g_pad;
    T g_x1min, g_x1max, g_inv_dx1, g_inv_dth, g_inv_dph;
    T g_gm1;        // gamma_ad - 1
    T g_ne_unit;    // m_unit / (L^3 (m_p + m_e))      [cm^-3 per code density]
    T g_b_unit;     // c sqrt(4 pi m_unit / L^3)       [gauss per code field]
    T g_th_unit;    // (m_p / m_e)(gamma_ad - 1)
    T g_r_high, g_r_low, g_sigma_cut;
    // FP32 pass of the mixed modes (0 elsewhere): relative distances from the emission model's
    // discontinuities (the magnetisation cut b^2/rho = sigma_cut, the disk's inner edge r_in) within
    // which a sample flags its ray for the high-precision re-trace
    T e_sig, e_rin;
};
using SynchConst = SynchConstT<double>;
using SynchConstF = SynchConstT<float>;

// The float copy (every value rounded to nearest).
inline SynchConstF synch_to_float(const SynchConst& d)
{
    SynchConstF f;
    f.ne0 = (float)d.ne0; f.th0 = (float)d.th0; f.b0 = (float)d.b0; f.ne_s = (float)d.ne_s;
    f.te_s = (float)d.te_s; f.b_s = (float)d.b_s; f.inv_2w2 = (float)d.inv_2w2;
    f.r_in = (float)d.r_in; f.bz = (float)d.bz; f.bnorm = (float)d.bnorm;
    f.LCj = (float)d.LCj; f.CB = (float)d.CB; f.nu_obs = (float)d.nu_obs; f.xB = (float)d.xB;
    f.invKB = (float)d.invKB; f.LCV = (float)d.LCV; f.LCQ = (float)d.LCQ;
    f.grid = d.grid;
    f.g_n1 = d.g_n1; f.g_n2 = d.g_n2; f.g_n3 = d.g_n3; f.g_pad = d.g_pad;
    f.g_x1min = (float)d.g_x1min; f.g_x1max = (float)d.g_x1max;
    f.g_inv_dx1 = (float)d.g_inv_dx1; f.g_inv_dth = (float)d.g_inv_dth;
    f.g_inv_dph = (float)d.g_inv_dph; f.g_gm1 = (float)d.g_gm1;
    f.g_ne_unit = (float)d.g_ne_unit; f.g_b_unit = (float)d.g_b_unit;
    f.g_th_unit = (float)d.g_th_unit; f.g_r_high = (float)d.g_r_high;
    f.g_r_low = (float)d.g_r_low; f.g_sigma_cut = (float)d.g_sigma_cut;
    f.e_sig = (float)d.e_sig; f.e_rin = (float)d.e_rin;
    return f;
}

template <class Q>
ART_HD Q horner7(Q t, Q c0, Q c1, Q c2, Q c3, Q c4, Q c5, Q c6)
{
    return fmad(t, fmad(t, fmad(t, fmad(t, fmad(t, fmad(t, c6, c5), c4), c3), c2), c1), c0);
}

// K_0, K_1, K_2 (the polynomials of Abramowitz & Stegun 9.8.1-9.8.8).  For x > 2 they are returned
// scaled by e^x (K_n(x) e^x, so that FP32 stays finite for cold plasma, large x) and the function
// returns true; for x <= 2 unscaled (false), which spares the exponential there: the caller's
// e^-X^1/3 / K_2 takes the factor e^x exactly when the K_n carry it.
// ix = 1/x and lx = log(x) are passed in (the caller has them), which spares divisions and a
// logarithm on GB300's FP64 pipe.
template <class Q>
ART_HD bool bessel_k012(Q x, Q ix, Q lx, Q& K0, Q& K1, Q& K2)
{
    const bool scaled = x > Q(2);
    if (!scaled) {
        Q t = x * Q(1.0 / 3.75), t2 = t * t;
        Q i0 = horner7<Q>(t2, Q(1), Q(3.5156229), Q(3.0899424), Q(1.2067492), Q(0.2659732),
                          Q(0.0360768), Q(0.0045813));
        Q i1 = x * horner7<Q>(t2, Q(0.5), Q(0.87890594), Q(0.51498869), Q(0.15084934),
                              Q(0.02658733), Q(0.00301532), Q(0.00032411));
        Q y = Q(0.25) * x * x, lg = lx - Q(0.69314718055994530942);
        K0 = fmad(-lg, i0, horner7<Q>(y, Q(-0.57721566), Q(0.42278420), Q(0.23069756),
                                      Q(0.03488590), Q(0.00262698), Q(0.00010750),
                                      Q(0.0000074)));
        K1 = fmad(lg, i1, ix * horner7<Q>(y, Q(1), Q(0.15443144), Q(-0.67278579),
                                                  Q(-0.18156897), Q(-0.01919402),
                                                  Q(-0.00110404), Q(-0.00004686)));
    } else {
        Q y = Q(2) * ix, pre = sqrt(ix);
        K0 = pre * horner7<Q>(y, Q(1.25331414), Q(-0.07832358), Q(0.02189568), Q(-0.01062446),
                              Q(0.00587872), Q(-0.00251540), Q(0.00053208));
        K1 = pre * horner7<Q>(y, Q(1.25331414), Q(0.23498619), Q(-0.03655620), Q(0.01504268),
                              Q(-0.00780353), Q(0.00325614), Q(-0.00068245));
    }
    K2 = fmad(Q(2), K1 * ix, K0);
    return scaled;
}

// Minkowski + Kerr-Schild pieces at a point: F = 2 r^3 / (r^4 + a^2 z^2), L (outgoing l = (1,-L)).
template <class Q>
struct KSPoint {
    Q F, Lx, Ly, Lz;
    ART_HD Q ldot(const Q* v) const { return v[0] - fmad(Lz, v[3], fmad(Ly, v[2], Lx * v[1])); }
    ART_HD Q dot(const Q* u, const Q* v) const
    {
        return fmad(F * ldot(u), ldot(v),
                    fmad(u[3], v[3], fmad(u[2], v[2], fmad(u[1], v[1], -(u[0] * v[0])))));
    }
    // raise a covector: w^t = -w_t + F lw, w^i = w_i + F L_i lw, lw = l^mu w_mu = -w_t - L.w
    ART_HD void raise(const Q* w, Q* up) const
    {
        Q lw = -w[0] - fmad(Lz, w[3], fmad(Ly, w[2], Lx * w[1]));
        up[0] = fmad(F, lw, -w[0]);
        up[1] = fmad(F * Lx, lw, w[1]);
        up[2] = fmad(F * Ly, lw, w[2]);
        up[3] = fmad(F * Lz, lw, w[3]);
    }
};

// ir = 1/r (the caller has it).
template <class Q>
ART_HD KSPoint<Q> ks_point(Q x, Q y, Q z, Q r, Q ir, Q a, Q a2)
{
    KSPoint<Q> P;
    Q r2 = r * r;
    P.F = Q(2) * r2 * r / fmad(r2, r2, a2 * z * z);
    Q ira2 = Q(1) / (r2 + a2);
    P.Lx = fmad(r, x, -(a * y)) * ira2;
    P.Ly = fmad(r, y, a * x) * ira2;
    P.Lz = z * ir;
    return P;
}

// 4x4 determinant det[A; B; C; D] of contravariant components (sqrt(-g) = 1 in these coordinates).
template <class Q>
ART_HD Q det4(const Q* A, const Q* B, const Q* C, const Q* D)
{
    Q m01 = fmad(C[0], D[1], -(C[1] * D[0])), m02 = fmad(C[0], D[2], -(C[2] * D[0]));
    Q m03 = fmad(C[0], D[3], -(C[3] * D[0])), m12 = fmad(C[1], D[2], -(C[2] * D[1]));
    Q m13 = fmad(C[1], D[3], -(C[3] * D[1])), m23 = fmad(C[2], D[3], -(C[3] * D[2]));
    Q c0 = fmad(B[3], m12, fmad(B[1], m23, -(B[2] * m13)));
    Q c1 = fmad(B[3], m02, fmad(B[0], m23, -(B[2] * m03)));
    Q c2 = fmad(B[3], m01, fmad(B[0], m13, -(B[1] * m03)));
    Q c3 = fmad(B[2], m01, fmad(B[0], m12, -(B[1] * m02)));
    return fmad(-A[3], c3, fmad(A[2], c2, fmad(A[0], c0, -(A[1] * c1))));
}

// Thermal-synchrotron coefficients of a fluid element (velocity u, unit field direction b in its
// frame, density ne [cm^-3], temperature Th and its reciprocal iTh, field Bm [G]) seen by the ray
// with covariant k (kt, s.k) and fluid-frame frequency ratio nu = k.u > 0; f (nullable) is the
// transported covector.  J4, K7 in code units, in the (e_N, e_E) basis of f.
template <class Q>
ART_HD void synch_coeffs(const KSPoint<Q>& G, const RayState<Q>& s, Q kt, const Q* u, const Q* b,
                         Q nu, Q ne, Q Th, Q iTh, Q Bm, const Q* f, const SynchConstT<Q>& S,
                         Q* J4, Q* K7)
{
    Q kc[4] = {kt, s.kx, s.ky, s.kz}, ku[4];
    G.raise(kc, ku);
    // unit propagation direction in the fluid frame: -(k + nu u)/|k + nu u| (nu > 0; the
    // integrated k is null only to the truncation error)
    Q d[4];
    for (int m = 0; m < 4; ++m) d[m] = fmad(nu, u[m], ku[m]);
    Q dn = -rsqrt(G.dot(d, d));
    for (int m = 0; m < 4; ++m) d[m] *= dn;
    Q cth = G.dot(d, b);
    cth = cth > Q(1) ? Q(1) : (cth < Q(-1) ? Q(-1) : cth);
    Q sth2 = fmad(-cth, cth, Q(1));
    Q sth = sqrt(sth2);
    // coefficients in the E-vector frame; K_n e^x keeps 1/K_2 finite for large x, where
    // e^(x - X^1/3) recombines (bessel_k012)
    const Q lTh = log_q<Q>(Th);
    Q x = iTh, K0, K1, K2;
    const bool kscaled = bessel_k012<Q>(x, Th, -lTh, K0, K1, K2);
    // 1/nu, 1/nu_s and 1/K2 from one division
    const bool emits = sth > Q(1e-12);
    const Q nus = emits ? Q(2.0 / 9.0) * Q(S.CB) * Bm * Th * Th * sth : Q(1);
    const Q nuK2 = nu * K2;
    const Q idv = Q(1) / (nuK2 * nus);
    const Q inu = (nus * K2) * idv, inus = nuK2 * idv, iK2 = (nu * nus) * idv;
    Q jI = Q(0), jQ = Q(0);
    if (emits) {
        Q X = Q(S.nu_obs) * nu * inus;
        Q x3 = cbrt(X), x6 = sqrt(x3), x2 = x3 * x6;  // X^1/3, X^1/6, X^1/2
        Q pre = Q(S.LCj) * ne * nus * exp(kscaled ? x - x3 : -x3) * (inu * inu) * iK2;
        Q t96 = exp(Q(0.96) * lTh);
        Q q = fmad(Q(7), t96, Q(35)) / fmad(Q(10), t96, Q(75));
        const Q k1112 = Q(1.8877486253633868);  // 2^(11/12)
        Q vi = fmad(k1112, x6, x2), vq = fmad(q * k1112, x6, x2);
        jI = pre * vi * vi;
        jQ = pre * vq * vq;
    }
    Q kir = expm1(Q(S.xB) * nu * x) * Q(S.invKB);  // nu^3 / B_nu in code units
    J4[0] = jI;
    K7[0] = jI * kir;
    if (!f) return;
    Q rV = Q(S.LCV) * ne * Bm * cth * inu * (K0 * iK2);
    Q rQ = Q(S.LCQ) * ne * Bm * Bm * sth2 * (inu * inu) * fmad(Q(6), Th, K1 * iK2);
    // polarization basis from the transported covector
    Q fu_[4];
    G.raise(f, fu_);
    Q fuu = G.dot(fu_, u), fud = G.dot(fu_, d), eN[4];
    for (int m = 0; m < 4; ++m) eN[m] = fmad(-fud, d[m], fmad(fuu, u[m], fu_[m]));
    Q nN = Q(1) / sqrt(G.dot(eN, eN));
    for (int m = 0; m < 4; ++m) eN[m] *= nN;
    Q bN = G.dot(b, eN);
    Q bE = -det4<Q>(b, u, d, eN);
    Q bp2 = fmad(bE, bE, bN * bN);
    Q c2 = Q(1), s2 = Q(0);
    if (bp2 > Q(0)) {
        // E-vector at angle chi from north: cos chi = -bE/|b_perp|, sin chi = bN/|b_perp|
        const Q ibp2 = Q(1) / bp2;
        c2 = fmad(bE, bE, -(bN * bN)) * ibp2;
        s2 = Q(-2) * bE * bN * ibp2;
    }
    J4[1] = jQ * c2;
    J4[2] = jQ * s2;
    K7[1] = jQ * kir * c2;
    K7[2] = jQ * kir * s2;
    K7[4] = rQ * c2;
    K7[5] = rQ * s2;
    K7[6] = rV;
}

// Emission J4 and K7 = {aI,aQ,aU,aV,rQ,rU,rV} of the synchrotron disk at one point, code units.
// f (nullable) is the transported covector; without it only the I terms are returned.
template <class Q>
ART_HD void emission_synch(const RayState<Q>& s, Q r, Q kt, const Q* f, const DevJob& J,
                           const SynchConstT<Q>& S, Q* J4, Q* K7, int* edge = nullptr)
{
    for (int i = 0; i < 4; ++i) J4[i] = Q(0);
    for (int i = 0; i < 7; ++i) K7[i] = Q(0);
    // a sample within rounding of the inner edge (in the emitting layer) may fall on either side
    // of it in another precision: the ray's intensity then jumps by a whole segment's emission
    if (edge && S.e_rin > Q(0) && fabs(r - Q(S.r_in)) < Q(S.e_rin) * Q(S.r_in)) {
        const Q c0 = s.z / r;
        if (c0 * c0 * Q(S.inv_2w2) < Q(20)) *edge = 1;
    }
    if (r < jq<Q>(J.r_in_stop, J.f_r_in_stop) || r < Q(S.r_in)) return;
    const Q a = jq<Q>(J.a, J.f_a), a2 = jq<Q>(J.a2, J.f_a2);
    const Q ir = Q(1) / r;
    Q ct = s.z * ir, ct2 = ct * ct, r2 = r * r;
    // Keplerian flow (Omega at Boyer-Lindquist r, theta)
    Q st2 = Q(1) - ct2;
    Q iSig = Q(1) / (r2 + a2 * ct2);
    Q gtt = -(Q(1) - Q(2) * r * iSig);
    Q gtp = -Q(2) * a * r * st2 * iSig;
    Q gpp = fmad(Q(2) * a2 * r * st2, iSig, r2 + a2) * st2;
    Q Om = Q(1) / fmad(r, sqrt(r), a);
    Q nrm = -fmad(Om * Om, gpp, fmad(Q(2) * Om, gtp, gtt));
    if (!(nrm > Q(0))) return;
    Q ut = Q(1) / sqrt(nrm);
    Q u[4] = {ut, -Om * s.y * ut, Om * s.x * ut, Q(0)};
    Q nu = ut * fmad(Om, fmad(s.x, s.ky, -(s.y * s.kx)), kt);
    if (!(nu > Q(0))) return;
    Q lr = log(r);
    Q ne = Q(S.ne0) * exp(fmad(Q(S.ne_s), lr, -(ct2 * Q(S.inv_2w2))));
    Q Th = Q(S.th0) * exp(Q(S.te_s) * lr);
    Q Bm = Q(S.b0) * exp(Q(S.b_s) * lr);
    if (!(ne > Q(0))) return;
    KSPoint<Q> G = ks_point<Q>(s.x, s.y, s.z, r, ir, a, a2);
    // field direction (e_phi + q e_z)/sqrt(1 + q^2) in the fluid frame
    Q ephi[4] = {Q(0), -s.y, s.x, Q(0)};
    Q pu = G.dot(u, ephi);
    for (int m = 0; m < 4; ++m) ephi[m] = fmad(pu, u[m], ephi[m]);
    Q nph = Q(1) / sqrt(G.dot(ephi, ephi));
    for (int m = 0; m < 4; ++m) ephi[m] *= nph;
    Q ez[4] = {Q(0), Q(0), Q(0), Q(1)};
    Q pz = G.dot(u, ez), pe = G.dot(ephi, ez);
    for (int m = 0; m < 4; ++m) ez[m] = fmad(-pe, ephi[m], fmad(pz, u[m], ez[m]));
    Q nz = Q(1) / sqrt(G.dot(ez, ez));
    Q b[4];
    for (int m = 0; m < 4; ++m) b[m] = fmad(Q(S.bz) * nz, ez[m], ephi[m]) * Q(S.bnorm);
    synch_coeffs<Q>(G, s, kt, u, b, nu, ne, Th, Q(1) / Th, Bm, f, S, J4, K7);
}

// Parallel transport of the covector f along the geodesic (outgoing Kerr-Schild form):
// df_mu/dlambda = 1/2 [T1_mu + T2_mu - T3_mu] with, for g = eta + F l l, lf = l.f, lk = l.k,
// Jm_ij = d_i L_j, gF_i = d_i F (contravariant k and f):
//   T1_i = gF_i lf lk - F ((Jm f)_i lk + lf (Jm k)_i),                            T1_t = 0,
//   T2_mu = (k.gF) lf l_mu - F (k.Jm.f) l_mu + F lf Dk(l_mu),  Dk(l_j) = -(k.Jm)_j, Dk(l_t) = 0,
//   T3_mu = (f.gF) lk l_mu - F (f.Jm.k) l_mu + F lk Df(l_mu),  Df(l_j) = -(f.Jm)_j.
template <class Q>
ART_HD Q dot3(Q a0, Q b0, Q a1, Q b1, Q a2, Q b2)
{
    return fmad(a2, b2, fmad(a1, b1, a0 * b0));
}

template <class Q>
ART_HD void transport_rhs(const RayState<Q>& s, Q kt, const Q* f, Q a, Q a2, Q* df)
{
    const Q x = s.x, y = s.y, z = s.z;
    Q z2 = z * z, a2z2 = a2 * z2;
    Q bb = (fmad(y, y, x * x) + z2) - a2;
    Q r2 = Q(0.5) * (bb + sqrt(fmad(bb, bb, Q(4) * a2z2)));
    Q r = sqrt(r2), ir = Q(1) / r;
    Q r4 = r2 * r2, iQ = Q(1) / (r4 + a2z2);
    Q F = Q(2) * r2 * r * iQ;
    Q ira2 = Q(1) / (r2 + a2);
    Q Lx = fmad(r, x, -(a * y)) * ira2, Ly = fmad(r, y, a * x) * ira2, Lz = z * ir;
    Q iSig = r2 * iQ;
    Q dr[3] = {x * r * iSig, y * r * iSig, z * (r2 + a2) * ir * iSig};
    Q B = F * ir * fmad(Q(-4) * r4, iQ, Q(3));
    Q gF[3] = {B * dr[0], B * dr[1], fmad(B, dr[2], -(Q(2) * F * a2 * z * iQ))};
    // Jm[i][j] = d_i L_j
    Q Jm[3][3];
    for (int i = 0; i < 3; ++i) {
        const Q tr = Q(-2) * r * dr[i];
        Jm[i][0] = (fmad(tr, Lx, x * dr[i]) + ((i == 0 ? r : Q(0)) - (i == 1 ? a : Q(0)))) * ira2;
        Jm[i][1] = (fmad(tr, Ly, y * dr[i]) + ((i == 1 ? r : Q(0)) + (i == 0 ? a : Q(0)))) * ira2;
        Jm[i][2] = fmad(-z * dr[i], ir * ir, (i == 2 ? ir : Q(0)));
    }
    // contravariant k and f
    Q lkc = -kt - dot3(Lx, s.kx, Ly, s.ky, Lz, s.kz);
    Q ku[4] = {fmad(F, lkc, -kt), fmad(F * Lx, lkc, s.kx), fmad(F * Ly, lkc, s.ky),
               fmad(F * Lz, lkc, s.kz)};
    Q lfc = -f[0] - dot3(Lx, f[1], Ly, f[2], Lz, f[3]);
    Q fu[4] = {fmad(F, lfc, -f[0]), fmad(F * Lx, lfc, f[1]), fmad(F * Ly, lfc, f[2]),
               fmad(F * Lz, lfc, f[3])};
    Q lk = ku[0] - dot3(Lx, ku[1], Ly, ku[2], Lz, ku[3]);
    Q lf = fu[0] - dot3(Lx, fu[1], Ly, fu[2], Lz, fu[3]);
    Q Jf[3], Jk[3], kJ[3], fJ[3];
    for (int i = 0; i < 3; ++i) {
        Jf[i] = dot3(Jm[i][0], fu[1], Jm[i][1], fu[2], Jm[i][2], fu[3]);
        Jk[i] = dot3(Jm[i][0], ku[1], Jm[i][1], ku[2], Jm[i][2], ku[3]);
        kJ[i] = dot3(ku[1], Jm[0][i], ku[2], Jm[1][i], ku[3], Jm[2][i]);
        fJ[i] = dot3(fu[1], Jm[0][i], fu[2], Jm[1][i], fu[3], Jm[2][i]);
    }
    Q kgF = dot3(ku[1], gF[0], ku[2], gF[1], ku[3], gF[2]);
    Q fgF = dot3(fu[1], gF[0], fu[2], gF[1], fu[3], gF[2]);
    Q kJf = dot3(ku[1], Jf[0], ku[2], Jf[1], ku[3], Jf[2]);
    Q fJk = dot3(fu[1], Jk[0], fu[2], Jk[1], fu[3], Jk[2]);
    Q l[4] = {Q(1), -Lx, -Ly, -Lz};
    Q c2 = fmad(kgF, lf, -(F * kJf));   // T2 = c2 l_mu + F lf Dk(l_mu)
    Q c3 = fmad(fgF, lk, -(F * fJk));   // T3 = c3 l_mu + F lk Df(l_mu)
    df[0] = Q(0.5) * (c2 - c3);
    for (int i = 0; i < 3; ++i) {
        Q t1 = fmad(gF[i] * lf, lk, -(F * fmad(Jf[i], lk, lf * Jk[i])));
        Q t2 = fmad(c2, l[i + 1], -(F * lf * kJ[i]));
        Q t3 = fmad(c3, l[i + 1], -(F * lk * fJ[i]));
        df[i + 1] = Q(0.5) * ((t1 + t2) - t3);
    }
}

// psi_n(x) = int_0^1 t^n e^{-x t} dt = sum_k (-x)^k / (k! (n + k + 1)) for small x (18 terms,
// Horner form with the coefficients 1/(k! (n + k + 1)) fixed at compile time), closed forms
// otherwise.
template <int N, int K>
struct PsiCoef {
    static constexpr double fact = PsiCoef<N, K - 1>::fact * K;
    static constexpr double v = 1.0 / (fact * (N + K + 1));
};
template <int N>
struct PsiCoef<N, 0> {
    static constexpr double fact = 1.0;
    static constexpr double v = 1.0 / (N + 1);
};

template <class Q, int N, int K>
ART_HD Q psi_series(Q mx)
{
    if constexpr (K == 17)
        return Q(PsiCoef<N, K>::v);
    else
        return fmad(mx, psi_series<Q, N, K + 1>(mx), Q(PsiCoef<N, K>::v));
}

template <class Q, int N>
ART_HD Q psi_n(Q x)
{
    if (x < Q(1.5)) return psi_series<Q, N, 0>(-x);
    Q e = exp(-x), x2 = x * x;
    if (N == 1) return (Q(1) - e * (Q(1) + x)) / x2;
    if (N == 2) return (Q(2) - e * (x2 + Q(2) * x + Q(2))) / (x2 * x);
    return (Q(6) - e * (x2 * x + Q(3) * x2 + Q(6) * x + Q(6))) / (x2 * x2);
}

// (1 - e^{-x})/x for real x >= 0 and its complex counterpart for z = x + i y
template <class Q>
ART_HD Q phi_r(Q x)
{
    return x > Q(1e-6) ? -expm1(-x) / x : Q(1) - Q(0.5) * x;
}

template <class Q>
ART_HD void phi_c(Q x, Q y, Q& re, Q& im)
{
    Q d = fmad(y, y, x * x);
    if (d < Q(1e-12)) {  // 1 - z/2
        re = Q(1) - Q(0.5) * x;
        im = Q(-0.5) * y;
        return;
    }
    Q e = exp(-x), sh = sin(Q(0.5) * y);
    // numerator 1 - e^{-x}(cos y - i sin y), with 1 - e^{-x} cos y = -expm1(-x) cos y + 2 sin^2(y/2)
    Q nr = fmad(Q(2) * sh, sh, -expm1(-x) * cos(y));
    Q ni = e * sin(y);
    re = fmad(ni, y, nr * x) / d;
    im = fmad(ni, x, -(nr * y)) / d;
}

// K' v for the traceless polarized part of K.
template <class Q>
ART_HD void kprime_v(const Q* K7, const Q* v, Q* o)
{
    const Q aQ = K7[1], aU = K7[2], aV = K7[3], rQ = K7[4], rU = K7[5], rV = K7[6];
    o[0] = fmad(aV, v[3], fmad(aU, v[2], aQ * v[1]));
    o[1] = fmad(-rU, v[3], fmad(rV, v[2], aQ * v[0]));
    o[2] = fmad(rQ, v[3], fmad(-rV, v[1], aU * v[0]));
    o[3] = fmad(-rQ, v[2], fmad(rU, v[1], aV * v[0]));
}

// row-vector times K' (P K' for one row of P)
template <class Q>
ART_HD void v_kprime(const Q* K7, const Q* v, Q* o)
{
    const Q aQ = K7[1], aU = K7[2], aV = K7[3], rQ = K7[4], rU = K7[5], rV = K7[6];
    o[0] = fmad(v[3], aV, fmad(v[2], aU, v[1] * aQ));
    o[1] = fmad(v[3], rU, fmad(-v[2], rV, v[0] * aQ));
    o[2] = fmad(-v[3], rQ, fmad(v[1], rV, v[0] * aU));
    o[3] = fmad(v[2], rQ, fmad(-v[1], rU, v[0] * aV));
}

// One constant-coefficient Stokes segment of length h: adds P X to acc (4 Stokes) and replaces the
// accumulated propagator P (row-major, camera <- segment start) by P exp(-K h).  The hyperbolic
// functions are carried with the attenuation exp(-aI h) folded in, so optically thick segments
// cannot overflow (aI >= L1 for physical coefficients).
template <class Q>
ART_HD void segment_pol(const Q* K7, const Q* J4, Q h, Q* P, Q* acc)
{
    const Q tiny = Q(sizeof(Q) == 4 ? 1e-3 : 1e-7);
    const Q aI = K7[0];
    Q al2 = fmad(K7[3], K7[3], fmad(K7[2], K7[2], K7[1] * K7[1]));
    Q rh2 = fmad(K7[6], K7[6], fmad(K7[5], K7[5], K7[4] * K7[4]));
    Q ar = fmad(K7[3], K7[6], fmad(K7[2], K7[5], K7[1] * K7[4]));
    Q t = Q(0.5) * (al2 - rh2), sq = sqrt(fmad(ar, ar, t * t));
    Q L1 = sqrt(fmax(t + sq, Q(0))), L2 = sqrt(fmax(sq - t, Q(0)));
    const Q L11 = L1 * L1, L22 = L2 * L2;
    Q D = L11 + L22;
    Q a = L1 * h, b = L2 * h, Dh2 = D * h * h;
    const Q ea = exp(-aI * h);
    Q C0, C1, C2, C3;  // exp(-K h) = C0 + C1 K' + C2 K'^2 + C3 K'^3 (attenuation included)
    Q X0, X1, X2, X3;  // source integral = X0 J + X1 K'J + X2 K'^2 J + X3 K'^3 J
    if (Dh2 < tiny * tiny) {
        // weakly polarizing segment (the common case of an optically thin flow): the series of
        // exp(-K' s) to third order; only the attenuation's functions are needed
        const Q x = aI * h;
        C0 = ea;
        C1 = -h * ea;
        C2 = Q(0.5) * h * h * ea;
        C3 = -h * h * h * ea / Q(6);
        X0 = h * phi_r<Q>(x);
        X1 = -h * h * psi_n<Q, 1>(x);
        X2 = Q(0.5) * h * h * h * psi_n<Q, 2>(x);
        X3 = -h * h * h * h * psi_n<Q, 3>(x) / Q(6);
    } else {
        // ea cosh(a), ea sinh(a)/a, ea sinh^2(a/2)
        Q eCh, eSha, eSa2;
        if (a < Q(20)) {
            Q sa2 = sinh(Q(0.5) * a);
            eCh = ea * cosh(a);
            eSha = ea * (a < tiny ? Q(1) + a * a / Q(6) : sinh(a) / a);
            eSa2 = ea * sa2 * sa2;
        } else {
            Q e1 = exp(-(aI - L1) * h), e2 = exp(-(aI + L1) * h);
            eCh = Q(0.5) * (e1 + e2);
            eSha = Q(0.5) * (e1 - e2) / a;
            eSa2 = Q(0.5) * (eCh - ea);
        }
        Q cb = cos(b), sb2 = sin(Q(0.5) * b);
        Q sbb = b < tiny ? Q(1) - b * b / Q(6) : sin(b) / b;
        C0 = fmad(L22, eCh, L11 * ea * cb) / D;
        C1 = -h * fmad(L22, eSha, L11 * ea * sbb) / D;
        C2 = Q(2) * fmad(ea * sb2, sb2, eSa2) / D;
        if (a * a + b * b < Q(0.1) && a < Q(20)) {
            Q a2_ = a * a, b2_ = b * b;
            C3 = -h * h * h * ea *
                 (Q(1) / Q(6) + (a2_ - b2_) / Q(120) + (a2_ * a2_ - a2_ * b2_ + b2_ * b2_) / Q(5040));
        } else {
            C3 = -h * (eSha - ea * sbb) / D;
        }
        // source coefficients: the same functions of s integrated against exp(-aI s)
        Q r1 = fmax((aI - L1) * h, Q(0)), r2 = (aI + L1) * h;
        Q p1 = phi_r<Q>(r1), p2 = phi_r<Q>(r2);
        Q Ic = Q(0.5) * h * (p1 + p2);
        Q IsL1 = a < tiny ? h * h * psi_n<Q, 1>(aI * h) : Q(0.5) * h * (p1 - p2) / L1;
        Q pcr, pci;
        phi_c<Q>(aI * h, -b, pcr, pci);
        Q Icos = h * pcr;
        Q IsinL2 = b < tiny ? h * h * psi_n<Q, 1>(aI * h) : h * pci / L2;
        X0 = fmad(L22, Ic, L11 * Icos) / D;
        X1 = -fmad(L22, IsL1, L11 * IsinL2) / D;
        X2 = (Ic - Icos) / D;
        X3 = -(IsL1 - IsinL2) / D;
    }
    // X = X0 J + X1 K'J + X2 K'^2 J + X3 K'^3 J
    Q v1[4], v2[4], v3[4], Xv[4];
    kprime_v<Q>(K7, J4, v1);
    kprime_v<Q>(K7, v1, v2);
    kprime_v<Q>(K7, v2, v3);
    for (int i = 0; i < 4; ++i) Xv[i] = fmad(X3, v3[i], fmad(X2, v2[i], fmad(X1, v1[i], X0 * J4[i])));
    // acc += P X ;  P <- P exp(-K h)
    for (int i = 0; i < 4; ++i) {
        Q* row = P + 4 * i;
        acc[i] += fmad(row[3], Xv[3], fmad(row[2], Xv[2], fmad(row[1], Xv[1], row[0] * Xv[0])));
        Q w1[4], w2[4], w3[4];
        v_kprime<Q>(K7, row, w1);
        v_kprime<Q>(K7, w1, w2);
        v_kprime<Q>(K7, w2, w3);
        for (int j = 0; j < 4; ++j)
            row[j] = fmad(C3, w3[j], fmad(C2, w2[j], fmad(C1, w1[j], C0 * row[j])));
    }
}

}  // namespace art
