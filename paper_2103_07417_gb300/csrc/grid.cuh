// grid.cuh -- emission from a fluid snapshot on a spherical Kerr-Schild grid (a GRMHD-like
// model, Sec. 4.2 and 5 of the paper: electron temperatures from the R_high prescription and a
// magnetisation cut).
//
// Lookup: the snapshot holds eight FP32 primitives per cell (rho, u, u^r, u^theta, u^phi, B^r,
// B^theta, B^phi; contravariant Kerr-Schild spherical components) as two float4, cell-centred on
// a uniform grid in (ln r, theta, phi).  A sample at (ln r, theta, phi) is the trilinear
// interpolant of the eight surrounding cells: per axis f = (coordinate - start)/spacing - 1/2;
// ln r and theta clamp f to [0, n - 1], phi wraps; points with ln r outside the grid do not emit.
// A sample reads 8 cells x 32 B = 256 B through the read-only data path; consecutive samples of a
// ray fall in the same or neighbouring cells, so most of them hit in L1/L2.
//
// Fluid reconstruction (Gammie, McKinney & Toth 2003 for b):
//   u^t = q / (sqrt(p^2 - g_tt q) - p),  q = 1 + g_ij u^i u^j,  p = g_ti u^i
//     (the positive root of g_mu nu u^mu u^nu = -1 that stays continuous through g_tt = 0);
//   b^t = g_{i mu} B^i u^mu,  b^i = (B^i + b^t u^i)/u^t;
//   T_i/T_e = (R_high beta^2 + R_low)/(1 + beta^2), beta = (gamma - 1) u / (b^2/2)
//     (Moscibrodzka, Falcke & Shiokawa 2016), Theta_e = (m_p/m_e)(gamma - 1) u/(rho (1 + T_i/T_e));
//   n_e = rho * ne_unit, |B| = sqrt(b^2) * b_unit;  no emission where b^2/rho > sigma_cut.
// In outgoing Cartesian Kerr-Schild form g_tt = F - 1, g_ti = -F L_i, g_ij = delta_ij + F L_i L_j.
#pragma once
#include "synch.cuh"

namespace art {

// float -> double on the integer units.  GB300 converts between the two precisions at the FP64
// rate (a warp instruction per 64 cycles on a scheduler), its integer units issue every cycle,
// and a sample widens 64 cell values.  For zeros and normal numbers the exponent is rebiased
// (127 -> 1023) and the significand moved into place: the conversion's exact result.  The other
// values (subnormal, infinite, NaN) are flagged by widen_special; a sample holding one takes the
// conversion instruction for all its cells.
ART_FM_DEV double widen(float f)
{
    const uint32_t u = fm_f32bits(f), au = u & 0x7fffffffu;
    const uint32_t hi = au != 0u ? (au >> 3) + (896u << 20) : 0u;
    const uint32_t lo = au << 29;
    return fm_double((int64_t)(((uint64_t)(hi | (u & 0x80000000u)) << 32) | (uint64_t)lo));
}

ART_FM_DEV unsigned widen_special(float f)
{
    const uint32_t au = fm_f32bits(f) & 0x7fffffffu;
    return (unsigned)(au != 0u) & (unsigned)(au - 0x00800000u >= 0x7f000000u);
}

// Two float4 of a snapshot cell through the read-only data path (a plain load on the host, where
// the same code is built for the accuracy checks).
ART_FM_DEV float4 grid_load(const float4* p)
{
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

template <class Q>
ART_HD void grid_axis_clamped(Q f, int n, int& i0, Q& w)
{
    f = f < Q(0) ? Q(0) : (f > Q(n - 1) ? Q(n - 1) : f);
    int i = int(floor(f));
    i = i > n - 2 ? n - 2 : i;
    i = i < 0 ? 0 : i;
    i0 = i;
    w = n > 1 ? f - Q(i) : Q(0);
}

// Emission of the grid model at one point (J4, K7 as emission_synch).  f nullable.  ks
// (nullable): 1/r, F, Lx, Ly, Lz at the point, as the geodesic's right-hand side computed them
// (spares a division and the Kerr-Schild pieces of ks_point).
template <class Q>
ART_FM_DEV void emission_grid(const RayState<Q>& s, Q r, Q kt, const Q* f,
                                              const Q* ks, const DevJob& J,
                                              const SynchConstT<Q>& S, Q* J4, Q* K7,
                                              int* edge = nullptr)
{
    for (int i = 0; i < 4; ++i) J4[i] = Q(0);
    for (int i = 0; i < 7; ++i) K7[i] = Q(0);
    if (r < jq<Q>(J.r_in_stop, J.f_r_in_stop)) return;
    const Q lr = log_q<Q>(r);
    if (!(lr >= Q(S.g_x1min) && lr <= Q(S.g_x1max))) return;
    const Q a = jq<Q>(J.a, J.f_a), a2 = jq<Q>(J.a2, J.f_a2);
    const Q ir = ks ? ks[0] : Q(1) / r;
    Q ct = s.z * ir;
    ct = ct > Q(1) ? Q(1) : (ct < Q(-1) ? Q(-1) : ct);
    const Q th = acos(ct);
    const Q twopi = Q(6.283185307179586476925);
    // phi = arg(x + i y) + arg(r + i a) = arg((x + i y)(r + i a)): one arctangent, and its cosine
    // and sine from the product's parts instead of evaluating them (on the axis, x = y = 0, the
    // first argument is taken as 0)
    const Q px = fmad(s.x, r, -(s.y * a)), py = fmad(s.y, r, s.x * a);
    const Q pp = fmad(px, px, py * py);
    Q ph, sp, cp;
    if (pp > Q(0)) {
        ph = atan2(py, px);
        const Q ip = rsqrt(pp);
        cp = px * ip;
        sp = py * ip;
    } else {
        const Q ira = rsqrt(fmad(r, r, a2));
        ph = atan2(a, r);
        cp = r * ira;
        sp = a * ira;
    }
    if (ph < Q(0)) ph += twopi;
    if (ph >= twopi) ph -= twopi;
    const int n1 = S.g_n1, n2 = S.g_n2, n3 = S.g_n3;
    int i0, j0;
    Q w1, w2;
    grid_axis_clamped<Q>(fmad(lr - Q(S.g_x1min), Q(S.g_inv_dx1), Q(-0.5)), n1, i0, w1);
    grid_axis_clamped<Q>(fmad(th, Q(S.g_inv_dth), Q(-0.5)), n2, j0, w2);
    const int i1 = n1 > 1 ? i0 + 1 : i0, j1 = n2 > 1 ? j0 + 1 : j0;
    Q f3 = fmad(ph, Q(S.g_inv_dph), Q(-0.5));
    Q fl = floor(f3);
    Q w3 = f3 - fl;
    int k0 = int(fl);
    k0 = ((k0 % n3) + n3) % n3;
    const int k1 = k0 + 1 == n3 ? 0 : k0 + 1;
    Q P[8];
    // P = sum over the eight cells of weight x value; conv takes a cell value into Q and returns
    // whether it was one that widen does not cover
    auto trilinear = [&](auto conv) {
        unsigned special = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) P[q] = Q(0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int ii = (c & 1) ? i1 : i0, jj = (c & 2) ? j1 : j0, kk = (c & 4) ? k1 : k0;
            const Q wt = ((c & 1) ? w1 : Q(1) - w1) * ((c & 2) ? w2 : Q(1) - w2) *
                         ((c & 4) ? w3 : Q(1) - w3);
            const float4* cell = S.grid + 2 * (((int64_t)kk * n2 + jj) * n1 + ii);
            const float4 v0 = grid_load(cell), v1 = grid_load(cell + 1);
            P[0] = fmad(wt, conv(v0.x, special), P[0]);
            P[1] = fmad(wt, conv(v0.y, special), P[1]);
            P[2] = fmad(wt, conv(v0.z, special), P[2]);
            P[3] = fmad(wt, conv(v0.w, special), P[3]);
            P[4] = fmad(wt, conv(v1.x, special), P[4]);
            P[5] = fmad(wt, conv(v1.y, special), P[5]);
            P[6] = fmad(wt, conv(v1.z, special), P[6]);
            P[7] = fmad(wt, conv(v1.w, special), P[7]);
        }
        return special;
    };
    if constexpr (std::is_same<Q, double>::value) {
        // integer widening; a sample with a value it does not cover is summed again with the
        // conversion instruction (the same cells, still in L1)
        if (trilinear([](float v, unsigned& sp) {
                sp |= widen_special(v);
                return widen(v);
            }))
            trilinear([](float v, unsigned&) { return (double)v; });
    } else {
        trilinear([](float v, unsigned&) { return v; });
    }
    const Q rho = P[0], ug = P[1];
    if (!(rho > Q(0)) || !(ug > Q(0))) return;
    // d(x, y, z)/d(r, theta, phi) of x + i y = (r - i a) sin(theta) e^{i phi}, z = r cos(theta)
    const Q st = sqrt(Q(1) - ct * ct);
    const Q Jm[3][3] = {{st * cp, ct * fmad(r, cp, a * sp), -s.y},
                        {st * sp, ct * fmad(r, sp, -(a * cp)), s.x},
                        {ct, -r * st, Q(0)}};
    Q u[4], B[4];
    u[0] = B[0] = Q(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        u[1 + i] = fmad(Jm[i][2], P[4], fmad(Jm[i][1], P[3], Jm[i][0] * P[2]));
        B[1 + i] = fmad(Jm[i][2], P[7], fmad(Jm[i][1], P[6], Jm[i][0] * P[5]));
    }
    KSPoint<Q> G;
    if (ks) {
        G.F = ks[1];
        G.Lx = ks[2];
        G.Ly = ks[3];
        G.Lz = ks[4];
    } else {
        G = ks_point<Q>(s.x, s.y, s.z, r, ir, a, a2);
    }
    const Q Lu = fmad(G.Lz, u[3], fmad(G.Ly, u[2], G.Lx * u[1]));
    const Q LB = fmad(G.Lz, B[3], fmad(G.Ly, B[2], G.Lx * B[1]));
    const Q uu = fmad(u[3], u[3], fmad(u[2], u[2], u[1] * u[1]));
    const Q qn = fmad(G.F * Lu, Lu, Q(1) + uu);
    const Q pn = -G.F * Lu;
    const Q D = fmad(pn, pn, -((G.F - Q(1)) * qn));
    if (!(D >= Q(0))) return;
    const Q den = sqrt(D) - pn;
    if (!(den > Q(0))) return;
    // u^t = qn / den and 1/u^t = den / qn from one reciprocal
    const Q iqd = Q(1) / (qn * den);
    u[0] = qn * qn * iqd;
    const Q Bu = fmad(B[3], u[3], fmad(B[2], u[2], B[1] * u[1]));
    Q b[4];
    b[0] = fmad(G.F * LB, Lu - u[0], Bu);
    const Q iut = den * den * iqd;
#pragma unroll
    for (int i = 1; i < 4; ++i) b[i] = fmad(b[0], u[i], B[i]) * iut;
    // b^mu b_mu = (g_ij B^i B^j + (b^t)^2) / (u^t)^2 (from b^mu = (B^mu + b^t u^mu)/u^t and
    // u.u = -1): two positive terms, where the four-vector contraction -(b^t)^2 + ... cancels
    // (by whole factors in FP32 for fast flows, which then moved points across the sigma cut)
    const Q BB = fmad(B[3], B[3], fmad(B[2], B[2], B[1] * B[1]));
    const Q b2 = fmad(b[0], b[0], fmad(G.F * LB, LB, BB)) * (iut * iut);
    if (!(b2 > Q(0))) return;
    // a sample within rounding of the cut may keep or lose its emission in another precision
    if (edge && S.e_sig > Q(0) &&
        fabs(b2 - Q(S.g_sigma_cut) * rho) < Q(S.e_sig) * Q(S.g_sigma_cut) * rho)
        *edge = 1;
    if (b2 > Q(S.g_sigma_cut) * rho) return;
    const Q pg = Q(S.g_gm1) * ug, pm = Q(0.5) * b2;
    const Q pg2 = pg * pg, pm2 = pm * pm;
    Q Th, iTh;
    if constexpr (std::is_same<Q, double>::value) {
        // Theta_e = nm / dn and its reciprocal from one division: with s2 = pg^2 + pm^2,
        // nm = th_unit u s2, dn = rho (s2 + r_high pg^2 + r_low pm^2) (T_i/T_e = (dn/rho - s2)/s2)
        const Q s2 = pg2 + pm2;
        const Q nm = Q(S.g_th_unit) * ug * s2;
        const Q dn = rho * (s2 + fmad(Q(S.g_r_high), pg2, Q(S.g_r_low) * pm2));
        const Q inv = Q(1) / (nm * dn);
        Th = nm * nm * inv;
        iTh = dn * dn * inv;
    } else {
        // (single precision: nm dn can leave the range; its divisions are cheap)
        const Q trat = fmad(Q(S.g_r_high), pg2, Q(S.g_r_low) * pm2) / (pg2 + pm2);
        Th = Q(S.g_th_unit) * ug / (rho * (Q(1) + trat));
        iTh = Q(1) / Th;
    }
    const Q ne = Q(S.g_ne_unit) * rho;
    const Q ib = rsqrt(b2);
    const Q bm = b2 * ib;
    const Q Bm = Q(S.g_b_unit) * bm;
#pragma unroll
    for (int m = 0; m < 4; ++m) b[m] *= ib;
    const Q nu = fmad(s.kz, u[3], fmad(s.ky, u[2], fmad(s.kx, u[1], kt * u[0])));
    if (!(nu > Q(0))) return;
    synch_coeffs<Q>(G, s, kt, u, b, nu, ne, Th, iTh, Bm, f, S, J4, K7);
}

}  // namespace art
