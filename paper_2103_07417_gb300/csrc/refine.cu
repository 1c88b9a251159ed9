// refine.cu -- the adaptive-refinement kernels of Sec. 3.2: base-grid queue, I_bar_int, the fused
// criterion + interpolation + ray-queue compaction of one level, the truth gather (refinement
// run on a precomputed image) and the image metrics of Sec. 4.1.
//
// Layout: the image is the final nodal grid (planes x ny x nx doubles).  Level k points are the
// sub-lattice of stride s = 2^(N-k); a point is new at level k when (i/s, j/s) are not both even,
// and it reads only level-(k-1) points (stride 2s).  So no per-level copies exist and the new
// points of a level never read each other: one kernel per level decides, interpolates and
// compacts the rays to trace into the queue.  All of it is HBM/L2-bound stencil work.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace art {

// --------------------------------------------------------------------------------------------
// level 0
// --------------------------------------------------------------------------------------------

__global__ void enqueue_base_kernel(DevJob J, int32_t* queue, unsigned long long* counters)
{
    const int S0 = 1 << J.levels;
    const int n0x = (J.nx - 1) / S0 + 1, n0y = (J.ny - 1) / S0 + 1;
    const int64_t n = (int64_t)n0x * n0y;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        int ii = (int)(q % n0x), jj = (int)(q / n0x);
        queue[q] = jj * S0 * J.nx + ii * S0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counters[C_QUEUE] = (unsigned long long)n;
        counters[C_LEVEL0] = (unsigned long long)n;
    }
}

cudaError_t launch_enqueue_base(const DevJob& J, int32_t* queue, unsigned long long* counters,
                                cudaStream_t st)
{
    const int S0 = 1 << J.levels;
    int64_t n = (int64_t)((J.nx - 1) / S0 + 1) * ((J.ny - 1) / S0 + 1);
    int grid = (int)((n + 255) / 256);
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    enqueue_base_kernel<<<grid, 256, 0, st>>>(J, queue, counters);
    return cudaGetLastError();
}

// Refinement on a precomputed image: "tracing" a queued pixel copies it from `truth`.
__global__ void gather_truth_kernel(int planes, int64_t npix, const int32_t* queue,
                                    const unsigned long long* count, const double* truth,
                                    double* img, uint8_t* mask)
{
    const unsigned long long n = *count;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        int32_t p = queue[q];
        if (p < 0 || p >= npix) continue;
        for (int c = 0; c < planes; ++c) img[c * npix + p] = truth[c * npix + p];
        if (mask) mask[p] = ART_MASK_TRACED;
    }
}

cudaError_t launch_gather_truth(const DevJob& J, const int32_t* queue,
                                const unsigned long long* count, const double* truth,
                                double* img, uint8_t* mask, int64_t cap, cudaStream_t st)
{
    int grid = (int)((cap + 255) / 256);
    if (grid < 1) grid = 1;
    if (grid > 8192) grid = 8192;
    gather_truth_kernel<<<grid, 256, 0, st>>>(J.planes, (int64_t)J.nx * J.ny, queue, count, truth,
                                              img, mask);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------------
// I_bar_int: mean of the bilinear interpolant of the base samples = trapezoid weights
// (1/2 on the edges of each axis); one block, fixed reduction order (deterministic).
// norm3[0] = the criterion's normalisation (I_bar_int or the peak), [1] = I_bar_int, [2] = peak.
// --------------------------------------------------------------------------------------------

constexpr int NORM_THREADS = 1024;

__global__ void __launch_bounds__(NORM_THREADS)
    norm_kernel(const double* img, int nx, int ny, int stride, int abs_norm, double* norm3)
{
    const int n0x = (nx - 1) / stride + 1, n0y = (ny - 1) / stride + 1;
    const int64_t n = (int64_t)n0x * n0y;
    double s = 0.0, w = 0.0, mx = -INFINITY;
    for (int64_t q = threadIdx.x; q < n; q += NORM_THREADS) {
        int ii = (int)(q % n0x), jj = (int)(q / n0x);
        double wx = (n0x > 1 && (ii == 0 || ii == n0x - 1)) ? 0.5 : 1.0;
        double wy = (n0y > 1 && (jj == 0 || jj == n0y - 1)) ? 0.5 : 1.0;
        double v = img[(int64_t)jj * stride * nx + (int64_t)ii * stride];
        s += wx * wy * v;
        w += wx * wy;
        mx = fmax(mx, v);
    }
    __shared__ double ss[NORM_THREADS], sw[NORM_THREADS], sm[NORM_THREADS];
    ss[threadIdx.x] = s;
    sw[threadIdx.x] = w;
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int h = NORM_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            ss[threadIdx.x] += ss[threadIdx.x + h];
            sw[threadIdx.x] += sw[threadIdx.x + h];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double ibar = ss[0] / sw[0];
        norm3[1] = ibar;
        norm3[2] = sm[0];
        norm3[0] = abs_norm == ART_NORM_PEAK ? sm[0] : ibar;
    }
}

cudaError_t launch_norm(const DevJob& J, const double* img, int nx, int ny, int stride,
                        double* norm3, cudaStream_t st)
{
    norm_kernel<<<1, NORM_THREADS, 0, st>>>(img, nx, ny, stride, J.abs_norm, norm3);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------------
// criterion + interpolation + compaction of one level
// --------------------------------------------------------------------------------------------

// High-word FP32 value of a double; ok = false for |x| >= 2^128, infinities and NaN.
__device__ __forceinline__ float hiword_f32(double x, bool& ok)
{
    const int hi = __double2hiint(x);
    const int e = (hi >> 20) & 0x7ff;
    if (e > 1150) {
        ok = false;
        return 0.f;
    }
    if (e < 897) return 0.f;
    return __int_as_float((hi & 0x80000000) | ((e - 896) << 23) | ((hi & 0xfffff) << 3));
}

// Where the stencil functions below read the criterion plane (fine-grid coordinates i, j of a
// point of the coarser lattice): straight from the image (GlobalSrc), or from a block's shared-
// memory tile of that lattice (TileSrc, the level kernel).  Both hold the image's own doubles, so
// every decision and interpolant is the same bits either way.
template <class IX>
struct GlobalSrc {
    const double* img;  // the criterion plane
    int nx;
    __device__ __forceinline__ double at(int i, int j) const { return __ldg(img + (IX)j * nx + i); }
    __device__ __forceinline__ float at_f(int i, int j, bool& ok) const
    {
        return hiword_f32(at(i, j), ok);
    }
    __device__ __forceinline__ const double* plane() const { return img; }
};

// Sum of the two central second differences along one line through the point (inner
// neighbours at -/+ d, outer at -/+ 3d): I(-3) - I(-1) - I(+1) + I(+3); where one outer point is
// outside the image, twice the one second difference available; where none is, ok = false.
template <class Src>
__device__ __forceinline__ double second_diff_sum(const Src& V, int nx, int ny, int i, int j,
                                                  int di, int dj, double Im, double Ip, bool& ok)
{
    const int iom = i - 3 * di, jom = j - 3 * dj, iop = i + 3 * di, jop = j + 3 * dj;
    const bool has_m = iom >= 0 && iom < nx && jom >= 0 && jom < ny;
    const bool has_p = iop >= 0 && iop < nx && jop >= 0 && jop < ny;
    if (has_m && has_p) {
        double Om = V.at(iom, jom), Op = V.at(iop, jop);
        return ((Om - Im) - Ip) + Op;
    }
    if (has_m) return 2.0 * ((V.at(iom, jom) - 2.0 * Im) + Ip);
    if (has_p) return 2.0 * ((V.at(iop, jop) - 2.0 * Ip) + Im);
    ok = false;
    return 0.0;
}

// Estimated errors of Eqs. (epabs), (eprel), Appendix A, for the new point (i, j) of the level
// with stride s.  Linear: eps_abs = |S_out - S_in| / (16 norm) [centre] or / (8 norm) [edge
// midpoints, the 1-D form], eps_rel = |S_out - S_in| / (4 |S_in|), interpolant S_in/4 or S_in/2.
// Nearest: sqrt(((I4-I1)/2)^2 + ((I3-I2)/2)^2) [centre] or |I2-I1|/2 [midpoints] over norm and
// over |I1|, interpolant I1.  Decision: trace iff eps_abs > R_abs && eps_rel > R_rel (strict);
// NaN traces; a line without any outer point gives +inf.
template <class IX, class Src>
__device__ __forceinline__ bool decide(const DevJob& J, const Src& V, int i, int j, int s,
                                      double norm, int cat, double& w1, double& w2, IX& p1, IX& p2,
                                      IX& p3, IX& p4, double& ea, double& er)
{
    const double* img = V.plane();
    const int nx = J.nx, ny = J.ny;
    bool ok = true;
    double num, sin_, i1, den;
    if (cat == 4) {
        p1 = (IX)(j - s) * nx + (i - s);  // point 1
        p4 = (IX)(j + s) * nx + (i + s);  // point 4 (opposite 1)
        p2 = (IX)(j + s) * nx + (i - s);  // point 2
        p3 = (IX)(j - s) * nx + (i + s);  // point 3 (opposite 2)
        double I1 = V.at(i - s, j - s), I4 = V.at(i + s, j + s), I2 = V.at(i - s, j + s),
               I3 = V.at(i + s, j - s);
        sin_ = ((I1 + I2) + I3) + I4;
        i1 = I1;
        if (J.interp == ART_INTERP_NEAREST) {
            double d41 = I4 - I1, d32 = I3 - I2;
            num = sqrt(__dadd_rn(__dmul_rn(__dmul_rn(0.25, d41), d41), __dmul_rn(__dmul_rn(0.25, d32), d32)));
            w1 = 1.0;
            w2 = 0.0;
            den = fabs(i1);
        } else {
            double dA = second_diff_sum(V, nx, ny, i, j, s, s, I1, I4, ok);
            double dB = second_diff_sum(V, nx, ny, i, j, s, -s, I2, I3, ok);
            num = fabs(dA + dB) / 16.0;
            w1 = 0.25;
            w2 = 0.25;
            den = fabs(sin_) / 4.0;
        }
    } else {
        const int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
        p1 = (IX)(j - dj) * nx + (i - di);
        p2 = (IX)(j + dj) * nx + (i + di);
        p3 = p4 = -1;
        double I1 = V.at(i - di, j - dj), I2 = V.at(i + di, j + dj);
        sin_ = I1 + I2;
        i1 = I1;
        if (J.interp == ART_INTERP_NEAREST) {
            num = fabs(I2 - I1) / 2.0;
            w1 = 1.0;
            w2 = 0.0;
            den = fabs(i1);
        } else {
            double d = second_diff_sum(V, nx, ny, i, j, di, dj, I1, I2, ok);
            num = fabs(d) / 8.0;
            w1 = 0.5;
            w2 = 0.5;
            den = fabs(sin_) / 2.0;
        }
    }
    if (!ok && J.interp == ART_INTERP_LINEAR) {
        ea = er = INFINITY;
    } else {
        ea = num / norm;
        er = (den == 0.0) ? (num == 0.0 ? 0.0 : INFINITY) : num / den;
    }
    bool tr = (ea > J.R_abs) && (er > J.R_rel);
    if (isnan(ea) || isnan(er) || isnan(sin_) || isnan(i1)) tr = true;
    if (!tr && J.criterion == ART_CRIT_STOKES_ANY && J.stokes == 4) {
        // Sec. 6, "replacing I by Q, U, V": Q, U and V each through the same estimator (same
        // stencil and divisors), eps_abs over the same normalisation, eps_rel over I's
        // denominator (Q, U, V may vanish or change sign); the point is traced if any asks
        const int64_t npix = (int64_t)nx * ny;
        for (int c = 1; c < 4 && !tr; ++c) {
            const double* pl = img + c * npix;
            const GlobalSrc<IX> P{pl, nx};
            double nc;
            if (cat == 4) {
                const double I1 = __ldg(pl + p1), I4 = __ldg(pl + p4), I2 = __ldg(pl + p2),
                             I3 = __ldg(pl + p3);
                if (J.interp == ART_INTERP_NEAREST) {
                    const double d41 = I4 - I1, d32 = I3 - I2;
                    nc = sqrt(__dadd_rn(__dmul_rn(__dmul_rn(0.25, d41), d41),
                                        __dmul_rn(__dmul_rn(0.25, d32), d32)));
                } else {
                    bool okc = true;
                    const double dA = second_diff_sum(P, nx, ny, i, j, s, s, I1, I4, okc);
                    const double dB = second_diff_sum(P, nx, ny, i, j, s, -s, I2, I3, okc);
                    nc = fabs(dA + dB) / 16.0;
                }
            } else {
                const int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
                const double I1 = __ldg(pl + p1), I2 = __ldg(pl + p2);
                if (J.interp == ART_INTERP_NEAREST) {
                    nc = fabs(I2 - I1) / 2.0;
                } else {
                    bool okc = true;
                    nc = fabs(second_diff_sum(P, nx, ny, i, j, di, dj, I1, I2, okc)) / 8.0;
                }
            }
            const double eac = nc / norm;
            const double erc = (den == 0.0) ? (nc == 0.0 ? 0.0 : INFINITY) : nc / den;
            tr = (eac > J.R_abs && erc > J.R_rel) || isnan(eac) || isnan(erc);
        }
    }
    if (J.edge_mode == ART_EDGE_TRACE) {
        const int di = (cat == 2) ? 0 : s, dj = (cat == 3) ? 0 : s;
        if (i - 3 * di < 0 || i + 3 * di >= nx || j - 3 * dj < 0 || j + 3 * dj >= ny) tr = true;
    }
    return tr;
}

// ---- FP32 screen of the linear criterion ------------------------------------------------------
// GB300 issues FP64 at 1/64 of the FP32 rate, and a decision in FP64 (two divisions plus the
// stencil sums) made this HBM-bound pass FP64-bound.  The screen evaluates the same sums in FP32
// from the high words of the doubles with a rigorous error bound and decides only where the
// estimate clears both thresholds by more than that bound; every other point (and every point
// of the nearest-neighbour scheme, of a non-positive or non-finite normalisation, or with a value
// outside the FP32 range) takes the FP64 decision above, so the decisions are those of decide()
// for every point.
//   Value: the double's high word gives sign, exponent and 20 mantissa bits, a truncation with
//   relative error < 2^-20; magnitudes below 2^-126 are taken as 0 (absolute error < 2^-126).
//   Sums of c_k v_k in FP32 (|c_k| <= 4, at most 8 operations): |error| <= 2^-19 C + 2^-120 with
//   C = sum |c_k v_k|; the screen uses twice that.
// Linear scheme, X = |S_out - S_in| (the sum of the available second differences): eps_abs >
// R_abs <=> X > 16 R_abs norm (centre) or 8 R_abs norm (edge midpoints); eps_rel > R_rel <=>
// X > 4 R_rel |S_in| in both cases.
struct Screen {
    float tabs4, tabs2, rrel4;
    float bup, bdn;         // 1 +/- the band of the exact-decision mode (1, 1 otherwise)
    bool abs_any, rel_any;  // negative tolerance: every estimate exceeds it
    bool on;
};

__device__ __forceinline__ Screen make_screen(const DevJob& J, double norm, double band = 0.0)
{
    Screen sc;
    sc.bup = (float)(1.0 + band);
    sc.bdn = (float)(1.0 - band);
    sc.on = J.interp == ART_INTERP_LINEAR && norm > 0.0 && norm < 1e300 &&
            !(J.criterion == ART_CRIT_STOKES_ANY && J.stokes == 4);
    sc.abs_any = J.R_abs < 0.0;
    sc.rel_any = J.R_rel < 0.0;
    const double t4 = 16.0 * J.R_abs * norm, t2 = 8.0 * J.R_abs * norm, r4 = 4.0 * J.R_rel;
    // thresholds must be zero or normal FP32 numbers
    auto fits = [](double v) { double m = fabs(v); return m == 0.0 || (m > 1e-37 && m < 1e37); };
    if (!sc.abs_any && !(fits(t4) && fits(t2))) sc.on = false;
    if (!sc.rel_any && !fits(r4)) sc.on = false;
    sc.tabs4 = (float)t4;
    sc.tabs2 = (float)t2;
    sc.rrel4 = (float)r4;
    return sc;
}

// FP32 second-difference sum along one line (as second_diff_sum) and its sum of |c_k v_k|.
template <class Src>
__device__ __forceinline__ float second_diff_f(const Src& V, int nx, int ny, int i, int j,
                                               int di, int dj, float Im, float Ip, float& C,
                                               bool& ok)
{
    const int iom = i - 3 * di, jom = j - 3 * dj, iop = i + 3 * di, jop = j + 3 * dj;
    const bool has_m = iom >= 0 && iom < nx && jom >= 0 && jom < ny;
    const bool has_p = iop >= 0 && iop < nx && jop >= 0 && jop < ny;
    if (has_m && has_p) {
        float Om = V.at_f(iom, jom, ok);
        float Op = V.at_f(iop, jop, ok);
        C += ((fabsf(Om) + fabsf(Im)) + fabsf(Ip)) + fabsf(Op);
        return ((Om - Im) - Ip) + Op;
    }
    if (has_m) {
        float Om = V.at_f(iom, jom, ok);
        C += 2.f * fabsf(Om) + 4.f * fabsf(Im) + 2.f * fabsf(Ip);
        return 2.f * ((Om - 2.f * Im) + Ip);
    }
    if (has_p) {
        float Op = V.at_f(iop, jop, ok);
        C += 2.f * fabsf(Op) + 4.f * fabsf(Ip) + 2.f * fabsf(Im);
        return 2.f * ((Op - 2.f * Ip) + Im);
    }
    ok = false;
    return 0.f;
}

// Screened decision: 1 = trace, 0 = interpolate, -1 = undecided (take the FP64 decision).
template <class Src>
__device__ __forceinline__ int screen_decide(const Screen& sc, const Src& V, int nx, int ny,
                                             int i, int j, int s, int cat)
{
    if (!sc.on) return -1;
    bool ok = true;
    float X, C = 0.f, Sin, Cin;
    float tabs;
    if (cat == 4) {
        float I1 = V.at_f(i - s, j - s, ok);
        float I4 = V.at_f(i + s, j + s, ok);
        float I2 = V.at_f(i - s, j + s, ok);
        float I3 = V.at_f(i + s, j - s, ok);
        Sin = ((I1 + I2) + I3) + I4;
        Cin = ((fabsf(I1) + fabsf(I2)) + fabsf(I3)) + fabsf(I4);
        float dA = second_diff_f(V, nx, ny, i, j, s, s, I1, I4, C, ok);
        float dB = second_diff_f(V, nx, ny, i, j, s, -s, I2, I3, C, ok);
        X = fabsf(dA + dB);
        tabs = sc.tabs4;
    } else {
        const int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
        float I1 = V.at_f(i - di, j - dj, ok);
        float I2 = V.at_f(i + di, j + dj, ok);
        Sin = I1 + I2;
        Cin = fabsf(I1) + fabsf(I2);
        X = fabsf(second_diff_f(V, nx, ny, i, j, di, dj, I1, I2, C, ok));
        tabs = sc.tabs2;
    }
    if (!ok) return -1;
    const float E = 0x1p-18f * C + 0x1p-118f;
    const float Es = 0x1p-18f * Cin + 0x1p-118f;
    const float up = (1.f + 0x1p-18f) * sc.bup, dn = (1.f - 0x1p-18f) * sc.bdn;
    bool abs_t, abs_f, rel_t, rel_f;
    if (sc.abs_any) {
        abs_t = true;
        abs_f = false;
    } else {
        abs_t = X - E > tabs * up;
        abs_f = X + E < tabs * dn;
    }
    if (sc.rel_any) {
        rel_t = true;
        rel_f = false;
    } else {
        const float lo = fabsf(Sin) - Es, hi = fabsf(Sin) + Es;
        rel_t = X - E > sc.rrel4 * hi * up;
        rel_f = lo > 0.f && X + E < sc.rrel4 * lo * dn;
    }
    if (abs_f || rel_f) return 0;
    if (abs_t && rel_t) return 1;
    return -1;
}

// Whether the linear scheme's whole stencil of a point (parents and outer points) holds one finite
// value, bit for bit, with every outer point inside the image: then both second differences are
// exactly 0, eps_abs = 0 / norm = 0 for a positive finite norm, and with R_abs >= 0 the FP64
// decision is "interpolate" whatever R_rel is.  The dark background of a wide field takes this
// exit on the integer pipes.
template <class Src>
__device__ __forceinline__ bool uniform_stencil(const Src& V, int nx, int ny, int i, int j,
                                                int s, int cat)
{
    int di1, dj1, di2 = 0, dj2 = 0;  // the one or two lines of the stencil
    if (cat == 4) {
        di1 = s; dj1 = s; di2 = s; dj2 = -s;
    } else {
        di1 = (cat == 3) ? s : 0;
        dj1 = (cat == 2) ? s : 0;
    }
    const int ri = 3 * (di1 > di2 ? di1 : di2), rj = 3 * s * (cat != 3);
    if (i - ri < 0 || i + ri >= nx || j - rj < 0 || j + rj >= ny) return false;
    const long long v = __double_as_longlong(V.at(i - di1, j - dj1));
    if (((v >> 52) & 0x7ff) == 0x7ff) return false;
    auto same = [&](int ii, int jj) { return __double_as_longlong(V.at(ii, jj)) == v; };
    if (!same(i + di1, j + dj1) || !same(i - 3 * di1, j - 3 * dj1) || !same(i + 3 * di1, j + 3 * dj1))
        return false;
    if (cat == 4 && (!same(i - di2, j - dj2) || !same(i + di2, j + dj2) ||
                     !same(i - 3 * di2, j - 3 * dj2) || !same(i + 3 * di2, j + 3 * dj2)))
        return false;
    return true;
}

// v * 2^-k (k = 1, 2), bit-identical to the FP64 product: for a normal v whose result stays
// normal the product only lowers the exponent, done here on the integer pipes (GB300's FP64 pipe
// issues 2 operations per SM and cycle); zeros, subnormal results, infinities and NaN multiply.
__device__ __forceinline__ double scale_pow2(double v, int k)
{
    const int hi = __double2hiint(v), lo = __double2loint(v);
    const int e = (hi >> 20) & 0x7ff;
    if (e > k && e < 0x7ff) return __hiloint2double(hi - (k << 20), lo);
    return v * (k == 1 ? 0.5 : 0.25);
}

// Stencil of the interpolant of a new point (the points decide() names 1..4; nearest: point 1).
template <class IX>
__device__ __forceinline__ void interp_parents(int nx, int i, int j, int s, int cat, IX& p1, IX& p2,
                                               IX& p3, IX& p4)
{
    if (cat == 4) {
        p1 = (IX)(j - s) * nx + (i - s);
        p4 = (IX)(j + s) * nx + (i + s);
        p2 = (IX)(j + s) * nx + (i - s);
        p3 = (IX)(j - s) * nx + (i + s);
    } else {
        const int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
        p1 = (IX)(j - dj) * nx + (i - di);
        p2 = (IX)(j + dj) * nx + (i + di);
        p3 = p4 = -1;
    }
}

// The interpolant of a new point in every plane (linear: mean of the 2 or 4 parents; nearest:
// point 1).  The one definition used by the criterion pass and by the exact-decision passes, so
// that an interpolant recomputed from the same parents is the same bits.
template <class IX>
__device__ __forceinline__ void write_interp(const DevJob& J, double* img, IX pix, IX p1, IX p2,
                                             IX p3, IX p4, int cat, int64_t npix)
{
    const bool nearest = J.interp == ART_INTERP_NEAREST;
    for (int c = 0; c < J.planes; ++c) {
        const double* pl = img + c * npix;
        double v;
        if (nearest) {
            v = __ldg(pl + p1);
        } else if (cat == 4) {
            const double v1 = __ldg(pl + p1), v2 = __ldg(pl + p2), v3 = __ldg(pl + p3),
                         v4 = __ldg(pl + p4);
            const long long b1 = __double_as_longlong(v1);
            // equal parents (the dark background): ((v + v) + v) + v = 4 v and 4 v / 4 = v exactly
            // (|v| < 2^1021: no overflow; NaN stays NaN); compared on the bits, which spares the
            // FP64 pipe
            if (b1 == __double_as_longlong(v2) && b1 == __double_as_longlong(v3) &&
                b1 == __double_as_longlong(v4) && ((b1 >> 52) & 0x7ff) < 0x7fc)
                v = v1;
            else
                v = scale_pow2(((v1 + v2) + v3) + v4, 2);
        } else {
            const double v1 = __ldg(pl + p1), v2 = __ldg(pl + p2);
            const long long b1 = __double_as_longlong(v1);
            if (b1 == __double_as_longlong(v2) && ((b1 >> 52) & 0x7ff) < 0x7fc)
                v = v1;  // (v + v) / 2 = v exactly
            else
                v = scale_pow2(v1 + v2, 1);
        }
        img[c * npix + pix] = v;
    }
}

// write_interp for a one-plane image, the parents read through V: the same operations on the
// same values, so the same bits.
template <class Src>
__device__ __forceinline__ void write_interp_v(const DevJob& J, const Src& V, double* out, int i,
                                               int j, int s, int cat)
{
    double v;
    if (cat == 4) {
        const double v1 = V.at(i - s, j - s);
        if (J.interp == ART_INTERP_NEAREST) {
            *out = v1;
            return;
        }
        const double v2 = V.at(i - s, j + s), v3 = V.at(i + s, j - s), v4 = V.at(i + s, j + s);
        const long long b1 = __double_as_longlong(v1);
        if (b1 == __double_as_longlong(v2) && b1 == __double_as_longlong(v3) &&
            b1 == __double_as_longlong(v4) && ((b1 >> 52) & 0x7ff) < 0x7fc)
            v = v1;
        else
            v = scale_pow2(((v1 + v2) + v3) + v4, 2);
    } else {
        const int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
        const double v1 = V.at(i - di, j - dj);
        if (J.interp == ART_INTERP_NEAREST) {
            *out = v1;
            return;
        }
        const double v2 = V.at(i + di, j + dj);
        const long long b1 = __double_as_longlong(v1);
        if (b1 == __double_as_longlong(v2) && ((b1 >> 52) & 0x7ff) < 0x7fc)
            v = v1;
        else
            v = scale_pow2(v1 + v2, 1);
    }
    *out = v;
}

// Exact-decision mode (ART_MIXED_EXACT): per-pixel exactness bytes, the borderline list and the
// band within which an FP64 decision on FP32-traced values is not trusted.
struct CertArgs {
    uint8_t* xst;
    double band;
};

// Whether every value decide() reads for the point (parents, and for the linear scheme the outer
// points inside the image) is exact.
__device__ __forceinline__ bool stencil_exact(const DevJob& J, const uint8_t* xst, int i, int j,
                                              int s, int cat)
{
    const int nx = J.nx, ny = J.ny;
    auto ex = [&](int ii, int jj) {
        if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) return true;  // outside: not read
        return (xst[(int64_t)jj * nx + ii] & XS_EXACT) != 0;
    };
    const bool lin = J.interp == ART_INTERP_LINEAR;
    if (cat == 4) {
        if (!ex(i - s, j - s) || !ex(i + s, j + s) || !ex(i - s, j + s) || !ex(i + s, j - s))
            return false;
        if (lin && (!ex(i - 3 * s, j - 3 * s) || !ex(i + 3 * s, j + 3 * s) ||
                    !ex(i - 3 * s, j + 3 * s) || !ex(i + 3 * s, j - 3 * s)))
            return false;
        return true;
    }
    const int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
    if (!ex(i - di, j - dj) || !ex(i + di, j + dj)) return false;
    if (lin && (!ex(i - 3 * di, j - 3 * dj) || !ex(i + 3 * di, j + 3 * dj))) return false;
    return true;
}

// Whether an FP64 decision on values with FP32 rounding in them can be trusted: every estimate
// that decides it clears its tolerance by the relative band.  Negative tolerances are exceeded by
// every estimate; infinite or NaN estimates trace whatever the values.
__device__ __forceinline__ bool decision_robust(const DevJob& J, double ea, double er, double band)
{
    if (!(ea == ea) || !(er == er) || isinf(ea) || isinf(er)) return true;
    const bool a_hi = J.R_abs < 0.0 || ea > J.R_abs * (1.0 + band);
    const bool r_hi = J.R_rel < 0.0 || er > J.R_rel * (1.0 + band);
    const bool a_lo = J.R_abs >= 0.0 && ea < J.R_abs * (1.0 - band);
    const bool r_lo = J.R_rel >= 0.0 && er < J.R_rel * (1.0 - band);
    return a_lo || r_lo || (a_hi && r_hi);
}

// One new point of a level: decide (screen, else FP64), then mark it for tracing or write its
// interpolant into every plane.  Returns 1 when the point is to be traced, 0 when interpolated.
// Learned path (spec = true): a point the criterion traces whose ray was already traced
// speculatively (mask MASK_SPEC_DONE) is marked traced and not queued again (return 2).
// Diagnostics planes (nullable) receive the mean of the interpolation parents.
// CERT (exact decisions): a decision within the band of a tolerance whose stencil is not all
// exact is left to the exact-decision passes (return 3, nothing written); an interpolated point
// whose parents are exact is marked exact.
// V reads the criterion plane (plane J.cplane of img).
template <class IX, bool CERT, class Src>
__device__ __forceinline__ int refine_point_s(const DevJob& J, const Screen& sc, const Src& V,
                                              double* img, uint8_t* mask, int i, int j, int s,
                                              int cat, double norm, int64_t npix, bool spec,
                                              float* aminr, float* aturn, const CertArgs* ca)
{
    double w1, w2;
    IX p1, p2, p3, p4;
    // a uniform stencil decides "interpolate" exactly; under CERT only where the tolerance
    // leaves room for rounding of the values (R_abs > 0)
    const bool flat = sc.on && !sc.abs_any && J.interp == ART_INTERP_LINEAR &&
                      (!CERT || J.R_abs > 0.0) && uniform_stencil(V, J.nx, J.ny, i, j, s, cat);
    const int scr = flat ? 0 : screen_decide(sc, V, J.nx, J.ny, i, j, s, cat);
    bool trace;
    if (scr < 0) {
        double ea, er;
        trace = decide<IX>(J, V, i, j, s, norm, cat, w1, w2, p1, p2, p3, p4, ea, er);
        if constexpr (CERT) {
            if (!decision_robust(J, ea, er, ca->band) && !stencil_exact(J, ca->xst, i, j, s, cat))
                return 3;
        }
    } else {
        trace = scr == 1;
        if (J.edge_mode == ART_EDGE_TRACE) {
            const int di = (cat == 2) ? 0 : s, dj = (cat == 3) ? 0 : s;
            if (i - 3 * di < 0 || i + 3 * di >= J.nx || j - 3 * dj < 0 || j + 3 * dj >= J.ny)
                trace = true;
        }
        interp_parents<IX>(J.nx, i, j, s, cat, p1, p2, p3, p4);
        w1 = w2 = 0.5;
    }
    const IX pix = (IX)j * J.nx + i;
    if (trace) {
        if (mask) {
            const bool done = spec && mask[pix] == MASK_SPEC_DONE;
            mask[pix] = ART_MASK_TRACED;
            if (done) return 2;
        }
        return 1;
    }
    if (aminr) {
        if (cat == 4) {
            aminr[pix] = 0.25f * (((aminr[p1] + aminr[p2]) + aminr[p3]) + aminr[p4]);
            aturn[pix] = 0.25f * (((aturn[p1] + aturn[p2]) + aturn[p3]) + aturn[p4]);
        } else {
            aminr[pix] = 0.5f * (aminr[p1] + aminr[p2]);
            aturn[pix] = 0.5f * (aturn[p1] + aturn[p2]);
        }
    }
    (void)w1;
    (void)w2;
    if (J.planes == 1)
        write_interp_v(J, V, img + pix, i, j, s, cat);
    else
        write_interp<IX>(J, img, pix, p1, p2, p3, p4, cat, npix);
    if (mask) mask[pix] = ART_MASK_INTERP;
    if constexpr (CERT) {
        const uint8_t* x = ca->xst;
        bool ex = (x[p1] & XS_EXACT) != 0;
        if (J.interp == ART_INTERP_LINEAR) {
            ex = ex && (x[p2] & XS_EXACT);
            if (cat == 4) ex = ex && (x[p3] & XS_EXACT) && (x[p4] & XS_EXACT);
        }
        // (a point traced speculatively in FP64 and interpolated after all loses its exactness
        // unless its parents are exact)
        ca->xst[pix] = ex ? XS_EXACT : 0;
    }
    return 0;
}

template <class IX, bool CERT = false>
__device__ __forceinline__ int refine_point(const DevJob& J, const Screen& sc, double* img,
                                            uint8_t* mask, int i, int j, int s, int cat,
                                            double norm, int64_t npix, bool spec, float* aminr,
                                            float* aturn, const CertArgs* ca = nullptr)
{
    const GlobalSrc<IX> V{img + (IX)J.cplane * npix, J.nx};  // the plane the criterion reads
    return refine_point_s<IX, CERT>(J, sc, V, img, mask, i, j, s, cat, norm, npix, spec, aminr,
                                    aturn, ca);
}

// The level kernel works on tiles of the coarser (level k-1) lattice.  A block holds RT_X x RT_Y
// coarse cells, one per thread; a cell owns the (up to) three new points at its right edge
// midpoint (category 3), lower edge midpoint (2) and centre (4).  Their stencils reach one coarse
// point before and two after the tile along each axis, so the block first copies that
// (RT_X + 3) x (RT_Y + 3) window of the criterion plane into shared memory, once, with the FP32
// high words the screen reads beside it; every stencil value is then a shared-memory read
// instead of a global load per use (a coarse point is read by up to twelve stencils).
constexpr int RT_X = 32, RT_Y = 8;
constexpr int RT_HX = RT_X + 3, RT_HY = RT_Y + 3;

struct TileSrc {
    const double* v;    // [RT_HY][RT_HX] values of the criterion plane
    const float* f;     // their FP32 high words, NaN where hiword_f32 reports not ok
    const double* img;  // the criterion plane in global memory
    int sh, ox, oy;     // coarse index = fine >> sh; coarse index of v[0][0]
    __device__ __forceinline__ int idx(int i, int j) const
    {
        return ((j >> sh) - oy) * RT_HX + ((i >> sh) - ox);
    }
    __device__ __forceinline__ double at(int i, int j) const { return v[idx(i, j)]; }
    __device__ __forceinline__ float at_f(int i, int j, bool& ok) const
    {
        const float x = f[idx(i, j)];
        if (x != x) {
            ok = false;
            return 0.f;
        }
        return x;
    }
    __device__ __forceinline__ const double* plane() const { return img; }
};

// Copy the window of coarse points [X0 - 1, X0 + RT_X + 1] x [Y0 - 1, Y0 + RT_Y + 1] of the
// criterion plane and their FP32 high words into the block's tile (all threads take part).
__device__ __forceinline__ void load_refine_tile(const double* plane, int nx, int ncx, int ncy,
                                                 int sh, int X0, int Y0, double* tv, float* tf)
{
    for (int q = threadIdx.x; q < RT_HY * RT_HX; q += blockDim.x) {
        const int hy = q / RT_HX, hx = q - hy * RT_HX;
        const int cx = X0 - 1 + hx, cy = Y0 - 1 + hy;
        double v = 0.0;  // outside the lattice: never read (the stencils check the image edge)
        if (cx >= 0 && cx < ncx && cy >= 0 && cy < ncy)
            v = __ldg(plane + ((int64_t)cy << sh) * nx + ((int64_t)cx << sh));
        bool ok = true;
        const float f = hiword_f32(v, ok);
        tv[q] = v;
        tf[q] = ok ? f : __int_as_float(0x7fffffff);
    }
}

template <bool CERT>
__global__ void __launch_bounds__(RT_X * RT_Y)
    refine_kernel(DevJob J, int level, const double* __restrict__ norm_ptr, double* img,
                  uint8_t* mask, int32_t* queue, unsigned long long* qcount, float* aminr,
                  float* aturn, unsigned long long* counters, CertArgs ca, int32_t* border,
                  unsigned long long* cert_counters, unsigned long long border_cap)
{
    const int s = 1 << (J.levels - level);
    const int sh = J.levels - level + 1;  // coarse stride 2 s = 1 << sh
    const int ncx = (J.nx - 1) / (2 * s) + 1, ncy = (J.ny - 1) / (2 * s) + 1;
    const int64_t npix = (int64_t)J.nx * J.ny;
    const double* plane = img + (int64_t)J.cplane * npix;
    const double norm = *norm_ptr;
    // the screen's thresholds once per block: made per thread, the compiler recomputed their
    // FP64 products inside the loop (to save registers), which kept GB300's FP64 pipe 75 % busy
    __shared__ Screen sc_s;
    __shared__ double tv[RT_HY * RT_HX];
    __shared__ float tf[RT_HY * RT_HX];
    if (threadIdx.x == 0) sc_s = make_screen(J, norm, CERT ? ca.band : 0.0);
    const int lane = threadIdx.x & 31, tx = threadIdx.x % RT_X, ty = threadIdx.x / RT_X;
    // exact decisions on a degenerate image: every value is FP64 from here on, so a speculative
    // (FP32) ray the criterion asks for is traced again
    const bool spec_ok = counters != nullptr && !(CERT && cert_counters[C_DEGEN] != 0);
    const int X0 = blockIdx.x * RT_X;
    for (int Y0 = blockIdx.y * RT_Y; Y0 < ncy; Y0 += gridDim.y * RT_Y) {
        __syncthreads();  // the previous tile is read; the screen is written
        load_refine_tile(plane, J.nx, ncx, ncy, sh, X0, Y0, tv, tf);
        __syncthreads();
        const Screen sc = sc_s;
        const TileSrc V{tv, tf, plane, sh, X0 - 1, Y0 - 1};
        const int cx = X0 + tx, cy = Y0 + ty;
#pragma unroll 1
        for (int t = 0; t < 3; ++t) {
            const int oi = t != 1, oj = t != 0;  // t = 0: category 3, 1: category 2, 2: category 4
            const bool act = cx + oi < ncx && cy + oj < ncy;
            bool trace = false, used = false, bord = false;
            int32_t pix = 0;
            int i = 0, j = 0, cat = 0;
            if (act) {
                i = (2 * cx + oi) * s;
                j = (2 * cy + oj) * s;
                cat = (oi && oj) ? 4 : (oi ? 3 : 2);
                const int r = refine_point_s<int, CERT>(J, sc, V, img, mask, i, j, s, cat, norm,
                                                        npix, spec_ok, aminr, aturn, &ca);
                trace = r == 1;
                used = r == 2;
                bord = r == 3;
                pix = j * J.nx + i;
            }
            if constexpr (CERT) {
                // borderline points join the exact-decision list; where it is full they are
                // decided here after all (counted)
                const unsigned bb = __ballot_sync(0xffffffffu, bord);
                if (bb) {
                    unsigned long long w = 0;
                    if (lane == 0)
                        w = atomicAdd(cert_counters + C_BORDER, (unsigned long long)__popc(bb));
                    w = __shfl_sync(0xffffffffu, w, 0);
                    if (bord) {
                        const unsigned long long slot = w + __popc(bb & ((1u << lane) - 1u));
                        if (slot < border_cap) {
                            border[slot] = pix;
                            if (mask) mask[pix] = MASK_PENDING;
                        } else {
                            atomicAdd(cert_counters + C_CERTOVF, 1ull);
                            const int r = refine_point_s<int, false>(J, sc, V, img, mask, i, j, s,
                                                                     cat, norm, npix, spec_ok,
                                                                     aminr, aturn, nullptr);
                            trace = r == 1;
                            used = r == 2;
                            if (r == 0) ca.xst[pix] = 0;  // an interpolant of unchecked parents
                        }
                    }
                }
            }
            // warp-aggregated append to the ray queue (ballot -> popc -> one atomic per warp)
            const unsigned b = __ballot_sync(0xffffffffu, trace);
            if (b) {
                unsigned long long w = 0;
                if (lane == 0) w = atomicAdd(qcount, (unsigned long long)__popc(b));
                w = __shfl_sync(0xffffffffu, w, 0);
                if (trace) queue[w + __popc(b & ((1u << lane) - 1u))] = pix;
            }
            if (counters) {
                const unsigned u = __ballot_sync(0xffffffffu, used);
                if (u && lane == 0) {
                    atomicAdd(counters + C_SPECUSED, (unsigned long long)__popc(u));
                    atomicAdd(counters + C_LEVEL0 + level, (unsigned long long)__popc(u));
                }
            }
        }
    }
}

// Launch shape of the level kernel: the tiles of a row of the coarse lattice over blockIdx.x, its
// rows of tiles over blockIdx.y (a grid-stride loop past 65535).
static dim3 refine_tile_grid(const DevJob& J, int level)
{
    const int s = 1 << (J.levels - level);
    const int ncx = (J.nx - 1) / (2 * s) + 1, ncy = (J.ny - 1) / (2 * s) + 1;
    int gy = (ncy + RT_Y - 1) / RT_Y;
    if (gy > 65535) gy = 65535;
    return dim3((ncx + RT_X - 1) / RT_X, gy);
}

cudaError_t launch_refine(const DevJob& J, int level, const double* norm, double* img,
                          uint8_t* mask, int32_t* queue, unsigned long long* count,
                          cudaStream_t st, float* aux_minr, float* aux_turn,
                          unsigned long long* spec_counters)
{
    refine_kernel<false><<<refine_tile_grid(J, level), RT_X * RT_Y, 0, st>>>(
        J, level, norm, img, mask, queue, count, aux_minr, aux_turn, spec_counters,
        CertArgs{nullptr, 0.0}, nullptr, nullptr, 0);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------------
// Exact decisions (ART_MIXED_EXACT).  The FP32-traced values a decision reads differ from the FP64
// render's by rounding, so a decision whose estimates lie within a band of a tolerance may differ
// from the FP64 render's.  Those borderline points are decided here on exact values instead: the
// values their stencil reads are made exact (FP64 re-traces of FP32-traced points, recomputed
// interpolants of interpolated ones, down to exact values), then the point is decided in FP64.
// The base level is traced in FP64, so I_bar_int and every closure end in exact values.
// --------------------------------------------------------------------------------------------

cudaError_t launch_refine_cert(const DevJob& J, int level, const double* norm, double* img,
                               uint8_t* mask, int32_t* queue, unsigned long long* count,
                               cudaStream_t st, float* aux_minr, float* aux_turn,
                               unsigned long long* spec_counters, uint8_t* xst, double band,
                               int32_t* border, unsigned long long* counters,
                               unsigned long long border_cap)
{
    refine_kernel<true><<<refine_tile_grid(J, level), RT_X * RT_Y, 0, st>>>(
        J, level, norm, img, mask, queue, count, aux_minr, aux_turn, spec_counters,
        CertArgs{xst, band}, border, counters, border_cap);
    return cudaGetLastError();
}

// Level at which pixel (i, j) of the final grid is new (0: base lattice) and its stride there.
__device__ __forceinline__ int pixel_level(int i, int j, int N, int& s)
{
    int k = N;
    while (k > 0) {
        const int st = 1 << (N - k + 1);  // stride of level k - 1
        if ((i % st) != 0 || (j % st) != 0) break;
        --k;
    }
    s = 1 << (N - k);
    return k;
}

// Base lattice points are exact (traced in FP64).
__global__ void cert_mark_base_kernel(DevJob J, uint8_t* xst)
{
    const int S0 = 1 << J.levels;
    const int n0x = (J.nx - 1) / S0 + 1, n0y = (J.ny - 1) / S0 + 1;
    const int64_t n = (int64_t)n0x * n0y;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int ii = (int)(q % n0x), jj = (int)(q / n0x);
        xst[(int64_t)jj * S0 * J.nx + (int64_t)ii * S0] = XS_EXACT;
    }
}

// counters[C_SPECN] = counters[C_QUEUE] - counters[C_LEVEL0]: the speculative part of the base
// level's queue (band rays), traced in FP32 after the FP64 base rays.
__global__ void cert_spec_count_kernel(unsigned long long* counters)
{
    const unsigned long long q = counters[C_QUEUE], b = counters[C_LEVEL0];
    counters[C_SPECN] = q > b ? q - b : 0;
}

// Claim pixel p for the closure (true when this thread claimed it and it is not exact).
__device__ __forceinline__ bool cert_claim(uint8_t* xst, int64_t p)
{
    if (xst[p] & (XS_EXACT | XS_CLAIM)) return false;
    unsigned* w = reinterpret_cast<unsigned*>(xst + (p & ~(int64_t)3));
    const unsigned bit = (unsigned)XS_CLAIM << (8 * (int)(p & 3));
    const unsigned old = atomicOr(w, bit);
    const unsigned prev = (old >> (8 * (int)(p & 3))) & 0xffu;
    return (prev & (XS_EXACT | XS_CLAIM)) == 0;
}

constexpr int CERT_STACK = 96;

// Closure of the borderline points: every non-exact value their decision reads is claimed once;
// FP32-traced ones join the FP64 queue, interpolated ones the recompute list (with their level)
// and their own parents are searched in turn.  The borderline points themselves join the FP64
// queue too unless already traced in FP64 (traced speculatively: their decision may ask for
// them).
__global__ void cert_closure_kernel(DevJob J, const int32_t* border, const unsigned long long* counters_ro,
                                    unsigned long long* counters, uint8_t* xst, const uint8_t* mask,
                                    int32_t* xq, unsigned long long xq_cap, uint64_t* fixq,
                                    unsigned long long fix_cap, int level)
{
    const unsigned long long nb = counters_ro[C_BORDER];
    const int nx = J.nx, ny = J.ny, N = J.levels;
    const bool lin = J.interp == ART_INTERP_LINEAR;
    for (unsigned long long b = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; b < nb;
         b += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t p = border[b];
        if (!(xst[p] & XS_EXACT)) {  // not already traced in FP64 (a band ray)
            const unsigned long long w = atomicAdd(counters + C_XQ, 1ull);
            if (w < xq_cap) xq[w] = p;
            else atomicAdd(counters + C_CERTERR, 1ull);
        }
        int32_t stk[CERT_STACK];
        int top = 0;
        auto push = [&](int ii, int jj) {
            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) return;
            if (top < CERT_STACK) stk[top++] = jj * nx + ii;
            else atomicAdd(counters + C_CERTERR, 1ull);
        };
        // the stencil decide() reads at the borderline point's level
        const int i = p % nx, j = p / nx, s = 1 << (N - level);
        const int oi = (i / s) & 1, oj = (j / s) & 1;
        const int cat = (oi && oj) ? 4 : (oi ? 3 : 2);
        if (cat == 4) {
            push(i - s, j - s); push(i + s, j + s); push(i - s, j + s); push(i + s, j - s);
            if (lin) {
                push(i - 3 * s, j - 3 * s); push(i + 3 * s, j + 3 * s);
                push(i - 3 * s, j + 3 * s); push(i + 3 * s, j - 3 * s);
            }
        } else {
            const int di = (cat == 3) ? s : 0, dj = (cat == 2) ? s : 0;
            push(i - di, j - dj); push(i + di, j + dj);
            if (lin) { push(i - 3 * di, j - 3 * dj); push(i + 3 * di, j + 3 * dj); }
        }
        while (top > 0) {
            const int32_t q = stk[--top];
            if (!cert_claim(xst, q)) continue;
            if (mask[q] == ART_MASK_INTERP) {
                const int qi = q % nx, qj = q / nx;
                int qs;
                const int ql = pixel_level(qi, qj, N, qs);
                const unsigned long long w = atomicAdd(counters + C_FIXQ, 1ull);
                if (w < fix_cap) fixq[w] = ((uint64_t)ql << 32) | (uint32_t)q;
                else atomicAdd(counters + C_CERTERR, 1ull);
                const int qoi = (qi / qs) & 1, qoj = (qj / qs) & 1;
                const int qc = (qoi && qoj) ? 4 : (qoi ? 3 : 2);
                if (qc == 4) {
                    push(qi - qs, qj - qs);
                    if (lin) { push(qi + qs, qj + qs); push(qi - qs, qj + qs); push(qi + qs, qj - qs); }
                } else {
                    const int di = (qc == 3) ? qs : 0, dj = (qc == 2) ? qs : 0;
                    push(qi - di, qj - dj);
                    if (lin) push(qi + di, qj + dj);
                }
            } else {
                // traced in FP32 (or at a level with speculation): re-trace in FP64
                const unsigned long long w = atomicAdd(counters + C_XQ, 1ull);
                if (w < xq_cap) xq[w] = q;
                else atomicAdd(counters + C_CERTERR, 1ull);
            }
        }
    }
}

// After an FP64 pass: its pixels are exact; C_XRAYS counts them.
__global__ void cert_mark_traced_kernel(const int32_t* xq, unsigned long long* counters,
                                        unsigned long long xq_cap, uint8_t* xst, int count_idx)
{
    unsigned long long n = counters[count_idx];
    if (n > xq_cap) n = xq_cap;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x)
        xst[xq[q]] = XS_EXACT;
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[C_XRAYS] += n;
}

// An image whose normalisation lies far outside FP32's range (a plane that is dark at every
// base point, say) has tolerances that FP32-traced values cannot resolve: its later levels are
// traced in FP64 (C_DEGEN).
constexpr double CERT_NORM_MIN = 1e-25, CERT_NORM_MAX = 1e25;

__global__ void cert_check_norm_kernel(const double* norm3, unsigned long long* counters)
{
    const double n = fabs(norm3[0]);
    counters[C_DEGEN] = (n >= CERT_NORM_MIN && n <= CERT_NORM_MAX) ? 0ull : 1ull;
}

// The level's queue goes to the FP32 pass, or to the FP64 pass on a degenerate image.
__global__ void cert_split_kernel(unsigned long long* counters)
{
    const unsigned long long q = counters[C_QUEUE];
    const bool d = counters[C_DEGEN] != 0;
    counters[C_QF32] = d ? 0ull : q;
    counters[C_QF64] = d ? q : 0ull;
}

// Rays handed on to FP64 (slots of `queue` in the list, counters[count_idx] of them): a
// speculative one (slot at or beyond *spec_from) is left for its own level (mask unset); the
// others join the FP64 queue of this level's exact decisions.
__global__ void cert_take_uncertain_kernel(const int32_t* queue, const int32_t* reroute2,
                                           unsigned long long* counters, int count_idx,
                                           const unsigned long long* spec_from, uint8_t* mask,
                                           int32_t* xq, unsigned long long xq_cap)
{
    const unsigned long long n = counters[count_idx];
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t slot = reroute2[q];
        const int32_t p = queue[slot];
        if (spec_from && (unsigned long long)slot >= *spec_from) {
            mask[p] = ART_MASK_UNSET;
            continue;
        }
        const unsigned long long w = atomicAdd(counters + C_XQ, 1ull);
        if (w < xq_cap) xq[w] = p;
        else atomicAdd(counters + C_CERTERR, 1ull);
    }
}

cudaError_t launch_cert_take_uncertain(const int32_t* queue, const int32_t* reroute2,
                                       unsigned long long* counters, int count_idx,
                                       const unsigned long long* spec_from, uint8_t* mask,
                                       int32_t* xq, unsigned long long xq_cap, cudaStream_t st)
{
    cert_take_uncertain_kernel<<<64, 256, 0, st>>>(queue, reroute2, counters, count_idx,
                                                   spec_from, mask, xq, xq_cap);
    return cudaGetLastError();
}

cudaError_t launch_cert_check_norm(const double* norm3, unsigned long long* counters,
                                   cudaStream_t st)
{
    cert_check_norm_kernel<<<1, 1, 0, st>>>(norm3, counters);
    return cudaGetLastError();
}

cudaError_t launch_cert_split(unsigned long long* counters, cudaStream_t st)
{
    cert_split_kernel<<<1, 1, 0, st>>>(counters);
    return cudaGetLastError();
}

// Recompute the interpolants of the listed points of level `lvl` from their (now exact) parents.
__global__ void cert_fixup_kernel(DevJob J, const uint64_t* fixq, unsigned long long* counters,
                                  unsigned long long fix_cap, int lvl, double* img, uint8_t* xst)
{
    unsigned long long n = counters[C_FIXQ];
    if (n > fix_cap) n = fix_cap;
    const int64_t npix = (int64_t)J.nx * J.ny;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t e = fixq[q];
        if ((int)(e >> 32) != lvl) continue;
        const int32_t p = (int32_t)(e & 0xffffffffu);
        const int i = p % J.nx, j = p / J.nx, s = 1 << (J.levels - lvl);
        const int oi = (i / s) & 1, oj = (j / s) & 1;
        const int cat = (oi && oj) ? 4 : (oi ? 3 : 2);
        int p1, p2, p3, p4;
        interp_parents<int>(J.nx, i, j, s, cat, p1, p2, p3, p4);
        bool ok = (xst[p1] & XS_EXACT) != 0;
        if (J.interp == ART_INTERP_LINEAR) {
            ok = ok && (xst[p2] & XS_EXACT);
            if (cat == 4) ok = ok && (xst[p3] & XS_EXACT) && (xst[p4] & XS_EXACT);
        }
        if (!ok) atomicAdd(counters + C_CERTERR, 1ull);
        write_interp<int>(J, img, p, p1, p2, p3, p4, cat, npix);
        xst[p] = XS_EXACT;
    }
}

// Decide the borderline points of `level` in FP64 on their exact stencils.  Those to be traced
// keep the FP64 ray traced for them (mask TRACED) and count as rays of the level; the others
// receive their interpolant.  All become exact.
__global__ void cert_redecide_kernel(DevJob J, int level, const double* __restrict__ norm_ptr,
                                     const int32_t* border, unsigned long long* counters,
                                     unsigned long long border_cap, double* img, uint8_t* mask,
                                     uint8_t* xst, float* aminr, float* aturn)
{
    unsigned long long n = counters[C_BORDER];
    if (n > border_cap) n = border_cap;
    const int64_t npix = (int64_t)J.nx * J.ny;
    const double norm = *norm_ptr;
    const int s = 1 << (J.levels - level);
    unsigned long long traced = 0;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t p = border[q];
        const int i = p % J.nx, j = p / J.nx;
        const int oi = (i / s) & 1, oj = (j / s) & 1;
        const int cat = (oi && oj) ? 4 : (oi ? 3 : 2);
        if (!stencil_exact(J, xst, i, j, s, cat)) atomicAdd(counters + C_CERTERR, 1ull);
        double w1, w2, ea, er;
        int p1, p2, p3, p4;
        const GlobalSrc<int> V{img + (int64_t)J.cplane * npix, J.nx};
        bool tr = decide<int>(J, V, i, j, s, norm, cat, w1, w2, p1,
                              p2, p3, p4, ea, er);
        if (J.edge_mode == ART_EDGE_TRACE) {
            const int di = (cat == 2) ? 0 : s, dj = (cat == 3) ? 0 : s;
            if (i - 3 * di < 0 || i + 3 * di >= J.nx || j - 3 * dj < 0 || j + 3 * dj >= J.ny)
                tr = true;
        }
        if (tr) {
            mask[p] = ART_MASK_TRACED;
            ++traced;
        } else {
            interp_parents<int>(J.nx, i, j, s, cat, p1, p2, p3, p4);
            if (aminr) {
                if (cat == 4) {
                    aminr[p] = 0.25f * (((aminr[p1] + aminr[p2]) + aminr[p3]) + aminr[p4]);
                    aturn[p] = 0.25f * (((aturn[p1] + aturn[p2]) + aturn[p3]) + aturn[p4]);
                } else {
                    aminr[p] = 0.5f * (aminr[p1] + aminr[p2]);
                    aturn[p] = 0.5f * (aturn[p1] + aturn[p2]);
                }
            }
            write_interp<int>(J, img, p, p1, p2, p3, p4, cat, npix);
            mask[p] = ART_MASK_INTERP;
        }
        xst[p] = XS_EXACT;
    }
    if (traced) atomicAdd(counters + C_LEVEL0 + level, traced);
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[C_BTOT] += n;
}

static int cert_grid(unsigned long long cap)
{
    unsigned long long g = (cap + 255) / 256;
    if (g > 1216) g = 1216;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_cert_mark_base(const DevJob& J, uint8_t* xst, cudaStream_t st)
{
    const int S0 = 1 << J.levels;
    const int64_t n = (int64_t)((J.nx - 1) / S0 + 1) * ((J.ny - 1) / S0 + 1);
    cert_mark_base_kernel<<<cert_grid((unsigned long long)n), 256, 0, st>>>(J, xst);
    return cudaGetLastError();
}

cudaError_t launch_cert_spec_count(unsigned long long* counters, cudaStream_t st)
{
    cert_spec_count_kernel<<<1, 1, 0, st>>>(counters);
    return cudaGetLastError();
}

cudaError_t launch_cert_closure(const DevJob& J, int level, const int32_t* border,
                                unsigned long long border_cap, unsigned long long* counters,
                                uint8_t* xst, const uint8_t* mask, int32_t* xq,
                                unsigned long long xq_cap, uint64_t* fixq,
                                unsigned long long fix_cap, cudaStream_t st)
{
    cert_closure_kernel<<<cert_grid(border_cap), 256, 0, st>>>(J, border, counters, counters, xst,
                                                               mask, xq, xq_cap, fixq, fix_cap,
                                                               level);
    return cudaGetLastError();
}

// Longest first (exact decisions).  An FP64 launch ends when its last ray does, and the rays of one
// launch differ several-fold in length (~300 RK4 steps near the photon ring, ~70 for a ray that
// escapes), so its queue is reordered longest first: a counting sort over LPT_BUCKETS buckets of
// 4 steps.  A ray's expected length is the steps its pixel's ray took in an earlier pass (mask
// traced or speculatively traced), else the longest of its interpolation parents' (0 where none
// of them has been traced).
__device__ __forceinline__ int lpt_key(const DevJob& J, int32_t p, const uint16_t* steps,
                                       const uint8_t* mask)
{
    const int64_t npix = (int64_t)J.nx * J.ny;
    if (p < 0 || p >= npix) return 0;
    auto traced = [&](int q) {
        const uint8_t m = mask[q];
        return (m == ART_MASK_TRACED || m == MASK_SPEC_DONE) ? (int)steps[q] : 0;
    };
    const uint8_t m = mask[p];
    if (m == ART_MASK_TRACED || m == MASK_SPEC_DONE) return steps[p];
    const int i = p % J.nx, j = p / J.nx;
    int s;
    if (pixel_level(i, j, J.levels, s) == 0) return 0;
    const int oi = (i / s) & 1, oj = (j / s) & 1;
    const int cat = (oi && oj) ? 4 : (oi ? 3 : 2);
    int p1, p2, p3, p4;
    interp_parents<int>(J.nx, i, j, s, cat, p1, p2, p3, p4);
    int k = max(traced(p1), traced(p2));
    if (cat == 4) k = max(k, max(traced(p3), traced(p4)));
    return k;
}

__device__ __forceinline__ int lpt_bucket(int key)
{
    const int b = key >> 2;
    return LPT_BUCKETS - 1 - (b < LPT_BUCKETS - 1 ? b : LPT_BUCKETS - 1);
}

__global__ void lpt_hist_kernel(DevJob J, const int32_t* q, const unsigned long long* count,
                                unsigned long long cap, const uint16_t* steps,
                                const uint8_t* mask, unsigned int* hist)
{
    __shared__ unsigned int h[LPT_BUCKETS];
    for (int b = threadIdx.x; b < LPT_BUCKETS; b += blockDim.x) h[b] = 0;
    __syncthreads();
    unsigned long long n = *count;
    if (n > cap) n = cap;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&h[lpt_bucket(lpt_key(J, q[k], steps, mask))], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < LPT_BUCKETS; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Exclusive prefix sum of the LPT_BUCKETS counts in place (one block of LPT_BUCKETS threads).
__global__ void __launch_bounds__(LPT_BUCKETS) lpt_scan_kernel(unsigned int* hist)
{
    __shared__ unsigned int t[LPT_BUCKETS];
    const int b = threadIdx.x;
    const unsigned int own = hist[b];
    t[b] = own;
    __syncthreads();
    for (int off = 1; off < LPT_BUCKETS; off <<= 1) {
        const unsigned int v = b >= off ? t[b - off] : 0u;
        __syncthreads();
        t[b] += v;
        __syncthreads();
    }
    hist[b] = t[b] - own;
}

__global__ void lpt_scatter_kernel(DevJob J, const int32_t* q_in, const unsigned long long* count,
                                   unsigned long long cap, const uint16_t* steps,
                                   const uint8_t* mask, int32_t* q_out, unsigned int* cursor)
{
    unsigned long long n = *count;
    if (n > cap) n = cap;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t p = q_in[k];
        const unsigned int pos = atomicAdd(&cursor[lpt_bucket(lpt_key(J, p, steps, mask))], 1u);
        q_out[pos] = p;
    }
}

cudaError_t launch_lpt_order(const DevJob& J, const int32_t* q_in,
                             const unsigned long long* count, unsigned long long cap,
                             const uint16_t* pix_steps, const uint8_t* mask, int32_t* q_out,
                             unsigned int* hist, int num_sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned int) * LPT_BUCKETS, st);
    if (e != cudaSuccess) return e;
    const int grid = 2 * num_sms;
    lpt_hist_kernel<<<grid, 256, 0, st>>>(J, q_in, count, cap, pix_steps, mask, hist);
    lpt_scan_kernel<<<1, LPT_BUCKETS, 0, st>>>(hist);
    lpt_scatter_kernel<<<grid, 256, 0, st>>>(J, q_in, count, cap, pix_steps, mask, q_out, hist);
    return cudaGetLastError();
}

cudaError_t launch_cert_mark_traced(const int32_t* xq, unsigned long long* counters,
                                    unsigned long long xq_cap, uint8_t* xst, cudaStream_t st,
                                    int count_idx)
{
    cert_mark_traced_kernel<<<cert_grid(xq_cap), 256, 0, st>>>(xq, counters, xq_cap, xst,
                                                               count_idx);
    return cudaGetLastError();
}

cudaError_t launch_cert_fixup(const DevJob& J, const uint64_t* fixq, unsigned long long* counters,
                              unsigned long long fix_cap, int lvl, double* img, uint8_t* xst,
                              cudaStream_t st)
{
    cert_fixup_kernel<<<cert_grid(fix_cap), 256, 0, st>>>(J, fixq, counters, fix_cap, lvl, img, xst);
    return cudaGetLastError();
}

cudaError_t launch_cert_redecide(const DevJob& J, int level, const double* norm,
                                 const int32_t* border, unsigned long long* counters,
                                 unsigned long long border_cap, double* img, uint8_t* mask,
                                 uint8_t* xst, float* aminr, float* aturn, cudaStream_t st)
{
    cert_redecide_kernel<<<cert_grid(border_cap), 256, 0, st>>>(J, level, norm, border, counters,
                                                                border_cap, img, mask, xst, aminr,
                                                                aturn);
    return cudaGetLastError();
}

// counters[C_LEVEL0 + level] += counters[C_QUEUE] (rays of the level: queued + consumed speculative)
__global__ void level_count_kernel(unsigned long long* counters, int level)
{
    counters[C_LEVEL0 + level] += counters[C_QUEUE];
}

cudaError_t launch_level_count(unsigned long long* counters, int level, cudaStream_t st)
{
    level_count_kernel<<<1, 1, 0, st>>>(counters, level);
    return cudaGetLastError();
}

// counters[C_SPECFROM] = counters[C_QUEUE]: speculative rays are appended after this slot
__global__ void spec_mark_kernel(unsigned long long* counters)
{
    counters[C_SPECFROM] = counters[C_QUEUE];
}

cudaError_t launch_spec_mark(unsigned long long* counters, cudaStream_t st)
{
    spec_mark_kernel<<<1, 1, 0, st>>>(counters);
    return cudaGetLastError();
}

// Appends reserve slots with atomics and skip those beyond the capacity; clamp the length.
__global__ void queue_clamp_kernel(unsigned long long* counters, unsigned long long cap)
{
    if (counters[C_QUEUE] > cap) counters[C_QUEUE] = cap;
}

__global__ void counter_clamp_kernel(unsigned long long* counters, int idx, unsigned long long cap)
{
    if (counters[idx] > cap) counters[idx] = cap;
}

cudaError_t launch_counter_clamp(unsigned long long* counters, int idx, unsigned long long cap,
                                 cudaStream_t st)
{
    counter_clamp_kernel<<<1, 1, 0, st>>>(counters, idx, cap);
    return cudaGetLastError();
}

cudaError_t launch_queue_clamp(unsigned long long* counters, unsigned long long cap,
                               cudaStream_t st)
{
    queue_clamp_kernel<<<1, 1, 0, st>>>(counters, cap);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------------
// batched forms: blockIdx.y selects the image; queue entries are (image << 32) | pixel and the
// rays of a level are also counted per image (img_counts[16 * image + level]).
// --------------------------------------------------------------------------------------------

__global__ void enqueue_base_batch_kernel(const DevJob* jobs, int64_t* queue,
                                          unsigned long long* qcount,
                                          unsigned long long* img_counts)
{
    const int img = blockIdx.y;
    const DevJob& J = jobs[img];
    const int S0 = 1 << J.levels;
    const int n0x = (J.nx - 1) / S0 + 1, n0y = (J.ny - 1) / S0 + 1;
    const int64_t n = (int64_t)n0x * n0y;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = base + threadIdx.x;
        const bool have = q < n;
        const unsigned b = __ballot_sync(0xffffffffu, have);
        unsigned long long w = 0;
        if (lane == 0 && b) w = atomicAdd(qcount, (unsigned long long)__popc(b));
        w = __shfl_sync(0xffffffffu, w, 0);
        if (have) {
            int ii = (int)(q % n0x), jj = (int)(q / n0x);
            int64_t pix = (int64_t)jj * S0 * J.nx + (int64_t)ii * S0;
            queue[w + __popc(b & ((1u << lane) - 1u))] = ((int64_t)img << 32) | pix;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) img_counts[16 * img] = (unsigned long long)n;
}

cudaError_t launch_enqueue_base_batch(const DevJob* jobs, int n, int max_base, int64_t* queue,
                                      unsigned long long* qcount, unsigned long long* img_counts,
                                      cudaStream_t st)
{
    int gx = (max_base + 255) / 256;
    if (gx < 1) gx = 1;
    if (gx > 1024) gx = 1024;
    enqueue_base_batch_kernel<<<dim3(gx, n), 256, 0, st>>>(jobs, queue, qcount, img_counts);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NORM_THREADS)
    norm_batch_kernel(const DevJob* jobs, double* const* imgs, double* norms)
{
    const DevJob& J = jobs[blockIdx.x];
    const int stride = 1 << J.levels, nx = J.nx, ny = J.ny;
    const double* img = imgs[blockIdx.x] + (int64_t)J.cplane * nx * ny;  // the criterion's plane
    const int n0x = (nx - 1) / stride + 1, n0y = (ny - 1) / stride + 1;
    const int64_t n = (int64_t)n0x * n0y;
    double s = 0.0, w = 0.0, mx = -INFINITY;
    for (int64_t q = threadIdx.x; q < n; q += NORM_THREADS) {
        int ii = (int)(q % n0x), jj = (int)(q / n0x);
        double wx = (n0x > 1 && (ii == 0 || ii == n0x - 1)) ? 0.5 : 1.0;
        double wy = (n0y > 1 && (jj == 0 || jj == n0y - 1)) ? 0.5 : 1.0;
        double v = img[(int64_t)jj * stride * nx + (int64_t)ii * stride];
        s += wx * wy * v;
        w += wx * wy;
        mx = fmax(mx, v);
    }
    __shared__ double ss[NORM_THREADS], sw[NORM_THREADS], sm[NORM_THREADS];
    ss[threadIdx.x] = s;
    sw[threadIdx.x] = w;
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int h = NORM_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            ss[threadIdx.x] += ss[threadIdx.x + h];
            sw[threadIdx.x] += sw[threadIdx.x + h];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double ibar = ss[0] / sw[0];
        double* o = norms + 4 * blockIdx.x;
        o[1] = ibar;
        o[2] = sm[0];
        o[0] = J.abs_norm == ART_NORM_PEAK ? sm[0] : ibar;
    }
}

cudaError_t launch_norm_batch(const DevJob* jobs, double* const* imgs, int n, double* norms,
                              cudaStream_t st)
{
    norm_batch_kernel<<<n, NORM_THREADS, 0, st>>>(jobs, imgs, norms);
    return cudaGetLastError();
}

// The batched level kernel: the tiled level kernel over the images of a batch (blockIdx.z), the
// rays appended as (image << 32) | pixel.
__global__ void __launch_bounds__(RT_X * RT_Y)
    refine_batch_kernel(const DevJob* jobs, int level, const double* __restrict__ norms,
                        double* const* imgs, uint8_t* const* masks, int64_t* queue,
                        unsigned long long* qcount, unsigned long long* img_counts,
                        unsigned long long* counters)
{
    const int im = blockIdx.z;
    const DevJob J = jobs[im];
    if (level > J.levels) return;  // the whole block: this image has no such level
    double* img = imgs[im];
    uint8_t* mask = masks[im];
    const int s = 1 << (J.levels - level);
    const int sh = J.levels - level + 1;
    const int ncx = (J.nx - 1) / (2 * s) + 1, ncy = (J.ny - 1) / (2 * s) + 1;
    const int X0 = blockIdx.x * RT_X;
    if (X0 >= ncx) return;  // the whole block: the image is narrower than the widest one
    const int64_t npix = (int64_t)J.nx * J.ny;
    const double* plane = img + (int64_t)J.cplane * npix;  // the criterion's plane
    const double norm = norms[4 * im];
    __shared__ Screen sc_s;  // once per block, as in refine_kernel
    __shared__ double tv[RT_HY * RT_HX];
    __shared__ float tf[RT_HY * RT_HX];
    if (threadIdx.x == 0) sc_s = make_screen(J, norm);
    const int lane = threadIdx.x & 31, tx = threadIdx.x % RT_X, ty = threadIdx.x / RT_X;
    for (int Y0 = blockIdx.y * RT_Y; Y0 < ncy; Y0 += gridDim.y * RT_Y) {
        __syncthreads();
        load_refine_tile(plane, J.nx, ncx, ncy, sh, X0, Y0, tv, tf);
        __syncthreads();
        const Screen sc = sc_s;
        const TileSrc V{tv, tf, plane, sh, X0 - 1, Y0 - 1};
        const int cx = X0 + tx, cy = Y0 + ty;
#pragma unroll 1
        for (int t = 0; t < 3; ++t) {
            const int oi = t != 1, oj = t != 0;
            const bool act = cx + oi < ncx && cy + oj < ncy;
            bool trace = false, used = false;
            int32_t pix = 0;
            if (act) {
                const int i = (2 * cx + oi) * s, j = (2 * cy + oj) * s;
                const int cat = (oi && oj) ? 4 : (oi ? 3 : 2);
                const int r = refine_point_s<int, false>(J, sc, V, img, mask, i, j, s, cat, norm,
                                                         npix, counters != nullptr, nullptr,
                                                         nullptr, nullptr);
                trace = r == 1;
                used = r == 2;
                pix = j * J.nx + i;
            }
            const unsigned b = __ballot_sync(0xffffffffu, trace);
            if (b) {
                unsigned long long w = 0;
                if (lane == 0) {
                    w = atomicAdd(qcount, (unsigned long long)__popc(b));
                    atomicAdd(img_counts + 16 * im + level, (unsigned long long)__popc(b));
                }
                w = __shfl_sync(0xffffffffu, w, 0);
                if (trace) queue[w + __popc(b & ((1u << lane) - 1u))] = ((int64_t)im << 32) | pix;
            }
            // speculative rays of this level the criterion asked for count as its rays
            if (counters) {
                const unsigned u = __ballot_sync(0xffffffffu, used);
                if (u && lane == 0) {
                    atomicAdd(counters + C_SPECUSED, (unsigned long long)__popc(u));
                    atomicAdd(img_counts + 16 * im + level, (unsigned long long)__popc(u));
                }
            }
        }
    }
}

cudaError_t launch_refine_batch(const DevJob* jobs, int n, int level, int max_kx, int max_ky,
                                const double* norms, double* const* imgs, uint8_t* const* masks,
                                int64_t* queue, unsigned long long* qcount,
                                unsigned long long* img_counts, cudaStream_t st,
                                unsigned long long* spec_counters)
{
    // tiles of the widest image's coarse lattice (max_kx, max_ky: the largest level lattice)
    const int ncx = (max_kx - 1) / 2 + 1, ncy = (max_ky - 1) / 2 + 1;
    int gy = (ncy + RT_Y - 1) / RT_Y;
    if (gy > 65535) gy = 65535;
    if (gy < 1) gy = 1;
    int gx = (ncx + RT_X - 1) / RT_X;
    if (gx < 1) gx = 1;
    refine_batch_kernel<<<dim3(gx, gy, n), RT_X * RT_Y, 0, st>>>(jobs, level, norms, imgs, masks,
                                                                 queue, qcount, img_counts,
                                                                 spec_counters);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------------
// A third sampling axis (frequency or time; Sec. 6 proposes adaptive sampling there): the new
// samples of one level of the axis are decided per pixel with the one-dimensional estimator of
// Sec. 3.2 along the axis (the category 2/3 form: inner samples f -/+ s, outer f -/+ 3s, one-sided
// where one outer sample is missing, infinite where both are), normalised by the mean I_bar_int of
// the base samples; interpolated pixels receive the mean of their two axis neighbours in every
// plane, traced ones join the ray queue.
// --------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(256)
    axis_refine_kernel(int64_t npix, int planes, double* const* imgs, int f, int s, int F,
                       double norm, double R_rel, double R_abs, int32_t* queue,
                       unsigned long long* qcount, uint8_t* amask)
{
    const double* lo1 = imgs[f - s];
    const double* hi1 = imgs[f + s];
    const double* lo3 = f - 3 * s >= 0 ? imgs[f - 3 * s] : nullptr;
    const double* hi3 = f + 3 * s < F ? imgs[f + 3 * s] : nullptr;
    double* out = imgs[f];
    const int lane = threadIdx.x & 31;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < npix;
         b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = b0 + threadIdx.x;
        bool trace = false;
        if (p < npix) {
            const double a1 = __ldg(lo1 + p), b1 = __ldg(hi1 + p);
            double d = 0.0;
            bool none = false;
            if (lo3 && hi3) d = ((__ldg(lo3 + p) - a1) - b1) + __ldg(hi3 + p);
            else if (lo3) d = 2.0 * ((__ldg(lo3 + p) - 2.0 * a1) + b1);
            else if (hi3) d = 2.0 * ((__ldg(hi3 + p) - 2.0 * b1) + a1);
            else none = true;
            const double sin_ = a1 + b1;
            const double num = fabs(d) / 8.0, den = fabs(sin_) / 2.0;
            double ea, er;
            if (none) {
                ea = er = INFINITY;
            } else {
                ea = num / norm;
                er = den == 0.0 ? (num == 0.0 ? 0.0 : INFINITY) : num / den;
            }
            trace = (ea > R_abs) && (er > R_rel);
            if (isnan(ea) || isnan(er) || isnan(sin_)) trace = true;
            if (!trace) {
                for (int c = 0; c < planes; ++c) {
                    const double v1 = __ldg(lo1 + c * npix + p), v2 = __ldg(hi1 + c * npix + p);
                    const long long bb = __double_as_longlong(v1);
                    out[c * npix + p] = (bb == __double_as_longlong(v2) && ((bb >> 52) & 0x7ff) < 0x7fc)
                                            ? v1
                                            : scale_pow2(v1 + v2, 1);
                }
            }
            if (amask) amask[(int64_t)f * npix + p] = trace ? ART_MASK_TRACED : ART_MASK_INTERP;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, trace);
        if (bal) {
            unsigned long long w = 0;
            if (lane == 0) w = atomicAdd(qcount, (unsigned long long)__popc(bal));
            w = __shfl_sync(0xffffffffu, w, 0);
            if (trace) queue[w + __popc(bal & ((1u << lane) - 1u))] = (int32_t)p;
        }
    }
}

cudaError_t launch_axis_refine(int64_t npix, int planes, double* const* imgs, int f, int s, int F,
                               double norm, double R_rel, double R_abs, int32_t* queue,
                               unsigned long long* qcount, uint8_t* amask, cudaStream_t st)
{
    int64_t g = (npix + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    axis_refine_kernel<<<(int)g, 256, 0, st>>>(npix, planes, imgs, f, s, F, norm, R_rel, R_abs,
                                               queue, qcount, amask);
    return cudaGetLastError();
}

// The axis estimate of pixel p at sample f (as axis_refine_kernel); true when it asks for a ray.
__device__ __forceinline__ bool axis_wants(double* const* imgs, int f, int s, int F, int64_t p,
                                           double norm, double R_rel, double R_abs)
{
    const double a1 = __ldg(imgs[f - s] + p), b1 = __ldg(imgs[f + s] + p);
    const bool lo = f - 3 * s >= 0, hi = f + 3 * s < F;
    if (!lo && !hi) return true;  // infinite estimate
    double d;
    if (lo && hi) d = ((__ldg(imgs[f - 3 * s] + p) - a1) - b1) + __ldg(imgs[f + 3 * s] + p);
    else if (lo) d = 2.0 * ((__ldg(imgs[f - 3 * s] + p) - 2.0 * a1) + b1);
    else d = 2.0 * ((__ldg(imgs[f + 3 * s] + p) - 2.0 * b1) + a1);
    const double sin_ = a1 + b1;
    const double num = fabs(d) / 8.0, den = fabs(sin_) / 2.0;
    const double ea = num / norm;
    const double er = den == 0.0 ? (num == 0.0 ? 0.0 : INFINITY) : num / den;
    bool trace = (ea > R_abs) && (er > R_rel);
    if (isnan(ea) || isnan(er) || isnan(sin_)) trace = true;
    return trace;
}

// The spatial queue of one level at a new axis sample f (counters[C_QUEUE] pixels): the pixels
// the axis estimate also asks for are kept (compacted into `out`, counters[C_AXQ]); the others
// receive the axis interpolant in every plane (mask ART_MASK_AXIS).
__global__ void __launch_bounds__(256)
    axis_filter_kernel(int64_t npix, int planes, double* const* imgs, int f, int s, int F,
                       double norm, double R_rel, double R_abs, const int32_t* queue,
                       unsigned long long* counters, int32_t* out, uint8_t* mask)
{
    const unsigned long long n = counters[C_QUEUE];
    const int lane = threadIdx.x & 31;
    double* dst = imgs[f];
    unsigned long long kept = 0, interp = 0;
    for (unsigned long long b0 = (unsigned long long)blockIdx.x * blockDim.x; b0 < n;
         b0 += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long q = b0 + threadIdx.x;
        bool keep = false;
        int32_t p = 0;
        if (q < n) {
            p = queue[q];
            keep = axis_wants(imgs, f, s, F, p, norm, R_rel, R_abs);
            if (!keep) {
                for (int c = 0; c < planes; ++c) {
                    const double v1 = __ldg(imgs[f - s] + c * npix + p);
                    const double v2 = __ldg(imgs[f + s] + c * npix + p);
                    const long long bb = __double_as_longlong(v1);
                    dst[c * npix + p] = (bb == __double_as_longlong(v2) && ((bb >> 52) & 0x7ff) < 0x7fc)
                                            ? v1
                                            : scale_pow2(v1 + v2, 1);
                }
                if (mask) mask[p] = ART_MASK_AXIS;
                ++interp;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (bal) {
            unsigned long long w = 0;
            if (lane == 0) w = atomicAdd(counters + C_AXQ, (unsigned long long)__popc(bal));
            w = __shfl_sync(0xffffffffu, w, 0);
            if (keep) out[w + __popc(bal & ((1u << lane) - 1u))] = p;
        }
        kept += keep ? 1 : 0;
    }
    if (kept) atomicAdd(counters + C_AXKEPT, kept);
    if (interp) atomicAdd(counters + C_AXINTERP, interp);
}

cudaError_t launch_axis_filter(int64_t npix, int planes, double* const* imgs, int f, int s, int F,
                               double norm, double R_rel, double R_abs, const int32_t* queue,
                               unsigned long long* counters, int32_t* out, uint8_t* mask,
                               int num_sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counters + C_AXQ, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    axis_filter_kernel<<<num_sms * 8, 256, 0, st>>>(npix, planes, imgs, f, s, F, norm, R_rel,
                                                     R_abs, queue, counters, out, mask);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------------
// metrics (Eqs. interpdef, fluxdef, msedef): per-block partial sums, then one block combines them
// in a fixed order.  Sums: [0] interpolated points, [1] F (trapezoid), [2] F_hat, [3] sum dI^2,
// [4] sum I^2, [5] sum I.
// --------------------------------------------------------------------------------------------

constexpr int MET_THREADS = 256;

__global__ void __launch_bounds__(MET_THREADS)
    metrics_partial_kernel(const double* truth, const double* img, const uint8_t* mask, int nx,
                           int ny, double* partials)
{
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const int64_t n = (int64_t)nx * ny;
    for (int64_t p = blockIdx.x * (int64_t)MET_THREADS + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * MET_THREADS) {
        int i = (int)(p % nx), j = (int)(p / nx);
        double wx = (nx > 1 && (i == 0 || i == nx - 1)) ? 0.5 : 1.0;
        double wy = (ny > 1 && (j == 0 || j == ny - 1)) ? 0.5 : 1.0;
        double t = truth[p], v = img[p], d = t - v;
        if (mask && mask[p] == ART_MASK_INTERP) acc[0] += 1.0;
        acc[1] += wx * wy * t;
        acc[2] += wx * wy * v;
        acc[3] += d * d;
        acc[4] += t * t;
        acc[5] += t;
    }
    __shared__ double sh[6][MET_THREADS];
    for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int h = MET_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int c = 0; c < 6; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 6) partials[blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void metrics_final_kernel(const double* partials, int nblocks, double* out6)
{
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b * 6 + threadIdx.x];
        out6[threadIdx.x] = s;
    }
}

cudaError_t launch_metrics(const double* truth, const double* img, const uint8_t* mask, int nx,
                           int ny, double* partials, int nblocks, double* out6, cudaStream_t st)
{
    metrics_partial_kernel<<<nblocks, MET_THREADS, 0, st>>>(truth, img, mask, nx, ny, partials);
    metrics_final_kernel<<<1, 32, 0, st>>>(partials, nblocks, out6);
    return cudaGetLastError();
}

}  // namespace art
