// vis.cu -- visibility-domain analysis of an image (Sec. 4.3 of the paper): the complex
// visibilities V(u, v) of a tapered image, the 2-D Fourier transform an interferometer samples,
// on the grid of an m x m FFT.
//
//   V(u, v) = dx^2 sum_{x, y} T(x, y) A(x, y) exp(-2 pi i (u X + v Y)),
//   X = (x - (nx - 1)/2) dx, Y = (y - (ny - 1)/2) dx (the image centre at the origin),
//   T = exp(-4 ln 2 (X^2 + Y^2) / fwhm^2) (a Gaussian taper of the given full width at half
//   maximum; none when fwhm <= 0), A = img, or img - ref for residual visibilities,
//   u = k_u / (m dx), v = k_v / (m dx) with k in [-m/2, m/2), stored at index k mod m.
//
// The image is zero-padded to m x m (which samples the same continuous transform more finely).
// FP64 throughout.  A row transform of length L <= 8192 runs in one CTA: the row is loaded into
// shared memory in bit-reversed order and transformed by log2(L) radix-2 butterfly stages.  Longer
// rows (m = 16384, 32768) are split four-step: m1 = m / 8192 interleaved sub-sequences of length
// 8192 are transformed in shared memory and multiplied by exp(-2 pi i n1 k2 / m), then a radix-m1
// pass combines them.  Rows, transpose, rows, transpose (with the centring phase and dx^2) give the
// 2-D transform.  GB300's FP64 pipe bounds the butterflies; the passes over the m x m array in HBM
// cost about as much again.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace art {

constexpr int VIS_SMEM_LEN = 8192;  // longest row transformed in one CTA
constexpr int VIS_THREADS = 512;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// Tables: twL[j] = exp(-2 pi i j / L) (j < L/2), twm[j] = exp(-2 pi i j / m) (j < m),
// pu[k] = exp(+2 pi i ks cx / m), pv[k] = exp(+2 pi i ks cy / m) (ks the signed frequency index),
// tx[x], ty[y] the taper factors.
__global__ void vis_tables_kernel(int m, int L, int nx, int ny, double dx, double fwhm,
                                  double2* twL, double2* twm, double2* pu, double2* pv, double* tx,
                                  double* ty)
{
    const double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1);
    const double a = fwhm > 0.0 ? 4.0 * log(2.0) * dx * dx / (fwhm * fwhm) : 0.0;
    const int n = m > L ? m : L;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s, c;
        if (j < L / 2) {
            sincospi(-2.0 * j / L, &s, &c);
            twL[j] = make_double2(c, s);
        }
        if (j < m) {
            sincospi(-2.0 * j / m, &s, &c);
            twm[j] = make_double2(c, s);
            const double ks = j < m / 2 ? (double)j : (double)(j - m);
            // reduce the phase argument ks c / m modulo 1 before sincospi (c may be large)
            const double fu = fmod(ks * cx, (double)m) / m, fv = fmod(ks * cy, (double)m) / m;
            sincospi(2.0 * fu, &s, &c);
            pu[j] = make_double2(c, s);
            sincospi(2.0 * fv, &s, &c);
            pv[j] = make_double2(c, s);
        }
        if (j < nx) tx[j] = exp(-a * (j - cx) * (j - cx));
        if (j < ny) ty[j] = exp(-a * (j - cy) * (j - cy));
    }
}

// The padded, tapered image (or residual) as complex rows of length m.
__global__ void vis_prepare_kernel(const double* img, const double* ref, int nx, int ny, int m,
                                   const double* tx, const double* ty, double2* out)
{
    const int64_t n = (int64_t)m * m;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(q / m), x = (int)(q % m);
        double v = 0.0;
        if (x < nx && y < ny) {
            const int64_t p = (int64_t)y * nx + x;
            v = ref ? img[p] - ref[p] : img[p];
            v *= tx[x] * ty[y];
        }
        out[q] = make_double2(v, 0.0);
    }
}

// One length-L transform per CTA, in shared memory.  sub == 0: row blockIdx.x of X, in place
// (L == m).  sub == 1 (L < m, m1 = m / L): sub-sequence n1 = blockIdx.x % m1 of row
// r = blockIdx.x / m1, elements X[r m + n1 + m1 n2]; the result times exp(-2 pi i n1 k2 / m) is
// written to Y[r m + n1 L + k2].
__global__ void __launch_bounds__(VIS_THREADS)
    vis_fft_rows_kernel(double2* X, double2* Y, int m, int L, int logL, int sub,
                        const double2* __restrict__ twL, const double2* __restrict__ twm)
{
    extern __shared__ double2 sbuf[];
    const int m1 = m / L;
    const int64_t r = sub ? blockIdx.x / m1 : blockIdx.x;
    const int n1 = sub ? (int)(blockIdx.x % m1) : 0;
    const double2* src = X + r * m + n1;
    const int stride = sub ? m1 : 1;
    for (int n = threadIdx.x; n < L; n += blockDim.x)
        sbuf[__brev((unsigned)n) >> (32 - logL)] = src[(int64_t)n * stride];
    __syncthreads();
    for (int h = 1; h < L; h <<= 1) {
        const int tstep = L / (2 * h);
        for (int b = threadIdx.x; b < L / 2; b += blockDim.x) {
            const int j = b & (h - 1);
            const int i0 = ((b - j) << 1) + j, i1 = i0 + h;
            const double2 u = sbuf[i0], v = cmul(sbuf[i1], __ldg(&twL[j * tstep]));
            sbuf[i0] = make_double2(u.x + v.x, u.y + v.y);
            sbuf[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    if (!sub) {
        double2* dst = X + r * m;
        for (int k = threadIdx.x; k < L; k += blockDim.x) dst[k] = sbuf[k];
    } else {
        double2* dst = Y + r * m + (int64_t)n1 * L;
        for (int k = threadIdx.x; k < L; k += blockDim.x)
            dst[k] = cmul(sbuf[k], __ldg(&twm[((int64_t)n1 * k) % m]));
    }
}

// Four-step combine: X[r m + k2 + L k1] = sum_n1 exp(-2 pi i n1 k1 / m1) Y[r m + n1 L + k2].
__global__ void vis_combine_kernel(const double2* Y, double2* X, int m, int L, int64_t rows)
{
    const int m1 = m / L;
    const int64_t n = rows * L;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / L;
        const int k2 = (int)(q % L);
        const double2* y = Y + r * m + k2;
        double2* x = X + r * m + k2;
        if (m1 == 2) {
            const double2 a = y[0], b = y[L];
            x[0] = make_double2(a.x + b.x, a.y + b.y);
            x[L] = make_double2(a.x - b.x, a.y - b.y);
        } else {  // m1 == 4: exp(-2 pi i n1 k1 / 4) = (-i)^(n1 k1)
            const double2 a = y[0], b = y[L], c = y[2 * L], d = y[3 * L];
            const double2 s0 = make_double2(a.x + c.x, a.y + c.y), s1 = make_double2(a.x - c.x, a.y - c.y);
            const double2 t0 = make_double2(b.x + d.x, b.y + d.y), t1 = make_double2(b.x - d.x, b.y - d.y);
            x[0] = make_double2(s0.x + t0.x, s0.y + t0.y);
            x[2 * L] = make_double2(s0.x - t0.x, s0.y - t0.y);
            // k1 = 1: a - i b - c + i d = s1 - i t1 ; k1 = 3: s1 + i t1
            x[L] = make_double2(s1.x + t1.y, s1.y - t1.x);
            x[3 * L] = make_double2(s1.x - t1.y, s1.y + t1.x);
        }
    }
}

// out[c][r] = in[r][c] (m x m), times pv[r] pu[c] dx^2 when `phase` is set (the last transpose:
// in[k_u][k_v] -> out[k_v][k_u]).
__global__ void vis_transpose_kernel(const double2* in, double2* out, int m, int phase,
                                     const double2* __restrict__ pu, const double2* __restrict__ pv,
                                     double scale)
{
    __shared__ double2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y)
        tile[j][threadIdx.x] = in[(int64_t)(by + j) * m + bx + threadIdx.x];
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int orow = bx + j, ocol = by + threadIdx.x;  // out[orow][ocol] = in[ocol][orow]
        double2 v = tile[threadIdx.x][j];
        if (phase) {
            // in rows are k_u (= ocol), columns k_v (= orow)
            v = cmul(cmul(v, pu[ocol]), pv[orow]);
            v.x *= scale;
            v.y *= scale;
        }
        out[(int64_t)orow * m + ocol] = v;
    }
}

int vis_table_doubles(int m, int nx, int ny)
{
    const int L = m < VIS_SMEM_LEN ? m : VIS_SMEM_LEN;
    return L + 2 * m + 2 * m + 2 * m + nx + ny;
}

static cudaError_t rows_fft(double2* X, double2* T, int m, const double2* twL, const double2* twm,
                            cudaStream_t st)
{
    const int L = m < VIS_SMEM_LEN ? m : VIS_SMEM_LEN;
    int logL = 0;
    while ((1 << logL) < L) ++logL;
    const size_t smem = sizeof(double2) * L;
    cudaError_t e = cudaFuncSetAttribute(vis_fft_rows_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (L == m) {
        vis_fft_rows_kernel<<<m, VIS_THREADS, smem, st>>>(X, nullptr, m, L, logL, 0, twL, twm);
        return cudaGetLastError();
    }
    const int m1 = m / L;
    vis_fft_rows_kernel<<<m * m1, VIS_THREADS, smem, st>>>(X, T, m, L, logL, 1, twL, twm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    vis_combine_kernel<<<152 * 16, 256, 0, st>>>(T, X, m, L, (int64_t)m);
    return cudaGetLastError();
}

// The whole transform: V (m x m complex, output) and Q (m x m complex scratch), tables
// (vis_table_doubles(m, nx, ny) doubles of scratch).
cudaError_t launch_visibilities(const double* img, const double* ref, int nx, int ny, double dx,
                                double fwhm, int m, double2* V, double2* Q, double* tables,
                                cudaStream_t st)
{
    const int L = m < VIS_SMEM_LEN ? m : VIS_SMEM_LEN;
    double2* twL = reinterpret_cast<double2*>(tables);
    double2* twm = twL + L / 2;
    double2* pu = twm + m;
    double2* pv = pu + m;
    double* tx = reinterpret_cast<double*>(pv + m);
    double* ty = tx + nx;
    const int nt = (m > L ? m : L) > nx ? (m > L ? m : L) : nx;
    const int ntab = nt > ny ? nt : ny;
    vis_tables_kernel<<<(ntab + 255) / 256, 256, 0, st>>>(m, L, nx, ny, dx, fwhm, twL, twm, pu, pv,
                                                          tx, ty);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vis_prepare_kernel<<<152 * 16, 256, 0, st>>>(img, ref, nx, ny, m, tx, ty, V);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = rows_fft(V, Q, m, twL, twm, st)) != cudaSuccess) return e;
    const dim3 tg(m / 32, m / 32), tb(32, 8);
    vis_transpose_kernel<<<tg, tb, 0, st>>>(V, Q, m, 0, pu, pv, 1.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = rows_fft(Q, V, m, twL, twm, st)) != cudaSuccess) return e;
    vis_transpose_kernel<<<tg, tb, 0, st>>>(Q, V, m, 1, pu, pv, dx * dx);
    return cudaGetLastError();
}

}  // namespace art
