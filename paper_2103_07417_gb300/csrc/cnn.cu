// cnn.cu -- the learned block proposal: a small convolutional network run and trained on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// The paper has no learned component.  The network predicts, from the completed level-k lattice
// (features: asinh(I / I_norm), 3 / max(r_min, 1), polar turns), which 4 x 4-cell blocks of that
// lattice the exact criterion of Sec. 3.2 will refine two levels later; those rays can then be
// traced early.  Layers: four 3x3 convolutions with 32 channels (strides 1, 1, 2, 2, pad 1, ReLU)
// and a 1x1 head with a logistic output; loss = mean binary cross-entropy.
//
// Every convolution is an implicit GEMM on the tensor cores:
//   forward  D[o][co]        = sum_{t, ci} X[s o + t - 1][ci] W[co][t][ci]        (M = output pixels)
//   dgrad    D[i][ci]        = sum_{t, co} dY[(i + 1 - t)/s][co] W[co][t][ci]     (M = input pixels)
//   wgrad    D[(t, ci)][co]  = sum_o X[s o + t - 1][ci] dY[o][co]                 (K = output pixels)
// with 128-row operand tiles in shared memory in the canonical K-major layout (umma.cuh): views
// of a staged input halo (the forward, and the stride-1 layer's dgrad as a forward convolution of
// dY with flipped taps), a gathered tile (the stride-2 dgrad), or one built from staged input rows
// (the wgrad); one thread issues the MMAs, completion through an mbarrier, and the epilogue reads D
// from tensor memory.  The weight gradient carries one extra row of ones so the same GEMM yields the bias
// gradient.  Activations are NHWC BF16 (32 channels, 64 B per pixel; the 3 input features padded
// to 8 channels); the head, the loss and the optimizer (Adam) run in FP32 on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.cuh"
#include "umma.cuh"

namespace art {

using bf16 = __nv_bfloat16;
constexpr int CH = 32;       // channels of every hidden layer
constexpr int CIN0 = 8;      // input features padded to 16 bytes per pixel
constexpr int NFEAT = 3;     // real input features
constexpr int K1 = 80;       // 9 x 8 = 72 padded to a multiple of 16
constexpr int KH = 288;      // 9 x 32
constexpr int GEMM_THREADS = 128;
constexpr int WG_PIX = 64;   // output pixels per weight-gradient stage (K of the stage)

// offsets of the parameter vector (FP32): W1, b1, W2, b2, W3, b3, W4, b4, w_head, b_head
constexpr int P_W1 = 0, P_B1 = P_W1 + CH * 9 * NFEAT, P_W2 = P_B1 + CH, P_B2 = P_W2 + CH * 9 * CH,
              P_W3 = P_B2 + CH, P_B3 = P_W3 + CH * 9 * CH, P_W4 = P_B3 + CH,
              P_B4 = P_W4 + CH * 9 * CH, P_WH = P_B4 + CH, P_BH = P_WH + CH, P_N = P_BH + 1;
static_assert(P_N == ART_CNN_PARAMS, "parameter layout");

struct ConvArgs {
    const bf16* src;    // forward: X (H x W x CIN); dgrad: dY (Ho x Wo x 32)
    const bf16* B;      // 32 x KPAD BF16 (forward [co][t CIN + ci], dgrad [ci][t 32 + co])
    const float* bias;  // forward only
    const bf16* mask;   // dgrad only: the forward input X (H x W x 32); output *= (X > 0)
    bf16* out;          // forward: Ho x Wo x 32; dgrad: H x W x 32
    int H, W, Ho, Wo, stride;
    int* err;
};

__device__ __forceinline__ uint4 bf16x8_zero() { return make_uint4(0, 0, 0, 0); }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Input gradient of a stride-2 layer as an implicit GEMM: 128-row tiles of input pixels, N = 32
// channels, K = KPAD (9 taps x 32 output channels of dY, gathered; the taps that do not land on an
// output pixel of the strided forward are zero).  The CTAs are persistent: the weights are loaded
// once per CTA, then tiles blockIdx.x, + gridDim.x, ...  Output: dX times the forward input's ReLU
// mask.
template <int CIN, int KPAD>
__global__ void __launch_bounds__(GEMM_THREADS) conv_dgrad_kernel(ConvArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    uint8_t* sA = smem;
    uint8_t* sB = smem + 128 * KPAD * 2;
    constexpr int KC = KPAD / 8, TAPC = CIN / 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rows = a.H * a.W;
    const int ntiles = (rows + 127) / 128;
    const int sW = a.Wo, sH = a.Ho;  // source grid (dY)
    const int rW = a.W;              // row grid width
    for (int q = tid; q < CH * KC; q += GEMM_THREADS) {
        const int r = q & 7, rest = q >> 3;
        const int kc = rest % KC, g = rest / KC;
        const int n = g * 8 + r;
        *reinterpret_cast<uint4*>(sB + umma::chunk_off(n, kc, KPAD)) =
            __ldg(reinterpret_cast<const uint4*>(a.B + (int64_t)n * KPAD) + kc);
    }
    if (tid == 0) umma::mbar_init(&bar);
    if (warp == 0) umma::tmem_alloc(&tslot, 32);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, phase ^= 1u) {
        const int p0 = tile * 128;
        // A: chunk (row m, column group kc); rows fastest within an 8-row group
        for (int q = tid; q < 128 * KC; q += GEMM_THREADS) {
            const int r = q & 7, rest = q >> 3;
            const int kc = rest % KC, g = rest / KC;
            const int m = g * 8 + r, p = p0 + m;
            uint4 v = bf16x8_zero();
            const int tap = kc / TAPC, cg = kc - tap * TAPC;
            if (p < rows && tap < 9) {
                const int py = p / rW, px = p - py * rW;
                const int ky = tap / 3, kx = tap - ky * 3;
                const int ny = py + 1 - ky, nx = px + 1 - kx;
                const int sy = ny / a.stride, sx = nx / a.stride;
                if (ny >= 0 && nx >= 0 && sy * a.stride == ny && sx * a.stride == nx && sy < sH &&
                    sx < sW)
                    v = __ldg(reinterpret_cast<const uint4*>(a.src + ((int64_t)sy * sW + sx) * CIN) + cg);
            }
            *reinterpret_cast<uint4*>(sA + umma::chunk_off(m, kc, KPAD)) = v;
        }
        umma::fence_smem_async();
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
        if (tid == 0) {
            const uint32_t ab = umma::smem_u32(sA), bb = umma::smem_u32(sB), sbo = KC * 128;
            for (int kb = 0; kb < KPAD / 16; ++kb)
                umma::mma(tmem, umma::desc(ab + kb * 256, 128, sbo),
                          umma::desc(bb + kb * 256, 128, sbo), umma::idesc_bf16(128, CH), kb > 0);
            umma::commit(&bar);
        }
        ok = __syncthreads_and(umma::wait(&bar, phase));
        umma::fence_after();
        if (ok) {
            float v[32];
            umma::ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
            const int p = p0 + warp * 32 + lane;
            if (p < rows) {
                uint32_t w[16];
                const uint4* mk = reinterpret_cast<const uint4*>(a.mask + (int64_t)p * CH);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    uint4 mv = __ldg(mk + c4);
                    const __nv_bfloat162* mh = reinterpret_cast<const __nv_bfloat162*>(&mv);
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        float2 f = __bfloat1622float2(mh[h]);
                        const int c = c4 * 8 + 2 * h;
                        w[c / 2] = pack_bf16x2(f.x > 0.f ? v[c] : 0.f, f.y > 0.f ? v[c + 1] : 0.f);
                    }
                }
                uint4* o = reinterpret_cast<uint4*>(a.out + (int64_t)p * CH);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4)
                    o[c4] = make_uint4(w[4 * c4], w[4 * c4 + 1], w[4 * c4 + 2], w[4 * c4 + 3]);
            }
        } else if (tid == 0) {
            atomicExch(a.err, 1);
        }
        // the tensor-memory reads and the shared-memory tile are done before the next tile
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
    }
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, 32);
}

// Forward convolution of a 32-channel layer (stride S = 1 or 2) from a halo tile: one CTA computes an
// output tile of 8 x 16 pixels (M = 128: row group g = output row y0 + g, row r = column x0 + r).
// The CTA loads the input rows and columns under the tile once (coalesced 16-byte chunks, zeros
// outside the image) into planes of 16-byte entries, one per (channel group of 8, column parity
// for S = 2); within a plane an input row is PITCH consecutive entries.  The A operand of tap
// (ky, kx) for channels 16 h .. 16 h + 15 is then the same tile viewed at an offset: start at row
// ky, entry kx / S of parity kx % S, core matrices 8 consecutive entries (the 8 output columns),
// K step (next channel group) = one parity-plane pair, M step (next output row) = S rows.  18 MMAs
// (9 taps x 2 K-halves) accumulate D in tensor memory, as the im2col kernel, with the same
// operand values in the same order.
template <int S, int CIN>
struct Halo {
    static constexpr int TW = 8, TH = 16;
    static constexpr int HR = S * (TH - 1) + 3, HC = S * (TW - 1) + 3;  // rows, columns of input
    static constexpr int NPAR = S, PITCH = (HC + S - 1) / S;            // entries per plane row
    static constexpr int PLANE = HR * PITCH * 16;                       // bytes per plane
    static constexpr int CG = CIN / 8;                                  // channel groups
    static constexpr int KPAD = CIN == CH ? KH : K1;
    static constexpr int ABYTES = CG * NPAR * PLANE;
    static constexpr int BOFF = (ABYTES + 1023) / 1024 * 1024;
    static constexpr int SMEM = BOFF + CH * KPAD * 2;
};

// CIN = 8 (the 3 input features, S = 1): one channel group per pixel, so a K = 16 slice holds two
// taps; its second core matrix is the next tap's view of the same plane (LBO = the taps' address
// difference, 16 B along a row), matching the weights' [tap][channel] columns.
// MODE 0: forward (bias, ReLU).  MODE 1 (stride 1, CIN = CH): the input gradient of a stride-1
// layer, which is the same convolution of dY with the taps flipped (B rows ci, columns
// t' 32 + co holding W[co][8 - t'][ci]) and, instead of bias and ReLU, the forward input's ReLU
// mask (a.mask > 0) at the output pixel.
template <int S, int CIN, int MODE = 0>
__global__ void __launch_bounds__(GEMM_THREADS) conv_halo_kernel(ConvArgs a)
{
    static_assert(CIN == CH || (CIN == CIN0 && S == 1), "halo convolution variants");
    static_assert(MODE == 0 || (S == 1 && CIN == CH), "input gradient of stride-1 layers only");
    using HT = Halo<S, CIN>;
    constexpr int CGR = HT::CG;
    constexpr int NQ = HT::HR * HT::HC * CGR;                    // 16-byte chunks of one halo
    constexpr int NPT = (NQ + GEMM_THREADS - 1) / GEMM_THREADS;  // per thread
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    uint8_t* sA = smem;
    uint8_t* sB = smem + HT::BOFF;
    constexpr int KC = HT::KPAD / 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (a.Wo + HT::TW - 1) / HT::TW;
    const int ntiles = tiles_x * ((a.Ho + HT::TH - 1) / HT::TH);
    // persistent: the weights once per CTA, then tiles blockIdx.x, + gridDim.x, ...; the next
    // tile's halo is fetched into registers while the current tile's MMAs run
    for (int q = tid; q < CH * KC; q += GEMM_THREADS) {
        const int r = q & 7, rest = q >> 3;
        const int kc = rest % KC, g = rest / KC;
        const int n = g * 8 + r;
        *reinterpret_cast<uint4*>(sB + umma::chunk_off(n, kc, HT::KPAD)) =
            __ldg(reinterpret_cast<const uint4*>(a.B + (int64_t)n * HT::KPAD) + kc);
    }
    // the gap between the halo and the weights is read (times zero weights) by the padding
    // slice of the 8-channel layer: keep it finite
    for (int q = HT::ABYTES / 16 + tid; q < HT::BOFF / 16; q += GEMM_THREADS)
        reinterpret_cast<uint4*>(sA)[q] = bf16x8_zero();
    if (tid == 0) umma::mbar_init(&bar);
    if (warp == 0) umma::tmem_alloc(&tslot, 32);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;
    // halo chunk q of the tile at (x0, y0): input rows S y0 - 1 .., columns S x0 - 1 ..; zeros
    // outside the image
    auto fetch = [&](int tile, uint4* R) {
        const int x0 = (tile % tiles_x) * HT::TW, y0 = (tile / tiles_x) * HT::TH;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int q = tid + k * GEMM_THREADS;
            uint4 v = bf16x8_zero();
            if (q < NQ) {
                const int cg = q % CGR, pe = q / CGR;
                const int yy = pe / HT::HC, cc = pe - yy * HT::HC;
                const int iy = S * y0 - 1 + yy, ix = S * x0 - 1 + cc;
                if (iy >= 0 && iy < a.H && ix >= 0 && ix < a.W)
                    v = __ldg(reinterpret_cast<const uint4*>(a.src + ((int64_t)iy * a.W + ix) * CIN) + cg);
            }
            R[k] = v;
        }
    };
    uint4 R[NPT];
    int tile = blockIdx.x;
    if (tile < ntiles) fetch(tile, R);
    uint32_t phase = 0;
    bool ok = true;
    for (; tile < ntiles && ok; tile += gridDim.x, phase ^= 1u) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int q = tid + k * GEMM_THREADS;
            if (q < NQ) {
                const int cg = q % CGR, pe = q / CGR;
                const int yy = pe / HT::HC, cc = pe - yy * HT::HC;
                const int par = cc % S, e = cc / S;
                *reinterpret_cast<uint4*>(sA + (cg * HT::NPAR + par) * HT::PLANE +
                                          (yy * HT::PITCH + e) * 16) = R[k];
            }
        }
        umma::fence_smem_async();
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
        if (tid == 0) {
            const uint32_t ab = umma::smem_u32(sA), bb = umma::smem_u32(sB);
            const uint32_t sbo = S * HT::PITCH * 16;
            auto tap_addr = [&](int t) {
                const int ky = t / 3, kx = t - 3 * ky, par = kx % S, eoff = kx / S;
                return ab + par * HT::PLANE + (ky * HT::PITCH + eoff) * 16;
            };
            if (CIN == CH) {
                const uint32_t lbo = HT::NPAR * HT::PLANE;
                for (int t = 0; t < 9; ++t)
                    for (int h = 0; h < 2; ++h)
                        umma::mma(tmem, umma::desc(tap_addr(t) + 2 * h * HT::NPAR * HT::PLANE, lbo, sbo),
                                  umma::desc(bb + (2 * t + h) * 256, 128, KC * 128),
                                  umma::idesc_bf16(128, CH), t > 0 || h > 0);
            } else {
                for (int j = 0; j < K1 / 16; ++j) {
                    const int t0 = 2 * j, t1 = 2 * j + 1;  // t1 = 9: the zero-weight padding
                    const uint32_t a0 = tap_addr(t0);
                    const uint32_t lbo = t1 < 9 ? tap_addr(t1) - a0 : 16;
                    umma::mma(tmem, umma::desc(a0, lbo, sbo),
                              umma::desc(bb + j * 256, 128, KC * 128),
                              umma::idesc_bf16(128, CH), j > 0);
                }
            }
            umma::commit(&bar);
        }
        const int next = tile + gridDim.x;
        if (next < ntiles) fetch(next, R);  // in flight during the MMAs
        ok = __syncthreads_and(umma::wait(&bar, phase));
        umma::fence_after();
        if (ok) {
            float v[32];
            umma::ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
            const int x0 = (tile % tiles_x) * HT::TW, y0 = (tile / tiles_x) * HT::TH;
            const int m = warp * 32 + lane;
            const int oy = y0 + (m >> 3), ox = x0 + (m & 7);
            if (oy < a.Ho && ox < a.Wo) {
                uint32_t w[16];
                if (MODE == 0) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        w[c] = pack_bf16x2(fmaxf(v[2 * c] + __ldg(a.bias + 2 * c), 0.f),
                                           fmaxf(v[2 * c + 1] + __ldg(a.bias + 2 * c + 1), 0.f));
                } else {
                    const uint4* mk =
                        reinterpret_cast<const uint4*>(a.mask + ((int64_t)oy * a.Wo + ox) * CH);
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {
                        const uint4 mv = __ldg(mk + c4);
                        const __nv_bfloat162* mh = reinterpret_cast<const __nv_bfloat162*>(&mv);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 m2 = __bfloat1622float2(mh[e]);
                            const int c = 8 * c4 + 2 * e;
                            w[c / 2] = pack_bf16x2(m2.x > 0.f ? v[c] : 0.f,
                                                   m2.y > 0.f ? v[c + 1] : 0.f);
                        }
                    }
                }
                uint4* o = reinterpret_cast<uint4*>(a.out + ((int64_t)oy * a.Wo + ox) * CH);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4)
                    o[c4] = make_uint4(w[4 * c4], w[4 * c4 + 1], w[4 * c4 + 2], w[4 * c4 + 3]);
            }
        } else if (tid == 0) {
            atomicExch(a.err, 1);
        }
        // the tensor-memory reads and the shared-memory tile are done before the next tile
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
    }
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, 32);
}

struct WgradArgs {
    const bf16* X;     // forward input, H x W x CIN
    const bf16* dY;    // Ho x Wo x 32
    float* part;       // per-CTA partial sums: [blockIdx.x][layer parameter]
    int w_off, b_off;  // offsets of this layer's W and b in the vector
    int cin_real;      // channels of the layer's real input (3 or 32)
    int H, W, Ho, Wo, stride;
    int pix_per_cta;   // output-row segments (of at most WG_PIX pixels) reduced by one CTA
    int* err;
};

// Weight and bias gradient: rows (t, ci) of one 128-row tile (blockIdx.y), N = the 32 output
// channels, K = output pixels, one segment of at most WG_PIX pixels of one output row per stage
// (this CTA's segments: a.pix_per_cta of them from blockIdx.x on).  Per stage the CTA copies the
// three input rows under the segment (the columns its taps reach, zeros outside the image) and the
// segment's dY into shared memory with 16-byte loads, then builds the canonical K-major operands
// from there; row 9 CIN is all ones and yields the bias gradient.  Partial sums per CTA.
template <int CIN, int S>
struct WgradSmem {
    static constexpr int XC = S * WG_PIX + 2;  // staged input columns per row: S x0 - 1 + [0, XC)
    static constexpr int A_BYTES = 128 * WG_PIX * 2, B_BYTES = CH * WG_PIX * 2;
    static constexpr int X_BYTES = 3 * XC * CIN * 2;
    static constexpr int BYTES = A_BYTES + B_BYTES + X_BYTES;
};

template <int CIN, int S>
__global__ void __launch_bounds__(GEMM_THREADS) conv_wgrad_kernel(WgradArgs a)
{
    using L = WgradSmem<CIN, S>;
    constexpr int KC = WG_PIX / 8, XC = L::XC, CG = CIN / 8;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + L::A_BYTES;
    bf16* xt = reinterpret_cast<bf16*>(smem + L::A_BYTES + L::B_BYTES);  // [ky][column][ci]
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nsx = (a.Wo + WG_PIX - 1) / WG_PIX, nseg = a.Ho * nsx;
    const int s_begin = blockIdx.x * a.pix_per_cta;
    if (s_begin >= nseg) return;  // uniform over the CTA
    const int s_end = min(nseg, s_begin + a.pix_per_cta);
    const int m0 = blockIdx.y * 128;
    if (tid == 0) umma::mbar_init(&bar);
    if (warp == 0) umma::tmem_alloc(&tslot, 32);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    int stage = 0;
    for (int sg = s_begin; sg < s_end; ++sg, ++stage) {
        const int oy = sg / nsx, x0 = (sg - oy * nsx) * WG_PIX;
        const int npx = min(WG_PIX, a.Wo - x0);
        const int cx0 = S * x0 - 1;  // input column of staged column 0
        // the three input rows under the segment, 16 bytes (8 channels) per load
        for (int q = tid; q < 3 * XC * CG; q += GEMM_THREADS) {
            const int g = q % CG, rest = q / CG, c = rest % XC, ky = rest / XC;
            const int iy = S * oy + ky - 1, ix = cx0 + c;
            uint4 v = bf16x8_zero();
            if (iy >= 0 && iy < a.H && ix >= 0 && ix < a.W)
                v = __ldg(reinterpret_cast<const uint4*>(a.X + ((int64_t)iy * a.W + ix) * CIN) + g);
            *reinterpret_cast<uint4*>(xt + (ky * XC + c) * CIN + 8 * g) = v;
        }
        // dY of the segment into the canonical B layout (rows co, K = pixels)
        for (int q = tid; q < WG_PIX * (CH / 8); q += GEMM_THREADS) {
            const int g = q & 3, px = q >> 2;
            uint4 v = bf16x8_zero();
            if (px < npx)
                v = __ldg(reinterpret_cast<const uint4*>(a.dY + ((int64_t)oy * a.Wo + x0 + px) * CH) + g);
            const uint16_t* h = reinterpret_cast<const uint16_t*>(&v);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                *reinterpret_cast<uint16_t*>(sB + umma::chunk_off(8 * g + e, px >> 3, WG_PIX) +
                                             (px & 7) * 2) = h[e];
        }
        __syncthreads();
        // A chunk (row m, pixel octet c8) from the staged rows
        for (int q = tid; q < 128 * KC; q += GEMM_THREADS) {
            const int r = q & 7, rest = q >> 3;
            const int c8 = rest % KC, g = rest / KC;
            const int m = m0 + g * 8 + r;
            uint32_t w[4] = {0, 0, 0, 0};
            if (m < 9 * CIN) {
                const int tap = m / CIN, ci = m - tap * CIN;
                const int ky = tap / 3, kx = tap - ky * 3;
                const uint16_t* row = reinterpret_cast<const uint16_t*>(xt) + ky * XC * CIN + ci;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int px = c8 * 8 + j;
                    const uint32_t h = px < npx ? row[(S * px + kx) * CIN] : 0u;
                    w[j >> 1] |= h << (16 * (j & 1));
                }
            } else if (m == 9 * CIN) {
                const uint32_t one = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c8 * 8 + j < npx) w[j >> 1] |= one << (16 * (j & 1));
            }
            *reinterpret_cast<uint4*>(sA + umma::chunk_off(g * 8 + r, c8, WG_PIX)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
        umma::fence_smem_async();
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
        if (tid == 0) {
            const uint32_t ab = umma::smem_u32(sA), bb = umma::smem_u32(sB), sbo = KC * 128;
            for (int kb = 0; kb < WG_PIX / 16; ++kb)
                umma::mma(tmem, umma::desc(ab + kb * 256, 128, sbo),
                          umma::desc(bb + kb * 256, 128, sbo), umma::idesc_bf16(128, CH),
                          stage > 0 || kb > 0);
            umma::commit(&bar);
        }
        ok = __syncthreads_and(umma::wait(&bar, stage & 1));
        umma::fence_after();
        if (!ok) break;
    }
    if (ok) {
        // this CTA's sums over its segments, reduced across CTAs in a fixed order afterwards
        // (wgrad_reduce_kernel), so that training is reproducible
        float v[32];
        umma::ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        const int m = m0 + warp * 32 + lane;
        float* part = a.part + (int64_t)blockIdx.x * (CH * 9 * a.cin_real + CH);
        if (m < 9 * CIN) {
            const int tap = m / CIN, ci = m - tap * CIN;
            if (ci < a.cin_real)
                for (int co = 0; co < CH; ++co) part[(co * 9 + tap) * a.cin_real + ci] = v[co];
        } else if (m == 9 * CIN) {
            for (int co = 0; co < CH; ++co) part[CH * 9 * a.cin_real + co] = v[co];
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, 32);
}

// grad[w_off + i] (i < 9 CH cin) or grad[b_off + i - 9 CH cin] += the sum over the CTAs' partials,
// in CTA order.
__global__ void wgrad_reduce_kernel(const float* part, int nblk, int cin_real, float* grad,
                                    int w_off, int b_off)
{
    const int nw = CH * 9 * cin_real, np = nw + CH;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * np + i];
    grad[i < nw ? w_off + i : b_off + (i - nw)] += s;
}

// BF16 GEMM operands from the FP32 parameters: forward B[co][t CIN + ci] per layer and the input
// gradient's B[ci][t 32 + co] for layers 2-4.
__global__ void cnn_prep_weights_kernel(const float* prm, bf16* f1, bf16* f2, bf16* f3, bf16* f4,
                                        bf16* d2, bf16* d3, bf16* d4, bf16* d2f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < CH * K1) {
        const int co = i / K1, k = i - co * K1, t = k / CIN0, ci = k - t * CIN0;
        const float v = (t < 9 && ci < NFEAT) ? prm[P_W1 + (co * 9 + t) * NFEAT + ci] : 0.f;
        f1[i] = __float2bfloat16_rn(v);
    }
    if (i < CH * KH) {
        const int r = i / KH, k = i - r * KH;
        {   // forward: r = co, k = t 32 + ci
            const int t = k / CH, ci = k - t * CH, idx = (r * 9 + t) * CH + ci;
            f2[i] = __float2bfloat16_rn(prm[P_W2 + idx]);
            f3[i] = __float2bfloat16_rn(prm[P_W3 + idx]);
            f4[i] = __float2bfloat16_rn(prm[P_W4 + idx]);
        }
        {   // input gradient: r = ci, k = t 32 + co
            const int t = k / CH, co = k - t * CH, idx = (co * 9 + t) * CH + r;
            d2[i] = __float2bfloat16_rn(prm[P_W2 + idx]);
            d3[i] = __float2bfloat16_rn(prm[P_W3 + idx]);
            d4[i] = __float2bfloat16_rn(prm[P_W4 + idx]);
        }
        {   // the stride-1 layer's input gradient as a forward convolution of dY: r = ci,
            // k = t' 32 + co with the tap flipped (t = 8 - t')
            const int tf = k / CH, co = k - tf * CH, idx = (co * 9 + (8 - tf)) * CH + r;
            d2f[i] = __float2bfloat16_rn(prm[P_W2 + idx]);
        }
    }
}

// FP32 features (H x W x 3) -> BF16 NHWC with 8 channels.
__global__ void cnn_input_kernel(const float* feat, int n, bf16* x0)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint4 v;
    v.x = pack_bf16x2(feat[3 * p], feat[3 * p + 1]);
    v.y = pack_bf16x2(feat[3 * p + 2], 0.f);
    v.z = 0u;
    v.w = 0u;
    reinterpret_cast<uint4*>(x0)[p] = v;
}

// Head (1x1 conv 32 -> 1 + logistic), the loss and, with a target, the head's backward pass:
// dY4 = (p - t)/n w_head (Y4 > 0) in BF16, gradients of w_head and b_head, loss sum.
constexpr int HEAD_THREADS = 256;
__global__ void __launch_bounds__(HEAD_THREADS)
    cnn_head_kernel(const bf16* y4, int n, const float* prm, const float* target, float* prob,
                    bf16* dy4, float* part)
{
    __shared__ float red[CH + 2][HEAD_THREADS / 32];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float h[CH];
    float dlog = 0.f, l = 0.f;
    if (p < n) {
        const uint4* src = reinterpret_cast<const uint4*>(y4 + (int64_t)p * CH);
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            uint4 v = src[c4];
            const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 f = __bfloat1622float2(hv[k]);
                h[c4 * 8 + 2 * k] = f.x;
                h[c4 * 8 + 2 * k + 1] = f.y;
            }
        }
        float z = prm[P_BH];
#pragma unroll
        for (int c = 0; c < CH; ++c) z += prm[P_WH + c] * h[c];
        const float pr = 1.f / (1.f + expf(-z));
        if (prob) prob[p] = pr;
        if (target) {
            const float t = target[p];
            l = fmaxf(z, 0.f) - z * t + log1pf(expf(-fabsf(z)));
            dlog = (pr - t) / (float)n;
            uint32_t w[16];
#pragma unroll
            for (int c = 0; c < 16; ++c)
                w[c] = pack_bf16x2(h[2 * c] > 0.f ? dlog * prm[P_WH + 2 * c] : 0.f,
                                   h[2 * c + 1] > 0.f ? dlog * prm[P_WH + 2 * c + 1] : 0.f);
            uint4* o = reinterpret_cast<uint4*>(dy4 + (int64_t)p * CH);
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4)
                o[c4] = make_uint4(w[4 * c4], w[4 * c4 + 1], w[4 * c4 + 2], w[4 * c4 + 3]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < CH; ++c) h[c] = 0.f;
    }
    if (!target) return;  // uniform over the grid
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    auto wsum = [&](float v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const float s = wsum(dlog * h[c]);
        if (lane == 0) red[c][wid] = s;
    }
    {
        const float s = wsum(dlog), s2 = wsum(l);
        if (lane == 0) {
            red[CH][wid] = s;
            red[CH + 1][wid] = s2;
        }
    }
    __syncthreads();
    // the block's sums of dL/dw_head (CH), dL/db_head and the loss, reduced over the blocks in a
    // fixed order by head_reduce_kernel
    if (threadIdx.x < CH + 2) {
        float s = 0.f;
        for (int w = 0; w < HEAD_THREADS / 32; ++w) s += red[threadIdx.x][w];
        part[(int64_t)blockIdx.x * (CH + 2) + threadIdx.x] = s;
    }
}

__global__ void head_reduce_kernel(const float* part, int nblk, float* grad, float* loss_sum)
{
    const int c = threadIdx.x;
    if (c >= CH + 2) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * (CH + 2) + c];
    if (c < CH)
        grad[P_WH + c] += s;
    else if (c == CH)
        grad[P_BH] += s;
    else
        *loss_sum = s;
}

// Adam (Kingma & Ba 2015) on the FP32 parameters; clears the gradients.
__global__ void cnn_adam_kernel(float* prm, float* grad, float* m, float* v, int n, float lr,
                                float b1t, float b2t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g, vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    prm[i] -= lr * (mi / (1.f - b1t)) / (sqrtf(vi / (1.f - b2t)) + 1e-8f);
    grad[i] = 0.f;
}

// --------------------------------------------------------------------------------------------
// host side: the network's device state and its passes
// --------------------------------------------------------------------------------------------

struct CnnState {
    float *prm = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    bf16 *f1 = nullptr, *f2 = nullptr, *f3 = nullptr, *f4 = nullptr, *d2 = nullptr, *d3 = nullptr,
         *d4 = nullptr, *d2f = nullptr;
    int* err = nullptr;
    int step = 0;
    bool weights_ready = false;
    // activations, sized for the largest lattice seen
    int64_t cap = 0;
    bf16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *a4 = nullptr;
    bf16 *g1 = nullptr, *g2 = nullptr, *g3 = nullptr, *g4 = nullptr;
    // per-CTA partial sums of the gradient kernels (reduced in a fixed order)
    float* part = nullptr;
    int64_t part_cap = 0;
};

static int conv_smem(int kpad) { return (128 + CH) * kpad * 2; }

template <int CIN, int KPAD>
static cudaError_t run_dgrad(const ConvArgs& a, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(conv_dgrad_kernel<CIN, KPAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, conv_smem(KPAD));
    if (e != cudaSuccess) return e;
    static int grid_cap = 0;  // resident CTAs of the device (persistent grid)
    if (!grid_cap) {
        int dev = 0, sms = 0, smem_sm = 0;
        cudaFuncAttributes fa;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv_dgrad_kernel<CIN, KPAD>);
        if (e != cudaSuccess) return e;
        int per = smem_sm / (conv_smem(KPAD) + (int)fa.sharedSizeBytes + 1024);
        if (per > 8) per = 8;  // 8 x 32 tensor-memory columns of 512
        grid_cap = sms * (per > 0 ? per : 1);
    }
    const int tiles = (a.H * a.W + 127) / 128;
    conv_dgrad_kernel<CIN, KPAD><<<tiles < grid_cap ? tiles : grid_cap, GEMM_THREADS,
                                  conv_smem(KPAD), st>>>(a);
    return cudaGetLastError();
}

// Forward convolution of stride S through the halo-tile kernel.
template <int S, int CIN, int MODE_ = 0>
static cudaError_t run_conv_halo(const ConvArgs& a, cudaStream_t st)
{
    using HT = Halo<S, CIN>;
    constexpr int MODE = MODE_;
    static bool attr = false;  // one device per process is the supported configuration
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv_halo_kernel<S, CIN, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             HT::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    static int grid_cap = 0;  // resident CTAs of the device (persistent grid)
    if (!grid_cap) {
        // CTAs per SM from the kernel's registers and shared memory (the occupancy query
        // answered 1 here)
        int dev = 0, sms = 0, smem_sm = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv_halo_kernel<S, CIN, MODE>);
        if (e != cudaSuccess) return e;
        const int by_smem = smem_sm / (HT::SMEM + (int)fa.sharedSizeBytes + 1024);
        const int by_regs = 65536 / ((fa.numRegs > 0 ? fa.numRegs : 255) * GEMM_THREADS);
        int per = by_smem < by_regs ? by_smem : by_regs;
        if (per > 8) per = 8;  // 8 x 32 tensor-memory columns of 512
        grid_cap = sms * (per > 0 ? per : 1);
    }
    const int tiles = ((a.Wo + HT::TW - 1) / HT::TW) * ((a.Ho + HT::TH - 1) / HT::TH);
    conv_halo_kernel<S, CIN, MODE><<<tiles < grid_cap ? tiles : grid_cap, GEMM_THREADS, HT::SMEM,
                                     st>>>(a);
    return cudaGetLastError();
}

// CTAs along the output-row segments of a weight-gradient launch: about 32 segments (2048 output
// pixels) each, at most WG_CTAS (their partial sums are reduced afterwards), every one with a
// non-empty range.
constexpr int WG_CTAS = 608;
static int wgrad_ctas(int Ho, int Wo, int* spc)
{
    const int nseg = Ho * ((Wo + WG_PIX - 1) / WG_PIX);
    int ctas = (nseg + 31) / 32;
    if (ctas < 1) ctas = 1;
    if (ctas > WG_CTAS) ctas = WG_CTAS;
    *spc = (nseg + ctas - 1) / ctas;
    return (nseg + *spc - 1) / *spc;
}

// Weight and bias gradients of one layer: the tensor-core partial sums, then their reduction into
// grad (a.part must hold wgrad_ctas() x (9 CH cin_real + CH) floats).
template <int CIN, int S>
static cudaError_t run_wgrad_s(WgradArgs a, float* grad, cudaStream_t st)
{
    using L = WgradSmem<CIN, S>;
    const int ctas = wgrad_ctas(a.Ho, a.Wo, &a.pix_per_cta);
    const int mtiles = (9 * CIN + 1 + 127) / 128;
    cudaError_t e = cudaFuncSetAttribute(conv_wgrad_kernel<CIN, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    if (e != cudaSuccess) return e;
    conv_wgrad_kernel<CIN, S><<<dim3(ctas, mtiles), GEMM_THREADS, L::BYTES, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int np = CH * 9 * a.cin_real + CH;
    wgrad_reduce_kernel<<<(np + 255) / 256, 256, 0, st>>>(a.part, ctas, a.cin_real, grad, a.w_off,
                                                          a.b_off);
    return cudaGetLastError();
}

template <int CIN>
static cudaError_t run_wgrad(WgradArgs a, float* grad, cudaStream_t st)
{
    return a.stride == 1 ? run_wgrad_s<CIN, 1>(a, grad, st) : run_wgrad_s<CIN, 2>(a, grad, st);
}

#define CKE(x)                                 \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

static cudaError_t ensure_state(CnnState*& s)
{
    if (s) return cudaSuccess;
    s = new CnnState();
    CKE(cudaMalloc(&s->prm, sizeof(float) * P_N));
    CKE(cudaMalloc(&s->grad, sizeof(float) * P_N));
    CKE(cudaMalloc(&s->m, sizeof(float) * P_N));
    CKE(cudaMalloc(&s->v, sizeof(float) * P_N));
    CKE(cudaMalloc(&s->loss, sizeof(float) * 2));
    CKE(cudaMalloc(&s->err, sizeof(int)));
    CKE(cudaMemset(s->err, 0, sizeof(int)));
    CKE(cudaMalloc(&s->f1, sizeof(bf16) * CH * K1));
    for (bf16** p : {&s->f2, &s->f3, &s->f4, &s->d2, &s->d3, &s->d4, &s->d2f})
        CKE(cudaMalloc(p, sizeof(bf16) * CH * KH));
    return cudaSuccess;
}

static cudaError_t ensure_acts(CnnState* s, int H, int W)
{
    const int64_t n = (int64_t)H * W;
    if (n <= s->cap) return cudaSuccess;
    for (bf16** p : {&s->x0, &s->a1, &s->a2, &s->a3, &s->a4, &s->g1, &s->g2, &s->g3, &s->g4}) {
        cudaFree(*p);
        *p = nullptr;
    }
    s->cap = 0;
    CKE(cudaMalloc(&s->x0, sizeof(bf16) * n * CIN0));
    for (bf16** p : {&s->a1, &s->a2, &s->a3, &s->a4, &s->g1, &s->g2, &s->g3, &s->g4})
        CKE(cudaMalloc(p, sizeof(bf16) * n * CH));
    s->cap = n;
    return cudaSuccess;
}

void cnn_destroy(CnnState* s)
{
    if (!s) return;
    for (float* p : {s->prm, s->grad, s->m, s->v, s->loss}) cudaFree(p);
    for (bf16* p : {s->f1, s->f2, s->f3, s->f4, s->d2, s->d3, s->d4, s->d2f, s->x0, s->a1, s->a2,
                    s->a3, s->a4, s->g1, s->g2, s->g3, s->g4})
        cudaFree(p);
    cudaFree(s->err);
    cudaFree(s->part);
    delete s;
}

cudaError_t cnn_load(CnnState*& s, const float* host_params, cudaStream_t st)
{
    CKE(ensure_state(s));
    CKE(cudaMemcpyAsync(s->prm, host_params, sizeof(float) * P_N, cudaMemcpyHostToDevice, st));
    CKE(cudaMemsetAsync(s->grad, 0, sizeof(float) * P_N, st));
    CKE(cudaMemsetAsync(s->m, 0, sizeof(float) * P_N, st));
    CKE(cudaMemsetAsync(s->v, 0, sizeof(float) * P_N, st));
    s->step = 0;
    s->weights_ready = false;
    return cudaStreamSynchronize(st);
}

cudaError_t cnn_read(CnnState* s, float* host_params, cudaStream_t st)
{
    CKE(cudaMemcpyAsync(host_params, s->prm, sizeof(float) * P_N, cudaMemcpyDeviceToHost, st));
    return cudaStreamSynchronize(st);
}

static cudaError_t prep_weights(CnnState* s, cudaStream_t st)
{
    if (s->weights_ready) return cudaSuccess;
    cnn_prep_weights_kernel<<<(CH * KH + 255) / 256, 256, 0, st>>>(
        s->prm, s->f1, s->f2, s->f3, s->f4, s->d2, s->d3, s->d4, s->d2f);
    CKE(cudaGetLastError());
    s->weights_ready = true;
    return cudaSuccess;
}

static inline int osz(int n, int s) { return (n - 1) / s + 1; }

// Forward from s->x0 (already filled); probabilities to prob (nullable); with target, the backward
// pass accumulates into s->grad and the loss sum into s->loss[0].
static cudaError_t forward_backward(CnnState* s, int H, int W, const float* target, float* prob,
                                    cudaStream_t st)
{
    CKE(prep_weights(s, st));
    const int H2 = osz(H, 2), W2 = osz(W, 2), H4 = osz(H2, 2), W4 = osz(W2, 2);
    ConvArgs c{};
    c.err = s->err;
    // c1, c2 (stride 1), c3, c4 (stride 2)
    c.src = s->x0; c.B = s->f1; c.bias = s->prm + P_B1; c.out = s->a1;
    c.H = H; c.W = W; c.Ho = H; c.Wo = W; c.stride = 1;
    CKE((run_conv_halo<1, CIN0>(c, st)));
    c.src = s->a1; c.B = s->f2; c.bias = s->prm + P_B2; c.out = s->a2;
    CKE((run_conv_halo<1, CH>(c, st)));
    c.src = s->a2; c.B = s->f3; c.bias = s->prm + P_B3; c.out = s->a3;
    c.Ho = H2; c.Wo = W2; c.stride = 2;
    CKE((run_conv_halo<2, CH>(c, st)));
    c.src = s->a3; c.B = s->f4; c.bias = s->prm + P_B4; c.out = s->a4;
    c.H = H2; c.W = W2; c.Ho = H4; c.Wo = W4;
    CKE((run_conv_halo<2, CH>(c, st)));
    const int n4 = H4 * W4;
    const int hblk = (n4 + HEAD_THREADS - 1) / HEAD_THREADS;
    if (target) {
        // partial-sum scratch: the head's blocks, and the largest weight-gradient launch
        int ppc;
        int64_t need = (int64_t)hblk * (CH + 2);
        need = std::max<int64_t>(need, (int64_t)wgrad_ctas(H, W, &ppc) * (CH * 9 * CH + CH));
        if (need > s->part_cap) {
            CKE(cudaStreamSynchronize(st));
            cudaFree(s->part);
            s->part = nullptr;
            s->part_cap = 0;
            CKE(cudaMalloc(&s->part, sizeof(float) * need));
            s->part_cap = need;
        }
    }
    cnn_head_kernel<<<hblk, HEAD_THREADS, 0, st>>>(s->a4, n4, s->prm, target, prob, s->g4,
                                                   s->part);
    CKE(cudaGetLastError());
    if (!target) return cudaSuccess;
    head_reduce_kernel<<<1, 64, 0, st>>>(s->part, hblk, s->grad, s->loss);
    CKE(cudaGetLastError());
    WgradArgs w{};
    w.part = s->part;
    w.err = s->err;
    ConvArgs d{};
    d.err = s->err;
    // layer 4: X = a3 (H2 x W2), dY = g4 (H4 x W4)
    w.X = s->a3; w.dY = s->g4; w.w_off = P_W4; w.b_off = P_B4; w.cin_real = CH;
    w.H = H2; w.W = W2; w.Ho = H4; w.Wo = W4; w.stride = 2;
    CKE(run_wgrad<CH>(w, s->grad, st));
    d.src = s->g4; d.B = s->d4; d.mask = s->a3; d.out = s->g3;
    d.H = H2; d.W = W2; d.Ho = H4; d.Wo = W4; d.stride = 2;
    CKE((run_dgrad<CH, KH>(d, st)));
    // layer 3: X = a2 (H x W), dY = g3 (H2 x W2)
    w.X = s->a2; w.dY = s->g3; w.w_off = P_W3; w.b_off = P_B3;
    w.H = H; w.W = W; w.Ho = H2; w.Wo = W2; w.stride = 2;
    CKE(run_wgrad<CH>(w, s->grad, st));
    d.src = s->g3; d.B = s->d3; d.mask = s->a2; d.out = s->g2;
    d.H = H; d.W = W; d.Ho = H2; d.Wo = W2; d.stride = 2;
    CKE((run_dgrad<CH, KH>(d, st)));
    // layer 2: X = a1, dY = g2 (stride 1)
    w.X = s->a1; w.dY = s->g2; w.w_off = P_W2; w.b_off = P_B2;
    w.Ho = H; w.Wo = W; w.stride = 1;
    CKE(run_wgrad<CH>(w, s->grad, st));
    // its input gradient: the forward halo kernel on dY with the flipped taps, ReLU mask of a1
    d.src = s->g2; d.B = s->d2f; d.mask = s->a1; d.out = s->g1;
    d.H = H; d.W = W; d.Ho = H; d.Wo = W; d.stride = 1;
    CKE((run_conv_halo<1, CH, 1>(d, st)));
    // layer 1: X = x0 (8 channels, 3 real), dY = g1
    w.X = s->x0; w.dY = s->g1; w.w_off = P_W1; w.b_off = P_B1; w.cin_real = NFEAT;
    CKE(run_wgrad<CIN0>(w, s->grad, st));
    return cudaSuccess;
}

static int check_err(CnnState* s, cudaStream_t st)
{
    int e = 0;
    if (cudaMemcpyAsync(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ART_ERR_CUDA;
    if (e) {
        cudaMemsetAsync(s->err, 0, sizeof(int), st);
        return ART_ERR_DEVICE;
    }
    return ART_OK;
}

int cnn_forward(CnnState* s, const float* feat, int H, int W, float* prob, cudaStream_t st)
{
    if (!s) return ART_ERR_ARG;
    if (ensure_acts(s, H, W) != cudaSuccess) return ART_ERR_OOM;
    cnn_input_kernel<<<(H * W + 255) / 256, 256, 0, st>>>(feat, H * W, s->x0);
    if (cudaGetLastError() != cudaSuccess) return ART_ERR_CUDA;
    if (forward_backward(s, H, W, nullptr, prob, st) != cudaSuccess) return ART_ERR_CUDA;
    return check_err(s, st);
}

// Forward from the BF16 input already in the state (used by the render's proposal step).
cudaError_t cnn_forward_x0(CnnState* s, int H, int W, float* prob, cudaStream_t st)
{
    return forward_backward(s, H, W, nullptr, prob, st);
}

cudaError_t cnn_ensure_input(CnnState* s, int H, int W, bf16** x0)
{
    CKE(ensure_acts(s, H, W));
    *x0 = s->x0;
    return cudaSuccess;
}

int cnn_grad(CnnState* s, const float* feat, int H, int W, const float* target, float* loss,
             float* grad_host, cudaStream_t st)
{
    if (!s) return ART_ERR_ARG;
    if (ensure_acts(s, H, W) != cudaSuccess) return ART_ERR_OOM;
    if (cudaMemsetAsync(s->grad, 0, sizeof(float) * P_N, st) != cudaSuccess) return ART_ERR_CUDA;
    cnn_input_kernel<<<(H * W + 255) / 256, 256, 0, st>>>(feat, H * W, s->x0);
    if (cudaGetLastError() != cudaSuccess) return ART_ERR_CUDA;
    if (forward_backward(s, H, W, target, nullptr, st) != cudaSuccess) return ART_ERR_CUDA;
    const int H4 = osz(osz(H, 2), 2), W4 = osz(osz(W, 2), 2);
    float lsum = 0.f;
    if (cudaMemcpyAsync(&lsum, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ART_ERR_CUDA;
    if (grad_host &&
        cudaMemcpyAsync(grad_host, s->grad, sizeof(float) * P_N, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return ART_ERR_CUDA;
    int rc = check_err(s, st);
    if (loss) *loss = lsum / (float)(H4 * W4);
    return rc;
}

int cnn_train_step(CnnState* s, const float* feat, int H, int W, const float* target, float lr,
                   float* loss, cudaStream_t st)
{
    float l = 0.f;
    int rc = cnn_grad(s, feat, H, W, target, &l, nullptr, st);
    if (loss) *loss = l;
    if (rc) return rc;
    if (!std::isfinite(l)) {  // a non-finite sample leaves the parameters unchanged
        if (cudaMemsetAsync(s->grad, 0, sizeof(float) * P_N, st) != cudaSuccess) return ART_ERR_CUDA;
        return ART_OK;
    }
    s->step += 1;
    const float b1t = powf(0.9f, (float)s->step), b2t = powf(0.999f, (float)s->step);
    cnn_adam_kernel<<<(P_N + 255) / 256, 256, 0, st>>>(s->prm, s->grad, s->m, s->v, P_N, lr, b1t, b2t);
    if (cudaGetLastError() != cudaSuccess) return ART_ERR_CUDA;
    s->weights_ready = false;
    return ART_OK;
}

// --------------------------------------------------------------------------------------------
// the learned path inside the render: features of a level lattice, the proposal, training targets
// --------------------------------------------------------------------------------------------

// Features of the level-`level` lattice (stride s of the final grid): asinh(I / (R_abs I_norm))
// (the intensity in units of the absolute tolerance, so one network serves every tolerance),
// 3 / max(r_min, 1), polar turns.  BF16 NHWC with 8 channels (x0) or FP32 with 3 (f32).
__global__ void cnn_features_kernel(const double* img, const float* minr, const float* turn,
                                    const double* norm, double r_abs, int nx, int ny, int s,
                                    bf16* x0, float* f32)
{
    const int kx = (nx - 1) / s + 1, ky = (ny - 1) / s + 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kx * ky) return;
    const int jj = q / kx, ii = q - jj * kx;
    const int64_t p = (int64_t)jj * s * nx + (int64_t)ii * s;
    const double scale = r_abs > 0.0 ? r_abs * *norm : *norm;
    const double x = img[p] / scale;
    const float f0 = (scale > 0.0 && isfinite(x)) ? (float)asinh(x) : 0.f;  // dark image: 0
    const float f1 = 3.f / fmaxf(minr[p], 1.f);
    const float f2 = turn[p];
    if (x0) {
        uint4 v;
        v.x = pack_bf16x2(f0, f1);
        v.y = pack_bf16x2(f2, 0.f);
        v.z = 0u;
        v.w = 0u;
        reinterpret_cast<uint4*>(x0)[q] = v;
    }
    if (f32) {
        f32[3 * q] = f0;
        f32[3 * q + 1] = f1;
        f32[3 * q + 2] = f2;
    }
}

static inline int head_dim(int n) { return osz(osz(n, 2), 2); }

int64_t cnn_head_cells(const DevJob& J, int level)
{
    const int s = 1 << (J.levels - level);
    return (int64_t)head_dim((J.nx - 1) / s + 1) * head_dim((J.ny - 1) / s + 1);
}

// One block per head cell (4 x 4 cells of the input lattice, level L, stride s_in): where the
// probability exceeds thr, every point of levels L+2 .. L+1+depth inside the block (lattice of
// stride s_t = s_in / 2^(depth+1), minus the level-(L+1) lattice of stride s_in / 2) whose mask is
// still unset and whose enclosing level-(L+1) cell has a traced corner (the refinement front of
// the exact criterion, just decided for level L+1) is queued for a speculative trace and marked
// pending.  Blocks are disjoint, so each
// point has one candidate thread; queue slots beyond `cap` are skipped.
__global__ void __launch_bounds__(256)
    cnn_propose_kernel(const float* prob, int hw, float thr, int nx, int ny, int s_in, int s_t,
                       uint8_t* mask, int32_t* queue, unsigned long long* counters,
                       unsigned long long cap)
{
    const int cell = blockIdx.x;
    if (!(prob[cell] > thr)) return;  // uniform over the block
    const int hy = cell / hw, hx = cell - hy * hw;
    const int side = 4 * s_in / s_t, half = s_in / 2;
    const int lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < side * side; c0 += 256) {
        const int c = c0 + threadIdx.x;
        const int cy = c / side, cx = c - cy * side;
        const int i = hx * 4 * s_in + cx * s_t, j = hy * 4 * s_in + cy * s_t;
        bool want = c < side * side && i < nx && j < ny && (i % half != 0 || j % half != 0);
        const int64_t pix = (int64_t)j * nx + i;
        if (want) want = mask[pix] == ART_MASK_UNSET;
        if (want) {
            // refinement front: a corner of the enclosing level-(L+1) cell (stride `half`) is
            // traced -- the exact criterion has just queued it or traced it earlier
            const int i0 = (i / half) * half, j0 = (j / half) * half;
            const int i1 = min(i0 + half, nx - 1), j1 = min(j0 + half, ny - 1);
            want = mask[(int64_t)j0 * nx + i0] == ART_MASK_TRACED ||
                   mask[(int64_t)j0 * nx + i1] == ART_MASK_TRACED ||
                   mask[(int64_t)j1 * nx + i0] == ART_MASK_TRACED ||
                   mask[(int64_t)j1 * nx + i1] == ART_MASK_TRACED;
        }
        const unsigned b = __ballot_sync(0xffffffffu, want);
        if (!b) continue;
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(counters + C_QUEUE, (unsigned long long)__popc(b));
        w = __shfl_sync(0xffffffffu, w, 0);
        if (want) {
            const unsigned long long slot = w + __popc(b & ((1u << lane) - 1u));
            if (slot < cap) {
                queue[slot] = (int32_t)pix;
                mask[pix] = MASK_SPEC_PENDING;
                atomicAdd(counters + C_SPEC, 1ull);
            }
        }
    }
}

cudaError_t cnn_propose(CnnState* s, const DevJob& J, int level_in, int depth, const double* img,
                        const float* minr, const float* turn, const double* norm, float thr,
                        float* prob, uint8_t* mask, int32_t* queue, unsigned long long* counters,
                        unsigned long long cap, cudaStream_t st)
{
    const int sin_ = 1 << (J.levels - level_in);
    const int H = (J.ny - 1) / sin_ + 1, W = (J.nx - 1) / sin_ + 1;
    const int last = level_in + 1 + depth < J.levels ? level_in + 1 + depth : J.levels;
    CKE(ensure_acts(s, H, W));
    cnn_features_kernel<<<(H * W + 255) / 256, 256, 0, st>>>(img, minr, turn, norm, J.R_abs, J.nx,
                                                             J.ny, sin_, s->x0, nullptr);
    CKE(cudaGetLastError());
    CKE(forward_backward(s, H, W, nullptr, prob, st));
    const int hh = head_dim(H), hw = head_dim(W);
    cnn_propose_kernel<<<hh * hw, 256, 0, st>>>(prob, hw, thr, J.nx, J.ny, sin_,
                                                1 << (J.levels - last), mask, queue, counters, cap);
    return cudaGetLastError();
}

cudaError_t cnn_features_f32(const DevJob& J, int level, const double* img, const float* minr,
                             const float* turn, const double* norm, float* feat, cudaStream_t st)
{
    const int s = 1 << (J.levels - level);
    const int H = (J.ny - 1) / s + 1, W = (J.nx - 1) / s + 1;
    cnn_features_kernel<<<(H * W + 255) / 256, 256, 0, st>>>(img, minr, turn, norm, J.R_abs, J.nx,
                                                             J.ny, s, nullptr, feat);
    return cudaGetLastError();
}

// Training target of each head cell of the level-L lattice (stride s): 1 if the exact method
// traced a point of level L + 2 or L + 3 inside the block (the levels a proposal made after
// level L + 1's criterion covers with the default depth 2), else 0.  Points of those levels lie on
// the lattice of stride s_t = max(s / 8, 1) and off the level-(L+1) lattice (stride s / 2).
__global__ void __launch_bounds__(256)
    cnn_targets_kernel(const uint8_t* mask, int nx, int ny, int hw, int s, float* target)
{
    const int cell = blockIdx.x;
    const int hy = cell / hw, hx = cell - hy * hw;
    const int st = s >= 8 ? s / 8 : 1, half = s / 2;
    const int side = 4 * s / st;
    int hit = 0;
    for (int c = threadIdx.x; c < side * side; c += 256) {
        const int cy = c / side, cx = c - cy * side;
        const int i = hx * 4 * s + cx * st, j = hy * 4 * s + cy * st;
        if (i < nx && j < ny && (i % half != 0 || j % half != 0) &&
            mask[(int64_t)j * nx + i] == ART_MASK_TRACED)
            hit = 1;
    }
    const int any = __syncthreads_or(hit);
    if (threadIdx.x == 0) target[cell] = any ? 1.f : 0.f;
}

cudaError_t cnn_targets(const DevJob& J, int level, const uint8_t* mask, float* target,
                        cudaStream_t st)
{
    const int s = 1 << (J.levels - level);
    const int H = (J.ny - 1) / s + 1, W = (J.nx - 1) / s + 1;
    cnn_targets_kernel<<<head_dim(H) * head_dim(W), 256, 0, st>>>(mask, J.nx, J.ny, head_dim(W), s,
                                                                  target);
    return cudaGetLastError();
}

}  // namespace art
