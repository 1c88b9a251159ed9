// peaks.cu -- measured throughput of the plain FP32 and FP64 fused multiply-add pipes, the
// denominators of the tracer's ALU roofline beside the peaks derived from unit counts and clocks.
//
// Every thread runs NCH independent dependent chains a <- a b + c (b just below 1, so the values
// stay normal and bounded); with NCH chains per thread and 8 warps per scheduler the pipes, not
// the chains' latency, bound the rate.  One fused multiply-add counts two flops.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.cuh"

namespace art {

constexpr int PEAK_NCH = 8;
constexpr int PEAK_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_chain_kernel(T b, T c, int iters, T* sink)
{
    T v[PEAK_NCH];
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k) v[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < PEAK_NCH; ++k) v[k] = fma(v[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < PEAK_NCH; ++k) s += v[k];
    // a store the compiler cannot drop, taken by no thread in practice (the chains tend to 1)
    if (s == T(-1)) sink[blockIdx.x * PEAK_THREADS + threadIdx.x] = s;
}

// Best of `reps` timed launches of `blocks` x PEAK_THREADS threads, in TFLOP/s.
template <class T>
static cudaError_t time_chains(int blocks, int iters, int reps, T* sink, cudaStream_t st,
                               double* tflops)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    const T b = T(0.999999), c = T(1e-6);
    fma_chain_kernel<T><<<blocks, PEAK_THREADS, 0, st>>>(b, c, iters, sink);  // warm-up
    double best = 0.0;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        fma_chain_kernel<T><<<blocks, PEAK_THREADS, 0, st>>>(b, c, iters, sink);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.f) {
            const double flops =
                2.0 * PEAK_NCH * 16.0 * iters * (double)blocks * PEAK_THREADS;
            const double t = flops / (ms * 1e-3) / 1e12;
            if (t > best) best = t;
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = best;
    return e;
}

cudaError_t measure_alu_peaks(int num_sms, cudaStream_t st, double* fp32_tflops,
                              double* fp64_tflops)
{
    const int blocks = num_sms * 8;  // 64 warps per SM: 16 per scheduler
    void* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(double) * blocks * PEAK_THREADS);
    if (e != cudaSuccess) return e;
    // about 21 GFLOP in FP32 and 0.65 GFLOP in FP64 per launch
    e = time_chains<float>(blocks, 256, 3, static_cast<float*>(sink), st, fp32_tflops);
    if (e == cudaSuccess)
        e = time_chains<double>(blocks, 8, 3, static_cast<double*>(sink), st, fp64_tflops);
    cudaFree(sink);
    return e;
}

// Issue cost of FP64 fused multiply-adds on one SM, read from the SM clock: one warp running one
// dependent chain (the latency of a chain), one warp running ISSUE_NCH independent chains (the
// rate one scheduler issues FP64 at), and one warp per scheduler (four) running ISSUE_NCH chains
// each (the rate of the SM).  out[w] = elapsed cycles of warp w.
constexpr int ISSUE_NCH = 8;
constexpr int ISSUE_ITERS = 512;

template <int NCH>
__global__ void fp64_issue_kernel(double b, double c, long long* out, double* sink)
{
    double v[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) v[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < ISSUE_ITERS; ++it) {
#pragma unroll
        for (int k = 0; k < NCH; ++k) v[k] = fma(v[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += v[k];
    const long long t1 = clock64();
    if ((threadIdx.x & 31) == 0) out[threadIdx.x >> 5] = t1 - t0;
    if (s == -1.0) sink[threadIdx.x] = s;
}

cudaError_t measure_fp64_issue(cudaStream_t st, double* cycles3)
{
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 64 * sizeof(long long) + 128 * sizeof(double));
    if (e != cudaSuccess) return e;
    long long* out = static_cast<long long*>(buf);
    double* sink = reinterpret_cast<double*>(out + 64);
    long long h[3][4] = {};
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // the first pass warms up
        fp64_issue_kernel<1><<<1, 32, 0, st>>>(0.999999, 1e-7, out, sink);
        fp64_issue_kernel<ISSUE_NCH><<<1, 32, 0, st>>>(0.999999, 1e-7, out + 4, sink);
        fp64_issue_kernel<ISSUE_NCH><<<1, 128, 0, st>>>(0.999999, 1e-7, out + 8, sink);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(buf);
    if (e != cudaSuccess) return e;
    long long w4 = 0;
    for (int w = 0; w < 4; ++w) w4 = h[2][w] > w4 ? h[2][w] : w4;
    cycles3[0] = (double)h[0][0] / ISSUE_ITERS;
    cycles3[1] = (double)h[1][0] / (ISSUE_ITERS * ISSUE_NCH);
    cycles3[2] = (double)w4 / (4.0 * ISSUE_ITERS * ISSUE_NCH);
    return cudaSuccess;
}

}  // namespace art
