// trace_kernels.cuh -- the persistent trace kernels, as templates over the geodesic arithmetic R,
// the sweep-angle routing of the FP32 pass, polarization and the emission kernel kind (analytic
// models or the fluid grid), plus the launch and occupancy dispatch over them.  Each translation
// unit instantiates one emission kind for the single-image (trace_kernel) or the batched
// (trace_batch_kernel) form: trace.cu, trace_batch.cu, trace_grid.cu, trace_grid_batch.cu.
//
// Single image: one job for every ray of the queue, camera staged in shared memory.
// Batched: one persistent launch traces the queued rays of many images at once (each queue entry
// names its image), so rays of uneven length from images of different spins, inclinations, fields
// of view and depths keep every SM busy; only where a ray's job, camera and output come from
// differs from the single-image kernel.
#pragma once
#include "trace_impl.cuh"

namespace art {

template <class R, bool SWEEP, bool POL, int EM>
__global__ void __launch_bounds__(TRACE_BLOCK) trace_kernel(TraceArgs A)
{
    __shared__ Camera cam_s;
    {
        const double* src = reinterpret_cast<const double*>(A.cam);
        double* dst = reinterpret_cast<double*>(&cam_s);
        for (int q = threadIdx.x; q < (int)(sizeof(Camera) / sizeof(double)); q += blockDim.x)
            dst[q] = src[q];
    }
    __syncthreads();
    const DevJob& J = A.job;
    const SynchConst& S = A.synch;
    const unsigned long long n = *A.count;
    const bool mixed32 = (A.reroute != nullptr);
    Tracer<R> t;
    bool active = false;
    auto fetch_next = [&]() {
        while (true) {
            unsigned long long q = warp_fetch(A.fetch);
            if (q >= n) return false;
            int64_t slot = A.indirect ? (int64_t)A.indirect[q] : (int64_t)q;
            int32_t pix = A.queue[slot];
            if (pix < 0 || (int64_t)pix >= A.npix) {
                atomicAdd(A.counters + C_BADIDX, 1ull);
                continue;
            }
            ray_init<R, POL, EM>(t, J, S, cam_s, pix);
            t.slot = slot;
            return true;
        }
    };
    active = fetch_next();
    while (__any_sync(0xffffffffu, active)) {
        if (active) {
            if (ray_step<R, SWEEP, POL, EM>(t, J, S)) {
                atomicAdd(A.counters + C_STEPS, (unsigned long long)t.steps);
                bool rer = mixed32 && (t.status == RAY_REROUTE || t.status == ART_RAY_NAN ||
                                       t.status == ART_RAY_CAP);
                if (rer) {
                    unsigned long long w = atomicAdd(A.reroute_count, 1ull);
                    A.reroute[w] = (int32_t)t.slot;
                } else {
                    if (t.status == ART_RAY_CAP) atomicAdd(A.counters + C_CAPPED, 1ull);
                    if (t.status == ART_RAY_NAN) atomicAdd(A.counters + C_NAN, 1ull);
                    if (A.indirect) atomicAdd(A.counters + C_FP64, 1ull);  // re-trace pass
                    const int np = J.planes;
#pragma unroll
                    for (int p = 0; p < MAXPL; ++p) {
                        if (p < np) {
                            if (A.img) A.img[(int64_t)p * A.npix + t.pix] = double(t.acc[p]);
                            if (A.out) A.out[t.slot * np + p] = double(t.acc[p]);
                        }
                    }
                    if (A.img && A.mask)
                        A.mask[t.pix] = (A.spec_from && (unsigned long long)t.slot >= *A.spec_from)
                                            ? MASK_SPEC_DONE
                                            : (uint8_t)ART_MASK_TRACED;
                    if (A.img && A.pix_minr) {
                        A.pix_minr[t.pix] = t.min_r;
                        A.pix_turn[t.pix] = (float)t.nturn;
                    }
                    if (A.aux_status) A.aux_status[t.slot] = t.status;
                    if (A.aux_steps) A.aux_steps[t.slot] = t.steps;
                    if (A.aux_nturn) A.aux_nturn[t.slot] = t.nturn;
                    if (A.aux_minr) A.aux_minr[t.slot] = t.min_r;
                }
                active = fetch_next();
            }
        }
    }
}

template <class R, bool SWEEP, bool POL, int EM>
__global__ void __launch_bounds__(TRACE_BLOCK) trace_batch_kernel(BatchTraceArgs A)
{
    const unsigned long long n = *A.count;
    const bool mixed32 = (A.reroute != nullptr);
    Tracer<R> t;
    bool active = false;
    auto fetch_next = [&]() {
        while (true) {
            unsigned long long q = warp_fetch(A.fetch);
            if (q >= n) return false;
            int64_t slot = A.indirect ? (int64_t)A.indirect[q] : (int64_t)q;
            int64_t e = A.queue[slot];
            int32_t img = (int32_t)(e >> 32), pix = (int32_t)(e & 0xffffffff);
            const DevJob& J = A.jobs[img];
            if (pix < 0 || (int64_t)pix >= (int64_t)J.nx * J.ny) {
                atomicAdd(A.counters + C_BADIDX, 1ull);
                continue;
            }
            ray_init<R, POL, EM>(t, J, A.synchs[img], A.cams[img], pix);
            t.img = img;
            t.slot = slot;
            return true;
        }
    };
    active = fetch_next();
    while (__any_sync(0xffffffffu, active)) {
        if (active) {
            const DevJob& J = A.jobs[t.img];
            if (ray_step<R, SWEEP, POL, EM>(t, J, A.synchs[t.img])) {
                atomicAdd(A.counters + C_STEPS, (unsigned long long)t.steps);
                bool rer = mixed32 && (t.status == RAY_REROUTE || t.status == ART_RAY_NAN ||
                                       t.status == ART_RAY_CAP);
                if (rer) {
                    unsigned long long w = atomicAdd(A.reroute_count, 1ull);
                    A.reroute[w] = (int32_t)t.slot;
                } else {
                    if (t.status == ART_RAY_CAP) atomicAdd(A.counters + C_CAPPED, 1ull);
                    if (t.status == ART_RAY_NAN) atomicAdd(A.counters + C_NAN, 1ull);
                    if (A.indirect) atomicAdd(A.counters + C_FP64, 1ull);
                    const int64_t npix = (int64_t)J.nx * J.ny;
                    double* img = A.imgs[t.img];
#pragma unroll
                    for (int p = 0; p < MAXPL; ++p)
                        if (p < A.planes) img[(int64_t)p * npix + t.pix] = double(t.acc[p]);
                    uint8_t* mask = A.masks[t.img];
                    if (mask) mask[t.pix] = ART_MASK_TRACED;
                }
                active = fetch_next();
            }
        }
    }
}

template <int EM, bool POL>
static cudaError_t launch_single(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st)
{
    switch (kind) {
    case TK_FP32:
        if (a.reroute)
            trace_kernel<float, true, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
        else
            trace_kernel<float, false, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    case TK_DF:
        trace_kernel<df, false, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    default:
        trace_kernel<double, false, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <int EM>
static cudaError_t launch_single_em(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st)
{
    return a.job.stokes == 4 ? launch_single<EM, true>(a, kind, grid, st)
                             : launch_single<EM, false>(a, kind, grid, st);
}

template <int EM, bool POL>
static cudaError_t occupancy_single(TraceKind kind, int* blocks_per_sm)
{
    int b1 = 0, b2 = 0;
    cudaError_t e;
    switch (kind) {
    case TK_FP32:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, trace_kernel<float, true, POL, EM>,
                                                          TRACE_BLOCK, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &b2, trace_kernel<float, false, POL, EM>, TRACE_BLOCK, 0);
        *blocks_per_sm = b1 < b2 ? b1 : b2;
        return e;
    case TK_DF:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, trace_kernel<df, false, POL, EM>, TRACE_BLOCK, 0);
    default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, trace_kernel<double, false, POL, EM>, TRACE_BLOCK, 0);
    }
}

template <int EM, bool POL>
static cudaError_t launch_batch(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st)
{
    switch (kind) {
    case TK_FP32:
        if (a.reroute)
            trace_batch_kernel<float, true, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
        else
            trace_batch_kernel<float, false, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    case TK_DF:
        trace_batch_kernel<df, false, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    default:
        trace_batch_kernel<double, false, POL, EM><<<grid, TRACE_BLOCK, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <int EM>
static cudaError_t launch_batch_em(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st)
{
    return a.stokes == 4 ? launch_batch<EM, true>(a, kind, grid, st)
                         : launch_batch<EM, false>(a, kind, grid, st);
}

template <int EM, bool POL>
static cudaError_t occupancy_batch(int kind, int* b)
{
    int b1 = 0, b2 = 0;
    cudaError_t e;
    switch (kind) {
    case TK_FP32:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b1, trace_batch_kernel<float, true, POL, EM>, TRACE_BLOCK, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &b2, trace_batch_kernel<float, false, POL, EM>, TRACE_BLOCK, 0);
        *b = b1 < b2 ? b1 : b2;
        return e;
    case TK_DF:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            b, trace_batch_kernel<df, false, POL, EM>, TRACE_BLOCK, 0);
    default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            b, trace_batch_kernel<double, false, POL, EM>, TRACE_BLOCK, 0);
    }
}

}  // namespace art
