// trace_batch.cu -- the batched trace kernel: one persistent launch traces the queued rays of many
// images at once (each queue entry names its image), so rays of uneven length from images of
// different spins, inclinations, fields of view and depths keep every SM busy.  The ray physics is
// shared with the single-image kernel (trace_impl.cuh); only where a ray's job, camera and output
// come from differs.
#include "trace_impl.cuh"

namespace art {

// params3 = n x {a, r_obs, incl_deg}
__global__ void camera_setup_batch_kernel(const double* params3, int n, Camera* cams)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) camera_compute(params3[3 * i], params3[3 * i + 1], params3[3 * i + 2], cams + i);
}

cudaError_t launch_camera_setup_batch(const DevJob*, const double* params3, int n, Camera* cams,
                                      cudaStream_t st)
{
    camera_setup_batch_kernel<<<(n + 31) / 32, 32, 0, st>>>(params3, n, cams);
    return cudaGetLastError();
}

template <class R, bool SWEEP, bool POL>
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
            ray_init<R, POL>(t, J, A.synchs[img], A.cams[img], pix);
            t.img = img;
            t.slot = slot;
            return true;
        }
    };
    active = fetch_next();
    while (__any_sync(0xffffffffu, active)) {
        if (active) {
            const DevJob& J = A.jobs[t.img];
            if (ray_step<R, SWEEP, POL>(t, J, A.synchs[t.img])) {
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

template <bool POL>
static cudaError_t launch_batch_pol(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st)
{
    switch (kind) {
    case TK_FP32:
        if (a.reroute)
            trace_batch_kernel<float, true, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
        else
            trace_batch_kernel<float, false, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    case TK_DF:
        trace_batch_kernel<df, false, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    default:
        trace_batch_kernel<double, false, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_trace_batch(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st)
{
    return a.stokes == 4 ? launch_batch_pol<true>(a, kind, grid, st)
                         : launch_batch_pol<false>(a, kind, grid, st);
}

template <bool POL>
static cudaError_t occ_batch_pol(int kind, int* b)
{
    int b1 = 0, b2 = 0;
    cudaError_t e;
    switch (kind) {
    case TK_FP32:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, trace_batch_kernel<float, true, POL>,
                                                          TRACE_BLOCK, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &b2, trace_batch_kernel<float, false, POL>, TRACE_BLOCK, 0);
        *b = b1 < b2 ? b1 : b2;
        return e;
    case TK_DF:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, trace_batch_kernel<df, false, POL>,
                                                             TRACE_BLOCK, 0);
    default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            b, trace_batch_kernel<double, false, POL>, TRACE_BLOCK, 0);
    }
}

cudaError_t trace_batch_occupancy(int kind, bool pol, int* blocks_per_sm)
{
    return pol ? occ_batch_pol<true>(kind, blocks_per_sm) : occ_batch_pol<false>(kind, blocks_per_sm);
}

}  // namespace art
