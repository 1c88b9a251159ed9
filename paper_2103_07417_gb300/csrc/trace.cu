// trace.cu -- the single-image trace kernel (one job for every ray of the queue; camera staged in
// shared memory) and the camera set-up kernel.  The ray physics is in trace_impl.cuh.
#include "trace_impl.cuh"

namespace art {

__global__ void camera_setup_kernel(double a, double r_obs, double incl_deg, Camera* cam)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) camera_compute(a, r_obs, incl_deg, cam);
}

cudaError_t launch_camera_setup(const art_job& job, Camera* cam, cudaStream_t st)
{
    camera_setup_kernel<<<1, 32, 0, st>>>(job.a, job.r_obs, job.incl_deg, cam);
    return cudaGetLastError();
}

template <class R, bool SWEEP, bool POL>
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
            ray_init<R, POL>(t, J, S, cam_s, pix);
            t.slot = slot;
            return true;
        }
    };
    active = fetch_next();
    while (__any_sync(0xffffffffu, active)) {
        if (active) {
            if (ray_step<R, SWEEP, POL>(t, J, S)) {
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
                    if (A.img && A.mask) A.mask[t.pix] = ART_MASK_TRACED;
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

template <bool POL>
static cudaError_t launch_trace_pol(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st)
{
    switch (kind) {
    case TK_FP32:
        if (a.reroute)
            trace_kernel<float, true, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
        else
            trace_kernel<float, false, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    case TK_DF:
        trace_kernel<df, false, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
        break;
    default:
        trace_kernel<double, false, POL><<<grid, TRACE_BLOCK, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_trace(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st)
{
    return a.job.stokes == 4 ? launch_trace_pol<true>(a, kind, grid, st)
                             : launch_trace_pol<false>(a, kind, grid, st);
}

template <bool POL>
static cudaError_t occupancy_pol(TraceKind kind, int* blocks_per_sm)
{
    int b1 = 0, b2 = 0;
    cudaError_t e;
    switch (kind) {
    case TK_FP32:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, trace_kernel<float, true, POL>,
                                                          TRACE_BLOCK, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, trace_kernel<float, false, POL>,
                                                              TRACE_BLOCK, 0);
        *blocks_per_sm = b1 < b2 ? b1 : b2;
        return e;
    case TK_DF:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, trace_kernel<df, false, POL>, TRACE_BLOCK, 0);
    default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, trace_kernel<double, false, POL>, TRACE_BLOCK, 0);
    }
}

cudaError_t trace_occupancy(TraceKind kind, bool pol, int* blocks_per_sm)
{
    return pol ? occupancy_pol<true>(kind, blocks_per_sm) : occupancy_pol<false>(kind, blocks_per_sm);
}

}  // namespace art
