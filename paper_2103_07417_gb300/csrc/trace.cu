// trace.cu -- the camera set-up kernels and the single-image trace kernels of the analytic
// emission models; the dispatch of every trace launch over emission kind and polarization.
#include "trace_kernels.cuh"

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

cudaError_t launch_trace(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st)
{
    if (a.job.emission == ART_EMIT_GRID)
        return a.synch.grid ? launch_trace_grid(a, kind, grid, st) : cudaErrorInvalidValue;
    return launch_single_em<EM_ANALYTIC>(a, kind, grid, st);
}

cudaError_t trace_occupancy(TraceKind kind, int variant, int* blocks_per_sm)
{
    if (variant & TV_GRID) return trace_occupancy_grid(kind, variant, blocks_per_sm);
    return (variant & TV_POL) ? occupancy_single<EM_ANALYTIC, true>(kind, blocks_per_sm)
                              : occupancy_single<EM_ANALYTIC, false>(kind, blocks_per_sm);
}

}  // namespace art
