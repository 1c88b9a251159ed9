// trace_grid.cu -- the single-image trace kernels of the fluid-grid emission model.
#include "trace_kernels.cuh"

namespace art {

cudaError_t launch_trace_grid(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st)
{
    return launch_single_em<EM_GRID>(a, kind, grid, st);
}

cudaError_t trace_occupancy_grid(TraceKind kind, int variant, int* blocks_per_sm)
{
    return (variant & TV_POL) ? occupancy_single<EM_GRID, true>(kind, blocks_per_sm)
                              : occupancy_single<EM_GRID, false>(kind, blocks_per_sm);
}

}  // namespace art
