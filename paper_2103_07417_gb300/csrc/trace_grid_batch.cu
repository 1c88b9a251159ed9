// trace_grid_batch.cu -- the batched trace kernels of the fluid-grid emission model.
#include "trace_kernels.cuh"

namespace art {

cudaError_t launch_trace_batch_grid(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st)
{
    return launch_batch_em<EM_GRID>(a, kind, grid, st);
}

cudaError_t trace_batch_occupancy_grid(int kind, int variant, int* blocks_per_sm)
{
    return (variant & TV_POL) ? occupancy_batch<EM_GRID, true>(kind, blocks_per_sm)
                              : occupancy_batch<EM_GRID, false>(kind, blocks_per_sm);
}

}  // namespace art
