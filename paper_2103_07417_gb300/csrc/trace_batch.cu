// trace_batch.cu -- the batched trace kernels of the analytic emission models and the dispatch of
// every batched trace launch over emission kind and polarization.
#include "trace_kernels.cuh"

namespace art {

cudaError_t launch_trace_batch(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st)
{
    if (a.emission == ART_EMIT_GRID) return launch_trace_batch_grid(a, kind, grid, st);
    return launch_batch_em<EM_ANALYTIC>(a, kind, grid, st);
}

cudaError_t trace_batch_occupancy(int kind, int variant, int* blocks_per_sm)
{
    if (variant & TV_GRID) return trace_batch_occupancy_grid(kind, variant, blocks_per_sm);
    return (variant & TV_POL) ? occupancy_batch<EM_ANALYTIC, true>(kind, blocks_per_sm)
                              : occupancy_batch<EM_ANALYTIC, false>(kind, blocks_per_sm);
}

}  // namespace art
