// internal.cuh -- declarations shared by the library's translation units (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/art.h"
#include "kerr.cuh"
#include "synch.cuh"

namespace art {

// Device counters of one context (one array of unsigned long long in device memory).
enum Counter {
    C_QUEUE = 0,     // length of the ray queue of the current level
    C_FETCH = 1,     // next queue slot to trace (persistent-kernel work counter)
    C_REROUTE = 2,   // length of the FP64 re-trace queue (mixed precision)
    C_FETCH2 = 3,    // work counter of the re-trace pass
    C_STEPS = 4,     // RK4 steps, summed over rays
    C_CAPPED = 5,    // rays that hit max_steps
    C_NAN = 6,       // rays stopped by a non-finite state
    C_BADIDX = 7,    // queue entries outside the image (skipped)
    C_FP64 = 8,      // rays re-traced by the high-precision pass of the mixed modes
    C_SPECFROM = 9,  // learned path: first queue slot of the speculative rays of this level
    C_SPEC = 10,     // learned path: rays queued speculatively (all levels)
    C_SPECUSED = 11, // learned path: speculative rays the exact criterion asked for
    C_SYNCERR = 12,  // warp-pair trace kernels: a hand-over wait that ran out of time
    C_BORDER = 13,   // exact decisions: borderline points of the current level
    C_XQ = 14,       // exact decisions: length of the FP64 queue of the current level
    C_FIXQ = 15,     // exact decisions: interpolated points to recompute at the current level
    C_LEVEL0 = 16,   // C_LEVEL0 + k: rays of level k (16 slots)
    C_CERTERR = 32,  // exact decisions: a stencil value was not exact when it was used
    C_XRAYS = 33,    // exact decisions: FP64 rays traced for them (all levels)
    C_BTOT = 34,     // exact decisions: borderline points (all levels)
    C_CERTOVF = 35,  // exact decisions: points decided without them (lists full)
    C_SPECN = 36,    // exact decisions: length of the speculative part of the base-level queue
    C_ZERO = 37,     // always 0
    C_DEGEN = 38,    // exact decisions: the normalisation is outside FP32's range (all FP64)
    C_QF32 = 39,     // exact decisions: rays of the level for the FP32 pass
    C_QF64 = 40,     // exact decisions: rays of the level for the FP64 pass (degenerate images)
    C_REROUTE2 = 41, // exact decisions: double-float rays handed on to FP64
    C_AXQ = 42,      // third axis: length of the level's queue after the axis filter
    C_AXKEPT = 43,   // third axis: rays kept by the filter (all levels)
    C_AXINTERP = 44, // third axis: points interpolated along the axis (all levels)
    C_MAXSTEP = 45,  // profiler: most RK4 steps of one ray since the last trace launch
    C_RAYCNT = 46,   // profiler: rays finished (or handed on), summed
    C_COUNT = 64
};

// Exact-decision state of a pixel (one byte per pixel, ART_MIXED_EXACT): its value equals the
// FP64 render's (FP64-traced, or interpolated from such values); claimed by the closure search.
constexpr uint8_t XS_EXACT = 1, XS_CLAIM = 2;
// Transient mask value of a borderline point whose decision waits for exact stencil values.
constexpr uint8_t MASK_PENDING = 10;

struct TraceArgs {
    DevJob job;
    SynchConst synch;
    SynchConstF synchf;  // its float copy (the FP32 and double-float kernels' transfer)
    const Camera* cam;
    const int32_t* queue;           // pixel indices
    const int32_t* indirect;        // nullable: slot -> queue position (re-trace pass)
    const unsigned long long* count;// number of slots to trace
    unsigned long long* fetch;      // work counter, zeroed before the launch
    unsigned long long* counters;   // the context's counter array
    double* img;                    // image mode: planes x npix (nullable)
    uint8_t* mask;                  // image mode: nullable
    double* out;                    // ray mode: [queue position][plane] (nullable)
    int32_t* reroute;               // mixed FP32 pass: queue positions to re-trace in FP64
    unsigned long long* reroute_count;
    int32_t* aux_status;
    int32_t* aux_steps;
    int32_t* aux_nturn;
    float* aux_minr;
    int64_t npix;
    // image mode, learned path: per-pixel diagnostics planes (nullable) and the first queue slot
    // of speculative rays (nullable; slots at or beyond it are marked MASK_SPEC_DONE)
    float* pix_minr;
    float* pix_turn;
    uint16_t* pix_steps;  // nullable: RK4 steps of each traced pixel's ray (saturated at 65535)
    const unsigned long long* spec_from;
    // kernel forms of the FP32 pass (trace_kernels.cuh): queues of at most quad_rays rays per
    // block take the four-warp form, of at most pair_rays the two-warp form (art_tune)
    int32_t quad_rays, pair_rays;
    // FP64 launches: queues of at most quad64_rays rays per block take the four-warp form
    int32_t quad64_rays;
};

// Transient mask values of the learned path (a render ends with every point TRACED or INTERP).
constexpr uint8_t MASK_SPEC_PENDING = 8, MASK_SPEC_DONE = 9;

// Batched rendering: the rays of many images share one queue whose entries are
// (image << 32) | pixel; each image's job, synchrotron constants, camera and output live in tables.
struct BatchTraceArgs {
    const DevJob* jobs;
    const SynchConst* synchs;
    const SynchConstF* synchfs;  // their float copies
    const Camera* cams;
    double* const* imgs;
    uint8_t* const* masks;           // table entries may be null
    const int64_t* queue;
    const int32_t* indirect;         // nullable: slot -> queue position (re-trace pass)
    const unsigned long long* count;
    unsigned long long* fetch;
    unsigned long long* counters;
    int32_t* reroute;
    unsigned long long* reroute_count;
    // first queue slot of the speculative (near-critical band) rays: slots at or beyond it are
    // marked MASK_SPEC_DONE (nullable)
    const unsigned long long* spec_from;
    int planes, stokes, precision, emission;
};

// Trace-kernel variants for occupancy queries: polarized and/or fluid-grid emission.
enum TraceVariant { TV_POL = 1, TV_GRID = 2, TV_COUNT = 4 };

// trace.cu / trace_batch.cu (dispatch) and trace_grid.cu / trace_grid_batch.cu (grid kernels)
cudaError_t launch_camera_setup_batch(const DevJob* jobs_host_unused, const double* params3,
                                      int n, Camera* cams, cudaStream_t st);
cudaError_t launch_trace_batch(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st);
cudaError_t trace_batch_occupancy(int kind, int variant, int* blocks_per_sm);
cudaError_t launch_trace_batch_grid(const BatchTraceArgs& a, int kind, int grid, cudaStream_t st);
cudaError_t trace_batch_occupancy_grid(int kind, int variant, int* blocks_per_sm);

// refine.cu (batched)
cudaError_t launch_enqueue_base_batch(const DevJob* jobs, int n, int max_base, int64_t* queue,
                                      unsigned long long* qcount, unsigned long long* img_counts,
                                      cudaStream_t st);
cudaError_t launch_norm_batch(const DevJob* jobs, double* const* imgs, int n, double* norms,
                              cudaStream_t st);
cudaError_t launch_refine_batch(const DevJob* jobs, int n, int level, int max_kx, int max_ky,
                                const double* norms, double* const* imgs, uint8_t* const* masks,
                                int64_t* queue, unsigned long long* qcount,
                                unsigned long long* img_counts, cudaStream_t st,
                                unsigned long long* spec_counters = nullptr);

// trace.cu
enum TraceKind { TK_FP64 = 0, TK_FP32 = 1, TK_DF = 2 };
cudaError_t launch_camera_setup(const art_job& job, Camera* cam, cudaStream_t st);
cudaError_t launch_trace(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st);
cudaError_t trace_occupancy(TraceKind kind, int variant, int* blocks_per_sm);
cudaError_t launch_trace_grid(const TraceArgs& a, TraceKind kind, int grid, cudaStream_t st);
cudaError_t trace_occupancy_grid(TraceKind kind, int variant, int* blocks_per_sm);
constexpr int TRACE_BLOCK = 128;

// refine.cu
cudaError_t launch_enqueue_base(const DevJob& J, int32_t* queue, unsigned long long* counters,
                                cudaStream_t st);
cudaError_t launch_gather_truth(const DevJob& J, const int32_t* queue,
                                const unsigned long long* count, const double* truth,
                                double* img, uint8_t* mask, int64_t cap, cudaStream_t st);
cudaError_t launch_norm(const DevJob& J, const double* img, int nx, int ny, int stride,
                        double* norm3, cudaStream_t st);
cudaError_t launch_refine(const DevJob& J, int level, const double* norm, double* img,
                          uint8_t* mask, int32_t* queue, unsigned long long* count,
                          cudaStream_t st, float* aux_minr = nullptr, float* aux_turn = nullptr,
                          unsigned long long* spec_used = nullptr);
cudaError_t launch_level_count(unsigned long long* counters, int level, cudaStream_t st);
// refine.cu: exact decisions (ART_MIXED_EXACT)
cudaError_t launch_refine_cert(const DevJob& J, int level, const double* norm, double* img,
                               uint8_t* mask, int32_t* queue, unsigned long long* count,
                               cudaStream_t st, float* aux_minr, float* aux_turn,
                               unsigned long long* spec_counters, uint8_t* xst, double band,
                               int32_t* border, unsigned long long* counters,
                               unsigned long long border_cap);
cudaError_t launch_cert_mark_base(const DevJob& J, uint8_t* xst, cudaStream_t st);
cudaError_t launch_cert_spec_count(unsigned long long* counters, cudaStream_t st);
cudaError_t launch_cert_closure(const DevJob& J, int level, const int32_t* border,
                                unsigned long long border_cap, unsigned long long* counters,
                                uint8_t* xst, const uint8_t* mask, int32_t* xq,
                                unsigned long long xq_cap, uint64_t* fixq,
                                unsigned long long fix_cap, cudaStream_t st);
cudaError_t launch_cert_mark_traced(const int32_t* xq, unsigned long long* counters,
                                    unsigned long long xq_cap, uint8_t* xst, cudaStream_t st,
                                    int count_idx = C_XQ);
cudaError_t launch_cert_check_norm(const double* norm3, unsigned long long* counters,
                                   cudaStream_t st);
cudaError_t launch_cert_split(unsigned long long* counters, cudaStream_t st);
cudaError_t launch_cert_take_uncertain(const int32_t* queue, const int32_t* reroute2,
                                       unsigned long long* counters, int count_idx,
                                       const unsigned long long* spec_from, uint8_t* mask,
                                       int32_t* xq, unsigned long long xq_cap, cudaStream_t st);
cudaError_t launch_cert_fixup(const DevJob& J, const uint64_t* fixq, unsigned long long* counters,
                              unsigned long long fix_cap, int lvl, double* img, uint8_t* xst,
                              cudaStream_t st);
cudaError_t launch_cert_redecide(const DevJob& J, int level, const double* norm,
                                 const int32_t* border, unsigned long long* counters,
                                 unsigned long long border_cap, double* img, uint8_t* mask,
                                 uint8_t* xst, float* aminr, float* aturn, cudaStream_t st);
cudaError_t launch_counter_clamp(unsigned long long* counters, int idx, unsigned long long cap,
                                 cudaStream_t st);
// refine.cu: a third sampling axis (art_render_axis)
cudaError_t launch_axis_refine(int64_t npix, int planes, double* const* imgs, int f, int s, int F,
                               double norm, double R_rel, double R_abs, int32_t* queue,
                               unsigned long long* qcount, uint8_t* amask, cudaStream_t st);
cudaError_t launch_axis_filter(int64_t npix, int planes, double* const* imgs, int f, int s, int F,
                               double norm, double R_rel, double R_abs, const int32_t* queue,
                               unsigned long long* counters, int32_t* out, uint8_t* mask,
                               int num_sms, cudaStream_t st);
cudaError_t launch_spec_mark(unsigned long long* counters, cudaStream_t st);
cudaError_t launch_queue_clamp(unsigned long long* counters, unsigned long long cap,
                               cudaStream_t st);
cudaError_t launch_metrics(const double* truth, const double* img, const uint8_t* mask, int nx,
                           int ny, double* partials, int nblocks, double* out6, cudaStream_t st);
constexpr int METRIC_BLOCKS = 304;

// vis.cu: visibilities of a (residual) image, V and Q m x m complex, tables of
// vis_table_doubles() doubles
int vis_table_doubles(int m, int nx, int ny);
cudaError_t launch_visibilities(const double* img, const double* ref, int nx, int ny, double dx,
                                double fwhm, int m, double2* V, double2* Q, double* tables,
                                cudaStream_t st);

// peaks.cu: measured FP32 / FP64 fused multiply-add throughput (TFLOP/s)
cudaError_t measure_alu_peaks(int num_sms, cudaStream_t st, double* fp32_tflops,
                              double* fp64_tflops);
cudaError_t measure_fp64_issue(cudaStream_t st, double* cycles3);
// Longest first: the pixels of q_in (count entries, at most cap) into q_out in descending order
// of their rays' expected RK4 steps (refine.cu); hist: LPT_BUCKETS + 1 scratch counters.
constexpr int LPT_BUCKETS = 256;
cudaError_t launch_lpt_order(const DevJob& J, const int32_t* q_in,
                             const unsigned long long* count, unsigned long long cap,
                             const uint16_t* pix_steps, const uint8_t* mask, int32_t* q_out,
                             unsigned int* hist, int num_sms, cudaStream_t st);

// cnn.cu
struct CnnState;
void cnn_destroy(CnnState* s);
cudaError_t cnn_load(CnnState*& s, const float* host_params, cudaStream_t st);
cudaError_t cnn_read(CnnState* s, float* host_params, cudaStream_t st);
int cnn_forward(CnnState* s, const float* feat, int H, int W, float* prob, cudaStream_t st);
int cnn_grad(CnnState* s, const float* feat, int H, int W, const float* target, float* loss,
             float* grad_host, cudaStream_t st);
int cnn_train_step(CnnState* s, const float* feat, int H, int W, const float* target, float lr,
                   float* loss, cudaStream_t st);
// learned path: features of a level lattice from the image and diagnostics planes (BF16 into the
// network's input, or FP32 for training), the proposal of speculative rays, training targets
cudaError_t cnn_propose(CnnState* s, const DevJob& J, int level_in, int depth, const double* img,
                        const float* minr, const float* turn, const double* norm, float thr,
                        float* prob_scratch, uint8_t* mask, int32_t* queue,
                        unsigned long long* counters, unsigned long long cap, cudaStream_t st);
cudaError_t cnn_features_f32(const DevJob& J, int level, const double* img, const float* minr,
                             const float* turn, const double* norm, float* feat, cudaStream_t st);
cudaError_t cnn_targets(const DevJob& J, int level, const uint8_t* mask, float* target,
                        cudaStream_t st);
int64_t cnn_head_cells(const DevJob& J, int level);
// band.cu
cudaError_t launch_band_propose(const DevJob& J, const Camera* cam, double band, uint8_t* mask,
                                int32_t* queue, unsigned long long* counters,
                                unsigned long long cap, int num_sms, cudaStream_t st);
cudaError_t launch_band_propose_batch(const DevJob* jobs, const Camera* cams, const float* bands,
                                      uint8_t* const* masks, int n, int64_t max_npix,
                                      int64_t* queue, unsigned long long* counters,
                                      unsigned long long cap, cudaStream_t st);

}  // namespace art
