// capi.cu -- the C-ABI of include/art.h: context, job validation, scratch management and the
// level loop of Sec. 3.2 driven entirely on the device (one stream, no host round trip between
// levels: queue lengths live in device counters that the persistent trace kernel reads).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"

using namespace art;

struct art_ctx {
    art_tune tune = {ART_TUNE_QUAD_DEFAULT, ART_TUNE_PAIR_DEFAULT, ART_TUNE_BLOCKS64_DEFAULT, 0,
                ART_TUNE_QUAD64_DEFAULT};
    // exact decisions in a batch (art_render_batch): sub-contexts, each with a stream of its own
    // and its own scratch, render the images concurrently; every image's counters and
    // normalisation are copied into xsnap on its sub-context's stream
    std::vector<art_ctx*> subs;
    bool owns_stream = false;
    cudaEvent_t sub_in = nullptr;
    std::vector<cudaEvent_t> sub_out;
    unsigned long long* xsnap = nullptr;
    int64_t xsnap_cap = 0;
    // exact decisions: each traced pixel's RK4 steps, the longest-first copy of an FP64 queue and
    // its sort's counters; cur_steps is what trace launches record into (null outside them)
    uint16_t* steps_map = nullptr;
    int64_t steps_cap = 0;
    int32_t* lptq = nullptr;
    int64_t lptq_cap = 0;
    unsigned int* lpt_hist = nullptr;
    uint16_t* cur_steps = nullptr;
    // bumped whenever a scratch buffer is (re)allocated: a captured graph holds the pointers of
    // its capture and is replayed only while this is unchanged
    uint64_t scratch_gen = 0;
    uint64_t ggen = 0, gbgen = 0;
    // CUDA-graph replay of the level loop (art_graph_render): the captured graph, the call it
    // replays, and a capture stream ordered against the context's stream by two events
    cudaGraphExec_t gexec = nullptr;
    art_job gjob = {};
    double* gimg = nullptr;
    uint8_t* gmask = nullptr;
    art_tune gtune = {};
    const float* ggrid = nullptr;
    double ggmeta[5] = {};  // grid dimensions and radial range baked into the captured launches
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    // the same for art_graph_render_batch: graph, the batch it replays and its host plan
    cudaGraphExec_t gbexec = nullptr;
    std::vector<art_job> gbjobs;
    std::vector<double*> gbimgs;
    std::vector<uint8_t*> gbmasks;
    const float* gbgrid = nullptr;
    double gbgmeta[5] = {};
    struct BatchPlan* gbplan = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int occ[3][TV_COUNT] = {};   // resident blocks per SM of the trace kernels [kind][variant]
    int occb[3][TV_COUNT] = {};  // the same for the batched trace kernels
    // fluid grid of ART_EMIT_GRID (art_load_grid): referenced, or owned when copied from the host
    const float* grid = nullptr;
    float* grid_owned = nullptr;
    int32_t g_n1 = 0, g_n2 = 0, g_n3 = 0;
    double g_x1min = 0.0, g_x1max = 0.0;
    // learned block proposal (cnn.cu): the network, per-pixel diagnostics planes of the last
    // render (min r, polar turns), a scratch mask and the proposal probabilities
    CnnState* cnn = nullptr;
    float* aux = nullptr;
    int64_t aux_cap = 0, aux_npix = 0;
    uint8_t* smask = nullptr;
    int64_t smask_cap = 0;
    // exact decisions (ART_MIXED_EXACT): per-pixel exactness bytes, the borderline list, the FP64
    // queue and the list of interpolants to recompute of the current level
    uint8_t* xst = nullptr;
    int64_t xst_cap = 0;
    int32_t* cborder = nullptr;
    int64_t cborder_cap = 0;
    int32_t* cxq = nullptr;
    int64_t cxq_cap = 0;
    uint64_t* cfixq = nullptr;
    int64_t cfixq_cap = 0;
    // visibilities (art_visibilities): m x m complex scratch and the transform's tables
    double2* vq = nullptr;
    int64_t vq_cap = 0;
    double* vtab = nullptr;
    int64_t vtab_cap = 0;
    // third sampling axis (art_render_axis): device table of the samples' images, ray counts
    double** atab = nullptr;
    int64_t atab_cap = 0;
    int32_t* aq = nullptr;  // a level's queue after the axis filter
    int64_t aq_cap = 0;
    float* prob = nullptr;
    int64_t prob_cap = 0;
    // batched rendering tables and queue (grown, never shrunk)
    DevJob* bjobs = nullptr;
    SynchConst* bsynch = nullptr;
    SynchConstF* bsynchf = nullptr;
    Camera* bcams = nullptr;
    double* bparams = nullptr;
    double** bimgs = nullptr;
    uint8_t** bmasks = nullptr;
    double* bnorms = nullptr;
    unsigned long long* bcounts = nullptr;
    unsigned long long* bcounts_host = nullptr;
    int bcap = 0;
    int64_t* bqueue = nullptr;
    int32_t* breroute = nullptr;
    int64_t bqcap = 0;
    float* bband = nullptr;      // per image: near-critical band width (0: none)
    uint8_t* bsmask = nullptr;   // scratch masks of band batches whose caller passed none
    int64_t bsmask_cap = 0;
    // scratch owned by the library
    int32_t* queue = nullptr;
    int32_t* reroute = nullptr;
    int32_t* reroute2 = nullptr;  // exact decisions: double-float rays handed on to FP64
    int64_t queue_cap = 0;
    unsigned long long* counters = nullptr;
    double* norm3 = nullptr;
    Camera* cam = nullptr;
    double* partials = nullptr;
    double* out6 = nullptr;
    double* himg = nullptr;   // art_render_host buffers
    uint8_t* hmask = nullptr;
    int64_t hcap = 0;
    unsigned long long* pinned = nullptr;  // host copy of the counters
    double* pinned_d = nullptr;
    int64_t launches = 0;                  // kernels launched by the current call
    // profiler
    static const int PROF_MAX = 256;
    bool prof_on = false;
    int prof_n = 0;
    cudaEvent_t ev[2 * PROF_MAX] = {};
    art_launch_record rec[PROF_MAX];
    unsigned long long* prof_steps = nullptr;  // device snapshots (steps, longest ray, rays) per launch
    int prof_level = -1;
};

struct BatchPlan;
static void destroy_plan(BatchPlan* p);

// Profiler brackets: prof_begin before a launch, prof_end after it.
static int prof_begin(art_ctx* c)
{
    ++c->launches;
    if (!c->prof_on || c->prof_n >= art_ctx::PROF_MAX) return -1;
    int k = c->prof_n;
    if (cudaEventRecord(c->ev[2 * k], c->stream) != cudaSuccess) return -1;
    return k;
}

static void prof_end(art_ctx* c, int k, int kind, int64_t items)
{
    if (k < 0) return;
    cudaEventRecord(c->ev[2 * k + 1], c->stream);
    c->rec[k].kind = kind;
    c->rec[k].level = c->prof_level;
    c->rec[k].ms = 0.f;
    c->rec[k].steps = 0;
    c->rec[k].items = items;
    if (kind == ART_K_TRACE_FP64 || kind == ART_K_TRACE_FP32 || kind == ART_K_TRACE_DF) {
        // snapshots of the summed steps and rays and of the launch's longest ray (reset after)
        unsigned long long* snap = c->prof_steps + 3 * k;
        cudaMemcpyAsync(snap, c->counters + C_STEPS, sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(snap + 1, c->counters + C_MAXSTEP, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, c->stream);
        cudaMemsetAsync(c->counters + C_MAXSTEP, 0, sizeof(unsigned long long), c->stream);
    }
    c->prof_n = k + 1;
}

#define CK(x)                                    \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return err_of(e_); \
    } while (0)

static int err_of(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? ART_ERR_OOM : ART_ERR_CUDA;
}

extern "C" const char* art_strerror(int code)
{
    switch (code) {
    case ART_OK: return "ok";
    case ART_ERR_ARG: return "invalid argument";
    case ART_ERR_CUDA: return "CUDA runtime error";
    case ART_ERR_OOM: return "device allocation failed";
    case ART_ERR_UNSUPPORTED: return "unsupported option";
    case ART_ERR_DEVICE: return "kernel reported an inconsistency";
    default: return "unknown error";
    }
}

extern "C" int art_image_size(const art_job* job, int32_t* nx, int32_t* ny)
{
    if (!job || !nx || !ny) return ART_ERR_ARG;
    if (job->n0x < 2 || job->n0y < 1 || job->levels < 0 || job->levels > 14) return ART_ERR_ARG;
    int64_t x = ((int64_t)1 << job->levels) * (job->n0x - 1) + 1;
    int64_t y = ((int64_t)1 << job->levels) * (job->n0y - 1) + 1;
    if (x * y >= ((int64_t)1 << 31)) return ART_ERR_ARG;
    *nx = (int32_t)x;
    *ny = (int32_t)y;
    return ART_OK;
}

extern "C" int art_planes(const art_job* job)
{
    if (!job) return ART_ERR_ARG;
    return (job->stokes == 4 ? 4 : 1) * (job->subrings > 0 ? job->subrings : 1);
}

static double horizon(double a) { return 1.0 + sqrt(1.0 - a * a); }

// Validate the job and derive the kernels' view of it.
static int make_devjob(const art_job* job, DevJob* J)
{
    if (!job) return ART_ERR_ARG;
    int32_t nx, ny;
    if (art_image_size(job, &nx, &ny) != ART_OK) return ART_ERR_ARG;
    if (!(fabs(job->a) < 1.0) || !(job->r_obs > 10.0) || !(job->fov > 0.0)) return ART_ERR_ARG;
    if (!(job->incl_deg > 0.0 && job->incl_deg < 180.0)) return ART_ERR_ARG;
    if (!(job->step_frac > 0.0 && job->step_frac <= 0.5) || !(job->h_min > 0.0)) return ART_ERR_ARG;
    if (job->max_steps < 1 || !(job->escape_frac > 1.0) || !(job->horizon_eps >= 0.0))
        return ART_ERR_ARG;
    if (!(job->escape_frac * job->r_obs <= 1e8)) return ART_ERR_ARG;  // the tracers form r^4 in FP32
    if (job->stokes != 1 && job->stokes != 4) return ART_ERR_UNSUPPORTED;
    if (job->subrings < 0 || job->subrings > 4) return ART_ERR_UNSUPPORTED;
    if (job->emission != ART_EMIT_ANALYTIC && job->emission != ART_EMIT_SYNCH_DISK &&
        job->emission != ART_EMIT_GRID)
        return ART_ERR_UNSUPPORTED;
    if (job->stokes == 4 && job->emission == ART_EMIT_ANALYTIC) return ART_ERR_UNSUPPORTED;
    if (job->emission == ART_EMIT_SYNCH_DISK &&
        (!(job->ne0 >= 0.0) || !(job->thetae0 > 0.0) || !(job->b0 > 0.0) || !(job->nu_hz > 0.0) ||
         !(job->length_cm > 0.0) || !(job->r_in >= 0.0)))
        return ART_ERR_ARG;
    if (job->emission == ART_EMIT_GRID &&
        (!(job->nu_hz > 0.0) || !(job->length_cm > 0.0) || !(job->gamma_ad > 1.0) ||
         !(job->m_unit > 0.0) || !(job->r_high > 0.0) || !(job->r_low > 0.0) ||
         !(job->sigma_cut > 0.0)))
        return ART_ERR_ARG;
    if (job->flow != ART_FLOW_KEPLER && job->flow != ART_FLOW_STATIC) return ART_ERR_ARG;
    if (job->interp != ART_INTERP_LINEAR && job->interp != ART_INTERP_NEAREST) return ART_ERR_ARG;
    if (job->edge_mode != ART_EDGE_ONESIDED && job->edge_mode != ART_EDGE_TRACE) return ART_ERR_ARG;
    if (job->abs_norm != ART_NORM_IBAR_INT && job->abs_norm != ART_NORM_PEAK) return ART_ERR_ARG;
    if (job->precision < ART_FP64 || job->precision > ART_MIXED_EXACT) return ART_ERR_ARG;
    if (!(job->disk_w > 0.0)) return ART_ERR_ARG;
    if (job->criterion != ART_CRIT_I && job->criterion != ART_CRIT_STOKES_ANY) return ART_ERR_ARG;
    if (job->criterion_plane < 0 || job->criterion_plane >= art_planes(job) ||
        (job->criterion == ART_CRIT_STOKES_ANY && job->criterion_plane != 0))
        return ART_ERR_ARG;
    if (job->criterion == ART_CRIT_STOKES_ANY && job->stokes == 4 &&
        job->precision == ART_MIXED_EXACT)
        return ART_ERR_UNSUPPORTED;
    if (!(job->fp64_sweep > 0.0)) return ART_ERR_ARG;
    J->a = job->a;
    J->a2 = job->a * job->a;
    J->r_obs = job->r_obs;
    J->pix = job->fov / (double)(nx - 1);
    J->step_frac = job->step_frac;
    J->h_min = job->h_min;
    J->r_in_stop = (1.0 + job->horizon_eps) * horizon(job->a);
    J->r_out_stop = job->escape_frac * job->r_obs;
    J->inv_2w2 = 1.0 / (2.0 * job->disk_w * job->disk_w);
    J->R_abs = job->R_abs;
    J->R_rel = job->R_rel;
    J->nx = nx;
    J->ny = ny;
    J->levels = job->levels;
    J->emission = job->emission;
    J->flow = job->flow;
    J->stokes = job->stokes;
    J->subrings = job->subrings;
    J->planes = art_planes(job);
    J->max_steps = job->max_steps;
    J->fp64_sweep = job->fp64_sweep;
    J->interp = job->interp;
    J->edge_mode = job->edge_mode;
    J->abs_norm = job->abs_norm;
    // exact decisions change the level loop only; the rays are traced as in ART_MIXED_DF
    J->precision = job->precision == ART_MIXED_EXACT ? ART_MIXED_DF : job->precision;
    J->criterion = job->criterion;
    J->cplane = job->criterion_plane;
    J->f_a = (float)J->a;
    J->f_a_lo = (float)(J->a - (double)J->f_a);
    J->f_a2 = (float)J->a2;
    J->f_a2_lo = (float)(J->a2 - (double)J->f_a2);
    J->f_step_frac = (float)J->step_frac;
    J->f_h_min = (float)J->h_min;
    J->f_r_in_stop = (float)J->r_in_stop;
    J->f_r_out_stop = (float)J->r_out_stop;
    J->f_fp64_sweep = (float)J->fp64_sweep;
    J->f_inv_2w2 = (float)J->inv_2w2;
    return ART_OK;
}

// Exact decisions (ART_MIXED_EXACT): relative band of a tolerance within which a decision on
// FP32-traced values is re-made on exact values.  FP32-traced intensities differ from FP64 by
// ~1e-5 relative (median; 1e-3 on lensed rays), and the estimates' cancellation (their numerators
// are second differences) magnifies that ~10-500 times near the tolerances.
constexpr double CERT_BAND = 2.5e-1;

// Relative tolerances of the mixed modes' discontinuity flags (SynchConst::e_sig, e_rin).
constexpr double EDGE_SIGMA_TOL = 1e-2, EDGE_RIN_TOL = 2e-3;
// The same for the double-float re-trace of exact decisions, whose positions are accurate to
// ~1e-14 but whose emission is evaluated in FP32 (~1e-6 relative in sigma).
constexpr double EDGE_SIGMA_TOL_DF = 1e-5, EDGE_RIN_TOL_DF = 1e-6;

// Constants of the synchrotron models in the scaled form the kernels use (cgs constants, CODATA).
// g: the context's fluid grid (ART_EMIT_GRID), null where there is none.
static void make_synch(const art_job* job, const art_ctx* g, SynchConst* S)
{
    const double e = 4.80320471e-10, me = 9.1093837015e-28, c = 2.99792458e10;
    const double hp = 6.62607015e-27, pi = 3.14159265358979323846, mp = 1.67262192369e-24;
    memset(S, 0, sizeof *S);
    if (job->emission != ART_EMIT_SYNCH_DISK && job->emission != ART_EMIT_GRID) return;
    const double L = job->length_cm, nu = job->nu_hz;
    if (job->emission == ART_EMIT_SYNCH_DISK) {
        S->ne0 = job->ne0;
        S->th0 = job->thetae0;
        S->b0 = job->b0;
        S->ne_s = job->ne_slope;
        S->te_s = job->te_slope;
        S->b_s = 0.5 * (job->ne_slope + job->te_slope);
        S->inv_2w2 = 1.0 / (2.0 * job->disk_w * job->disk_w);
        S->r_in = job->r_in;
        S->bz = job->bz_ratio;
        S->bnorm = 1.0 / sqrt(1.0 + job->bz_ratio * job->bz_ratio);
    } else if (g && g->grid) {
        const double L3 = L * L * L;
        S->grid = reinterpret_cast<const float4*>(g->grid);
        S->g_n1 = g->g_n1;
        S->g_n2 = g->g_n2;
        S->g_n3 = g->g_n3;
        S->g_x1min = g->g_x1min;
        S->g_x1max = g->g_x1max;
        S->g_inv_dx1 = g->g_n1 / (g->g_x1max - g->g_x1min);
        S->g_inv_dth = g->g_n2 / pi;
        S->g_inv_dph = g->g_n3 / (2.0 * pi);
        S->g_gm1 = job->gamma_ad - 1.0;
        S->g_ne_unit = job->m_unit / (L3 * (mp + me));
        S->g_b_unit = c * sqrt(4.0 * pi * job->m_unit / L3);
        S->g_th_unit = (mp / me) * (job->gamma_ad - 1.0);
        S->g_r_high = job->r_high;
        S->g_r_low = job->r_low;
        S->g_sigma_cut = job->sigma_cut;
    }
    if (job->precision == ART_MIXED || job->precision == ART_MIXED_DF ||
        job->precision == ART_MIXED_EXACT) {
        // the FP32 pass hands rays with a sample this close to a discontinuity of the emission
        // model to the high-precision re-trace (FP32 positions of lensed rays differ from FP64
        // by up to ~1e-3 in sigma, ~1e-5 in r)
        S->e_sig = EDGE_SIGMA_TOL;
        S->e_rin = EDGE_RIN_TOL;
    }
    S->LCj = L * sqrt(2.0) * pi * e * e / (3.0 * c);
    S->CB = e / (2.0 * pi * me * c);
    S->nu_obs = nu;
    S->xB = hp * nu / (me * c * c);
    S->invKB = c * c / (2.0 * hp * nu * nu * nu);
    S->LCV = L * e * e * e / (pi * me * me * c * c * nu * nu);
    S->LCQ = L * e * e * e * e / (4.0 * pi * pi * me * me * me * c * c * c * nu * nu * nu);
}

// A grid job needs the context's grid.
static int check_grid(const art_ctx* c, const art_job* job)
{
    return (job->emission == ART_EMIT_GRID && !c->grid) ? ART_ERR_ARG : ART_OK;
}

// Persistent grid of a trace launch: SMs x resident blocks per SM, capped by the tuned blocks
// per SM (0: as many as fit).  FP64 queues known to hold more than FP64_FULL_GRID_RAYS_PER_SM rays
// per SM take every resident block whatever the setting.
constexpr int FP64_FULL_GRID_RAYS_PER_SM = 4096;
static int trace_grid(const art_ctx* c, int occ, int tuned)
{
    return c->num_sms * (tuned > 0 && tuned < occ ? tuned : occ);
}

// Trace-kernel variant of a job (occupancy table index).
static int variant_of(const DevJob& J)
{
    return (J.stokes == 4 ? TV_POL : 0) | (J.emission == ART_EMIT_GRID ? TV_GRID : 0);
}

// The same validation for the allocation-free entry point (noalloc.cu).
int art_make_devjob(const art_job* job, DevJob* J) { return make_devjob(job, J); }
void art_make_synch(const art_job* job, SynchConst* S) { make_synch(job, nullptr, S); }

extern "C" int art_create(art_ctx** out, int device, void* stream)
{
    if (!out) return ART_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return ART_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return ART_ERR_CUDA;
    art_ctx* c = new art_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return ART_ERR_CUDA;
    }
    for (int kd = 0; kd < 3; ++kd)
        for (int v = 0; v < TV_COUNT; ++v) {
            if (trace_occupancy(TraceKind(kd), v, &c->occ[kd][v]) != cudaSuccess) {
                delete c;
                return ART_ERR_CUDA;
            }
            if (c->occ[kd][v] < 1) c->occ[kd][v] = 1;
            if (trace_batch_occupancy(kd, v, &c->occb[kd][v]) != cudaSuccess) {
                delete c;
                return ART_ERR_CUDA;
            }
            if (c->occb[kd][v] < 1) c->occb[kd][v] = 1;
        }
    *out = c;
    return ART_OK;
}

extern "C" void art_destroy(art_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    for (art_ctx* d : c->subs) art_destroy(d);
    if (c->sub_in) cudaEventDestroy(c->sub_in);
    for (cudaEvent_t e : c->sub_out)
        if (e) cudaEventDestroy(e);
    cudaFree(c->xsnap);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->steps_map);
    cudaFree(c->lptq);
    cudaFree(c->lpt_hist);
    if (c->gstream) cudaStreamSynchronize(c->gstream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gbexec) cudaGraphExecDestroy(c->gbexec);
    destroy_plan(c->gbplan);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->gev_in) cudaEventDestroy(c->gev_in);
    if (c->gev_out) cudaEventDestroy(c->gev_out);
    cudaFree(c->queue);
    cudaFree(c->reroute);
    cudaFree(c->reroute2);
    cudaFree(c->counters);
    cudaFree(c->norm3);
    cudaFree(c->cam);
    cudaFree(c->partials);
    cudaFree(c->out6);
    cudaFree(c->himg);
    cudaFree(c->hmask);
    cudaFreeHost(c->pinned);
    cudaFreeHost(c->pinned_d);
    cudaFree(c->prof_steps);
    cudaFree(c->bjobs);
    cudaFree(c->bsynch);
    cudaFree(c->bsynchf);
    cudaFree(c->bcams);
    cudaFree(c->bparams);
    cudaFree(c->bimgs);
    cudaFree(c->bmasks);
    cudaFree(c->bnorms);
    cudaFree(c->bcounts);
    cudaFreeHost(c->bcounts_host);
    cudaFree(c->bqueue);
    cudaFree(c->breroute);
    cudaFree(c->bband);
    cudaFree(c->bsmask);
    cudaFree(c->grid_owned);
    cnn_destroy(c->cnn);
    cudaFree(c->aux);
    cudaFree(c->smask);
    cudaFree(c->prob);
    cudaFree(c->xst);
    cudaFree(c->cborder);
    cudaFree(c->cxq);
    cudaFree(c->cfixq);
    cudaFree(c->vq);
    cudaFree(c->vtab);
    cudaFree(c->atab);
    cudaFree(c->aq);
    for (int k = 0; k < 2 * art_ctx::PROF_MAX; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->owns_stream) cudaStreamDestroy(c->stream);
    delete c;
}

// Fixed-size scratch (counters, camera, normalisation, metric partials, pinned mirrors).
static int ensure_fixed(art_ctx* c)
{
    if (c->counters) return ART_OK;
    ++c->scratch_gen;
    CK(cudaMalloc(&c->counters, sizeof(unsigned long long) * C_COUNT));
    CK(cudaMalloc(&c->norm3, sizeof(double) * 4));
    CK(cudaMalloc(&c->cam, sizeof(Camera)));
    CK(cudaMalloc(&c->partials, sizeof(double) * 6 * METRIC_BLOCKS));
    CK(cudaMalloc(&c->out6, sizeof(double) * 8));
    CK(cudaMallocHost(&c->pinned, sizeof(unsigned long long) * C_COUNT));
    CK(cudaMallocHost(&c->pinned_d, sizeof(double) * 8));
    return ART_OK;
}

// Ray queues large enough for `cap` entries (grown, never shrunk).
static int ensure_queue(art_ctx* c, int64_t cap)
{
    if (cap < 1) cap = 1;
    if (cap <= c->queue_cap) return ART_OK;
    ++c->scratch_gen;
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->queue);
    cudaFree(c->reroute);
    cudaFree(c->reroute2);
    c->queue = c->reroute = c->reroute2 = nullptr;
    c->queue_cap = 0;
    CK(cudaMalloc(&c->queue, sizeof(int32_t) * cap));
    CK(cudaMalloc(&c->reroute, sizeof(int32_t) * cap));
    CK(cudaMalloc(&c->reroute2, sizeof(int32_t) * cap));
    c->queue_cap = cap;
    return ART_OK;
}

// Grow a context-owned device buffer to at least `n` elements (synchronises first).
template <class T>
static int grow(art_ctx* c, T*& buf, int64_t& cap, int64_t n)
{
    if (n <= cap) return ART_OK;
    ++c->scratch_gen;
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(buf);
    buf = nullptr;
    cap = 0;
    CK(cudaMalloc(&buf, sizeof(T) * n));
    cap = n;
    return ART_OK;
}

// Largest number of rays one level can queue: the base grid or the new points of level N.
static int64_t max_level_rays(const DevJob& J)
{
    int64_t n0 = (int64_t)((J.nx - 1) / (1 << J.levels) + 1) * ((J.ny - 1) / (1 << J.levels) + 1);
    if (J.levels == 0) return n0;
    int64_t prev = (int64_t)((J.nx - 1) / 2 + 1) * ((J.ny - 1) / 2 + 1);
    int64_t last = (int64_t)J.nx * J.ny - prev;
    return n0 > last ? n0 : last;
}

// Trace the rays of the queue (length in counters[count_idx]) with the job's precision.
static int trace_queue(art_ctx* c, const art_job* job, const DevJob& J,
                       const unsigned long long* count, double* img, uint8_t* mask, double* out,
                       const art_rayaux* aux, float* pix_minr = nullptr, float* pix_turn = nullptr,
                       const unsigned long long* spec_from = nullptr,
                       const int32_t* qbuf = nullptr, bool exact = false,
                       bool skip_retrace = false, int64_t n_host = -1)
{
    TraceArgs a;
    memset(&a, 0, sizeof a);
    a.job = J;
    a.pix_steps = c->cur_steps;
    a.quad_rays = c->tune.quad_rays;
    a.pair_rays = c->tune.pair_rays;
    a.quad64_rays = c->tune.quad64_rays;
    a.pix_minr = pix_minr;
    a.pix_turn = pix_turn;
    a.spec_from = spec_from;
    make_synch(job, c, &a.synch);
    a.synchf = synch_to_float(a.synch);
    a.cam = c->cam;
    a.queue = qbuf ? qbuf : c->queue;
    a.count = count;
    a.counters = c->counters;
    a.img = img;
    a.mask = mask;
    a.out = out;
    a.npix = (int64_t)J.nx * J.ny;
    if (aux) {
        a.aux_status = aux->status;
        a.aux_steps = aux->steps;
        a.aux_nturn = aux->nturn;
        a.aux_minr = aux->min_r;
    }
    const int pl = variant_of(J);
    // a queue the host knows to be very long (a large base level) keeps every resident block:
    // there the pipe needs the latency hiding more than the launch's last rays need their SMs
    const bool long_queue = n_host > (int64_t)FP64_FULL_GRID_RAYS_PER_SM * c->num_sms;
    const int g64 = trace_grid(c, c->occ[TK_FP64][pl], long_queue ? 0 : c->tune.blocks64);
    const int g32 = trace_grid(c, c->occ[TK_FP32][pl], c->tune.blocks32);
    const int gdf = trace_grid(c, c->occ[TK_DF][pl], c->tune.blocks32);
    int k;
    if (J.precision == ART_FP64) {
        a.fetch = c->counters + C_FETCH;
        CK(cudaMemsetAsync(a.fetch, 0, sizeof(unsigned long long), c->stream));
        k = prof_begin(c);
        CK(launch_trace(a, TK_FP64, g64, c->stream));
        prof_end(c, k, ART_K_TRACE_FP64, -1);
        return ART_OK;
    }
    const bool mixed = J.precision == ART_MIXED || J.precision == ART_MIXED_DF;
    a.fetch = c->counters + C_FETCH;
    CK(cudaMemsetAsync(c->counters + C_FETCH, 0, sizeof(unsigned long long) * 3, c->stream));
    if (mixed) {
        a.reroute = c->reroute;
        a.reroute_count = c->counters + C_REROUTE;
    }
    k = prof_begin(c);
    CK(launch_trace(a, TK_FP32, g32, c->stream));
    prof_end(c, k, ART_K_TRACE_FP32, -1);
    if (mixed && !skip_retrace) {
        // high-precision re-trace of the near-critical rays the FP32 pass routed
        TraceArgs b = a;
        b.reroute = nullptr;
        b.reroute_count = nullptr;
        b.indirect = c->reroute;
        b.count = c->counters + C_REROUTE;
        b.fetch = c->counters + C_FETCH2;
        const bool dfp = J.precision == ART_MIXED_DF;
        if (exact && dfp) {
            // exact decisions: a double-float ray with a sample within FP32 rounding of a
            // discontinuity (its emission is evaluated in FP32) is handed on to FP64
            b.synch.e_sig = EDGE_SIGMA_TOL_DF;
            b.synch.e_rin = EDGE_RIN_TOL_DF;
            b.synchf.e_sig = (float)EDGE_SIGMA_TOL_DF;  // the copy the double-float transfer reads
            b.synchf.e_rin = (float)EDGE_RIN_TOL_DF;
            b.reroute = c->reroute2;
            b.reroute_count = c->counters + C_REROUTE2;
        }
        k = prof_begin(c);
        CK(launch_trace(b, dfp ? TK_DF : TK_FP64, dfp ? gdf : g64, c->stream));
        prof_end(c, k, dfp ? ART_K_TRACE_DF : ART_K_TRACE_FP64, -1);
    }
    return ART_OK;
}

static int read_counters(art_ctx* c)
{
    CK(cudaMemcpyAsync(c->pinned, c->counters, sizeof(unsigned long long) * C_COUNT,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->pinned_d, c->norm3, sizeof(double) * 3, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ART_OK;
}

extern "C" int art_trace_pixels(art_ctx* c, const art_job* job, const int32_t* pix_dev, int64_t n,
                                double* out_dev, const art_rayaux* aux)
{
    if (!c || (n > 0 && (!pix_dev || !out_dev)) || n < 0) return ART_ERR_ARG;
    DevJob J;
    int rc = make_devjob(job, &J);
    if (rc || (rc = check_grid(c, job))) return rc;
    if (n == 0) return ART_OK;
    CK(cudaSetDevice(c->device));
    if ((rc = ensure_fixed(c)) || (rc = ensure_queue(c, n))) return rc;
    CK(cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * C_COUNT, c->stream));
    CK(cudaMemcpyAsync(c->queue, pix_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
    unsigned long long nn = (unsigned long long)n;
    CK(cudaMemcpyAsync(c->counters + C_QUEUE, &nn, sizeof nn, cudaMemcpyHostToDevice, c->stream));
    c->launches = 0;
    int k = prof_begin(c);
    CK(launch_camera_setup(*job, c->cam, c->stream));
    prof_end(c, k, ART_K_OTHER, 1);
    if ((rc = trace_queue(c, job, J, c->counters + C_QUEUE, nullptr, nullptr, out_dev, aux))) return rc;
    if ((rc = read_counters(c))) return rc;
    if (c->pinned[C_BADIDX] || c->pinned[C_SYNCERR]) return ART_ERR_DEVICE;
    return ART_OK;
}

extern "C" int art_ibar_int(art_ctx* c, const double* img_dev, int32_t nx, int32_t ny,
                            int32_t stride, double* ibar_host, double* peak_host)
{
    if (!c || !img_dev || nx < 1 || ny < 1 || stride < 1 || (nx - 1) % stride || (ny - 1) % stride)
        return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    int rc = ensure_fixed(c);
    if (rc) return rc;
    DevJob J;
    memset(&J, 0, sizeof J);
    J.abs_norm = ART_NORM_IBAR_INT;
    CK(launch_norm(J, img_dev, nx, ny, stride, c->norm3, c->stream));
    CK(cudaMemcpyAsync(c->pinned_d, c->norm3, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (ibar_host) *ibar_host = c->pinned_d[1];
    if (peak_host) *peak_host = c->pinned_d[2];
    return ART_OK;
}

extern "C" int art_refine_level(art_ctx* c, const art_job* job, double* img_dev, uint8_t* mask_dev,
                                int32_t level, double norm, int32_t* queue_dev, int64_t* count_host)
{
    if (!c || !img_dev || !queue_dev) return ART_ERR_ARG;
    DevJob J;
    int rc = make_devjob(job, &J);
    if (rc) return rc;
    if (level < 1 || level > J.levels) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if ((rc = ensure_fixed(c))) return rc;
    CK(cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * C_COUNT, c->stream));
    c->pinned_d[3] = norm;
    CK(cudaMemcpyAsync(c->norm3, &c->pinned_d[3], sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(launch_refine(J, level, c->norm3, img_dev, mask_dev, queue_dev, c->counters + C_QUEUE,
                     c->stream));
    if ((rc = read_counters(c))) return rc;
    if (count_host) *count_host = (int64_t)c->pinned[C_QUEUE];
    return ART_OK;
}

// A render's statistics from a copy of its counters and its normalisation; ART_ERR_DEVICE when a
// kernel reported an inconsistency.
static int stats_from(const DevJob& J, const unsigned long long* cnt, double norm, int launches,
                      bool cert, bool ax, art_stats* stats)
{
    memset(stats, 0, sizeof *stats);
    for (int k = 0; k <= J.levels && k < 16; ++k) {
        stats->rays_per_level[k] = (int64_t)cnt[C_LEVEL0 + k];
        stats->rays_traced += stats->rays_per_level[k];
    }
    stats->rays_fp64 = (int64_t)cnt[C_FP64];
    stats->steps = (int64_t)cnt[C_STEPS];
    stats->rays_capped = (int64_t)cnt[C_CAPPED];
    stats->rays_nan = (int64_t)cnt[C_NAN];
    stats->norm = norm;
    stats->kernel_launches = launches;
    stats->rays_speculative = (int64_t)cnt[C_SPEC];
    stats->rays_spec_used = (int64_t)cnt[C_SPECUSED];
    if (ax) {
        // rays actually traced: the axis filter's kept points (per level: queued minus
        // axis-interpolated)
        stats->rays_traced = (int64_t)cnt[C_AXKEPT];
        stats->border_points = (int64_t)cnt[C_AXINTERP];
    }
    if (cert) {
        stats->rays_exact = (int64_t)cnt[C_XRAYS] + stats->rays_per_level[0];
        stats->border_points = (int64_t)cnt[C_BTOT];
        stats->border_overflow = (int64_t)cnt[C_CERTOVF];
    }
    if (cnt[C_BADIDX] || cnt[C_SYNCERR] || cnt[C_CERTERR]) return ART_ERR_DEVICE;
    return ART_OK;
}

// The spatial level loop at a new sample of a third axis (art_render_axis): every level's queue
// is filtered by the axis criterion, so a point is traced only where neither the spatial nor the
// axis interpolant is good enough (the rest take the axis interpolant, mask ART_MASK_AXIS).
struct AxisFilter {
    double* const* atab;  // device table of the samples' images
    int f, s, F;
    double norm, R_rel, R_abs;
};

static int render_impl(art_ctx* c, const art_job* job, const double* truth_dev, double* img_dev,
                       uint8_t* mask_dev, art_stats* stats, const AxisFilter* ax);

extern "C" int art_render(art_ctx* c, const art_job* job, const double* truth_dev, double* img_dev,
                          uint8_t* mask_dev, art_stats* stats)
{
    return render_impl(c, job, truth_dev, img_dev, mask_dev, stats, nullptr);
}

static int render_impl(art_ctx* c, const art_job* job, const double* truth_dev, double* img_dev,
                       uint8_t* mask_dev, art_stats* stats, const AxisFilter* ax)
{
    if (!c || !img_dev) return ART_ERR_ARG;
    DevJob J;
    int rc = make_devjob(job, &J);
    if (rc || (rc = check_grid(c, job))) return rc;
    const bool learned = job->proposal != 0;
    if (learned && (!c->cnn || truth_dev || !(job->proposal_p >= 0.0) || !(job->proposal_p <= 1.0) ||
                    job->proposal_depth < 1))
        return ART_ERR_ARG;
    const bool band = job->crit_band > 0.0;
    if (band && (truth_dev || !(job->crit_band < 1.0))) return ART_ERR_ARG;
    const bool spec_any = learned || band;
    const bool cert = job->precision == ART_MIXED_EXACT;
    if (cert && truth_dev) return ART_ERR_ARG;
    if (ax && (spec_any || cert || truth_dev || !mask_dev)) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    const int64_t cap = max_level_rays(J);
    // the learned path appends speculative rays of later levels to a level's queue
    const int64_t qcap = spec_any ? cap + std::min<int64_t>((int64_t)J.nx * J.ny, 4 * cap) : cap;
    if ((rc = ensure_fixed(c)) || (rc = ensure_queue(c, qcap))) return rc;
    cudaStream_t st = c->stream;
    const int64_t npix = (int64_t)J.nx * J.ny;
    // per-pixel diagnostics (network features) are recorded whenever a network is loaded
    float *aminr = nullptr, *aturn = nullptr;
    if (c->cnn && !truth_dev) {
        if ((rc = grow(c, c->aux, c->aux_cap, 2 * npix))) return rc;
        aminr = c->aux;
        aturn = c->aux + npix;
        c->aux_npix = npix;
    } else {
        c->aux_npix = 0;
    }
    uint8_t* mask = mask_dev;
    if (spec_any || cert) {
        if (!mask) {
            if ((rc = grow(c, c->smask, c->smask_cap, npix))) return rc;
            mask = c->smask;
        }
        CK(cudaMemsetAsync(mask, 0, npix, st));  // speculation claims points whose mask is unset
    }
    // exact decisions: list capacities (a full borderline list leaves further points to the
    // ordinary decision, counted in border_overflow; the closure lists hold every point at most
    // once and are sized to the image)
    unsigned long long bcap = 0, xcap = 0;
    if (cert) {
        const int64_t b = std::min<int64_t>(npix, std::max<int64_t>(65536, cap / 64));
        const int64_t x = std::min<int64_t>(npix, 16 * b);
        if ((rc = grow(c, c->xst, c->xst_cap, (npix + 3) / 4 * 4)) ||
            (rc = grow(c, c->cborder, c->cborder_cap, b)) || (rc = grow(c, c->cxq, c->cxq_cap, x)) ||
            (rc = grow(c, c->cfixq, c->cfixq_cap, x)))
            return rc;
        bcap = (unsigned long long)b;
        xcap = (unsigned long long)x;
        CK(cudaMemsetAsync(c->xst, 0, (npix + 3) / 4 * 4, st));
        const int64_t n0 = (int64_t)((J.nx - 1) / (1 << J.levels) + 1) * ((J.ny - 1) / (1 << J.levels) + 1);
        if (npix > c->steps_cap) {
            if ((rc = grow(c, c->steps_map, c->steps_cap, npix))) return rc;
            CK(cudaMemsetAsync(c->steps_map, 0, sizeof(uint16_t) * npix, st));
        }
        if ((rc = grow(c, c->lptq, c->lptq_cap, std::max<int64_t>(x, n0)))) return rc;
        if (!c->lpt_hist) CK(cudaMalloc(&c->lpt_hist, sizeof(unsigned int) * LPT_BUCKETS));
    }
    c->cur_steps = cert ? c->steps_map : nullptr;
    DevJob J64 = J;
    J64.precision = ART_FP64;
    if (ax && (rc = grow(c, c->aq, c->aq_cap, cap))) return rc;
    // axis filter of the queue of `level` (counters[C_QUEUE]) into c->aq (counters[C_AXQ])
    auto axis_filter = [&](int level) -> int {
        int kk = prof_begin(c);
        CK(launch_axis_filter(npix, J.planes, ax->atab, ax->f, ax->s, ax->F, ax->norm, ax->R_rel,
                              ax->R_abs, c->queue, c->counters, c->aq, mask, c->num_sms, st));
        prof_end(c, kk, ART_K_REFINE, -1);
        (void)level;
        return ART_OK;
    };
    if (learned) {
        int64_t pc = 1;
        for (int lv = 0; lv + 2 <= J.levels; ++lv) pc = std::max(pc, cnn_head_cells(J, lv));
        if ((rc = grow(c, c->prob, c->prob_cap, pc))) return rc;
    }
    c->launches = 0;
    CK(cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * C_COUNT, st));
    int k;
    c->prof_level = -1;
    if (!truth_dev) {
        k = prof_begin(c);
        CK(launch_camera_setup(*job, c->cam, st));
        prof_end(c, k, ART_K_OTHER, 1);
    }
    k = prof_begin(c);
    CK(launch_enqueue_base(J, c->queue, c->counters, st));
    prof_end(c, k, ART_K_OTHER, -1);
    for (int level = 0; level <= J.levels; ++level) {
        c->prof_level = level;
        bool spec = false;
        if (level == 0 && band && J.levels > 0) {
            // near-critical band of every finer level, traced with the base level
            CK(launch_spec_mark(c->counters, st));
            k = prof_begin(c);
            CK(launch_band_propose(J, c->cam, job->crit_band, mask, c->queue, c->counters,
                                   (unsigned long long)qcap, c->num_sms, st));
            prof_end(c, k, ART_K_PROPOSE, -1);
            CK(launch_queue_clamp(c->counters, (unsigned long long)qcap, st));
            spec = true;
        }
        if (level > 0) {
            const int s = 1 << (J.levels - level);
            CK(cudaMemsetAsync(c->counters + C_QUEUE, 0, sizeof(unsigned long long), st));
            k = prof_begin(c);
            if (cert) {
                CK(cudaMemsetAsync(c->counters + C_BORDER, 0, 3 * sizeof(unsigned long long), st));
                CK(launch_refine_cert(J, level, c->norm3, img_dev, mask, c->queue,
                                      c->counters + C_QUEUE, st, aminr, aturn,
                                      spec_any ? c->counters : nullptr, c->xst, CERT_BAND,
                                      c->cborder, c->counters, bcap));
            } else {
                CK(launch_refine(J, level, c->norm3, img_dev, mask, c->queue,
                                 c->counters + C_QUEUE, st, aminr, aturn,
                                 spec_any ? c->counters : nullptr));
            }
            prof_end(c, k, ART_K_REFINE, (int64_t)((J.nx - 1) / s + 1) * ((J.ny - 1) / s + 1));
            CK(launch_level_count(c->counters, level, st));
            if (learned && level + 1 <= J.levels && (level - 1) % job->proposal_depth == 0) {
                // every D = proposal_depth levels the network reads the completed level-(k-1)
                // lattice and proposes points of levels k+1 .. k+D, traced now together with
                // level k's rays; the D - 1 levels in between trace only what was not proposed
                CK(launch_spec_mark(c->counters, st));
                k = prof_begin(c);
                CK(cnn_propose(c->cnn, J, level - 1, job->proposal_depth, img_dev, aminr, aturn,
                               c->norm3,
                               (float)job->proposal_p, c->prob, mask, c->queue, c->counters,
                               (unsigned long long)qcap, st));
                prof_end(c, k, ART_K_PROPOSE, -1);
                CK(launch_queue_clamp(c->counters, (unsigned long long)qcap, st));
                spec = true;
            }
            if (cert) {
                // the level's rays: FP32 (+ double-float, whose uncertain rays join the FP64
                // queue), or FP64 on a degenerate image
                CK(launch_cert_split(c->counters, st));
                // the rays the FP32 pass hands over (near-critical ones, and samples near an
                // emission discontinuity) join this level's FP64 pass instead of a double-float
                // pass of their own
                if ((rc = trace_queue(c, job, J, c->counters + C_QF32, img_dev, mask, nullptr,
                                      nullptr, aminr, aturn,
                                      spec ? c->counters + C_SPECFROM : nullptr, nullptr, true,
                                      true)))
                    return rc;
                if ((rc = trace_queue(c, job, J64, c->counters + C_QF64, img_dev, mask, nullptr,
                                      nullptr, aminr, aturn)))
                    return rc;
                CK(launch_cert_mark_traced(c->queue, c->counters, (unsigned long long)qcap, c->xst,
                                           st, C_QF64));
                CK(launch_cert_take_uncertain(c->queue, c->reroute, c->counters, C_REROUTE,
                                              spec ? c->counters + C_SPECFROM : nullptr, mask,
                                              c->cxq, xcap, st));
                // the borderline points: exact stencils (FP64 re-traces, recomputed
                // interpolants, coarsest level first), then their FP64 decisions
                CK(launch_counter_clamp(c->counters, C_BORDER, bcap, st));
                k = prof_begin(c);
                CK(launch_cert_closure(J, level, c->cborder, bcap, c->counters, c->xst, mask,
                                       c->cxq, xcap, c->cfixq, xcap, st));
                CK(launch_counter_clamp(c->counters, C_XQ, xcap, st));
                CK(launch_counter_clamp(c->counters, C_FIXQ, xcap, st));
                prof_end(c, k, ART_K_OTHER, -1);
                // longest rays first (an FP64 launch ends with its last ray)
                CK(launch_lpt_order(J, c->cxq, c->counters + C_XQ, xcap, c->steps_map, mask,
                                    c->lptq, c->lpt_hist, c->num_sms, st));
                if ((rc = trace_queue(c, job, J64, c->counters + C_XQ, img_dev, mask, nullptr,
                                      nullptr, aminr, aturn, nullptr, c->lptq)))
                    return rc;
                k = prof_begin(c);
                CK(launch_cert_mark_traced(c->cxq, c->counters, xcap, c->xst, st));
                for (int lv = 1; lv < level; ++lv)
                    CK(launch_cert_fixup(J, c->cfixq, c->counters, xcap, lv, img_dev, c->xst, st));
                CK(launch_cert_redecide(J, level, c->norm3, c->cborder, c->counters, bcap, img_dev,
                                        mask, c->xst, aminr, aturn, st));
                prof_end(c, k, ART_K_OTHER, -1);
            }
        }
        if (truth_dev) {
            k = prof_begin(c);
            CK(launch_gather_truth(J, c->queue, c->counters + C_QUEUE, truth_dev, img_dev, mask_dev,
                                   cap, st));
            prof_end(c, k, ART_K_OTHER, -1);
        } else if (cert && level == 0) {
            // exact decisions: the base level in FP64 (exact I_bar_int and the exact ends of every
            // closure), the band's speculative rays of later levels in the mixed precision
            const int S0 = 1 << J.levels;
            const int64_t n0 = (int64_t)((J.nx - 1) / S0 + 1) * ((J.ny - 1) / S0 + 1);
            // the lengths of the base rays from an FP32 pass (its values are overwritten), then
            // the FP64 pass longest first
            DevJob J32 = J;
            J32.precision = ART_FP32;
            if ((rc = trace_queue(c, job, J32, c->counters + C_LEVEL0, img_dev, mask, nullptr,
                                  nullptr, aminr, aturn)))
                return rc;
            CK(launch_lpt_order(J, c->queue, c->counters + C_LEVEL0, (unsigned long long)n0,
                                c->steps_map, mask, c->lptq, c->lpt_hist, c->num_sms, st));
            if ((rc = trace_queue(c, job, J64, c->counters + C_LEVEL0, img_dev, mask, nullptr,
                                  nullptr, aminr, aturn, nullptr, c->lptq, false, false, n0)))
                return rc;
            k = prof_begin(c);
            CK(launch_cert_mark_base(J, c->xst, st));
            prof_end(c, k, ART_K_OTHER, -1);
            if (spec) {
                CK(launch_cert_spec_count(c->counters, st));
                CK(cudaMemsetAsync(c->counters + C_REROUTE2, 0, sizeof(unsigned long long), st));
                if ((rc = trace_queue(c, job, J, c->counters + C_SPECN, img_dev, mask, nullptr,
                                      nullptr, aminr, aturn, c->counters + C_ZERO,
                                      c->queue + n0, true)))
                    return rc;
                // speculative rays handed on to FP64 are traced at their own level instead
                CK(launch_cert_take_uncertain(c->queue + n0, c->reroute2, c->counters, C_REROUTE2,
                                              c->counters + C_ZERO, mask, c->cxq, 0, st));
            }
        } else if (cert) {
            // traced above, before the exact decisions of the level's borderline points
        } else if (ax) {
            if ((rc = axis_filter(level))) return rc;
            if ((rc = trace_queue(c, job, J, c->counters + C_AXQ, img_dev, mask, nullptr, nullptr,
                                  aminr, aturn, nullptr, c->aq)))
                return rc;
        } else {
            // at level 0 the host knows the base grid's size (a lower bound with speculation)
            const int64_t nb = level == 0 ? (int64_t)((J.nx - 1) / (1 << J.levels) + 1) *
                                                ((J.ny - 1) / (1 << J.levels) + 1)
                                          : -1;
            if ((rc = trace_queue(c, job, J, c->counters + C_QUEUE, img_dev, mask, nullptr, nullptr,
                                  aminr, aturn, spec ? c->counters + C_SPECFROM : nullptr, nullptr,
                                  false, false, nb)))
                return rc;
        }
        if (level == 0) {
            k = prof_begin(c);
            CK(launch_norm(J, img_dev + (int64_t)J.cplane * npix, J.nx, J.ny, 1 << J.levels,
                           c->norm3, st));
            if (cert) CK(launch_cert_check_norm(c->norm3, c->counters, st));
            prof_end(c, k, ART_K_OTHER, -1);
        }
    }
    c->prof_level = -1;
    if (stats) {
        if ((rc = read_counters(c))) return rc;
        return stats_from(J, c->pinned, c->pinned_d[0], c->launches, cert, ax != nullptr, stats);
    }
    return ART_OK;
}

extern "C" int art_render_host(art_ctx* c, const art_job* job, double* img_host, uint8_t* mask_host,
                               art_stats* stats)
{
    if (!c || !img_host) return ART_ERR_ARG;
    DevJob J;
    int rc = make_devjob(job, &J);
    if (rc || (rc = check_grid(c, job))) return rc;
    CK(cudaSetDevice(c->device));
    const int64_t npix = (int64_t)J.nx * J.ny;
    if (npix * J.planes > c->hcap) {
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->himg);
        cudaFree(c->hmask);
        c->himg = nullptr;
        c->hmask = nullptr;
        c->hcap = 0;
        CK(cudaMalloc(&c->himg, sizeof(double) * npix * J.planes));
        CK(cudaMalloc(&c->hmask, npix));
        c->hcap = npix * J.planes;
    }
    if ((rc = art_render(c, job, nullptr, c->himg, c->hmask, nullptr))) return rc;
    CK(cudaMemcpyAsync(img_host, c->himg, sizeof(double) * npix * J.planes, cudaMemcpyDeviceToHost,
                       c->stream));
    if (mask_host) CK(cudaMemcpyAsync(mask_host, c->hmask, npix, cudaMemcpyDeviceToHost, c->stream));
    if (stats) {
        if ((rc = read_counters(c))) return rc;
        memset(stats, 0, sizeof *stats);
        for (int k = 0; k <= J.levels && k < 16; ++k) {
            stats->rays_per_level[k] = (int64_t)c->pinned[C_LEVEL0 + k];
            stats->rays_traced += stats->rays_per_level[k];
        }
        stats->rays_fp64 = (int64_t)c->pinned[C_FP64];
        stats->steps = (int64_t)c->pinned[C_STEPS];
        stats->rays_capped = (int64_t)c->pinned[C_CAPPED];
        stats->rays_nan = (int64_t)c->pinned[C_NAN];
        stats->norm = c->pinned_d[0];
        stats->kernel_launches = c->launches;
    } else {
        CK(cudaStreamSynchronize(c->stream));
    }
    return ART_OK;
}

extern "C" int art_render_axis(art_ctx* c, const art_job* jobs, int32_t F, int32_t levels3,
                               double R_rel3, double R_abs3, const double* const* truth,
                               double* const* imgs, uint8_t* amask_dev, art_stats* stats)
{
    if (!c || !jobs || !imgs || F < 2 || levels3 < 1 || levels3 > 12) return ART_ERR_ARG;
    const int S = 1 << levels3;
    if ((F - 1) % S) return ART_ERR_ARG;
    DevJob J0;
    int rc = make_devjob(&jobs[0], &J0);
    if (rc) return rc;
    for (int f = 0; f < F; ++f) {
        DevJob Jf;
        if ((rc = make_devjob(&jobs[f], &Jf))) return rc;
        if (Jf.nx != J0.nx || Jf.ny != J0.ny || Jf.planes != J0.planes) return ART_ERR_ARG;
        if (jobs[f].precision == ART_MIXED_EXACT) return ART_ERR_UNSUPPORTED;
        if (!imgs[f] || (truth && !truth[f])) return ART_ERR_ARG;
        if (!truth && (rc = check_grid(c, &jobs[f]))) return rc;
    }
    CK(cudaSetDevice(c->device));
    const int64_t npix = (int64_t)J0.nx * J0.ny;
    if ((rc = ensure_fixed(c)) || (rc = ensure_queue(c, npix)) ||
        (rc = grow(c, c->atab, c->atab_cap, (int64_t)F)))
        return rc;
    cudaStream_t st = c->stream;
    if (stats) memset(stats, 0, sizeof(art_stats) * F);
    // the base samples: the ordinary adaptive render (or the truth)
    double nsum = 0.0;
    int nbase = 0;
    for (int f = 0; f < F; f += S) {
        if (truth) {
            CK(cudaMemcpyAsync(imgs[f], truth[f], sizeof(double) * npix * J0.planes,
                               cudaMemcpyDeviceToDevice, st));
            DevJob Jn = J0;
            Jn.abs_norm = ART_NORM_IBAR_INT;
            CK(launch_norm(Jn, truth[f], J0.nx, J0.ny, 1, c->norm3, st));
            CK(cudaMemcpyAsync(c->pinned_d, c->norm3, sizeof(double) * 3, cudaMemcpyDeviceToHost,
                               st));
            CK(cudaStreamSynchronize(st));
            nsum += c->pinned_d[0];
            if (stats) stats[f].rays_traced = npix;
            if (amask_dev)
                CK(cudaMemsetAsync(amask_dev + (int64_t)f * npix, ART_MASK_TRACED, npix, st));
        } else {
            art_stats bs;
            if ((rc = art_render(c, &jobs[f], nullptr, imgs[f],
                                 amask_dev ? amask_dev + (int64_t)f * npix : nullptr, &bs)))
                return rc;
            nsum += bs.norm;
            if (stats) stats[f] = bs;
        }
        ++nbase;
    }
    const double norm = nsum / nbase;
    CK(cudaMemcpyAsync(c->atab, imgs, sizeof(double*) * F, cudaMemcpyHostToDevice, st));
    for (int k = 1; k <= levels3; ++k) {
        const int s = 1 << (levels3 - k);
        for (int f = s; f < F; f += 2 * s) {
            if (truth) {
                // the axis logic alone: every pixel of the new sample decided along the axis
                CK(cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * C_COUNT, st));
                int kp = prof_begin(c);
                CK(launch_axis_refine(npix, J0.planes, c->atab, f, s, F, norm, R_rel3, R_abs3,
                                      c->queue, c->counters + C_QUEUE, amask_dev, st));
                prof_end(c, kp, ART_K_REFINE, npix);
                CK(launch_gather_truth(J0, c->queue, c->counters + C_QUEUE, truth[f], imgs[f],
                                       nullptr, npix, st));
                if (stats) {
                    if ((rc = read_counters(c))) return rc;
                    stats[f].rays_traced = (int64_t)c->pinned[C_QUEUE];
                    stats[f].norm = norm;
                }
                continue;
            }
            // the spatial scheme at sample f, each level's rays filtered by the axis criterion
            art_job jf = jobs[f];
            jf.crit_band = 0.0;
            jf.proposal = 0;
            uint8_t* mk = amask_dev ? amask_dev + (int64_t)f * npix : nullptr;
            if (!mk) {
                if ((rc = grow(c, c->smask, c->smask_cap, npix))) return rc;
                mk = c->smask;
            }
            const AxisFilter axf{c->atab, f, s, F, norm, R_rel3, R_abs3};
            art_stats fs;
            if ((rc = render_impl(c, &jf, nullptr, imgs[f], mk, &fs, &axf))) return rc;
            if (stats) stats[f] = fs;
        }
    }
    if (!stats) CK(cudaStreamSynchronize(st));
    return ART_OK;
}

extern "C" int art_visibilities(art_ctx* c, const double* img_dev, const double* ref_dev,
                                int32_t nx, int32_t ny, double dx, double taper_fwhm, int32_t m,
                                double* vis_dev)
{
    if (!c || !img_dev || !vis_dev || nx < 1 || ny < 1 || !(dx > 0.0) || !(taper_fwhm == taper_fwhm))
        return ART_ERR_ARG;
    if (m < 32 || m > 32768 || (m & (m - 1)) || m < nx || m < ny) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    int rc;
    if ((rc = grow(c, c->vq, c->vq_cap, (int64_t)m * m)) ||
        (rc = grow(c, c->vtab, c->vtab_cap, (int64_t)vis_table_doubles(m, nx, ny))))
        return rc;
    CK(launch_visibilities(img_dev, ref_dev, nx, ny, dx, taper_fwhm, m,
                           reinterpret_cast<double2*>(vis_dev), c->vq, c->vtab, c->stream));
    return ART_OK;
}

extern "C" int art_metrics(art_ctx* c, const double* truth_dev, const double* img_dev,
                           const uint8_t* mask_dev, int32_t nx, int32_t ny, double* out_host)
{
    if (!c || !truth_dev || !img_dev || !out_host || nx < 1 || ny < 1) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    int rc = ensure_fixed(c);
    if (rc) return rc;
    CK(launch_metrics(truth_dev, img_dev, mask_dev, nx, ny, c->partials, METRIC_BLOCKS, c->out6,
                      c->stream));
    double h[6];
    CK(cudaMemcpyAsync(c->pinned_d, c->out6, sizeof(double) * 6, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    memcpy(h, c->pinned_d, sizeof h);
    const double N = (double)nx * ny;
    const double mean = h[5] / N;
    out_host[0] = h[0] / N;
    out_host[1] = fabs(h[1] - h[2]) / fabs(h[1]);
    out_host[2] = h[3] / h[4];
    out_host[3] = h[3] / (N * mean * mean);
    return ART_OK;
}

extern "C" int art_profile(art_ctx* c, int enable)
{
    if (!c) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (!enable) {
        c->prof_on = false;
        return ART_OK;
    }
    if (!c->prof_steps) {
        CK(cudaMalloc(&c->prof_steps, 3 * sizeof(unsigned long long) * art_ctx::PROF_MAX));
        for (int k = 0; k < 2 * art_ctx::PROF_MAX; ++k) CK(cudaEventCreate(&c->ev[k]));
    }
    CK(cudaStreamSynchronize(c->stream));
    c->prof_on = true;
    c->prof_n = 0;
    return ART_OK;
}

extern "C" int art_measure_alu_peaks(art_ctx* c, double* fp32_tflops, double* fp64_tflops)
{
    if (!c || !fp32_tflops || !fp64_tflops) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    CK(measure_alu_peaks(c->num_sms, c->stream, fp32_tflops, fp64_tflops));
    return ART_OK;
}

extern "C" int art_measure_fp64_issue(art_ctx* c, double* cycles3)
{
    if (!c || !cycles3) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    CK(measure_fp64_issue(c->stream, cycles3));
    return ART_OK;
}

extern "C" int art_profile_read(art_ctx* c, art_launch_record* recs, int cap, int* n)
{
    if (!c || !n || (cap > 0 && !recs)) return ART_ERR_ARG;
    *n = 0;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    if (!c->prof_steps) return ART_OK;
    std::vector<unsigned long long> snap(3 * (size_t)art_ctx::PROF_MAX);
    CK(cudaMemcpy(snap.data(), c->prof_steps, 3 * sizeof(unsigned long long) * c->prof_n,
                  cudaMemcpyDeviceToHost));
    unsigned long long prev = 0, prevr = 0;
    int out = 0;
    for (int k = 0; k < c->prof_n; ++k) {
        art_launch_record r = c->rec[k];
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
        r.ms = ms;
        r.max_steps = 0;
        if (r.kind == ART_K_TRACE_FP64 || r.kind == ART_K_TRACE_FP32 || r.kind == ART_K_TRACE_DF) {
            // the counters restart with every call: a snapshot below the previous one belongs to
            // a new call
            const unsigned long long st = snap[3 * k], mx = snap[3 * k + 1], nr = snap[3 * k + 2];
            r.steps = (int64_t)(st >= prev ? st - prev : st);
            r.items = (int64_t)(nr >= prevr ? nr - prevr : nr);
            r.max_steps = (int64_t)mx;
            prev = st;
            prevr = nr;
        }
        if (r.kind == ART_K_OTHER && r.items == 1) prev = prevr = 0;  // camera set-up opens a call
        if (out < cap) recs[out++] = r;
    }
    *n = out;
    return ART_OK;
}

// --------------------------------------------------------------------------------------------
// batched rendering
// --------------------------------------------------------------------------------------------

static int ensure_batch(art_ctx* c, int n, int64_t qcap)
{
    if (n > c->bcap) {
        ++c->scratch_gen;
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->bjobs);
        cudaFree(c->bsynch);
        cudaFree(c->bsynchf);
        cudaFree(c->bcams);
        cudaFree(c->bparams);
        cudaFree(c->bimgs);
        cudaFree(c->bmasks);
        cudaFree(c->bnorms);
        cudaFree(c->bcounts);
        cudaFreeHost(c->bcounts_host);
        cudaFree(c->bband);
        c->bcap = 0;
        CK(cudaMalloc(&c->bjobs, sizeof(DevJob) * n));
        CK(cudaMalloc(&c->bsynch, sizeof(SynchConst) * n));
        CK(cudaMalloc(&c->bsynchf, sizeof(SynchConstF) * n));
        CK(cudaMalloc(&c->bcams, sizeof(Camera) * n));
        CK(cudaMalloc(&c->bparams, sizeof(double) * 3 * n));
        CK(cudaMalloc(&c->bimgs, sizeof(double*) * n));
        CK(cudaMalloc(&c->bmasks, sizeof(uint8_t*) * n));
        CK(cudaMalloc(&c->bnorms, sizeof(double) * 4 * n));
        CK(cudaMalloc(&c->bcounts, sizeof(unsigned long long) * 16 * n));
        CK(cudaMallocHost(&c->bcounts_host, sizeof(unsigned long long) * 16 * n));
        CK(cudaMalloc(&c->bband, sizeof(float) * n));
        c->bcap = n;
    }
    if (qcap > c->bqcap) {
        ++c->scratch_gen;
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->bqueue);
        cudaFree(c->breroute);
        c->bqcap = 0;
        CK(cudaMalloc(&c->bqueue, sizeof(int64_t) * qcap));
        CK(cudaMalloc(&c->breroute, sizeof(int32_t) * qcap));
        c->bqcap = qcap;
    }
    return ART_OK;
}

static int trace_queue_batch(art_ctx* c, const DevJob& J0, const unsigned long long* spec_from)
{
    BatchTraceArgs a;
    memset(&a, 0, sizeof a);
    a.spec_from = spec_from;
    a.jobs = c->bjobs;
    a.synchs = c->bsynch;
    a.synchfs = c->bsynchf;
    a.cams = c->bcams;
    a.imgs = c->bimgs;
    a.masks = c->bmasks;
    a.queue = c->bqueue;
    a.count = c->counters + C_QUEUE;
    a.counters = c->counters;
    a.planes = J0.planes;
    a.stokes = J0.stokes;
    a.precision = J0.precision;
    a.emission = J0.emission;
    const int pl = variant_of(J0);
    a.fetch = c->counters + C_FETCH;
    CK(cudaMemsetAsync(c->counters + C_FETCH, 0, sizeof(unsigned long long) * 3, c->stream));
    int k;
    if (J0.precision == ART_FP64) {
        k = prof_begin(c);
        CK(launch_trace_batch(a, TK_FP64, trace_grid(c, c->occb[TK_FP64][pl], c->tune.blocks64),
                              c->stream));
        prof_end(c, k, ART_K_TRACE_FP64, -1);
        return ART_OK;
    }
    const bool mixed = J0.precision == ART_MIXED || J0.precision == ART_MIXED_DF;
    if (mixed) {
        a.reroute = c->breroute;
        a.reroute_count = c->counters + C_REROUTE;
    }
    k = prof_begin(c);
    CK(launch_trace_batch(a, TK_FP32, trace_grid(c, c->occb[TK_FP32][pl], c->tune.blocks32),
                          c->stream));
    prof_end(c, k, ART_K_TRACE_FP32, -1);
    if (mixed) {
        BatchTraceArgs b = a;
        b.reroute = nullptr;
        b.reroute_count = nullptr;
        b.indirect = c->breroute;
        b.count = c->counters + C_REROUTE;
        b.fetch = c->counters + C_FETCH2;
        const int kd = J0.precision == ART_MIXED_DF ? TK_DF : TK_FP64;
        k = prof_begin(c);
        CK(launch_trace_batch(
            b, kd, trace_grid(c, c->occb[kd][pl], kd == TK_FP64 ? c->tune.blocks64 : c->tune.blocks32),
            c->stream));
        prof_end(c, k, kd == TK_DF ? ART_K_TRACE_DF : ART_K_TRACE_FP64, -1);
    }
    return ART_OK;
}

// A batch's host-side plan: validated device jobs, synchrotron constants, camera parameters,
// output tables, and the launch extents of every level.
struct BatchPlan {
    int n = 0;
    std::vector<DevJob> J;
    std::vector<SynchConst> S;
    std::vector<SynchConstF> SF;
    std::vector<double> p3;
    std::vector<double*> im;
    std::vector<uint8_t*> mk;
    int64_t qcap = 0;
    int max_base = 1, max_levels = 0;
    std::vector<int> kx, ky;  // per level >= 1: the largest lattice extents
    // near-critical band: per-image widths, and where the scratch masks of images without a
    // caller mask start in the context's scratch (-1: the caller's)
    bool band = false;
    std::vector<float> bands;
    std::vector<int64_t> smask_off;
    int64_t smask_bytes = 0, max_npix = 1;
};

static int plan_batch(art_ctx* c, const art_job* jobs, int32_t n, double* const* imgs,
                      uint8_t* const* masks, BatchPlan& P)
{
    P.n = n;
    P.J.assign(n, DevJob{});
    P.S.assign(n, SynchConst{});
    P.SF.assign(n, SynchConstF{});
    P.p3.assign(3 * (size_t)n, 0.0);
    P.im.assign(imgs, imgs + n);
    P.mk.assign(n, nullptr);
    P.qcap = 0;
    P.max_base = 1;
    P.max_levels = 0;
    P.band = false;
    P.bands.assign(n, 0.f);
    P.smask_off.assign(n, -1);
    P.smask_bytes = 0;
    P.max_npix = 1;
    for (int i = 0; i < n; ++i) {
        int rc = make_devjob(&jobs[i], &P.J[i]);
        if (rc) return rc;
        if (jobs[i].precision == ART_MIXED_EXACT) return ART_ERR_UNSUPPORTED;  // art_render only
        if (!imgs[i]) return ART_ERR_ARG;
        if (jobs[i].crit_band > 0.0) {
            if (!(jobs[i].crit_band < 1.0)) return ART_ERR_ARG;
            if (P.J[i].levels > 0) {
                P.bands[i] = (float)jobs[i].crit_band;
                P.band = true;
            }
        }
        if (P.J[i].stokes != P.J[0].stokes || P.J[i].subrings != P.J[0].subrings ||
            P.J[i].precision != P.J[0].precision ||
            (P.J[i].emission == ART_EMIT_GRID) != (P.J[0].emission == ART_EMIT_GRID))
            return ART_ERR_ARG;  // one kernel kind and one plane count per batch
        if ((rc = check_grid(c, &jobs[i]))) return rc;
        make_synch(&jobs[i], c, &P.S[i]);
        P.SF[i] = synch_to_float(P.S[i]);
        P.p3[3 * i] = jobs[i].a;
        P.p3[3 * i + 1] = jobs[i].r_obs;
        P.p3[3 * i + 2] = jobs[i].incl_deg;
        if (masks) P.mk[i] = masks[i];
        const int64_t cap = max_level_rays(P.J[i]), npix = (int64_t)P.J[i].nx * P.J[i].ny;
        // the band appends speculative rays of later levels to the base level's queue
        P.qcap += cap + (P.bands[i] > 0.f ? std::min<int64_t>(npix, 4 * cap) : 0);
        P.max_npix = std::max(P.max_npix, npix);
        int S0 = 1 << P.J[i].levels;
        int nb = ((P.J[i].nx - 1) / S0 + 1) * ((P.J[i].ny - 1) / S0 + 1);
        if (nb > P.max_base) P.max_base = nb;
        if (P.J[i].levels > P.max_levels) P.max_levels = P.J[i].levels;
    }
    P.kx.assign(P.max_levels + 1, 1);
    P.ky.assign(P.max_levels + 1, 1);
    for (int level = 1; level <= P.max_levels; ++level)
        for (int i = 0; i < n; ++i)
            if (P.J[i].levels >= level) {
                int s = 1 << (P.J[i].levels - level);
                P.kx[level] = std::max(P.kx[level], (P.J[i].nx - 1) / s + 1);
                P.ky[level] = std::max(P.ky[level], (P.J[i].ny - 1) / s + 1);
            }
    // speculation keeps its state in the masks: images without one get a scratch mask
    if (P.band)
        for (int i = 0; i < n; ++i)
            if (!P.mk[i]) {
                P.smask_off[i] = P.smask_bytes;
                P.smask_bytes += ((int64_t)P.J[i].nx * P.J[i].ny + 15) & ~(int64_t)15;
            }
    return ART_OK;
}

// Point the plan's missing masks at the context's scratch (grown to fit first).
static int bind_batch_scratch(art_ctx* c, BatchPlan& P)
{
    if (!P.smask_bytes) return ART_OK;
    int rc = grow(c, c->bsmask, c->bsmask_cap, P.smask_bytes);
    if (rc) return rc;
    for (int i = 0; i < P.n; ++i)
        if (P.smask_off[i] >= 0) P.mk[i] = c->bsmask + P.smask_off[i];
    return ART_OK;
}

// The plan's tables into the context's device tables (outside any graph: host sources).
static int upload_batch(art_ctx* c, const BatchPlan& P)
{
    cudaStream_t st = c->stream;
    const int n = P.n;
    CK(cudaMemcpyAsync(c->bjobs, P.J.data(), sizeof(DevJob) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->bsynch, P.S.data(), sizeof(SynchConst) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->bsynchf, P.SF.data(), sizeof(SynchConstF) * n, cudaMemcpyHostToDevice,
                       st));
    CK(cudaMemcpyAsync(c->bparams, P.p3.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->bimgs, P.im.data(), sizeof(double*) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->bmasks, P.mk.data(), sizeof(uint8_t*) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->bband, P.bands.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    return ART_OK;
}

// The device part of a batched render: memsets and launches only (capturable).
static int run_batch(art_ctx* c, const BatchPlan& P)
{
    cudaStream_t st = c->stream;
    const int n = P.n;
    int rc;
    CK(cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * C_COUNT, st));
    CK(cudaMemsetAsync(c->bcounts, 0, sizeof(unsigned long long) * 16 * n, st));
    c->prof_level = -1;
    int k = prof_begin(c);
    CK(launch_camera_setup_batch(c->bjobs, c->bparams, n, c->bcams, st));
    prof_end(c, k, ART_K_OTHER, 1);
    k = prof_begin(c);
    CK(launch_enqueue_base_batch(c->bjobs, n, P.max_base, c->bqueue, c->counters + C_QUEUE,
                                 c->bcounts, st));
    prof_end(c, k, ART_K_OTHER, -1);
    for (int level = 0; level <= P.max_levels; ++level) {
        c->prof_level = level;
        if (level > 0) {
            CK(cudaMemsetAsync(c->counters + C_QUEUE, 0, sizeof(unsigned long long), st));
            k = prof_begin(c);
            CK(launch_refine_batch(c->bjobs, n, level, P.kx[level], P.ky[level], c->bnorms,
                                   c->bimgs, c->bmasks, c->bqueue, c->counters + C_QUEUE,
                                   c->bcounts, st, P.band ? c->counters : nullptr));
            prof_end(c, k, ART_K_REFINE, -1);
        }
        bool spec = false;
        if (level == 0 && P.band) {
            // near-critical band of every finer level of every image, traced with the base level
            CK(launch_spec_mark(c->counters, st));
            k = prof_begin(c);
            CK(launch_band_propose_batch(c->bjobs, c->bcams, c->bband, c->bmasks, n, P.max_npix,
                                         c->bqueue, c->counters, (unsigned long long)P.qcap, st));
            prof_end(c, k, ART_K_PROPOSE, -1);
            CK(launch_queue_clamp(c->counters, (unsigned long long)P.qcap, st));
            spec = true;
        }
        if ((rc = trace_queue_batch(c, P.J[0], spec ? c->counters + C_SPECFROM : nullptr)))
            return rc;
        if (level == 0) {
            k = prof_begin(c);
            CK(launch_norm_batch(c->bjobs, c->bimgs, n, c->bnorms, st));
            prof_end(c, k, ART_K_OTHER, -1);
        }
    }
    c->prof_level = -1;
    return ART_OK;
}

static void destroy_plan(BatchPlan* p) { delete p; }

// Exact decisions keep per-image closure lists, so a batch of them runs the single-image level
// loop once per image.  Each level of an image ends in a short FP64 launch that lasts as long as
// its longest ray while the rest of the GPU idles, so the images run concurrently: image i on
// sub-context i mod EXACT_SUBS, each with its own stream and scratch, ordered after the caller's
// stream by one event and joined back into it by one event per sub-context.  Jobs with the
// learned proposal (whose network lives in this context) run one after the other here instead.
constexpr int EXACT_SUBS = 32;

static int ensure_subs(art_ctx* c)
{
    if (c->subs.empty()) {
        for (int k = 0; k < EXACT_SUBS; ++k) {
            art_ctx* d = new art_ctx();
            d->device = c->device;
            d->num_sms = c->num_sms;
            memcpy(d->occ, c->occ, sizeof c->occ);
            memcpy(d->occb, c->occb, sizeof c->occb);
            if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess) {
                delete d;
                return ART_ERR_CUDA;
            }
            d->owns_stream = true;
            c->subs.push_back(d);
        }
        CK(cudaEventCreateWithFlags(&c->sub_in, cudaEventDisableTiming));
        c->sub_out.assign(EXACT_SUBS, nullptr);
        for (cudaEvent_t& e : c->sub_out) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    for (art_ctx* d : c->subs) {  // the loaded snapshot (referenced) and the kernel-form tuning
        d->grid = c->grid;
        d->g_n1 = c->g_n1;
        d->g_n2 = c->g_n2;
        d->g_n3 = c->g_n3;
        d->g_x1min = c->g_x1min;
        d->g_x1max = c->g_x1max;
        d->tune = c->tune;
    }
    return ART_OK;
}

static int render_batch_exact(art_ctx* c, const art_job* jobs, int n, double* const* imgs,
                              uint8_t* const* masks, art_stats* stats)
{
    bool learned = false;
    for (int i = 0; i < n; ++i) {
        if (jobs[i].precision != ART_MIXED_EXACT) return ART_ERR_ARG;
        learned = learned || jobs[i].proposal != 0;
    }
    if (learned) {
        for (int i = 0; i < n; ++i) {
            const int rc = art_render(c, &jobs[i], nullptr, imgs[i], masks ? masks[i] : nullptr,
                                      stats ? &stats[i] : nullptr);
            if (rc) return rc;
        }
        return ART_OK;
    }
    std::vector<DevJob> J(n);
    for (int i = 0; i < n; ++i) {
        int rc = make_devjob(&jobs[i], &J[i]);
        if (rc || (rc = check_grid(c, &jobs[i]))) return rc;
        if (!imgs[i]) return ART_ERR_ARG;
    }
    CK(cudaSetDevice(c->device));
    int rc = ensure_subs(c);
    if (rc) return rc;
    constexpr int SNAP = C_COUNT + 1;  // counters, then the normalisation's bits
    if (stats && (int64_t)n * SNAP > c->xsnap_cap) {
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->xsnap);
        c->xsnap = nullptr;
        c->xsnap_cap = 0;
        CK(cudaMalloc(&c->xsnap, sizeof(unsigned long long) * SNAP * n));
        c->xsnap_cap = (int64_t)SNAP * n;
    }
    // the largest images first, so that a sub-context's scratch is sized by its first image
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (int64_t)J[a].nx * J[a].ny > (int64_t)J[b].nx * J[b].ny;
    });
    std::vector<int> launches(n, 0);
    CK(cudaEventRecord(c->sub_in, c->stream));
    for (art_ctx* d : c->subs) CK(cudaStreamWaitEvent(d->stream, c->sub_in, 0));
    for (int q = 0; q < n; ++q) {
        const int i = order[q];
        art_ctx* d = c->subs[q % EXACT_SUBS];
        if ((rc = render_impl(d, &jobs[i], nullptr, imgs[i], masks ? masks[i] : nullptr, nullptr,
                              nullptr)))
            return rc;
        launches[i] = d->launches;
        if (stats) {
            CK(cudaMemcpyAsync(c->xsnap + (int64_t)SNAP * i, d->counters,
                               sizeof(unsigned long long) * C_COUNT, cudaMemcpyDeviceToDevice,
                               d->stream));
            CK(cudaMemcpyAsync(c->xsnap + (int64_t)SNAP * i + C_COUNT, d->norm3, sizeof(double),
                               cudaMemcpyDeviceToDevice, d->stream));
        }
    }
    for (int k = 0; k < EXACT_SUBS; ++k) {
        CK(cudaEventRecord(c->sub_out[k], c->subs[k]->stream));
        CK(cudaStreamWaitEvent(c->stream, c->sub_out[k], 0));
    }
    if (!stats) return ART_OK;
    std::vector<unsigned long long> h((size_t)SNAP * n);
    CK(cudaMemcpyAsync(h.data(), c->xsnap, sizeof(unsigned long long) * SNAP * n,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int err = ART_OK;
    for (int i = 0; i < n; ++i) {
        double norm;
        memcpy(&norm, &h[(size_t)SNAP * i + C_COUNT], sizeof norm);
        const int r = stats_from(J[i], &h[(size_t)SNAP * i], norm, launches[i], true, false,
                                 &stats[i]);
        if (r && !err) err = r;
    }
    return err;
}

extern "C" int art_render_batch(art_ctx* c, const art_job* jobs, int32_t n, double* const* imgs,
                                uint8_t* const* masks, art_stats* stats)
{
    if (!c || !jobs || !imgs || n < 1) return ART_ERR_ARG;
    if (jobs[0].precision == ART_MIXED_EXACT) return render_batch_exact(c, jobs, n, imgs, masks, stats);
    BatchPlan P;
    int rc = plan_batch(c, jobs, n, imgs, masks, P);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    if ((rc = ensure_fixed(c)) || (rc = ensure_batch(c, n, P.qcap)) ||
        (rc = bind_batch_scratch(c, P)))
        return rc;
    cudaStream_t st = c->stream;
    c->launches = 0;
    if ((rc = upload_batch(c, P)) || (rc = run_batch(c, P))) return rc;
    if (stats) {
        if ((rc = read_counters(c))) return rc;
        std::vector<double> norms(4 * (size_t)n);
        CK(cudaMemcpyAsync(c->bcounts_host, c->bcounts, sizeof(unsigned long long) * 16 * n,
                           cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(norms.data(), c->bnorms, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost,
                           st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) {
            art_stats& o = stats[i];
            memset(&o, 0, sizeof o);
            for (int l = 0; l <= P.J[i].levels && l < 16; ++l) {
                o.rays_per_level[l] = (int64_t)c->bcounts_host[16 * i + l];
                o.rays_traced += o.rays_per_level[l];
            }
            o.norm = norms[4 * i];
            // batch totals
            o.steps = (int64_t)c->pinned[C_STEPS];
            o.rays_fp64 = (int64_t)c->pinned[C_FP64];
            o.rays_capped = (int64_t)c->pinned[C_CAPPED];
            o.rays_nan = (int64_t)c->pinned[C_NAN];
            o.rays_speculative = (int64_t)c->pinned[C_SPEC];
            o.rays_spec_used = (int64_t)c->pinned[C_SPECUSED];
            o.kernel_launches = c->launches;
        }
        if (c->pinned[C_BADIDX] || c->pinned[C_SYNCERR]) return ART_ERR_DEVICE;
    }
    return ART_OK;
}

extern "C" int art_load_grid(art_ctx* c, const float* grid, int32_t n1, int32_t n2, int32_t n3,
                             double logr_min, double logr_max)
{
    if (!c) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (!grid) {  // unload
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->grid_owned);
        c->grid_owned = nullptr;
        c->grid = nullptr;
        c->g_n1 = c->g_n2 = c->g_n3 = 0;
        return ART_OK;
    }
    if (n1 < 2 || n2 < 2 || n3 < 1 || !(logr_max > logr_min)) return ART_ERR_ARG;
    const int64_t cells = (int64_t)n1 * n2 * n3;
    if (cells > ((int64_t)1 << 30)) return ART_ERR_ARG;
    const size_t bytes = (size_t)cells * 8 * sizeof(float);
    cudaPointerAttributes at;
    memset(&at, 0, sizeof at);
    if (cudaPointerGetAttributes(&at, grid) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    const bool on_device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (on_device && at.device != c->device) return ART_ERR_ARG;
    if (on_device && (reinterpret_cast<uintptr_t>(grid) & 15)) return ART_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->grid_owned);
    c->grid_owned = nullptr;
    c->grid = nullptr;
    if (on_device) {
        c->grid = grid;
    } else {
        CK(cudaMalloc(&c->grid_owned, bytes));
        CK(cudaMemcpyAsync(c->grid_owned, grid, bytes, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->grid = c->grid_owned;
    }
    c->g_n1 = n1;
    c->g_n2 = n2;
    c->g_n3 = n3;
    c->g_x1min = logr_min;
    c->g_x1max = logr_max;
    return ART_OK;
}

// ---- learned block proposal -------------------------------------------------------------------

static bool cnn_dims_ok(int32_t H, int32_t W)
{
    return H >= 1 && W >= 1 && (int64_t)H * W <= ((int64_t)1 << 26);
}

extern "C" int art_cnn_load(art_ctx* c, const float* params_host)
{
    if (!c || !params_host) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cnn_load(c->cnn, params_host, c->stream));
    return ART_OK;
}

extern "C" int art_cnn_read(art_ctx* c, float* params_host)
{
    if (!c || !params_host || !c->cnn) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    CK(cnn_read(c->cnn, params_host, c->stream));
    return ART_OK;
}

extern "C" int art_cnn_forward(art_ctx* c, const float* feat_dev, int32_t H, int32_t W,
                               float* prob_dev)
{
    if (!c || !c->cnn || !feat_dev || !prob_dev || !cnn_dims_ok(H, W)) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    return cnn_forward(c->cnn, feat_dev, H, W, prob_dev, c->stream);
}

extern "C" int art_cnn_grad(art_ctx* c, const float* feat_dev, int32_t H, int32_t W,
                            const float* target_dev, float* loss_host, float* grad_host)
{
    if (!c || !c->cnn || !feat_dev || !target_dev || !cnn_dims_ok(H, W)) return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    return cnn_grad(c->cnn, feat_dev, H, W, target_dev, loss_host, grad_host, c->stream);
}

extern "C" int art_cnn_train_step(art_ctx* c, const float* feat_dev, int32_t H, int32_t W,
                                  const float* target_dev, float lr, float* loss_host)
{
    if (!c || !c->cnn || !feat_dev || !target_dev || !cnn_dims_ok(H, W) || !(lr > 0.f))
        return ART_ERR_ARG;
    CK(cudaSetDevice(c->device));
    return cnn_train_step(c->cnn, feat_dev, H, W, target_dev, lr, loss_host, c->stream);
}

extern "C" int art_cnn_sample(art_ctx* c, const art_job* job, const double* img_dev,
                              const uint8_t* mask_dev, int32_t level, float* feat_dev,
                              float* target_dev)
{
    if (!c || !img_dev || !mask_dev || !feat_dev || !target_dev) return ART_ERR_ARG;
    DevJob J;
    int rc = make_devjob(job, &J);
    if (rc) return rc;
    if (level < 0 || level + 2 > J.levels) return ART_ERR_ARG;
    const int64_t npix = (int64_t)J.nx * J.ny;
    if (!c->aux || c->aux_npix != npix) return ART_ERR_ARG;  // no diagnostics of this grid
    CK(cudaSetDevice(c->device));
    CK(cnn_features_f32(J, level, img_dev, c->aux, c->aux + npix, c->norm3, feat_dev, c->stream));
    CK(cnn_targets(J, level, mask_dev, target_dev, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ART_OK;
}

// --------------------------------------------------------------------------------------------
// kernel-form thresholds and their autotuner
// --------------------------------------------------------------------------------------------

static bool tune_valid(const art_tune* t)
{
    return t->quad_rays >= 0 && t->pair_rays >= t->quad_rays && t->pair_rays <= 4096 &&
           t->blocks64 >= 0 && t->blocks64 <= 64 && t->blocks32 >= 0 && t->blocks32 <= 64 &&
           t->quad64_rays >= 0 && t->quad64_rays <= 4096;
}

extern "C" int art_set_tune(art_ctx* c, const art_tune* t)
{
    if (!c) return ART_ERR_ARG;
    if (!t) {
        c->tune = {ART_TUNE_QUAD_DEFAULT, ART_TUNE_PAIR_DEFAULT, ART_TUNE_BLOCKS64_DEFAULT, 0,
                ART_TUNE_QUAD64_DEFAULT};
        return ART_OK;
    }
    if (!tune_valid(t)) return ART_ERR_ARG;
    c->tune = *t;
    return ART_OK;
}

extern "C" int art_get_tune(art_ctx* c, art_tune* t)
{
    if (!c || !t) return ART_ERR_ARG;
    *t = c->tune;
    return ART_OK;
}

extern "C" int art_autotune(art_ctx* c, const art_job* job, double* img_dev, uint8_t* mask_dev,
                            int32_t reps, art_tune* best, float* best_ms)
{
    if (!c || !job || !img_dev || reps < 1 || reps > 32) return ART_ERR_ARG;
    // candidates, one dimension at a time: the FP32 kernel-form thresholds (one-thread only, pair
    // only, quad/pair splits around the defaults), then with the best of them the persistent
    // grids' blocks per SM, of the FP64 launches (where the job has any: 0 = as many as fit, 1,
    // 2) and of the FP32 and double-float ones (0, then 1 or 2), then the FP64 launches' quad
    // threshold (0: never, 64)
    static const int forms[][2] = {{0, 0},   {0, 64},   {32, 64},  {32, 96},
                                   {64, 96}, {32, 128}, {64, 128}, {16, 64}};
    const bool has64 = job->precision != ART_FP32, has32 = job->precision != ART_FP64;
    CK(cudaSetDevice(c->device));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ART_ERR_CUDA;
    }
    const art_tune saved = c->tune;
    art_tune win = {ART_TUNE_QUAD_DEFAULT, ART_TUNE_PAIR_DEFAULT, ART_TUNE_BLOCKS64_DEFAULT, 0,
                ART_TUNE_QUAD64_DEFAULT};
    float win_ms = INFINITY;
    int rc = ART_OK;
    std::vector<float> t(reps);
    auto trial = [&](const art_tune& cand) {
        c->tune = cand;
        if ((rc = art_render(c, job, nullptr, img_dev, mask_dev, nullptr))) return;  // warm-up
        for (int r = 0; r < reps && rc == ART_OK; ++r) {
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) rc = ART_ERR_CUDA;
            if (!rc) rc = art_render(c, job, nullptr, img_dev, mask_dev, nullptr);
            if (!rc && cudaEventRecord(e1, c->stream) != cudaSuccess) rc = ART_ERR_CUDA;
            if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = ART_ERR_CUDA;
            if (!rc && cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess) rc = ART_ERR_CUDA;
        }
        if (rc) return;
        std::vector<float> srt(t);
        std::sort(srt.begin(), srt.end());
        const float med = srt[reps / 2];
        if (med < win_ms) {
            win_ms = med;
            win = cand;
        }
    };
    for (const auto& f : forms) {
        if (rc) break;
        if (has32 || (f[0] == ART_TUNE_QUAD_DEFAULT && f[1] == ART_TUNE_PAIR_DEFAULT))
            trial(art_tune{f[0], f[1], ART_TUNE_BLOCKS64_DEFAULT, 0, ART_TUNE_QUAD64_DEFAULT});
    }
    for (int b = 0; b <= 2 && has64 && !rc; ++b) {
        if (b == ART_TUNE_BLOCKS64_DEFAULT) continue;
        art_tune cand = win;
        cand.blocks64 = b;
        trial(cand);
    }
    const int best64 = win.blocks64;
    for (int b = 1; b <= 2 && has32 && !rc; ++b) {
        art_tune cand = win;
        cand.blocks64 = best64;
        cand.blocks32 = b;
        trial(cand);
    }
    static const int quad64[] = {0, 64};
    for (int k = 0; k < 2 && has64 && !rc; ++k) {
        art_tune cand = win;
        cand.quad64_rays = quad64[k];
        trial(cand);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune = rc == ART_OK ? win : saved;
    if (rc) return rc;
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return ART_OK;
}

// --------------------------------------------------------------------------------------------
// CUDA-graph replay of the level loop
// --------------------------------------------------------------------------------------------

extern "C" int art_graph_render(art_ctx* c, const art_job* job, double* img_dev, uint8_t* mask_dev)
{
    if (!c || !job || !img_dev) return ART_ERR_ARG;
    if (job->proposal) return ART_ERR_UNSUPPORTED;  // the network's weights may change between calls
    CK(cudaSetDevice(c->device));
    if (!c->gstream) {
        CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->gev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->gev_out, cudaEventDisableTiming));
    }
    const double gmeta[5] = {(double)c->g_n1, (double)c->g_n2, (double)c->g_n3, c->g_x1min,
                             c->g_x1max};
    const bool same = c->gexec && memcmp(&c->gjob, job, sizeof(art_job)) == 0 &&
                      c->gimg == img_dev && c->gmask == mask_dev &&
                      memcmp(&c->gtune, &c->tune, sizeof(art_tune)) == 0 && c->ggrid == c->grid &&
                      memcmp(c->ggmeta, gmeta, sizeof gmeta) == 0 && c->ggen == c->scratch_gen;
    if (!same) {
        // one ordinary render sizes every scratch buffer (no allocation or synchronisation may
        // happen while capturing), then the same call is captured on the capture stream
        int rc = art_render(c, job, nullptr, img_dev, mask_dev, nullptr);
        if (rc) return rc;
        CK(cudaStreamSynchronize(c->stream));
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        const bool prof = c->prof_on;
        cudaStream_t user = c->stream;
        c->prof_on = false;
        c->stream = c->gstream;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = art_render(c, job, nullptr, img_dev, mask_dev, nullptr);
            e = cudaStreamEndCapture(c->gstream, &graph);
        }
        c->stream = user;
        c->prof_on = prof;
        if (e == cudaSuccess && rc == ART_OK) e = cudaGraphInstantiate(&c->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (rc) return rc;
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            cudaGetLastError();
            return ART_ERR_UNSUPPORTED;
        }
        c->gjob = *job;
        c->gimg = img_dev;
        c->gmask = mask_dev;
        c->gtune = c->tune;
        c->ggrid = c->grid;
        memcpy(c->ggmeta, gmeta, sizeof gmeta);
        c->ggen = c->scratch_gen;
    }
    CK(cudaEventRecord(c->gev_in, c->stream));
    CK(cudaStreamWaitEvent(c->gstream, c->gev_in, 0));
    CK(cudaGraphLaunch(c->gexec, c->gstream));
    CK(cudaEventRecord(c->gev_out, c->gstream));
    CK(cudaStreamWaitEvent(c->stream, c->gev_out, 0));
    return ART_OK;
}

extern "C" int art_graph_render_batch(art_ctx* c, const art_job* jobs, int32_t n,
                                      double* const* imgs, uint8_t* const* masks)
{
    if (!c || !jobs || !imgs || n < 1) return ART_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (jobs[i].proposal) return ART_ERR_UNSUPPORTED;
    CK(cudaSetDevice(c->device));
    if (!c->gstream) {
        CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->gev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->gev_out, cudaEventDisableTiming));
    }
    const double gmeta[5] = {(double)c->g_n1, (double)c->g_n2, (double)c->g_n3, c->g_x1min,
                             c->g_x1max};
    bool same = c->gbexec && c->gbplan && (int)c->gbjobs.size() == n && c->gbgrid == c->grid &&
                memcmp(c->gbgmeta, gmeta, sizeof gmeta) == 0 && c->gbgen == c->scratch_gen &&
                memcmp(c->gbjobs.data(), jobs, sizeof(art_job) * n) == 0;
    for (int i = 0; same && i < n; ++i)
        same = c->gbimgs[i] == imgs[i] && c->gbmasks[i] == (masks ? masks[i] : nullptr);
    if (!same) {
        BatchPlan* P = new BatchPlan();
        int rc = plan_batch(c, jobs, n, imgs, masks, *P);
        // one ordinary batch render sizes the scratch; then the device part is captured
        if (!rc) rc = art_render_batch(c, jobs, n, imgs, masks, nullptr);
        if (!rc) rc = bind_batch_scratch(c, *P);
        if (rc) {
            delete P;
            return rc;
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            delete P;
            return ART_ERR_CUDA;
        }
        if (c->gbexec) {
            cudaGraphExecDestroy(c->gbexec);
            c->gbexec = nullptr;
        }
        destroy_plan(c->gbplan);
        c->gbplan = nullptr;
        const bool prof = c->prof_on;
        cudaStream_t user = c->stream;
        c->prof_on = false;
        c->stream = c->gstream;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = run_batch(c, *P);
            e = cudaStreamEndCapture(c->gstream, &graph);
        }
        c->stream = user;
        c->prof_on = prof;
        if (e == cudaSuccess && rc == ART_OK) e = cudaGraphInstantiate(&c->gbexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (rc || e != cudaSuccess) {
            delete P;
            c->gbexec = nullptr;
            cudaGetLastError();
            return rc ? rc : ART_ERR_UNSUPPORTED;
        }
        c->gbplan = P;
        c->gbjobs.assign(jobs, jobs + n);
        c->gbimgs.assign(imgs, imgs + n);
        c->gbmasks.assign(n, nullptr);
        if (masks) c->gbmasks.assign(masks, masks + n);
        c->gbgrid = c->grid;
        memcpy(c->gbgmeta, gmeta, sizeof gmeta);
        c->gbgen = c->scratch_gen;
    }
    // the job tables are re-uploaded every call (another batch call may have replaced them)
    int rc = upload_batch(c, *c->gbplan);
    if (rc) return rc;
    CK(cudaEventRecord(c->gev_in, c->stream));
    CK(cudaStreamWaitEvent(c->gstream, c->gev_in, 0));
    CK(cudaGraphLaunch(c->gbexec, c->gstream));
    CK(cudaEventRecord(c->gev_out, c->gstream));
    CK(cudaStreamWaitEvent(c->stream, c->gev_out, 0));
    return ART_OK;
}
