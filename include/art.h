/*
 * art.h -- C-ABI of the GB300-native adaptive ray tracer (libart_gb300.so).
 *
 * Adaptive ray tracing of Kerr black-hole images after Gelles et al. 2021, "The Role of Adaptive
 * Ray Tracing in Analyzing Black Hole Structure" (arXiv:2103.07417):
 *   - Sec. 3.2: a base grid of n0x x n0y rays is traced, then N times the grid is refined by a
 *     factor 2 to (2 n0 - 1); every new point is traced if BOTH estimated errors exceed their
 *     tolerances (eps_abs > R_abs and eps_rel > R_rel) and interpolated otherwise.  The final
 *     image has n = 2^N (n0 - 1) + 1 points per axis.
 *   - Eqs. (epabs), (eprel), Appendix A: the estimated errors (linear and nearest schemes) from the
 *     eight neighbours of the previous level, normalised by I_bar_int, the interpolated mean
 *     intensity after the first pass.
 *   - Eqs. (interpdef), (fluxdef), (msedef): interpolation fraction, flux error, MSE.
 * The intensity of one pixel is the covariant radiative transfer integrated along the null
 * geodesic traced backward from a static pinhole camera through the Kerr metric (the paper leaves
 * this to ipole; here: outgoing Cartesian Kerr-Schild Hamiltonian, RK4 with h = step_frac * r).
 *
 * Conventions for every call:
 *   - Every pointer named *_dev is a device pointer on the context's device; the caller owns it
 *     and it must stay valid until the work queued on the context's stream has finished.
 *     Pointers named *_host are ordinary host memory.  The library owns only its scratch (ray
 *     queues, counters), allocated on first use and grown when a larger job arrives.
 *   - Work is queued on the stream given to art_create; calls that return statistics to the host
 *     synchronise that stream before returning.
 *   - Images are planes x ny x nx, row-major (pixel p = j*nx + i; i runs along the screen's
 *     horizontal axis alpha, j along the vertical axis beta, which is the projected spin axis).
 *     Plane order is Stokes (I[,Q,U,V]) inside subring index: plane = n * stokes + s.
 *   - Return value: ART_OK (0) or a negative ART_ERR_* code; art_strerror() names it.  No call
 *     falls back to the CPU: without a CUDA device every compute call returns ART_ERR_CUDA.
 */
#ifndef ART_GB300_H
#define ART_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ART_OK 0
#define ART_ERR_ARG (-1)         /* invalid argument or job */
#define ART_ERR_CUDA (-2)        /* CUDA runtime error (no device, launch failure, ...) */
#define ART_ERR_OOM (-3)         /* device allocation of library scratch failed */
#define ART_ERR_UNSUPPORTED (-4) /* option combination not built */
#define ART_ERR_DEVICE (-5)      /* a kernel reported an internal inconsistency */

enum { ART_EMIT_ANALYTIC = 0, ART_EMIT_SYNCH_DISK = 1, ART_EMIT_GRID = 2 };
enum { ART_FLOW_KEPLER = 0, ART_FLOW_STATIC = 1 };
enum { ART_NORM_IBAR_INT = 0, ART_NORM_PEAK = 1 };
enum { ART_INTERP_LINEAR = 0, ART_INTERP_NEAREST = 1 };
enum { ART_EDGE_ONESIDED = 0, ART_EDGE_TRACE = 1 };
enum { ART_CRIT_I = 0, ART_CRIT_STOKES_ANY = 1 };
enum { ART_FP64 = 0, ART_MIXED = 1, ART_FP32 = 2, ART_MIXED_DF = 3, ART_MIXED_EXACT = 4 };
enum { ART_MASK_UNSET = 0, ART_MASK_TRACED = 1, ART_MASK_INTERP = 2, ART_MASK_AXIS = 3 };
enum { ART_RAY_ESCAPED = 0, ART_RAY_CAPTURED = 1, ART_RAY_CAP = 2, ART_RAY_NAN = 3 };

/* One rendering problem: camera, spacetime, emission model and the refinement parameters of
 * Sec. 3.2 (n0x, n0y, N, R_rel, R_abs, interpolation scheme). */
typedef struct art_job {
    double a;            /* dimensionless spin, |a| < 1 (M = 1 units) */
    double r_obs;        /* camera radius [M] */
    double incl_deg;     /* camera inclination [deg], 0 < incl < 180 */
    double fov;          /* horizontal field of view [M]; spacing fov/(nx-1) on both axes */
    int32_t n0x, n0y;    /* base grid, n0x >= 2, n0y >= 1 */
    int32_t levels;      /* N >= 0 refinement levels (<= 14) */
    double R_rel, R_abs; /* tolerances of Sec. 3.2 (strict '>' traces) */
    int32_t abs_norm;    /* ART_NORM_IBAR_INT (paper) or ART_NORM_PEAK (max of the base image) */
    int32_t interp;      /* ART_INTERP_LINEAR (paper default) or ART_INTERP_NEAREST */
    int32_t edge_mode;   /* ART_EDGE_ONESIDED or ART_EDGE_TRACE (trace points lacking a stencil) */
    int32_t emission;    /* ART_EMIT_* */
    int32_t flow;        /* ART_FLOW_* */
    int32_t stokes;      /* 1 (unpolarized) or 4 (I, Q, U, V; ART_EMIT_SYNCH_DISK or _GRID) */
    int32_t subrings;    /* 0, or the number of subring planes n = 0..subrings-1 */
    int32_t precision;   /* ART_FP64; ART_MIXED: FP32 with an FP64 re-trace of near-critical rays;
                          * ART_MIXED_DF: the same with the re-traced geodesic in double-float
                          * (float pairs, ~48-bit significand) on the FP32 pipes; ART_FP32;
                          * ART_MIXED_EXACT: ART_MIXED_DF with the refinement decisions of the
                          * FP64 render (art_render only): the base level is traced in FP64, and
                          * every point whose estimate lies within a relative band (0.25) of a
                          * tolerance is decided in FP64 on exact values of its stencil (FP64
                          * re-traces of the FP32-traced values it reads, recomputed interpolants
                          * of the interpolated ones), so its mask equals the FP64 render's wherever
                          * the FP32 values decide a point as the FP64 values would outside that
                          * band.  In both mixed modes the FP32 pass also hands over rays with a
                          * sample within rounding of a discontinuity of the emission model (the
                          * magnetisation cut, the disk's inner edge). */
    int32_t max_steps;   /* RK4 step cap per ray */
    double fp64_sweep;   /* ART_MIXED: re-trace in FP64 the rays whose position vector swept at
                          * least this angle [rad] about the hole (3 pi: a full loop of
                          * deflection beyond a straight pass), i.e. the near-critical rays
                          * whose errors the photon-orbit instability amplifies */
    double step_frac;    /* RK4 step h = step_frac * r */
    double h_min;        /* floor of h */
    double horizon_eps;  /* stop rays at r < (1 + horizon_eps) r_+ */
    double escape_frac;  /* stop rays at r > escape_frac * r_obs (at most 1e8 [M]) */
    double disk_w;       /* vertical Gaussian width of the emitter as a fraction of r */
    /* ART_EMIT_SYNCH_DISK: thermal-synchrotron thin disk, n_e = ne0 r^ne_slope
     * exp(-cos^2(theta)/(2 disk_w^2)) [cm^-3], Theta_e = thetae0 r^te_slope, |B| = b0
     * r^((ne_slope + te_slope)/2) [G] along (e_phi + bz_ratio e_z) in the fluid frame, Keplerian,
     * no emission inside r_in; observed at nu_hz for a hole with GM/c^2 = length_cm. */
    double ne0, thetae0, b0, nu_hz, ne_slope, te_slope, r_in, length_cm, bz_ratio;
    /* ART_EMIT_GRID: thermal synchrotron from the context's fluid grid (art_load_grid), the
     * GRMHD-image model of Sec. 4.2 and 5: Theta_e = (m_p/m_e)(gamma_ad - 1) u / (rho (1 + R)),
     * R = T_i/T_e = (r_high beta^2 + r_low)/(1 + beta^2) with beta = (gamma_ad - 1) u/(b^2/2);
     * n_e = rho m_unit/(length_cm^3 (m_p + m_e)), |B| = |b| c sqrt(4 pi m_unit / length_cm^3);
     * no emission where b^2/rho > sigma_cut; observed at nu_hz. */
    double gamma_ad, m_unit, r_high, r_low, sigma_cut;
    /* Learned path (not in the paper): with proposal = 1, after the criterion of every level
     * k = 1, 1 + D, 1 + 2D, ... (D = proposal_depth >= 1) the loaded network (art_cnn_load) reads
     * the completed level-(k-1) lattice, and in every block whose probability exceeds proposal_p
     * the points of levels k+1 .. k+D next to the refinement front (a corner of their level-k
     * cell is traced) are traced speculatively together with level k's rays.  The exact criterion still decides
     * every point: a speculative ray it asks for is used, one it does not ask for is discarded
     * (interpolated), so image and mask equal those of the same render without the proposal.
     * Requires a loaded network and no truth image (else ART_ERR_ARG); a scratch mask is used
     * when mask_dev is NULL. */
    int32_t proposal, proposal_depth;
    double proposal_p;
    /* Near-critical band (not in the paper; 0 = off, else 0 < crit_band < 1): every pixel of
     * levels 1..N whose camera ray has constants of motion (lambda, eta) within crit_band of the
     * Kerr critical curve (Bardeen 1973), measured as d = |R(r_m)| / r_m^4 with R the photon's
     * radial potential at its minimum r_m over the photon-orbit radii (|27 - eta - lambda^2|/27
     * for a = 0), is traced speculatively
     * with the base level, so the high-precision re-traces of the photon-ring rays of all levels
     * share one pass.  The exact criterion still decides every point: image and mask equal those
     * of the render without it.  Not with a truth image (ART_ERR_ARG).  art_render_batch applies
     * each job's band to its image, all in the batch's base-level pass.  With ART_MIXED_EXACT the
     * band's rays are traced in FP32 and double-float, and a borderline point still needs its
     * stencil's FP64 values at its own level, so there the band usually costs more than it saves
     * (the 16385^2 grid render: 60.7 ms with a band of 0.03, 58.7 ms without). */
    double crit_band;
    /* Criterion of polarized jobs (Sec. 6 proposes "replacing I by Q, U, V"): ART_CRIT_I decides
     * on I; ART_CRIT_STOKES_ANY traces a point when the criterion holds for any of I, Q, U, V
     * (Q, U, V through the same estimator, eps_abs over the same normalisation, eps_rel over the
     * magnitude of I's interpolant).  Ignored for stokes = 1; not with ART_MIXED_EXACT
     * (ART_ERR_UNSUPPORTED). */
    int32_t criterion;
    /* The plane the criterion reads (default 0): with subring planes, criterion_plane = n * stokes
     * decides on subring n's image (the paper renders each subring's image adaptively on its
     * own, Sec. 5.1).  0 <= criterion_plane < art_planes(job); 0 with ART_CRIT_STOKES_ANY. */
    int32_t criterion_plane;
} art_job;

/* Statistics of one render (host struct, filled on return). */
typedef struct art_stats {
    int64_t rays_traced;        /* rays whose result is in the image */
    int64_t rays_fp64;          /* mixed modes: rays re-traced at high precision */
    int64_t steps;              /* RK4 steps summed over all traced rays (incl. re-traces) */
    int64_t rays_capped;        /* rays that hit max_steps */
    int64_t rays_nan;           /* rays stopped by a non-finite state */
    int64_t rays_per_level[16]; /* rays traced at level 0..N */
    double norm;                /* I_bar_int (or the peak) used by the criterion */
    int64_t kernel_launches;    /* CUDA kernels this call launched */
    int64_t rays_speculative;   /* learned path: rays traced speculatively */
    int64_t rays_spec_used;     /* learned path: speculative rays the criterion asked for (these
                                 * are included in rays_traced; the rest were wasted) */
    int64_t rays_exact;         /* ART_MIXED_EXACT: FP64 rays traced for exact decisions (base
                                 * level, stencil re-traces, borderline points) */
    int64_t border_points;      /* ART_MIXED_EXACT: points decided on exact stencil values */
    int64_t border_overflow;    /* ART_MIXED_EXACT: borderline points decided without them
                                 * because the library's list was full (0 in normal use) */
} art_stats;

/* One kernel launch timed by the profiler (art_profile). */
enum { ART_K_TRACE_FP64 = 0, ART_K_TRACE_FP32 = 1, ART_K_REFINE = 2, ART_K_OTHER = 3,
       ART_K_TRACE_DF = 4, ART_K_PROPOSE = 5 };
typedef struct art_launch_record {
    int32_t kind;   /* ART_K_* */
    int32_t level;  /* refinement level of the launch (-1 outside a render) */
    float ms;       /* duration between CUDA events recorded around the launch on its stream */
    int64_t steps;  /* trace kernels: RK4 steps executed by this launch */
    int64_t items;  /* trace: rays it finished or handed on; refine: lattice points of the level */
    int64_t max_steps; /* trace kernels: RK4 steps of its longest ray */
} art_launch_record;

/* Per-ray diagnostics (device arrays, one entry per traced ray; nullable members). */
typedef struct art_rayaux {
    int32_t* status; /* ART_RAY_* */
    int32_t* steps;  /* RK4 steps */
    int32_t* nturn;  /* polar (theta) turning points = subring index of the last segment */
    float* min_r;    /* closest Kerr-Schild radius reached */
} art_rayaux;

typedef struct art_ctx art_ctx;

/* Create a context on CUDA device `device` that queues its work on `stream` (a cudaStream_t, or
 * NULL for the legacy default stream).  *out receives the context.  Errors: ART_ERR_ARG (null
 * out), ART_ERR_CUDA (no such device).  Allocates no device memory yet. */
int art_create(art_ctx** out, int device, void* stream);

/* Synchronise the stream and free the context's scratch.  Null is ignored. */
void art_destroy(art_ctx* ctx);

/* Static description of an error code. */
const char* art_strerror(int code);

/* Final image size n = 2^N (n0 - 1) + 1 (Sec. 3.2).  Errors: ART_ERR_ARG. */
int art_image_size(const art_job* job, int32_t* nx, int32_t* ny);

/* Number of planes of the image: stokes * max(subrings, 1). */
int art_planes(const art_job* job);

/* Trace the pixels pix_dev[0..n) (linear indices j*nx + i of the job's final grid) and write
 * their planes to out_dev[q*planes + plane] (ray-major).  aux (nullable, and each member
 * nullable) receives per-ray diagnostics.  The precision is the job's (ART_MIXED: FP32 trace
 * then an FP64 re-trace of the rays that swept >= fp64_sweep).  Errors: ART_ERR_ARG
 * (bad job, n < 0, pixel index not checked on the host: an index outside [0, nx*ny) is
 * skipped by the kernel and reported as ART_ERR_DEVICE), ART_ERR_CUDA, ART_ERR_OOM. */
int art_trace_pixels(art_ctx* ctx, const art_job* job, const int32_t* pix_dev, int64_t n,
                     double* out_dev, const art_rayaux* aux);

/* I_bar_int (Sec. 3.2): mean of the bilinear interpolant of the sub-lattice of stride `stride`
 * of the nx x ny plane img_dev, i.e. trapezoid weights; and the maximum of that sub-lattice.
 * Both are returned to the host (synchronises the stream). */
int art_ibar_int(art_ctx* ctx, const double* img_dev, int32_t nx, int32_t ny, int32_t stride,
                 double* ibar_host, double* peak_host);

/* One refinement level (Sec. 3.2, Eqs. epabs/eprel, Appendix A) on the job's final grid:
 * every new point of `level` (1..N) reads only points of level-1 in img_dev (plane 0 decides),
 * gets mask ART_MASK_TRACED and its index appended to queue_dev (capacity: the number of new
 * points of the level), or receives the interpolant in every plane and ART_MASK_INTERP.
 * `norm` is I_bar_int (or the peak).  *count_host receives the queue length (synchronises).
 * The queue's order is unspecified.  Errors: ART_ERR_ARG, ART_ERR_CUDA. */
int art_refine_level(art_ctx* ctx, const art_job* job, double* img_dev, uint8_t* mask_dev,
                     int32_t level, double norm, int32_t* queue_dev, int64_t* count_host);

/* The whole adaptive render (Sec. 3.2): trace the base grid, compute the normalisation, then
 * for each level refine and trace the queue on the device (no host round trip inside).
 * img_dev: planes x ny x nx doubles; mask_dev (nullable): ny x nx bytes (ART_MASK_*).
 * truth_dev (nullable): if given (planes x ny x nx), "tracing" a pixel copies it from there, so
 * the refinement logic can be run on any precomputed image (not with ART_MIXED_EXACT:
 * ART_ERR_ARG).  stats_host (nullable) is filled and the stream synchronised if it is given.
 * Errors: ART_ERR_ARG, ART_ERR_CUDA, ART_ERR_OOM, ART_ERR_DEVICE (ART_MIXED_EXACT also reports
 * a stencil value that was not exact when its decision was made, which would be a bug). */
int art_render(art_ctx* ctx, const art_job* job, const double* truth_dev, double* img_dev,
               uint8_t* mask_dev, art_stats* stats_host);

/* The batched form: render n images in one pass per level.  Every kernel of a level works on all
 * images that have that level, and the rays of all images share one device queue, so one
 * persistent trace launch per level packs rays of uneven length from images of different spins,
 * inclinations, fields of view, grids and depths.  jobs[i] may differ in everything except
 * stokes, subrings, precision and whether the emission is ART_EMIT_GRID (one kernel kind and one
 * plane count per batch; else ART_ERR_ARG); grid jobs all use the context's grid.  imgs is a
 * HOST array of n device pointers (planes x ny_i x nx_i doubles each); masks (nullable, entries
 * nullable) a host array of n device pointers.  Jobs with crit_band > 0 speculate as in
 * art_render (an image without a mask then uses a context-owned scratch mask).  stats_host
 * (nullable) receives n entries: rays per level and the normalisation per image; steps,
 * re-traced, capped, NaN and speculative rays and kernel launches are batch totals repeated in
 * every entry.  Synchronises when stats are requested.  Jobs with precision ART_MIXED_EXACT
 * (all of them, else ART_ERR_ARG) are rendered one after the other by art_render, with per-image
 * stats.  Errors as art_render. */
int art_render_batch(art_ctx* ctx, const art_job* jobs, int32_t n, double* const* imgs,
                     uint8_t* const* masks, art_stats* stats_host);

/* Adaptive sampling along a third axis: frequency or time (Sec. 6 proposes extending the method
 * "to selectively sample the time and frequency domains").  jobs[f], f = 0 .. F-1, is the problem
 * at axis sample f (an observing frequency nu_hz, or a movie frame's snapshot); all jobs share the
 * pixel grid and plane count.  F = 2^levels3 (F0 - 1) + 1.  The images of the base samples
 * (f a multiple of 2^levels3) are rendered by art_render (adaptive in x and y).  Then, for
 * k = 1 .. levels3, every new sample f (an odd multiple of s = 2^(levels3 - k)) is
 * rendered with the spatial scheme of Sec. 3.2, and every point that scheme would trace is decided
 * again along the axis with the same one-dimensional estimator, on plane 0: inner samples f -/+ s
 * and outer f -/+ 3s of level k-1 (complete images; one-sided where one outer sample is missing,
 * infinite where both are), eps_abs = |d| / (8 I_bar), eps_rel = |d| / (2 |S_in|) with I_bar the
 * mean of the base samples' I_bar_int.  The point is traced with jobs[f] only if both exceed
 * R_abs3, R_rel3 (strict); otherwise it receives the mean of its two axis neighbours in every plane
 * (mask ART_MASK_AXIS).  A point is thus traced only where neither the spatial nor the axis
 * interpolant is good enough.  The new samples' renders take no speculation (crit_band and the
 * proposal are ignored there).
 * imgs: HOST array of F device images (planes x ny x nx doubles), written.  truth (nullable): HOST
 * array of F device images; if given, the axis logic alone runs on them: base samples copy
 * truth[f] (their I_bar_int is that image's trapezoid mean), every pixel of a new sample is decided
 * along the axis, and "tracing" copies from truth[f].  amask_dev (nullable): F x ny x nx bytes,
 * the samples' masks (ART_MASK_TRACED / INTERP / AXIS; all TRACED for base samples with truth).
 * stats_host (nullable): F entries (rays_traced = rays actually traced for the sample,
 * border_points = its points interpolated along the axis).  Not with ART_MIXED_EXACT
 * (ART_ERR_UNSUPPORTED).  Synchronises the context's stream.  Errors as art_render. */
int art_render_axis(art_ctx* ctx, const art_job* jobs, int32_t F, int32_t levels3, double R_rel3,
                    double R_abs3, const double* const* truth, double* const* imgs,
                    uint8_t* amask_dev, art_stats* stats_host);

/* Visibility-domain analysis (Sec. 4.3): the complex visibilities of one image plane, the 2-D
 * Fourier transform that an interferometer baseline (u, v) samples,
 *   V(u, v) = dx^2 sum_{x,y} T(x, y) A(x, y) exp(-2 pi i (u X + v Y)),
 *   X = (x - (nx-1)/2) dx, Y = (y - (ny-1)/2) dx (origin at the image centre),
 *   T = exp(-4 ln 2 (X^2 + Y^2) / taper_fwhm^2) (the paper's Gaussian taper; none if <= 0),
 *   A = img, or img - ref when ref_dev is given (the Fourier amplitudes of the residual image),
 * on the grid u = k_u / (m dx), v = k_v / (m dx), k in [-m/2, m/2), of an m x m FFT of the
 * zero-padded image.  The paper doubles the field of view and the pixel count before the taper
 * (same resolution): render the job with fov * 2 and n0 -> 2 n0 - 1 for that.
 * img_dev, ref_dev (nullable): ny x nx doubles, row-major (one plane of an art_render image).
 * vis_dev: caller-owned m x m complex doubles (re, im interleaved), row k_v, column k_u, each
 * frequency index stored at k mod m.  m: a power of two, 32 <= m <= 32768, m >= nx, ny.  The
 * library holds m x m complex doubles of scratch (grown, never shrunk).  FP64 throughout.
 * Errors: ART_ERR_ARG, ART_ERR_OOM, ART_ERR_CUDA.  Asynchronous on the context's stream. */
int art_visibilities(art_ctx* ctx, const double* img_dev, const double* ref_dev, int32_t nx,
                     int32_t ny, double dx, double taper_fwhm, int32_t m, double* vis_dev);

/* art_render into HOST buffers: the image and mask are rendered into context-owned device
 * buffers and copied to img_host (planes x ny x nx doubles) and mask_host (nullable, ny x nx
 * bytes).  Synchronises the stream. */
int art_render_host(art_ctx* ctx, const art_job* job, double* img_host, uint8_t* mask_host,
                    art_stats* stats_host);

/* Scheduling of the trace launches (the paper has no counterpart: choices of this
 * implementation).  Kernel forms of the FP32 pass: a level's FP32 launch whose queue holds at most
 * quad_rays rays per block of the persistent grid splits each step over four warps per 32 rays
 * (geodesic, two warps for the emission coefficients of alternate steps, segment); at most
 * pair_rays, over two warps (geodesic, transfer); longer queues run one thread per ray.  FP64
 * launches take the four-warp form when their queue holds at most quad64_rays rays per block, the
 * two-warp form otherwise (an FP64 warp instruction costs a scheduler 64 cycles whatever its
 * active lanes, so a lone ray's step lasts as long as its slowest warp's FP64 chain).  Grid size:
 * the persistent grids of the FP64 launches hold blocks64 blocks of 128 threads per SM, those of
 * the FP32 and double-float launches blocks32 (0: as many as fit; a larger value is capped there).
 * The forms and grids give bit-identical rays, so the setting changes speed only.  Defaults
 * ART_TUNE_QUAD_DEFAULT, ART_TUNE_PAIR_DEFAULT, ART_TUNE_BLOCKS64_DEFAULT (one block of four
 * warps per SM: one warp per scheduler, which is all the FP64 pipe takes), 0,
 * ART_TUNE_QUAD64_DEFAULT; valid settings have 0 <= quad_rays <= pair_rays <= 4096,
 * 0 <= quad64_rays <= 4096 and 0 <= blocks64, blocks32 <= 64. */
#define ART_TUNE_QUAD_DEFAULT 32
#define ART_TUNE_PAIR_DEFAULT 64
#define ART_TUNE_BLOCKS64_DEFAULT 1
#define ART_TUNE_QUAD64_DEFAULT 32
typedef struct art_tune {
    int32_t quad_rays;
    int32_t pair_rays;
    int32_t blocks64;
    int32_t blocks32;
    int32_t quad64_rays;
} art_tune;

/* Set the context's scheduling setting (t == NULL restores the defaults), or read it.
 * Errors: ART_ERR_ARG (null context, invalid setting). */
int art_set_tune(art_ctx* ctx, const art_tune* t);
int art_get_tune(art_ctx* ctx, art_tune* t_out);

/* Autotuner: renders `job` (as art_render, into img_dev / mask_dev) with each candidate setting,
 * once to warm up and `reps` times timed with CUDA events on the context's stream, one dimension at
 * a time (eight FP32 kernel-form threshold pairs with the default grids; then, from the best,
 * blocks64 in {0, 1, 2} if the job has FP64 launches; then blocks32 in {1, 2} if it has FP32
 * ones; then quad64_rays in {0, 64} if it has FP64 launches), keeps the setting with the lowest
 * median time in the context and returns it in *best (nullable) with that median in *best_ms
 * (nullable).  img_dev and mask_dev hold the job's image
 * afterwards (the same for every setting).  Synchronises the stream.  Errors: ART_ERR_ARG (reps
 * outside 1..32, or as art_render), and those of art_render, after which the previous setting is
 * kept. */
int art_autotune(art_ctx* ctx, const art_job* job, double* img_dev, uint8_t* mask_dev,
                 int32_t reps, art_tune* best, float* best_ms);

/* art_render replayed from a CUDA graph (no stats; the paper has no counterpart).  The first call
 * for a given job, image and mask pointers, kernel-form setting and fluid grid renders once
 * normally (which sizes every scratch buffer), then captures the whole level loop (every launch
 * and memset of art_render) on a stream of the context's own and instantiates it; that call and
 * every later call with the same key launch the graph, ordered after prior work on the context's
 * stream and before later work (two events).  A different key captures again, replacing the
 * graph, as does any scratch buffer the context reallocated since the capture.  Since the first
 * call of a key synchronises the context's stream and captures, it must not itself be made while
 * that stream is being captured.  Jobs with the learned proposal return
 * ART_ERR_UNSUPPORTED (the network's weights may change between calls), as does a capture the
 * driver refuses.  Other errors as art_render. */
int art_graph_render(art_ctx* ctx, const art_job* job, double* img_dev, uint8_t* mask_dev);

/* art_render_batch replayed from a CUDA graph (no stats), on the same terms as art_graph_render:
 * the first call for a given batch (job structs, image and mask pointers) and fluid grid renders
 * it once normally, then captures its device part (every memset and launch of the level loop) and
 * instantiates it; every call uploads the batch's job tables (from a host copy the context keeps)
 * and launches the graph.  A scratch buffer reallocated by any later call of the context makes the
 * next call capture again.  Learned jobs: ART_ERR_UNSUPPORTED. */
int art_graph_render_batch(art_ctx* ctx, const art_job* jobs, int32_t n, double* const* imgs,
                           uint8_t* const* masks);

/* Per-launch profiling.  With enable != 0 every kernel launch of the following calls is
 * bracketed by CUDA events on the context's stream (and the trace kernels' step counters are
 * snapshotted), for at most 256 launches; enable == 0 stops recording.  art_profile_read
 * synchronises the stream and copies up to `cap` records of the launches since the last
 * art_profile(ctx, 1) into recs_host, *n receiving their number.  Errors: ART_ERR_ARG,
 * ART_ERR_CUDA, ART_ERR_OOM. */
int art_profile(art_ctx* ctx, int enable);
int art_profile_read(art_ctx* ctx, art_launch_record* recs_host, int cap, int* n);

/* Measured peaks of the plain arithmetic pipes (not in the paper; the denominators of the tracer's
 * roofline): fused multiply-add throughput in TFLOP/s (one FMA = 2 flops) of FP32 and FP64
 * chains on every SM, the best of three CUDA-event timed launches each, written to *fp32_tflops
 * and *fp64_tflops (host pointers).  Synchronises the context's stream first; allocates and
 * frees a small device buffer.  Errors: ART_ERR_ARG (null pointer), ART_ERR_CUDA. */
int art_measure_alu_peaks(art_ctx* ctx, double* fp32_tflops, double* fp64_tflops);

/* Issue cost of FP64 fused multiply-adds on one SM (not in the paper; it sets how the tracer splits
 * an FP64 ray's work between warps), in SM clock cycles per instruction, written to cycles3[0..2]
 * (host array): [0] one warp, one dependent chain; [1] one warp, eight independent chains;
 * [2] four warps (one per scheduler), eight chains each, per warp instruction of the SM.
 * Synchronises the context's stream first; allocates and frees a small device buffer.
 * Errors: ART_ERR_ARG (null pointer), ART_ERR_CUDA. */
int art_measure_fp64_issue(art_ctx* ctx, double* cycles3);

/* art_trace_pixels for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant.  Some callers cannot let a library call cudaMalloc:
 * a process whose device memory is reserved up front by its own allocator (a render service with
 * a fixed budget per GPU), code running while another framework owns allocation, or a caller that
 * must avoid the implicit synchronisation cudaMalloc and cudaFree can cause.  This call allocates
 * nothing and needs no context: it traces on the current device and on `stream` (a cudaStream_t
 * of the current device, else ART_ERR_ARG; NULL = legacy default stream), with the same
 * arguments, output layout and precision handling as art_trace_pixels.  Its scratch (camera, counters, FP64 re-trace queue) is one static device
 * array of about 4.2 MB, which every GPU that loads the library holds until the process exits.
 *   - n may be at most ART_NOALLOC_MAX_RAYS; larger n returns ART_ERR_ARG before any GPU work.
 *   - The first call on a device resolves the array's device address (cudaGetSymbolAddress) and
 *     the launch geometry.
 *   - Every call copies the ray count from the host stack to the array and synchronises `stream`
 *     before returning, so a call cannot be made while `stream` is being captured into a CUDA
 *     graph.
 *   - Every call shares the one array and clears its counters first; calls that overlap on the GPU
 *     (on different streams, or from several host threads) race on it and must be serialised.
 *   - Errors as art_trace_pixels. */
#define ART_NOALLOC_MAX_RAYS (1 << 20)
int art_trace_pixels_noalloc(const art_job* job, const int32_t* pix_dev, int64_t n,
                             double* out_dev, const art_rayaux* aux, void* stream);

/* The fluid snapshot of ART_EMIT_GRID jobs (Sec. 4.2: images of GRMHD snapshots; the lookup is
 * this library's).  grid holds n3 x n2 x n1 cells of eight FP32 primitives, cell (k, j, i) at
 * grid[((k * n2 + j) * n1 + i) * 8 + q], q = rho, u (internal energy), u^r, u^theta, u^phi
 * (contravariant four-velocity), B^r, B^theta, B^phi (B^i = *F^{it}), all in Kerr-Schild spherical
 * coordinates of the job's spin (x + i y = (r - i a) sin(theta) e^{i phi}, z = r cos(theta)),
 * code units (G = c = M = 1; Heaviside-Lorentz field units, magnetic pressure b^2/2).
 * Cell centres: ln r = logr_min + (i + 1/2)(logr_max - logr_min)/n1, theta = (j + 1/2) pi/n2,
 * phi = (k + 1/2) 2 pi/n3.  Samples are trilinear in (ln r, theta, phi); ln r and theta clamp to
 * the outer cell centres, phi is periodic, and points with ln r outside [logr_min, logr_max] do
 * not emit.  u^t follows from u.u = -1.
 *   - grid may be a device pointer on the context's device (16-byte aligned; referenced, not
 *     copied: the caller keeps it alive and unchanged while jobs use it) or host memory (copied
 *     into context-owned device memory before the call returns).
 *   - grid == NULL unloads.  Loading replaces the previous grid (synchronises the stream first).
 *   - n1, n2 >= 2, n3 >= 1, logr_max > logr_min, at most 2^30 cells; else ART_ERR_ARG (also
 *     for a device pointer on another device or misaligned).  ART_ERR_OOM, ART_ERR_CUDA.
 * Grid jobs on a context without a grid return ART_ERR_ARG; art_trace_pixels_noalloc has no
 * context and returns ART_ERR_UNSUPPORTED for them. */
int art_load_grid(art_ctx* ctx, const float* grid, int32_t n1, int32_t n2, int32_t n3,
                  double logr_min, double logr_max);

/* ---- Learned block proposal (not in the paper) -------------------------------------------
 * A small convolutional network predicts, from the completed level-k lattice, which blocks the
 * exact criterion of Sec. 3.2 will refine two levels later (the learned path traces them early;
 * the exact criterion still decides every point).  Network: features f = (asinh(I / I_norm),
 * 3 / max(r_min, 1), polar turns) per lattice point; four 3x3 convolutions with 32 channels
 * (strides 1, 1, 2, 2, zero padding 1, bias, ReLU) and a 1x1 head with a logistic output: one
 * probability per 4 x 4 lattice cells, i.e. an output grid of ceil(ceil(H/2)/2) x
 * ceil(ceil(W/2)/2).  Runs on the tensor cores in BF16 with FP32 accumulation; head, loss
 * (mean binary cross-entropy) and Adam in FP32.
 * Parameters: ART_CNN_PARAMS floats, in this order: W1 [32][3][3][3], b1 [32], W2 [32][3][3][32],
 * b2, W3, b3, W4, b4 (conv weights indexed [out][ky][kx][in]), w_head [32], b_head [1].
 * Feature maps are H x W x 3 FP32 device arrays (row-major, features fastest); probabilities and
 * targets are Ho x Wo FP32 device arrays.  Every call is stream-ordered on the context's stream
 * and synchronises it.  Errors: ART_ERR_ARG (no network loaded, H or W < 1 or H W > 2^26),
 * ART_ERR_OOM, ART_ERR_CUDA, ART_ERR_DEVICE (a tensor-core wait timed out). */
#define ART_CNN_PARAMS 28673
/* Load (host FP32 parameters) and reset the optimizer state. */
int art_cnn_load(art_ctx* ctx, const float* params_host);
/* Copy the current parameters to the host. */
int art_cnn_read(art_ctx* ctx, float* params_host);
/* Forward pass: probabilities of the blocks of one lattice. */
int art_cnn_forward(art_ctx* ctx, const float* feat_dev, int32_t H, int32_t W, float* prob_dev);
/* Loss and gradients (no update): *loss_host = mean cross-entropy against target_dev (0/1),
 * grad_host (nullable) receives ART_CNN_PARAMS gradient entries. */
int art_cnn_grad(art_ctx* ctx, const float* feat_dev, int32_t H, int32_t W,
                 const float* target_dev, float* loss_host, float* grad_host);
/* One Adam step (learning rate lr, beta1 0.9, beta2 0.999, eps 1e-8) on one lattice. */
int art_cnn_train_step(art_ctx* ctx, const float* feat_dev, int32_t H, int32_t W,
                       const float* target_dev, float lr, float* loss_host);

/* Training sample from the context's last render of `job` (which recorded per-pixel ray
 * diagnostics because a network was loaded): feat_dev (H x W x 3 FP32) = the features of the
 * level-`level` lattice of img_dev, target_dev (Ho x Wo FP32) = 1 where that render's mask traced
 * a point of level level + 2 or level + 3 inside the block, else 0.  level + 2 <= levels.  ART_ERR_ARG if the
 * last render did not record diagnostics for this grid. */
int art_cnn_sample(art_ctx* ctx, const art_job* job, const double* img_dev,
                   const uint8_t* mask_dev, int32_t level, float* feat_dev, float* target_dev);

/* Image metrics of plane 0 (Eqs. interpdef, fluxdef, msedef): out_host[0] = interpolation
 * fraction (mask_dev nullable -> 0), [1] = flux error with the trapezoid flux, [2] = MSE
 * sum|I - I_hat|^2 / sum|I|^2, [3] = sum|I - I_hat|^2 / (N mean(I)^2).  Synchronises. */
int art_metrics(art_ctx* ctx, const double* truth_dev, const double* img_dev,
                const uint8_t* mask_dev, int32_t nx, int32_t ny, double* out_host);

#ifdef __cplusplus
}
#endif
#endif
