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
#include <type_traits>

#include "trace_impl.cuh"

namespace art {

// Outputs of a finished ray of the single-image kernels: the re-trace list (FP32 pass of the mixed
// modes), else its planes, mask, diagnostics and counters.
template <class Q>
__device__ __forceinline__ void finish_ray(const TraceArgs& A, int status, int steps,
                                           const XferState<Q>& x, int32_t pix, int64_t slot)
{
    atomicAdd(A.counters + C_STEPS, (unsigned long long)steps);
    atomicMax(A.counters + C_MAXSTEP, (unsigned long long)steps);
    atomicAdd(A.counters + C_RAYCNT, 1ull);
    const bool rer = A.reroute != nullptr && (status == RAY_REROUTE || status == ART_RAY_NAN ||
                                              status == ART_RAY_CAP || x.edge);
    if (rer) {
        unsigned long long w = atomicAdd(A.reroute_count, 1ull);
        A.reroute[w] = (int32_t)slot;
        return;
    }
    if (status == ART_RAY_CAP) atomicAdd(A.counters + C_CAPPED, 1ull);
    if (status == ART_RAY_NAN) atomicAdd(A.counters + C_NAN, 1ull);
    if (A.indirect) atomicAdd(A.counters + C_FP64, 1ull);  // re-trace pass
    const int np = A.job.planes;
#pragma unroll
    for (int p = 0; p < MAXPL; ++p) {
        if (p < np) {
            if (A.img) A.img[(int64_t)p * A.npix + pix] = double(x.acc[p]);
            if (A.out) A.out[slot * np + p] = double(x.acc[p]);
        }
    }
    if (A.img && A.mask)
        A.mask[pix] = (A.spec_from && (unsigned long long)slot >= *A.spec_from)
                          ? MASK_SPEC_DONE
                          : (uint8_t)ART_MASK_TRACED;
    if (A.img && A.pix_steps) A.pix_steps[pix] = (uint16_t)(steps < 65535 ? steps : 65535);
    if (A.img && A.pix_minr) {
        A.pix_minr[pix] = x.min_r;
        A.pix_turn[pix] = (float)x.nturn;
    }
    if (A.aux_status) A.aux_status[slot] = status;
    if (A.aux_steps) A.aux_steps[slot] = steps;
    if (A.aux_nturn) A.aux_nturn[slot] = x.nturn;
    if (A.aux_minr) A.aux_minr[slot] = x.min_r;
}

// Queue position of the q-th ray a launch fetches.
__device__ __forceinline__ int64_t fetch_slot(const TraceArgs& A, unsigned long long q)
{
    return A.indirect ? (int64_t)A.indirect[q] : (int64_t)q;
}

// One-thread form: each lane traces its ray's whole step and refills itself from the queue.
template <class R, bool SWEEP, bool POL, int EM>
__device__ __forceinline__ void trace_lanes(const TraceArgs& A, const Camera& cam_s)
{
    const DevJob& J = A.job;
    const auto& S = synch_of<typename Aux<R>::Q>(A.synch, A.synchf);
    const unsigned long long n = *A.count;
    Tracer<R> t;
    bool active = false;
    auto fetch_next = [&]() {
        while (true) {
            unsigned long long q = warp_fetch(A.fetch);
            if (q >= n) return false;
            int64_t slot = fetch_slot(A, q);
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
                finish_ray(A, t.status, t.g.steps, t.x, t.pix, t.slot);
                active = fetch_next();
            }
        }
    }
}

// --------------------------------------------------------------------------------------------
// Warp-pair form.  The trace kernels are latency-bound on most levels: a level's few thousand to
// few tens of thousands of rays leave most schedulers with one warp or none, so a step costs its
// whole dependent instruction chain.  Here each pair of warps shares 32 rays: the even warp
// integrates their geodesics (geo_step), the odd warp their transfer (xfer_step) one step behind,
// so the two halves of a step overlap.  The geodesic warp hands each step's end point over through
// a two-slot ring in shared memory guarded by mbarriers (full: written by the geodesic warp;
// empty: released by the transfer warp).  Records per lane: a new ray (its start point, pixel and
// queue slot), a step (its end point and the ray's status after it) or idle; the geodesic warp
// marks the record after which none follows.  Every wait is bounded in time: when a wait runs out
// on any lane, the warp counts C_SYNCERR and leaves its loop, and the other warp of the pair then
// runs out of time on its next wait and leaves too.  The arithmetic is that of the one-thread form
// (the same geo_step and xfer_step, compiled without automatic contraction), so both forms give
// bit-identical rays.
// --------------------------------------------------------------------------------------------

constexpr int REC_IDLE = -3, REC_INIT = -2;
constexpr int SPLIT_SLOTS = 2;
constexpr long long SPLIT_WAIT_CYCLES = 1ll << 32;  // about 2 s at the SM clock

__device__ __forceinline__ void pair_bar_init(uint64_t* bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(count));
}

__device__ __forceinline__ void pair_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}

// Wait for the phase of parity `parity` to complete; false once SPLIT_WAIT_CYCLES have passed.
__device__ __forceinline__ bool pair_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > SPLIT_WAIT_CYCLES) return false;
    }
}

// Fields of an end-point record: x y z kx ky kz kt r h f0..f3, then either the point's Kerr-Schild
// pieces (StepPoint::ks: CarryRhs kernels) or, when the transfer half transports the covector, the
// NSTG stage values.
constexpr int REC_EXTRA = 13, REC_KS = 5;

// Shared memory of the warp-pair form: the hand-over rings and their mbarriers.
template <class Q, int NF>
struct PairRing {
    static constexpr int NPAIR = TRACE_BLOCK / 64;
    static constexpr int STG = REC_EXTRA;  // first stage field (read only with NF > REC_EXTRA + REC_KS)
    Q v[NPAIR][SPLIT_SLOTS][NF][32];
    int32_t code[NPAIR][SPLIT_SLOTS][32], pix[NPAIR][SPLIT_SLOTS][32], img[NPAIR][SPLIT_SLOTS][32];
    int64_t slot[NPAIR][SPLIT_SLOTS][32];
    int32_t last[NPAIR][SPLIT_SLOTS];
    uint64_t full[NPAIR][SPLIT_SLOTS], empty[NPAIR][SPLIT_SLOTS];
};

template <class Ring>
__device__ __forceinline__ void pair_ring_init(Ring& sm)
{
    if (threadIdx.x == 0)
        for (int p = 0; p < Ring::NPAIR; ++p)
            for (int k = 0; k < SPLIT_SLOTS; ++k) {
                pair_bar_init(&sm.full[p][k], 32);
                pair_bar_init(&sm.empty[p][k], 32);
            }
}

// Outputs of a finished ray of the batched kernels: as finish_ray, into the ray's own image.
template <class Q>
__device__ __forceinline__ void finish_batch_ray(const BatchTraceArgs& A, int status, int steps,
                                                 const XferState<Q>& x, int32_t pix, int64_t slot,
                                                 int32_t img)
{
    atomicAdd(A.counters + C_STEPS, (unsigned long long)steps);
    atomicMax(A.counters + C_MAXSTEP, (unsigned long long)steps);
    atomicAdd(A.counters + C_RAYCNT, 1ull);
    const bool rer = A.reroute != nullptr && (status == RAY_REROUTE || status == ART_RAY_NAN ||
                                              status == ART_RAY_CAP || x.edge);
    if (rer) {
        unsigned long long w = atomicAdd(A.reroute_count, 1ull);
        A.reroute[w] = (int32_t)slot;
        return;
    }
    if (status == ART_RAY_CAP) atomicAdd(A.counters + C_CAPPED, 1ull);
    if (status == ART_RAY_NAN) atomicAdd(A.counters + C_NAN, 1ull);
    if (A.indirect) atomicAdd(A.counters + C_FP64, 1ull);
    const DevJob& J = A.jobs[img];
    const int64_t npix = (int64_t)J.nx * J.ny;
    double* out = A.imgs[img];
#pragma unroll
    for (int p = 0; p < MAXPL; ++p)
        if (p < A.planes) out[(int64_t)p * npix + pix] = double(x.acc[p]);
    uint8_t* mask = A.masks[img];
    if (mask)
        mask[pix] = (A.spec_from && (unsigned long long)slot >= *A.spec_from)
                        ? MASK_SPEC_DONE
                        : (uint8_t)ART_MASK_TRACED;
}

// Where the rays of a launch come from and where their results go, for the forms that hand a
// ray's step between warps: one image (job, constants and camera shared by every ray) or a batch
// (each queue entry names its image).  next() takes the next valid queue entry (warp-aggregated;
// false once the queue is drained), finish() writes a finished ray.
struct SingleSource {
    const TraceArgs& A;
    const Camera& cam;
    unsigned long long n;
    __device__ const DevJob& job(int32_t) const { return A.job; }
    template <class Q>
    __device__ const SynchConstT<Q>& synch(int32_t) const
    {
        return synch_of<Q>(A.synch, A.synchf);
    }
    __device__ const Camera& camera(int32_t) const { return cam; }
    __device__ unsigned long long* counters() const { return A.counters; }
    __device__ bool next(int64_t& slot, int32_t& pix, int32_t& img) const
    {
        while (true) {
            const unsigned long long q = warp_fetch(A.fetch);
            if (q >= n) return false;
            const int64_t sq = fetch_slot(A, q);
            const int32_t px = A.queue[sq];
            if (px < 0 || (int64_t)px >= A.npix) {
                atomicAdd(A.counters + C_BADIDX, 1ull);
                continue;
            }
            slot = sq;
            pix = px;
            img = 0;
            return true;
        }
    }
    template <class Q>
    __device__ void finish(int status, int steps, const XferState<Q>& x, int32_t pix, int64_t slot,
                           int32_t) const
    {
        finish_ray(A, status, steps, x, pix, slot);
    }
};

struct BatchSource {
    const BatchTraceArgs& A;
    unsigned long long n;
    __device__ const DevJob& job(int32_t img) const { return A.jobs[img]; }
    template <class Q>
    __device__ const SynchConstT<Q>& synch(int32_t img) const
    {
        return synch_of<Q>(A.synchs[img], A.synchfs[img]);
    }
    __device__ const Camera& camera(int32_t img) const { return A.cams[img]; }
    __device__ unsigned long long* counters() const { return A.counters; }
    __device__ bool next(int64_t& slot, int32_t& pix, int32_t& img) const
    {
        while (true) {
            const unsigned long long q = warp_fetch(A.fetch);
            if (q >= n) return false;
            const int64_t sq = A.indirect ? (int64_t)A.indirect[q] : (int64_t)q;
            const int64_t e = A.queue[sq];
            const int32_t im = (int32_t)(e >> 32), px = (int32_t)(e & 0xffffffff);
            const DevJob& J = A.jobs[im];
            if (px < 0 || (int64_t)px >= (int64_t)J.nx * J.ny) {
                atomicAdd(A.counters + C_BADIDX, 1ull);
                continue;
            }
            slot = sq;
            pix = px;
            img = im;
            return true;
        }
    }
    template <class Q>
    __device__ void finish(int status, int steps, const XferState<Q>& x, int32_t pix, int64_t slot,
                           int32_t img) const
    {
        finish_batch_ray(A, status, steps, x, pix, slot, img);
    }
};

// Warp-pair form (the ring's mbarriers initialised and the block synchronised before the call).
template <class R, bool POL, int EM>
using PairRingOf =
    PairRing<typename Aux<R>::Q, !XportOnGeo<R, POL>::value ? REC_EXTRA + NSTG
                                 : CarryRhs<R, POL, EM>::value ? REC_EXTRA + REC_KS
                                                               : REC_EXTRA>;

template <class R, bool SWEEP, bool POL, int EM, class Src>
__device__ __forceinline__ void trace_pairs(const Src& src, PairRingOf<R, POL, EM>& sm)
{
    using Q = typename Aux<R>::Q;
    constexpr bool KS = CarryRhs<R, POL, EM>::value;
    constexpr int NSL = SPLIT_SLOTS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, pr = warp >> 1;
    if ((warp & 1) == 0) {
        // geodesic warp
        GeoState<R> g;
        bool has = false, drained = false;
        int32_t pix = 0, img = 0;
        int64_t slot = 0;
        for (int it = 0;; ++it) {
            const int sl = it % NSL;
            const uint32_t ph = (uint32_t)(it / NSL) & 1u;
            if (it >= NSL &&
                !__all_sync(0xffffffffu, pair_wait(&sm.empty[pr][sl], ph ^ 1u))) {
                if (lane == 0) atomicAdd(src.counters() + C_SYNCERR, 1ull);
                return;
            }
            StepPoint<Q> pt;
            int code = REC_IDLE;
            if (has) {
                code = geo_step<R, SWEEP, POL, EM>(g, src.job(img), pt,
                                                   &sm.v[pr][sl][PairRingOf<R, POL, EM>::STG][lane], 32);
                if (code != RAY_GOING) has = false;
            } else if (!drained) {
                int64_t sq;
                int32_t px, im;
                if (src.next(sq, px, im)) {
                    geo_init<R, POL, EM>(g, src.job(im), src.camera(im), px, pt);
                    pix = px;
                    img = im;
                    slot = sq;
                    has = true;
                    code = REC_INIT;
                } else {
                    drained = true;
                }
            }
            if (code != REC_IDLE) {
                Q* v = &sm.v[pr][sl][0][lane];
                v[0 * 32] = pt.q.x;
                v[1 * 32] = pt.q.y;
                v[2 * 32] = pt.q.z;
                v[3 * 32] = pt.q.kx;
                v[4 * 32] = pt.q.ky;
                v[5 * 32] = pt.q.kz;
                v[6 * 32] = pt.kt;
                v[7 * 32] = pt.r;
                v[8 * 32] = pt.h;
                if (POL)
                    for (int m = 0; m < 4; ++m) v[(9 + m) * 32] = pt.f[m];
                if constexpr (KS)
                    for (int m = 0; m < REC_KS; ++m) v[(REC_EXTRA + m) * 32] = pt.ks[m];
            }
            sm.code[pr][sl][lane] = code;
            sm.pix[pr][sl][lane] = pix;
            sm.img[pr][sl][lane] = img;
            sm.slot[pr][sl][lane] = slot;
            const bool last = __all_sync(0xffffffffu, code == REC_IDLE && drained);
            if (lane == 0) sm.last[pr][sl] = last ? 1 : 0;
            __syncwarp();
            pair_arrive(&sm.full[pr][sl]);
            if (last) return;
        }
    } else {
        // transfer warp
        XferState<Q> x;
        int32_t pix = 0, img = 0;
        int64_t slot = 0;
        int steps = 0;
        for (int it = 0;; ++it) {
            const int sl = it % NSL;
            const uint32_t ph = (uint32_t)(it / NSL) & 1u;
            if (!__all_sync(0xffffffffu, pair_wait(&sm.full[pr][sl], ph))) {
                if (lane == 0) atomicAdd(src.counters() + C_SYNCERR, 1ull);
                return;
            }
            const int code = sm.code[pr][sl][lane];
            const bool last = sm.last[pr][sl] != 0;
            StepPoint<Q> pt;
            if (code != REC_IDLE) {
                const Q* v = &sm.v[pr][sl][0][lane];
                pt.q.x = v[0 * 32];
                pt.q.y = v[1 * 32];
                pt.q.z = v[2 * 32];
                pt.q.kx = v[3 * 32];
                pt.q.ky = v[4 * 32];
                pt.q.kz = v[5 * 32];
                pt.kt = v[6 * 32];
                pt.r = v[7 * 32];
                pt.h = v[8 * 32];
                if (POL)
                    for (int m = 0; m < 4; ++m) pt.f[m] = v[(9 + m) * 32];
                if constexpr (KS)
                    for (int m = 0; m < REC_KS; ++m) pt.ks[m] = v[(REC_EXTRA + m) * 32];
            }
            if (code == REC_INIT) {
                pix = sm.pix[pr][sl][lane];
                img = sm.img[pr][sl][lane];
                slot = sm.slot[pr][sl][lane];
            }
            const DevJob& J = src.job(img);
            const bool moving = code != REC_IDLE && code != REC_INIT && code != ART_RAY_NAN &&
                                code != RAY_REROUTE;
            if (!XportOnGeo<R, POL>::value && moving)
                xfer_transport<Q>(x, pt, &sm.v[pr][sl][PairRingOf<R, POL, EM>::STG][lane], 32, J);
            __syncwarp();
            pair_arrive(&sm.empty[pr][sl]);
            if (code == REC_INIT) {
                xfer_init<Q, POL, EM, KS>(x, pt, J, src.template synch<Q>(img));
                steps = 0;
            } else if (code != REC_IDLE) {
                ++steps;
                if (moving) xfer_step<Q, POL, EM, KS>(x, pt, J, src.template synch<Q>(img));
                if (code != RAY_GOING) src.finish(code, steps, x, pix, slot, img);
            }
            if (last) return;
        }
    }
}

// --------------------------------------------------------------------------------------------
// Warp-quad form (FP32 and FP64 kernels).  In the warp-pair form the transfer warp is the slower
// half: the emission coefficients at a point are a long dependent chain, but a pure function of the point,
// so consecutive steps' coefficients can be computed at the same time.  Here a block's four warps
// share 32 rays: warp 0 integrates the geodesics (and transports the covector), warps 1 and 2
// compute the coefficients at the end points of the even and the odd steps, and warp 3 applies
// the segments in order and finishes the rays.  Ring A (four slots) carries the geodesic warp's
// records to the coefficient warp of that step's parity and to the segment warp (its slot is free
// once both have read it); ring C (four slots) carries the coefficients to the segment warp.  The
// geodesic warp ends with two records marked last, one for each coefficient warp; the segment
// warp leaves after the second.  Waits are bounded as in the pair form.  The arithmetic is that of
// the other forms (the same geo_step, coefficients and xfer_apply), so the rays are identical.
// --------------------------------------------------------------------------------------------

constexpr int QUAD_SLOTS = 4;
// FP32 kernels: queues of up to A.quad_rays rays per block take the quad form (one group of 32
// rays per block at once; longer queues are drained by the same warps in turn), up to
// A.pair_rays the pair form, longer ones the one-thread form (defaults 32 and 64, set per context
// by art_set_tune or art_autotune).  FP64 kernels: up to A.quad64_rays rays per block the quad
// form, longer queues the pair form (default 32).

template <class Q>
struct QuadRing {
    Q a[QUAD_SLOTS][REC_EXTRA + REC_KS][32];  // end point records (fields as in the pair form)
    int32_t code[QUAD_SLOTS][32], pix[QUAD_SLOTS][32];
    int64_t slot[QUAD_SLOTS][32];
    int32_t last[QUAD_SLOTS];
    Q c[QUAD_SLOTS][12][32];  // J1 (4), K1 (7) and the discontinuity flag at the record's point
    uint64_t a_full[QUAD_SLOTS], a_empty[QUAD_SLOTS], c_full[QUAD_SLOTS], c_empty[QUAD_SLOTS];
};

template <class Q>
__device__ __forceinline__ void quad_ring_init(QuadRing<Q>& sm)
{
    if (threadIdx.x == 0)
        for (int k = 0; k < QUAD_SLOTS; ++k) {
            pair_bar_init(&sm.a_full[k], 32);
            pair_bar_init(&sm.a_empty[k], 64);  // the coefficient warp of the step and the segment warp
            pair_bar_init(&sm.c_full[k], 32);
            pair_bar_init(&sm.c_empty[k], 32);
        }
}

template <class Q, bool POL, bool KS>
__device__ __forceinline__ void quad_read_point(const QuadRing<Q>& sm, int sl, int lane,
                                                StepPoint<Q>& pt)
{
    pt.q.x = sm.a[sl][0][lane];
    pt.q.y = sm.a[sl][1][lane];
    pt.q.z = sm.a[sl][2][lane];
    pt.q.kx = sm.a[sl][3][lane];
    pt.q.ky = sm.a[sl][4][lane];
    pt.q.kz = sm.a[sl][5][lane];
    pt.kt = sm.a[sl][6][lane];
    pt.r = sm.a[sl][7][lane];
    pt.h = sm.a[sl][8][lane];
    if (POL)
        for (int m = 0; m < 4; ++m) pt.f[m] = sm.a[sl][9 + m][lane];
    if (KS)
        for (int m = 0; m < REC_KS; ++m) pt.ks[m] = sm.a[sl][REC_EXTRA + m][lane];
}

// Warp-quad form (ring mbarriers initialised and the block synchronised before the call).
template <class R, bool SWEEP, bool POL, int EM>
__device__ __forceinline__ void trace_quads(const TraceArgs& A, const Camera& cam_s,
                                            QuadRing<R>& sm)
{
    static_assert(std::is_same<R, float>::value || std::is_same<R, double>::value,
                  "the quad form carries FP32 or FP64 rays");
    using Q = R;
    constexpr int NSL = QUAD_SLOTS;
    constexpr bool KS = CarryRhs<R, POL, EM>::value;
    const DevJob& J = A.job;
    const SynchConstT<Q>& S = synch_of<Q>(A.synch, A.synchf);
    const unsigned long long n = *A.count;
    const int lane = threadIdx.x & 31, role = threadIdx.x >> 5;
    if (role == 0) {
        // geodesic warp
        GeoState<R> g;
        bool has = false, drained = false;
        int32_t pix = 0;
        int64_t slot = 0;
        int nlast = 0;
        for (int it = 0;; ++it) {
            const int sl = it % NSL;
            const uint32_t ph = (uint32_t)(it / NSL) & 1u;
            if (it >= NSL && !__all_sync(0xffffffffu, pair_wait(&sm.a_empty[sl], ph ^ 1u))) {
                if (lane == 0) atomicAdd(A.counters + C_SYNCERR, 1ull);
                return;
            }
            StepPoint<Q> pt;
            int code = REC_IDLE;
            if (has) {
                code = geo_step<R, SWEEP, POL, EM>(g, J, pt, nullptr, 0);
                if (code != RAY_GOING) has = false;
            } else if (!drained) {
                while (true) {
                    const unsigned long long q = warp_fetch(A.fetch);
                    if (q >= n) {
                        drained = true;
                        break;
                    }
                    const int64_t sq = fetch_slot(A, q);
                    const int32_t px = A.queue[sq];
                    if (px < 0 || (int64_t)px >= A.npix) {
                        atomicAdd(A.counters + C_BADIDX, 1ull);
                        continue;
                    }
                    geo_init<R, POL, EM>(g, J, cam_s, px, pt);
                    pix = px;
                    slot = sq;
                    has = true;
                    code = REC_INIT;
                    break;
                }
            }
            if (code != REC_IDLE) {
                sm.a[sl][0][lane] = pt.q.x;
                sm.a[sl][1][lane] = pt.q.y;
                sm.a[sl][2][lane] = pt.q.z;
                sm.a[sl][3][lane] = pt.q.kx;
                sm.a[sl][4][lane] = pt.q.ky;
                sm.a[sl][5][lane] = pt.q.kz;
                sm.a[sl][6][lane] = pt.kt;
                sm.a[sl][7][lane] = pt.r;
                sm.a[sl][8][lane] = pt.h;
                if (POL)
                    for (int m = 0; m < 4; ++m) sm.a[sl][9 + m][lane] = pt.f[m];
                if (KS)
                    for (int m = 0; m < REC_KS; ++m) sm.a[sl][REC_EXTRA + m][lane] = pt.ks[m];
            }
            sm.code[sl][lane] = code;
            sm.pix[sl][lane] = pix;
            sm.slot[sl][lane] = slot;
            const bool last = __all_sync(0xffffffffu, code == REC_IDLE && drained);
            if (lane == 0) sm.last[sl] = last ? 1 : 0;
            __syncwarp();
            pair_arrive(&sm.a_full[sl]);
            if (last && ++nlast == 2) return;  // one last record for each coefficient warp
        }
    } else if (role < 3) {
        // coefficient warp of the even (role 1) or odd (role 2) steps
        for (int it = role - 1;; it += 2) {
            const int sl = it % NSL;
            const uint32_t ph = (uint32_t)(it / NSL) & 1u;
            if (!__all_sync(0xffffffffu, pair_wait(&sm.a_full[sl], ph))) {
                if (lane == 0) atomicAdd(A.counters + C_SYNCERR, 1ull);
                return;
            }
            const int code = sm.code[sl][lane];
            const bool last = sm.last[sl] != 0;
            StepPoint<Q> pt;
            const bool need = code == REC_INIT ||
                              (code != REC_IDLE && code != ART_RAY_NAN && code != RAY_REROUTE);
            if (need) quad_read_point<Q, POL, KS>(sm, sl, lane, pt);
            __syncwarp();
            pair_arrive(&sm.a_empty[sl]);
            Q J1[4], K1[7];
            int e1 = 0;
            if (need) coefficients<Q, POL, EM, KS>(pt, J, S, J1, K1, e1);
            if (it >= NSL && !__all_sync(0xffffffffu, pair_wait(&sm.c_empty[sl], ph ^ 1u))) {
                if (lane == 0) atomicAdd(A.counters + C_SYNCERR, 1ull);
                return;
            }
            if (need) {
                for (int i = 0; i < 4; ++i) sm.c[sl][i][lane] = J1[i];
                for (int i = 0; i < 7; ++i) sm.c[sl][4 + i][lane] = K1[i];
                sm.c[sl][11][lane] = Q(e1);
            }
            __syncwarp();
            pair_arrive(&sm.c_full[sl]);
            if (last) return;
        }
    } else {
        // segment warp
        XferState<Q> x;
        int32_t pix = 0;
        int64_t slot = 0;
        int steps = 0;
        bool prev_last = false;
        for (int it = 0;; ++it) {
            const int sl = it % NSL;
            const uint32_t ph = (uint32_t)(it / NSL) & 1u;
            if (!__all_sync(0xffffffffu, pair_wait(&sm.a_full[sl], ph))) {
                if (lane == 0) atomicAdd(A.counters + C_SYNCERR, 1ull);
                return;
            }
            const int code = sm.code[sl][lane];
            const bool last = sm.last[sl] != 0;
            const bool moving = code != REC_IDLE && code != REC_INIT && code != ART_RAY_NAN &&
                                code != RAY_REROUTE;
            StepPoint<Q> pt;
            if (code == REC_INIT || moving) quad_read_point<Q, POL, false>(sm, sl, lane, pt);
            if (code == REC_INIT) {
                pix = sm.pix[sl][lane];
                slot = sm.slot[sl][lane];
            }
            __syncwarp();
            pair_arrive(&sm.a_empty[sl]);
            if (!__all_sync(0xffffffffu, pair_wait(&sm.c_full[sl], ph))) {
                if (lane == 0) atomicAdd(A.counters + C_SYNCERR, 1ull);
                return;
            }
            Q J1[4], K1[7];
            int e1 = 0;
            if (code == REC_INIT || moving) {
                for (int i = 0; i < 4; ++i) J1[i] = sm.c[sl][i][lane];
                for (int i = 0; i < 7; ++i) K1[i] = sm.c[sl][4 + i][lane];
                e1 = sm.c[sl][11][lane] != Q(0);
            }
            __syncwarp();
            pair_arrive(&sm.c_empty[sl]);
            if (code == REC_INIT) {
                xfer_init_with<Q, POL>(x, pt, J1, K1, e1);
                steps = 0;
            } else if (code != REC_IDLE) {
                ++steps;
                if (moving) xfer_apply<Q, POL>(x, pt, J1, K1, J, e1);
                if (code != RAY_GOING) finish_ray(A, code, steps, x, pix, slot);
            }
            if (last) {
                if (prev_last) return;
                prev_last = true;
            }
        }
    }
}

// The single-image trace kernel.  The form follows the queue length (uniform over the grid): short
// queues (the latency-bound regime of most levels) take the warp-quad (FP32) or warp-pair form, a
// longer queue, where throughput counts, the one-thread form with the most rays in flight.  The
// double-float and FP64 kernels take the pair form whenever their queue fits the grid's pairs
// (GB300's FP64 pipe issues a warp instruction every 16 cycles, so an FP64 step is long even for
// one warp per scheduler, and splitting it over two warps halves a launch's tail).
template <class R, bool SWEEP, bool POL, int EM>
__global__ void __launch_bounds__(TRACE_BLOCK) trace_kernel(TraceArgs A)
{
    using Q = typename Aux<R>::Q;
    __shared__ Camera cam_s;
    {
        const double* src = reinterpret_cast<const double*>(A.cam);
        double* dst = reinterpret_cast<double*>(&cam_s);
        for (int q = threadIdx.x; q < (int)(sizeof(Camera) / sizeof(double)); q += blockDim.x)
            dst[q] = src[q];
    }
    {
        // The rings of the two split forms share one buffer: the queue length, and so the form,
        // is uniform over the grid, and only the chosen form's mbarriers are initialised.
        using PRing = PairRingOf<R, POL, EM>;
        using QRing = QuadRing<Q>;
        constexpr bool HAS_QUAD = !std::is_same<R, df>::value;
        constexpr size_t RING_BYTES =
            HAS_QUAD && sizeof(QRing) > sizeof(PRing) ? sizeof(QRing) : sizeof(PRing);
        __shared__ __align__(16) unsigned char rings[RING_BYTES];
        const unsigned long long n = *A.count, blocks = gridDim.x;
        const unsigned long long pair_lanes = blocks * PRing::NPAIR * 32ull;
        // 2: quad form, 1: pair form, 0: one thread per ray.  FP32: by the tuned thresholds.
        // FP64: the pair form at least.  GB300's FP64 pipe takes a warp instruction per 64 cycles
        // on one scheduler whatever its ILP and active lanes (about 16 cycles per SM across the
        // four), so a ray's latency is its slowest warp's FP64 instruction count: the pair halves
        // it, the quad (emission coefficients of alternate steps on two warps) cuts the transfer
        // half again, which shortens the launches whose longest rays finish last; the SM-wide
        // rate (the throughput bound) is the same in every form.  Double-float: the pair form
        // while the queue fits the grid's pairs.
        int form;
        if constexpr (std::is_same<R, float>::value)
            form = n <= blocks * (unsigned long long)A.quad_rays   ? 2
                   : n <= blocks * (unsigned long long)A.pair_rays ? 1
                                                                   : 0;
        else if constexpr (std::is_same<R, double>::value)
            form = n <= blocks * (unsigned long long)A.quad64_rays ? 2 : 1;
        else
            form = n <= pair_lanes ? 1 : 0;
        if constexpr (HAS_QUAD)
            if (form == 2) quad_ring_init(*reinterpret_cast<QRing*>(rings));
        if (form == 1) pair_ring_init(*reinterpret_cast<PRing*>(rings));
        __syncthreads();
        if constexpr (HAS_QUAD)
            if (form == 2) {
                trace_quads<R, SWEEP, POL, EM>(A, cam_s, *reinterpret_cast<QRing*>(rings));
                return;
            }
        if (form == 1)
            trace_pairs<R, SWEEP, POL, EM>(SingleSource{A, cam_s, n},
                                           *reinterpret_cast<PRing*>(rings));
        else
            trace_lanes<R, SWEEP, POL, EM>(A, cam_s);
    }
}

template <class R, bool SWEEP, bool POL, int EM>
__global__ void __launch_bounds__(TRACE_BLOCK) trace_batch_kernel(BatchTraceArgs A)
{
    const unsigned long long n = *A.count;
    if constexpr (std::is_same<R, df>::value) {
        // the double-float re-trace holds few rays (the near-critical ones of the whole batch):
        // the warp-pair form whenever the queue fits the grid's pairs, as for a single image
        __shared__ __align__(16) PairRingOf<R, POL, EM> ring;
        pair_ring_init(ring);
        __syncthreads();
        if (n <= (unsigned long long)gridDim.x * PairRingOf<R, POL, EM>::NPAIR * 32ull) {
            trace_pairs<R, SWEEP, POL, EM>(BatchSource{A, n}, ring);
            return;
        }
    }
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
            ray_init<R, POL, EM>(t, J, synch_of<typename Aux<R>::Q>(A.synchs[img], A.synchfs[img]),
                                 A.cams[img], pix);
            t.img = img;
            t.slot = slot;
            return true;
        }
    };
    active = fetch_next();
    while (__any_sync(0xffffffffu, active)) {
        if (active) {
            const DevJob& J = A.jobs[t.img];
            if (ray_step<R, SWEEP, POL, EM>(
                    t, J, synch_of<typename Aux<R>::Q>(A.synchs[t.img], A.synchfs[t.img]))) {
                finish_batch_ray(A, t.status, t.g.steps, t.x, t.pix, t.slot, t.img);
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
