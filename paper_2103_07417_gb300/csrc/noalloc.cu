// noalloc.cu -- art_trace_pixels_noalloc: the pixel tracer for callers that cannot allocate.
//
// art_trace_pixels keeps its scratch (work counters, the camera, the FP64 re-trace queue) in
// device memory that the context allocates on first use.  Some callers cannot let a library call
// cudaMalloc: a process whose device memory is fully reserved up front by its own allocator (a
// render service that pins a fixed budget per GPU), code that runs while another framework owns
// allocation, or a caller that must not trigger the implicit synchronisation cudaMalloc/cudaFree
// can cause.  This entry point allocates nothing: its scratch is the file-scope device array
// below, of a fixed size that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.cuh"

using namespace art;

namespace {

constexpr int64_t NOALLOC_MAX_RAYS = ART_NOALLOC_MAX_RAYS;
constexpr size_t OFF_CAM = 0;
constexpr size_t OFF_CNT = 256;                                    // after the camera (152 B)
constexpr size_t OFF_REROUTE = OFF_CNT + 8 * C_COUNT + 256;        // 256-byte aligned
constexpr size_t SCRATCH_BYTES = OFF_REROUTE + 4 * NOALLOC_MAX_RAYS;
static_assert(sizeof(Camera) <= OFF_CNT, "camera does not fit its slot");
static_assert(OFF_REROUTE % 256 == 0, "re-trace queue must stay 256-byte aligned");

}  // namespace

// The whole scratch of art_trace_pixels_noalloc: camera | counters | FP64 re-trace queue.
static __device__ __align__(256) unsigned char art_noalloc_scratch[SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
struct DeviceSlot {
    std::once_flag once;
    int rc = ART_ERR_CUDA;
    unsigned char* ptr = nullptr;  // device address of art_noalloc_scratch on that device
    int num_sms = 0;
    int occ[3][2] = {};  // resident blocks per SM [kind][polarized]
};
DeviceSlot g_slots[MAX_DEVICES];

// Once per device, with that device current: resolve the array's device address (its name in
// host code is only a host-side stand-in) and the launch geometry.
void setup_device(int dev)
{
    DeviceSlot& s = g_slots[dev];
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, art_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        s.rc = ART_ERR_CUDA;
        return;
    }
    if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        s.rc = ART_ERR_CUDA;
        return;
    }
    for (int kd = 0; kd < 3; ++kd)
        for (int pl = 0; pl < 2; ++pl) {
            if (trace_occupancy(TraceKind(kd), pl != 0, &s.occ[kd][pl]) != cudaSuccess) {
                cudaGetLastError();
                s.rc = ART_ERR_CUDA;
                return;
            }
            if (s.occ[kd][pl] < 1) s.occ[kd][pl] = 1;
        }
    s.ptr = static_cast<unsigned char*>(p);
    s.rc = ART_OK;
}

}  // namespace

// Job validation and synchrotron constants shared with the context path live in capi.cu.
int art_make_devjob(const art_job* job, DevJob* J);
void art_make_synch(const art_job* job, SynchConst* S);

extern "C" int art_trace_pixels_noalloc(const art_job* job, const int32_t* pix_dev, int64_t n,
                                        double* out_dev, const art_rayaux* aux, void* stream)
{
    if (n < 0 || (n > 0 && (!pix_dev || !out_dev))) return ART_ERR_ARG;
    if (n > NOALLOC_MAX_RAYS) return ART_ERR_ARG;  // beyond the static scratch
    DevJob J;
    int rc = art_make_devjob(job, &J);
    if (rc) return rc;
    if (J.emission == ART_EMIT_GRID) return ART_ERR_UNSUPPORTED;  // the grid lives in a context
    if (n == 0) return ART_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return ART_ERR_CUDA;
    std::call_once(g_slots[dev].once, setup_device, dev);
    const DeviceSlot& s = g_slots[dev];
    if (s.rc != ART_OK) return s.rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st) {
        // the scratch array's address is this device's: a stream of another device is an error
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return ART_ERR_ARG;
        }
        if (sdev != dev) return ART_ERR_ARG;
    }

    Camera* cam = reinterpret_cast<Camera*>(s.ptr + OFF_CAM);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(s.ptr + OFF_CNT);
    int32_t* reroute = reinterpret_cast<int32_t*>(s.ptr + OFF_REROUTE);

    // the counters keep the previous call's values: clear them, then store the ray count
    if (cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * C_COUNT, st) != cudaSuccess)
        return ART_ERR_CUDA;
    unsigned long long nn = static_cast<unsigned long long>(n);
    if (cudaMemcpyAsync(counters + C_QUEUE, &nn, sizeof nn, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return ART_ERR_CUDA;
    if (launch_camera_setup(*job, cam, st) != cudaSuccess) return ART_ERR_CUDA;

    TraceArgs a;
    memset(&a, 0, sizeof a);
    a.job = J;
    a.quad_rays = ART_TUNE_QUAD_DEFAULT;
    a.pair_rays = ART_TUNE_PAIR_DEFAULT;
    a.quad64_rays = ART_TUNE_QUAD64_DEFAULT;
    art_make_synch(job, &a.synch);
    a.synchf = synch_to_float(a.synch);
    a.cam = cam;
    a.queue = pix_dev;
    a.count = counters + C_QUEUE;
    a.counters = counters;
    a.out = out_dev;
    a.npix = (int64_t)J.nx * J.ny;
    if (aux) {
        a.aux_status = aux->status;
        a.aux_steps = aux->steps;
        a.aux_nturn = aux->nturn;
        a.aux_minr = aux->min_r;
    }
    const bool fp32_first = J.precision != ART_FP64;
    const bool mixed = J.precision == ART_MIXED || J.precision == ART_MIXED_DF;
    a.fetch = counters + C_FETCH;
    if (mixed) {
        a.reroute = reroute;
        a.reroute_count = counters + C_REROUTE;
    }
    const int pl = J.stokes == 4 ? 1 : 0;
    if (launch_trace(a, fp32_first ? TK_FP32 : TK_FP64,
                     s.num_sms * s.occ[fp32_first ? TK_FP32 : TK_FP64][pl], st) != cudaSuccess)
        return ART_ERR_CUDA;
    if (mixed) {
        TraceArgs b = a;
        b.reroute = nullptr;
        b.reroute_count = nullptr;
        b.indirect = reroute;
        b.count = counters + C_REROUTE;
        b.fetch = counters + C_FETCH2;
        const bool dfp = J.precision == ART_MIXED_DF;
        if (launch_trace(b, dfp ? TK_DF : TK_FP64, s.num_sms * s.occ[dfp ? TK_DF : TK_FP64][pl],
                         st) != cudaSuccess)
            return ART_ERR_CUDA;
    }
    // counters C_BADIDX .. C_SYNCERR: skipped queue entries and timed-out hand-overs
    unsigned long long bad[C_SYNCERR - C_BADIDX + 1] = {};
    if (cudaMemcpyAsync(bad, counters + C_BADIDX, sizeof bad, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ART_ERR_CUDA;
    return (bad[0] || bad[C_SYNCERR - C_BADIDX]) ? ART_ERR_DEVICE : ART_OK;
}
