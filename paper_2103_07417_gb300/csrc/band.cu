// band.cu -- speculation of the near-critical band: the pixels whose rays pass close to the
// photon shell, found from the Kerr critical curve in closed form, are traced with the base level.
//
// A ray's constants of motion lambda = L_z/E and eta = Q/E^2 (Carter 1968) follow from its initial
// covariant momentum at the camera.  The rays that orbit the hole before escaping are those with
// (lambda, eta) close to the critical curve of the spherical photon orbits (Bardeen 1973), whose
// radii lie between the prograde and retrograde equatorial orbits,
//   r_pro, r_ret = 2 (1 + cos(2/3 arccos(-+|a|))).
// On the curve the radial potential R(r) (below) has a double root at the orbit's radius: its
// minimum over [r_pro, r_ret] is zero, slightly positive for rays just inside the shadow and
// slightly negative for rays just outside.  The distance used here is that minimum over r^4 at
// the minimiser, d = |R(r_m)| / r_m^4: for a = 0, |27 - eta - lambda^2| / 27, the relative
// deviation of the impact parameter squared from 27.  Unlike a distance along eta at fixed
// lambda, it stays proportional to the offset at the two ends of the curve, where it meets the
// equatorial orbits (eta = 0) with a vertical tangent; those ends are in view for observers near
// the equatorial plane.  These are exactly the rays the FP32 pass hands to the double-float
// re-trace; tracing every unset pixel of the finer levels with d < band in the same launch as the
// base level puts all their re-traces into one double-float pass, instead of one latency-bound
// pass per level.  The exact criterion still decides every point (a speculative ray it does not
// ask for is overwritten by its interpolant), so images do not change; the band is a scheduling
// hint evaluated in FP32.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace art {

// Radial potential of a photon with constants (lambda, eta) in Boyer-Lindquist r (M = E = 1):
// R(r) = (r^2 + a^2 - a lambda)^2 - Delta (eta + (lambda - a)^2), Delta = r^2 - 2 r + a^2; the
// photon moves where R >= 0.
__device__ __forceinline__ float radial_potential(float a, float lam, float eta, float r)
{
    const float A = r * r + a * a - a * lam, D = r * r - 2.f * r + a * a, lm = lam - a;
    return A * A - D * (eta + lm * lm);
}

// Distance of (lambda, eta) from the critical curve of spin a (see above): |R| at its minimum
// over the photon-orbit radii [r_pro, r_ret] (golden-section search), over r^4 there.
__device__ __forceinline__ float crit_distance(float a, float lam, float eta)
{
    const float aa = fabsf(a);
    float lo = 2.f * (1.f + cosf(2.f / 3.f * acosf(-aa)));  // prograde photon orbit
    float hi = 2.f * (1.f + cosf(2.f / 3.f * acosf(aa)));   // retrograde photon orbit
    const float rl = lo, rh = hi;
    const float g = 0.618034f;
    float x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    float f1 = radial_potential(a, lam, eta, x1), f2 = radial_potential(a, lam, eta, x2);
    for (int it = 0; it < 24; ++it) {
        if (f1 < f2) {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - g * (hi - lo);
            f1 = radial_potential(a, lam, eta, x1);
        } else {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + g * (hi - lo);
            f2 = radial_potential(a, lam, eta, x2);
        }
    }
    float rm = 0.5f * (lo + hi), fm = radial_potential(a, lam, eta, rm);
    const float fl = radial_potential(a, lam, eta, rl), fh = radial_potential(a, lam, eta, rh);
    if (fl < fm) {
        fm = fl;
        rm = rl;
    }
    if (fh < fm) {
        fm = fh;
        rm = rh;
    }
    const float r2 = rm * rm;
    return fabsf(fm) / (r2 * r2);
}

// The camera quantities the band test needs, in FP32: the covariant tetrad, the position and its
// Kerr-Schild radius and polar angle.
struct BandCam {
    float E[4][4], x0[3], r0, ct, st;
};

__device__ __forceinline__ void band_cam_setup(const Camera* cam, float a, BandCam& c)
{
    if (threadIdx.x < 16) c.E[threadIdx.x / 4][threadIdx.x % 4] = (float)cam->E[threadIdx.x / 4][threadIdx.x % 4];
    if (threadIdx.x < 3) c.x0[threadIdx.x] = (float)cam->x0[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        const float q = c.x0[0] * c.x0[0] + c.x0[1] * c.x0[1] + c.x0[2] * c.x0[2] - a * a;
        c.r0 = sqrtf(0.5f * (q + sqrtf(q * q + 4.f * a * a * c.x0[2] * c.x0[2])));
        c.ct = c.x0[2] / c.r0;
        c.st = sqrtf(fmaxf(1.f - c.ct * c.ct, 1e-12f));
    }
    __syncthreads();
}

// Whether pixel (i, j) of a job lies within `band` of the critical curve.
__device__ __forceinline__ bool in_band(const DevJob& J, const BandCam& c, float band, int i, int j)
{
    const float a = (float)J.a, ro = (float)J.r_obs, pix = (float)J.pix;
    const float al = (i - 0.5f * (J.nx - 1)) * pix, be = (j - 0.5f * (J.ny - 1)) * pix;
    // the critical curve of every spin and inclination lies at impact parameters between 2 M and
    // 7 M (prograde and retrograde photon orbits of an extremal hole); the pinhole's screen
    // radius approximates the impact parameter, so screen radii outside (0.5 M, 20 M) are
    // rejected before the bisection
    const float b2 = al * al + be * be;
    if (!(b2 > 0.25f && b2 < 400.f)) return false;
    const float sc = rsqrtf(1.f + (al * al + be * be) / (ro * ro));
    float k[4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
        k[m] = -c.E[0][m] + sc * (-c.E[1][m] + (al / ro) * c.E[3][m] + (be / ro) * c.E[2][m]);
    const float Een = k[0];
    const float L = -(c.x0[0] * k[2] - c.x0[1] * k[1]);
    const float pth = -((c.x0[0] * k[1] + c.x0[1] * k[2]) * c.ct / c.st - c.r0 * c.st * k[3]);
    const float Q = pth * pth + c.ct * c.ct * (-a * a * Een * Een + L * L / (c.st * c.st));
    const float lam = L / Een, eta = Q / (Een * Een);
    return crit_distance(a, lam, eta) < band;
}

// Every pixel off the base lattice whose mask is unset and whose camera ray lies within `band` of
// the critical curve is queued for a speculative trace and marked pending (grid-stride over the
// final grid; slots beyond `cap` are skipped).
__global__ void __launch_bounds__(256)
    band_propose_kernel(DevJob J, const Camera* cam, float band, uint8_t* mask, int32_t* queue,
                        unsigned long long* counters, unsigned long long cap)
{
    __shared__ BandCam c;
    band_cam_setup(cam, (float)J.a, c);
    const int S0 = 1 << J.levels;
    const int64_t npix = (int64_t)J.nx * J.ny;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npix;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = base + threadIdx.x;
        bool want = false;
        if (p < npix) {
            const int i = (int)(p % J.nx), j = (int)(p / J.nx);
            want = (i % S0 != 0 || j % S0 != 0) && mask[p] == ART_MASK_UNSET &&
                   in_band(J, c, band, i, j);
        }
        const unsigned b = __ballot_sync(0xffffffffu, want);
        if (!b) continue;
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(counters + C_QUEUE, (unsigned long long)__popc(b));
        w = __shfl_sync(0xffffffffu, w, 0);
        if (want) {
            const unsigned long long slot = w + __popc(b & ((1u << lane) - 1u));
            if (slot < cap) {
                queue[slot] = (int32_t)p;
                mask[p] = MASK_SPEC_PENDING;
                atomicAdd(counters + C_SPEC, 1ull);
            }
        }
    }
}

// Batched form: blockIdx.y is the image (band[image] <= 0: none), queue entries
// (image << 32) | pixel.  The kernel also initialises every mask: each pixel of each image is
// written, pending where queued and unset elsewhere, so no separate clear is needed.
__global__ void __launch_bounds__(256)
    band_propose_batch_kernel(const DevJob* jobs, const Camera* cams, const float* bands,
                              uint8_t* const* masks, int64_t* queue,
                              unsigned long long* counters, unsigned long long cap)
{
    const int im = blockIdx.y;
    const DevJob J = jobs[im];
    const float band = bands[im];
    uint8_t* mask = masks[im];
    __shared__ BandCam c;
    band_cam_setup(cams + im, (float)J.a, c);
    const int S0 = 1 << J.levels;
    const int64_t npix = (int64_t)J.nx * J.ny;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npix;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = base + threadIdx.x;
        bool want = false;
        if (p < npix) {
            const int i = (int)(p % J.nx), j = (int)(p / J.nx);
            want = band > 0.f && J.levels > 0 && (i % S0 != 0 || j % S0 != 0) &&
                   in_band(J, c, band, i, j);
        }
        const unsigned b = __ballot_sync(0xffffffffu, want);
        bool queued = false;
        if (b) {
            unsigned long long w = 0;
            if (lane == 0) w = atomicAdd(counters + C_QUEUE, (unsigned long long)__popc(b));
            w = __shfl_sync(0xffffffffu, w, 0);
            if (want) {
                const unsigned long long slot = w + __popc(b & ((1u << lane) - 1u));
                if (slot < cap) {
                    queue[slot] = ((int64_t)im << 32) | p;
                    queued = true;
                    atomicAdd(counters + C_SPEC, 1ull);
                }
            }
        }
        if (p < npix) mask[p] = queued ? MASK_SPEC_PENDING : (uint8_t)ART_MASK_UNSET;
    }
}

cudaError_t launch_band_propose(const DevJob& J, const Camera* cam, double band, uint8_t* mask,
                                int32_t* queue, unsigned long long* counters,
                                unsigned long long cap, int num_sms, cudaStream_t st)
{
    band_propose_kernel<<<num_sms * 8, 256, 0, st>>>(J, cam, (float)band, mask, queue, counters, cap);
    return cudaGetLastError();
}

cudaError_t launch_band_propose_batch(const DevJob* jobs, const Camera* cams, const float* bands,
                                      uint8_t* const* masks, int n, int64_t max_npix,
                                      int64_t* queue, unsigned long long* counters,
                                      unsigned long long cap, cudaStream_t st)
{
    int64_t gx = (max_npix + 255) / 256;
    if (gx > 64) gx = 64;
    if (gx < 1) gx = 1;
    band_propose_batch_kernel<<<dim3((unsigned)gx, n), 256, 0, st>>>(jobs, cams, bands, masks, queue,
                                                                    counters, cap);
    return cudaGetLastError();
}

}  // namespace art
