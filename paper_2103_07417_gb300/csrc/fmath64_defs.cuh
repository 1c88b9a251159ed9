// fmath64_defs.cuh -- qualifiers and bit casts of fmath64.cuh: device functions and tables under
// nvcc's device pass, plain host ones elsewhere (the host build of the same source is what the
// accuracy checks against extended precision compile).
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDA_ARCH__
#define ART_FM_DEV __device__ __forceinline__
#define ART_FM_TABLE __device__
#else
#define ART_FM_DEV inline
#define ART_FM_TABLE static
#endif

namespace art {

ART_FM_DEV int64_t fm_bits(double x)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    int64_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

ART_FM_DEV double fm_double(int64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

ART_FM_DEV uint32_t fm_f32bits(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

}  // namespace art
