// fmath64.cuh -- FP64 elementary functions with fewer FP64 instructions than the general library
// ones, for the emission code of the FP64 tracer.  GB300 issues an FP64 warp instruction every 64
// cycles on a scheduler and an integer one every cycle, so these move the argument reduction onto
// the integer units and look the rest up in small tables.
//
// log_fp64: the natural logarithm by Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4),
// 1990).  With x = 2^k m, m in [1, 2) (exponent and significand split on the integer units),
// F = 1 + j/128 the nearest point of a 1/128 grid and f = m - F (exact, |f| <= 1/256):
//   ln x = k ln 2 + ln F + ln(1 + u),  u = f / F  (here f times the rounded reciprocal of F),
// where ln(1 + u) is its Taylor polynomial through u^7 (truncation below |u|^8 / 8 <= 2^-67) and
// k ln2 + ln F is summed exactly from leads that are multiples of 2^-42 (log_table.cuh).  Error
// about one unit in the last place (checked against extended precision by the host build of this
// file).  Finite positive normal arguments only; others go to the library logarithm.
#pragma once
#include <cmath>

#include "fmath64_defs.cuh"
#include "log_table.cuh"

namespace art {

ART_FM_DEV double log_fp64(double x)
{
    const int64_t b = fm_bits(x);
    const int hi = (int)(b >> 32);
    const int e = (hi >> 20) & 0x7ff;
    if (b < 0 || e == 0 || e == 0x7ff) return log(x);  // <= 0, subnormal, infinite or NaN
    const int k = e - 1023;
    // m = x 2^-k in [1, 2); j = nearest multiple of 1/128 (the 7 leading fraction bits, rounded)
    const int64_t mb = (b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL;
    const int j = (int)(((b >> 44) & 0xff) + 1) >> 1;  // 0 .. 128
    const double m = fm_double(mb);
    const double F = fm_double(0x3ff0000000000000LL + ((int64_t)j << 45));
#ifdef __CUDA_ARCH__
    const double* t = LOG_TABLE[j];
    const double lead = __ldg(t), trail = __ldg(t + 1), invF = __ldg(t + 2);
    const double kd = __int2double_rn(k);
#else
    const double lead = LOG_TABLE[j][0], trail = LOG_TABLE[j][1], invF = LOG_TABLE[j][2];
    const double kd = (double)k;
#endif
    const double f = m - F;
    const double u = f * invF;
    const double u2 = u * u;
    // ln(1 + u) = u + u^2 (-1/2 + u (1/3 + u (-1/4 + u (1/5 + u (-1/6 + u / 7)))))
    double q = fma(u, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(u, q, 0.2);
    q = fma(u, q, -0.25);
    q = fma(u, q, 1.0 / 3.0);
    q = fma(u, q, -0.5);
    const double p = fma(u2, q, u);
    const double head = fma(kd, LOG_LN2_LEAD, lead);  // exact: both multiples of 2^-42
    const double tail = fma(kd, LOG_LN2_TRAIL, trail) + p;
    return head + tail;
}

// ln x in the arithmetic Q: log_fp64 for FP64, the library logarithm otherwise.
template <class Q>
ART_FM_DEV Q log_q(Q x)
{
    return log(x);
}
template <>
ART_FM_DEV double log_q<double>(double x)
{
    return log_fp64(x);
}

}  // namespace art
