// gq_math.cuh -- FP64 logarithm and reciprocal for the direct-interaction
// kernels, which are bound by GB300's FP64 pipe: both use fewer FP64
// instructions than the IEEE-exact library routines while staying within a
// few units in the last place (checked against CUDA's log and division by
// tests/test_gpu_math.py).
#pragma once

#include <math.h>

// ---------------------------------------------------------------- logarithm
// Table-driven method of P. T. P. Tang, "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990:
// write x = 2^k m with m in [1, 2); let j be the leading 7 fraction bits of m
// and t_j the FP64 value nearest 1 / (1 + (j + 1/2)/128).  Then
//     log x = k log 2 + log(1/t_j) + log1p(r),   r = m t_j - 1,
// with r formed by one fused multiply-add (m t_j is exact in the FMA), |r| < 2^-8,
// and log1p(r) = r - r^2/2 + ... + r^7/7 (the truncation is below 2^-64/8).
// log(1/t_j) is tabulated to full FP64 precision.
struct GqLogTable {
    double t[128];       // t_j
    double logc[128];    // log(1 / t_j)
};

#ifndef __CUDACC_RTC__
inline void gq_log_table_host(GqLogTable *T) {
    for (int j = 0; j < 128; ++j) {
        long double c = 1.0L + (j + 0.5L) / 128.0L;
        double t = (double)(1.0L / c);
        T->t[j] = t;
        T->logc[j] = (double)(-logl((long double)t));
    }
}
#endif

__device__ __forceinline__ double gq_log(double x, const double *__restrict__ tt, const double *__restrict__ tl) {
    if (!(x >= 0x1p-1000 && x <= 0x1p1000)) return log(x);   // zero, subnormal, huge, inf, nan
    long long bits = __double_as_longlong(x);
    int k = (int)(bits >> 52) - 1023;
    int j = (int)((bits >> 45) & 0x7f);
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    double r = fma(m, tt[j], -1.0);
    double a = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    a = fma(r, a, 1.0 / 5.0);
    a = fma(r, a, -0.25);
    a = fma(r, a, 1.0 / 3.0);
    a = fma(r, a, -0.5);
    a = fma(r, a, 1.0);
    double p = r * a;
    const double ln2 = 0.693147180559945309417232121458176568;
    return fma((double)k, ln2, tl[j] + p);
}

// ---------------------------------------------------------------- reciprocal
// 1/x from the FP32 reciprocal of x (relative error < 2^-23) refined by two
// Newton steps y <- y + y (1 - x y), each squaring the relative error, so the
// result is within about one unit in the last place.  Outside [2^-120, 2^120]
// the library division is used.
__device__ __forceinline__ double gq_rcp(double x) {
    double ax = fabs(x);
    if (!(ax >= 0x1p-120 && ax <= 0x1p120)) return 1.0 / x;
    double y = (double)__frcp_rn(__double2float_rn(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
