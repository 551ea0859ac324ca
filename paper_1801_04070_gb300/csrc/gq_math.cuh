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
// write x = 2^k m with m in [1, 2); let j be the leading 9 fraction bits of m
// and t_j the FP64 value nearest 1 / (1 + (j + 1/2)/512).  Then
//     log x = k log 2 + log(1/t_j) + log1p(r),   r = m t_j - 1,
// with r formed by one fused multiply-add (m t_j is exact in the FMA), |r| < 2^-10,
// and log1p(r) = r - r^2/2 + r^3/3 - r^4/4 (the truncation is below 2^-53).
// The kernels need log|w| from |w|^2, so the primitive is (1/2) log x, with
// the halving folded into the tables and the coefficients; (k/2) log 2 is a
// third table indexed by the biased exponent (no integer-to-FP64 conversion).
// The two table terms are added first and the polynomial r a(r) enters
// through the final multiply-add.
// The range test looks at the exponent bits only (integer pipe).
constexpr int kGqLogJ = 512;
constexpr int kGqLogN = 2 * kGqLogJ + 2048;   // doubles in GqLogTable
struct GqLogTable {
    double t[kGqLogJ];    // t_j
    double hl[kGqLogJ];   // (1/2) log(1 / t_j)
    double hk[2048];      // (e - 1023) (log 2)/2 for the biased exponent e
};

#ifndef __CUDACC_RTC__
inline void gq_log_table_host(GqLogTable *T) {
    for (int j = 0; j < kGqLogJ; ++j) {
        long double c = 1.0L + (j + 0.5L) / (long double)kGqLogJ;
        double t = (double)(1.0L / c);
        T->t[j] = t;
        T->hl[j] = (double)(-0.5L * logl((long double)t));
    }
    for (int e = 0; e < 2048; ++e) T->hk[e] = (double)((long double)(e - 1023) * 0.5L * logl(2.0L));
}
#endif

// (1/2) log x; T points to a GqLogTable
__device__ __forceinline__ double gq_log_half(double x, const double *__restrict__ T) {
    long long bits = __double_as_longlong(x);
    unsigned long long e = (unsigned long long)bits >> 52;    // biased exponent, sign bit above it
    if (e - 23ull > 2000ull) return 0.5 * log(x);             // outside [2^-1000, 2^1001): zero, subnormal, huge, inf, nan, x < 0
    int j = (int)((bits >> 43) & (kGqLogJ - 1));
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    double r = fma(m, T[j], -1.0);
    double a = fma(r, -0.125, 1.0 / 6.0);
    a = fma(r, a, -0.25);
    a = fma(r, a, 0.5);
    return fma(r, a, T[2 * kGqLogJ + (int)e] + T[kGqLogJ + j]);
}

__device__ __forceinline__ double gq_log(double x, const double *__restrict__ T) { return 2.0 * gq_log_half(x, T); }

// FP32 copy of x built from its bits with integer operations only (no FP64
// conversion instruction): the leading 24 significant bits (truncated, so
// relative error below 2^-23), with the exponent lowered so that
// x = f * 2^(ebias - 1023).  Values with |f| below 2^-126 (and zeros,
// subnormals) give 0; the caller keeps |x| <= 2^(ebias - 1023 + 127).
__device__ __forceinline__ float gq_f32_rebased(double x, int ebias) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
    int e = (int)((hi >> 20) & 0x7ff) - ebias + 127;
    unsigned int f = (hi & 0x80000000u) | ((unsigned int)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return e > 0 ? __uint_as_float(f) : 0.0f;
}

// (1/2) log x as h + tail with fewer FP64 instructions: log1p(r)/2 =
// r/2 - r^2/4 + r^3 (1/6 - r/8); the first two terms and the table terms stay
// in FP64 (h, two FMAs after r), the tail, below 2^-32 in magnitude, is formed
// in FP32 from r's FP32 copy (relative error about 2^-21, so below 2^-53
// absolute).  The caller sums tails in FP32 and adds them once at the end.
// x = 0 gives h = 0 and tail = 0 (a coincident source contributes nothing).
__device__ __forceinline__ double gq_log_half_split(double x, const double *__restrict__ T, float &tail) {
    long long bits = __double_as_longlong(x);
    unsigned long long e = (unsigned long long)bits >> 52;
    if (e - 23ull > 2000ull) {                                 // rare: see gq_log_half
        tail = 0.0f;
        return x == 0.0 ? 0.0 : 0.5 * log(x);
    }
    int j = (int)((bits >> 43) & (kGqLogJ - 1));
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    double r = fma(m, T[j], -1.0);
    float rf = gq_f32_rebased(r, 1023);
    tail = rf * rf * (rf * fmaf(rf, -0.125f, 0.16666667f));
    double u = fma(r, -0.25, 0.5);
    return fma(r, u, T[2 * kGqLogJ + (int)e] + T[kGqLogJ + j]);
}

// 2^(e - 1023) for a biased exponent 1 <= e <= 2046 (0 for e = 0)
__device__ __forceinline__ double gq_pow2_biased(int e) {
    return e > 0 ? __longlong_as_double((long long)e << 52) : 0.0;
}

// ---------------------------------------------------------------- reciprocal
// 1/x from the hardware's approximate FP64 reciprocal (PTX rcp.approx.ftz.f64,
// which works on the upper mantissa bits; no conversions through FP32) refined
// by one third-order step: with e = 1 - x y, 1/x = y / (1 - e) = y (1 + e + e^2 + ...),
// so y (1 + e + e^2) has relative error e^3 -- below 2^-60 for a seed good to
// 20 bits -- and the result is within about half a unit in the last place
// after the final rounding; three FMAs instead of the four of two Newton
// steps.  Outside [2^-120, 2^121) (tested on the exponent bits) the library
// division is used.
__device__ __forceinline__ double gq_rcp(double x) {
    unsigned long long ex = ((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff;
    if (ex - 903ull > 240ull) return 1.0 / x;                 // |x| outside [2^-120, 2^121)
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}
