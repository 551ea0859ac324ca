// gq_dfl.cuh -- double-FP32 ("float-float") arithmetic for the split-precision
// direct-interaction kernels.  GB300 issues FP32 instructions 64 times as fast
// as FP64 ones, so carrying about 48 significant bits as an unevaluated sum
// hi + lo of two FP32 numbers is several times cheaper than FP64 even at ten to
// twenty FP32 instructions per operation.
//
// Exact building blocks: Knuth's two-sum (the rounding error of a + b),
// Dekker's fast two-sum (the same when |a| >= |b|) and the two-product
// a*b = p + e with e = fma(a, b, -p) (T. J. Dekker, "A floating-point technique
// for extending the available precision", Numer. Math. 18, 1971; the FMA form
// of the product is exact for FP32 operands).  Every operation renormalises so
// that |lo| <= ulp(hi)/2, except the lazy accumulator, which keeps the error
// terms of a running sum in lo and is normalised once at the end.  Sums and
// products whose rounding the error terms capture are written with the _rn
// intrinsics, which the compiler never fuses into multiply-adds.
#pragma once

#include <math.h>

struct dfl {
    float hi, lo;
};
struct dflc {
    dfl re, im;
};

__device__ __forceinline__ dfl dfl_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    return dfl{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl dfl_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    return dfl{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfl dfl_from_double(double x) {
    float h = __double2float_rn(x);
    return dfl{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dfl_to_double(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl dfl_neg(dfl a) { return dfl{-a.hi, -a.lo}; }

__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
    dfl s = dfl_two_sum(a.hi, b.hi);
    return dfl_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfl dfl_add_f(dfl a, float b) {
    dfl s = dfl_two_sum(a.hi, b);
    return dfl_fast_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dfl_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl dfl_mul_f(dfl a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return dfl_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl dfl_sqr(dfl a) {
    float p = __fmul_rn(a.hi, a.hi);
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(2.0f * a.hi, a.lo, e);
    return dfl_fast_two_sum(p, e);
}

// 1/x: FP32 seed y0 and one Newton step y0 + y0 (1 - x y0), whose residual is
// formed exactly up to the x.lo term; relative error about 2^-46.
__device__ __forceinline__ dfl dfl_rcp(dfl x) {
    float y0 = __frcp_rn(x.hi);
    float p = __fmul_rn(x.hi, y0);
    float e = fmaf(x.hi, y0, -p);
    float d = fmaf(-x.lo, y0, __fsub_rn(__fsub_rn(1.0f, p), e));
    return dfl_fast_two_sum(y0, y0 * d);
}

// Complex product with the real and imaginary parts each formed as one
// two-term sum of exact products plus the first-order cross terms.
__device__ __forceinline__ dfl dfl_dot2(float ah, float al, float bh, float bl, float ch, float cl, float dh, float dl) {
    // a b + c d
    float p1 = __fmul_rn(ah, bh), p2 = __fmul_rn(ch, dh);
    float e1 = fmaf(ah, bh, -p1), e2 = fmaf(ch, dh, -p2);
    dfl s = dfl_two_sum(p1, p2);
    float lo = s.lo + (e1 + e2);
    lo = fmaf(ah, bl, lo);
    lo = fmaf(al, bh, lo);
    lo = fmaf(ch, dl, lo);
    lo = fmaf(cl, dh, lo);
    return dfl_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ dflc dflc_mul(dflc a, dflc b) {
    return dflc{dfl_dot2(a.re.hi, a.re.lo, b.re.hi, b.re.lo, -a.im.hi, -a.im.lo, b.im.hi, b.im.lo),
                dfl_dot2(a.re.hi, a.re.lo, b.im.hi, b.im.lo, a.im.hi, a.im.lo, b.re.hi, b.re.lo)};
}

// Lazy accumulator: hi carries the running FP32 sum, lo the exact rounding
// errors of the hi additions plus the low parts of the summands.  With n
// summands lo stays below about n ulp(hi), so its own rounding costs about
// n 2^-48 relative; the directs sums here have at most a few hundred terms a lane.
__device__ __forceinline__ void dfl_acc(dfl &acc, dfl t) {
    dfl s = dfl_two_sum(acc.hi, t.hi);
    acc.hi = s.hi;
    acc.lo += s.lo + t.lo;
}
__device__ __forceinline__ void dflc_acc(dflc &acc, dflc t) {
    dfl_acc(acc.re, t.re);
    dfl_acc(acc.im, t.im);
}
// acc += c a (c = ch + cl, a = ah + al) into a lazy accumulator: the product's
// high part p = fl(ch ah) enters the running sum by a two-sum, its error
// fma(ch, ah, -p) and the cross terms ch al + cl ah go to lo (12 FP32 operations).
__device__ __forceinline__ void dfl_mac_lazy(dfl &acc, float ch, float cl, float ah, float al) {
    float p = __fmul_rn(ch, ah);
    float e = fmaf(ch, ah, -p);
    e = fmaf(ch, al, e);
    e = fmaf(cl, ah, e);
    dfl s = dfl_two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + e;
}

// ---------------------------------------------------------------- logarithm
// Tang's table-driven reduction (ACM TOMS 16(4), 1990) carried out in FP32
// pairs: x = 2^k m, j = the leading 7 fraction bits of m, t_j the FP32 number
// nearest 1/(1 + (j + 1/2)/128); then r = m t_j - 1 is formed exactly from the
// two-product of m.hi and t_j, |r| < 2^-8, and
//     log x = k log 2 + log(1/t_j) + r - r^2/2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6 + r^4/7),
// the first three terms in pairs, the cubic tail in FP32 (it is below 2^-24,
// so FP32 carries it to about 2^-48), truncation below 2^-67.  log(1/t_j)
// is tabulated as a pair; log 2 is split into a 16-bit head (so that k log 2
// is exact in FP32 for |k| < 256) and an FP32 pair.
struct GqDflLogTable {
    float t[128];
    float lhi[128];
    float llo[128];
};

#ifndef __CUDACC_RTC__
inline void gq_dfl_log_table_host(GqDflLogTable *T) {
    for (int j = 0; j < 128; ++j) {
        double c = 1.0 + (j + 0.5) / 128.0;
        float t = (float)(1.0 / c);
        long double L = -logl((long double)t);
        float h = (float)L;
        T->t[j] = t;
        T->lhi[j] = h;
        T->llo[j] = (float)(L - (long double)h);
    }
}
#endif

constexpr double kGqLn2 = 0.6931471805599453094172321214581765680755;
constexpr float kGqLn2A = 0.693145751953125f;   // 45426 / 2^16
constexpr float kGqLn2B = (float)(kGqLn2 - 0.693145751953125);
constexpr float kGqLn2C = (float)(kGqLn2 - 0.693145751953125 - (double)(float)(kGqLn2 - 0.693145751953125));

// x positive with x.hi a normal FP32 number in [2^-126, 2^126].
__device__ __forceinline__ dfl dfl_log(dfl x, const float *__restrict__ tt, const float *__restrict__ th,
                                       const float *__restrict__ tl) {
    int bits = __float_as_int(x.hi);
    int k = (bits >> 23) - 127;
    int j = (bits >> 16) & 0x7f;
    float mh = __int_as_float((bits & 0x007fffff) | 0x3f800000);
    float ml = x.lo * __int_as_float((127 - k) << 23);   // x.lo 2^-k
    float t = tt[j];
    float p = __fmul_rn(mh, t);
    float e = fmaf(mh, t, -p);
    dfl r = dfl_two_sum(__fsub_rn(p, 1.0f), fmaf(ml, t, e));
    dfl r2 = dfl_sqr(r);
    float rh = r.hi;
    float tail = fmaf(rh, fmaf(rh, fmaf(rh, fmaf(rh, 1.0f / 7.0f, -1.0f / 6.0f), 0.2f), -0.25f), 1.0f / 3.0f);
    tail *= rh * r2.hi;
    dfl l1p = dfl_add(r, dfl_add_f(dfl{-0.5f * r2.hi, -0.5f * r2.lo}, tail));
    float kf = (float)k;
    dfl kl = dfl_add(dfl{__fmul_rn(kf, kGqLn2A), 0.0f}, dfl_mul_f(dfl{kGqLn2B, kGqLn2C}, kf));
    return dfl_add(dfl_add(kl, dfl{th[j], tl[j]}), l1p);
}
