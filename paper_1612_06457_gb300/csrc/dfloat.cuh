// dfloat.cuh -- double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits (unit roundoff near 2^-48 ~ 3.6e-15).  On GB300 a
// dependent FP64 operation costs about 64 cycles and FP64 issues at 1/64 of
// the FP32 rate, so the single-CTA eigensolve carries its FP64-class
// quantities in this form instead.
//
// The building blocks are the classical error-free transformations:
//   two_sum       (Knuth; Moller)        s + e = a + b exactly
//   fast_two_sum  (Dekker, |a| >= |b|)   s + e = a + b exactly
//   two_prod      (with a fused multiply-add)  p + e = a * b exactly
// and the double-word algorithms analysed by M. Joldes, J.-M. Muller and
// V. Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017: the accurate sum of two
// double-words, the product of two double-words, and the product of a
// double-word by a float.  Division and reciprocal square root take a float
// estimate and one correction step computed in double-float.
#pragma once

#include <stdint.h>

namespace cva {

struct df {
    float hi, lo;
};

__device__ inline df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }
__device__ inline df df_from(float a) { return df_make(a, 0.0f); }

__device__ inline df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

__device__ inline df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

__device__ inline df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return df_make(p, e);
}

// Accurate sum of two double-words (relative error <= 3 u^2).
__device__ inline df df_add(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    const float c = __fadd_rn(s.lo, t.hi);
    const df v = fast_two_sum(s.hi, c);
    const float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}

__device__ inline df df_neg(df x) { return df_make(-x.hi, -x.lo); }
__device__ inline df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// Product of two double-words (relative error <= 5 u^2 with an FMA).
__device__ inline df df_mul(df x, df y)
{
    const df c = two_prod(x.hi, y.hi);
    const float tl = __fmul_rn(x.hi, y.lo);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl);
    const float cl3 = __fadd_rn(c.lo, cl2);
    return fast_two_sum(c.hi, cl3);
}

// Product of a double-word by a float (relative error <= 2 u^2).
__device__ inline df df_mulf(df x, float y)
{
    const df c = two_prod(x.hi, y);
    const float cl3 = __fmaf_rn(x.lo, y, c.lo);
    return fast_two_sum(c.hi, cl3);
}

// z - x * y
__device__ inline df df_fms(df z, df x, df y) { return df_add(z, df_neg(df_mul(x, y))); }
// z + x * y
__device__ inline df df_fma(df z, df x, df y) { return df_add(z, df_mul(x, y)); }

// 1 / y: float reciprocal q1, remainder r = 1 - q1 y in double-float, q1 + q1 r.
__device__ inline df df_rcp(df y)
{
    const float q1 = __frcp_rn(y.hi);
    const df r = df_sub(df_from(1.0f), df_mulf(y, q1));
    return fast_two_sum(q1, __fmul_rn(q1, r.hi));
}

// x / y: q1 = x.hi / y.hi, remainder r = x - q1 y, q1 + r.hi / y.hi.
__device__ inline df df_div(df x, df y)
{
    const float inv = __frcp_rn(y.hi);
    const float q1 = __fmul_rn(x.hi, inv);
    const df r = df_sub(x, df_mulf(y, q1));
    return fast_two_sum(q1, __fmul_rn(r.hi, inv));
}

// 1 / sqrt(x) for x > 0: float estimate r0, one Newton step
// r = r0 + r0 (1 - x r0^2) / 2 with the residual in double-float.
__device__ inline df df_rsqrt(df x)
{
    const float r0 = rsqrtf(x.hi);
    const df e = df_sub(df_from(1.0f), df_mulf(df_mulf(x, r0), r0));
    return fast_two_sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), e.hi));
}

__device__ inline bool df_gt(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ inline bool df_ge(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
__device__ inline df df_abs(df a) { return (a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f)) ? df_neg(a) : a; }

// Powers of two as floats (exact), for exponents in the normal range.
__device__ inline float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Non-negative 64-bit integer to double-float: the top 24 bits (truncated,
// exact as a float) plus the float nearest the exact remainder.
__device__ inline df df_from_u64(unsigned long long v)
{
    if (v < (1ull << 24)) return df_from(static_cast<float>(static_cast<uint32_t>(v)));
    const int nb = 64 - __clzll(v);
    const int s = nb - 24;
    const unsigned long long top = v >> s;
    const float h = __fmul_rn(static_cast<float>(static_cast<uint32_t>(top)), pow2f(s));
    const unsigned long long rem = v - (top << s);
    float l;
    if (rem < (1ull << 24)) {
        l = static_cast<float>(static_cast<uint32_t>(rem));
    } else {
        const int nb2 = 64 - __clzll(rem);
        const int s2 = nb2 - 24;
        l = __fmul_rn(static_cast<float>(static_cast<uint32_t>(rem >> s2)), pow2f(s2));
    }
    return fast_two_sum(h, l);
}

// Signed 128-bit integer to double-float (same scheme, 48 leading bits).
__device__ inline df df_from_i128(__int128 v)
{
    const bool neg = v < 0;
    unsigned __int128 u = neg ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
    const unsigned long long hi64 = static_cast<unsigned long long>(u >> 64);
    df r;
    if (hi64 == 0) {
        r = df_from_u64(static_cast<unsigned long long>(u));
    } else {
        const int nb = 128 - __clzll(hi64);  // bit length, > 64
        const int s = nb - 48;               // keep the leading 48 bits, exactly
        const unsigned long long top = static_cast<unsigned long long>(u >> s);
        r = df_mulf(df_from_u64(top), pow2f(s));
    }
    return neg ? df_neg(r) : r;
}

// Double-float to double (exact: 48 bits fit in 53) and back.
__device__ inline double df_to_double(df a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

}  // namespace cva
