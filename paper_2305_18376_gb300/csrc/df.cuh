// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, giving about 48 significant bits.
// The error-free transformations are Knuth's TwoSum, Dekker's Fast2Sum and
// the FMA-based TwoProduct (as collected in Hida, Li and Bailey's
// double-double work); they need round-to-nearest FP32 without
// reassociation, which nvcc guarantees without fast-math flags.
//
// On GB300 FP64 arithmetic runs at about 1/57 of the FP32 rate, so the
// per-slice summaries of the mixed-precision path (c_k, D_k of Eqs. 15-16 and
// the refinement of the W solve, Eq. 12) are kept and updated in this format
// instead of FP64.
#pragma once
#include <cuda_runtime.h>

namespace dash {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

// a + b with b a single FP32 number: one TwoSum, the low part added, one
// Fast2Sum (the double-float + float sum of the same collection)
__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a + b·c with b, c double-float
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(a, df_mul(b, c)); }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// Square root, reciprocal and reciprocal square root: an FP32 approximation
// refined by one Newton step whose residual is formed exactly with the
// error-free product (Karp and Markstein's scheme), about 44 bits.
__device__ __forceinline__ df df_sqrt(df a) {
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float x = sqrtf(a.hi);
    const df r = df_sub(a, two_prod(x, x));            // a − x², small
    return fast_two_sum(x, r.hi * (0.5f / x));
}
__device__ __forceinline__ df df_recip(df a) {
    const float x = 1.0f / a.hi;
    const df e = df_sub(df_make(1.0f), df_mul_f(a, x));  // 1 − a·x, small
    return fast_two_sum(x, x * e.hi);
}
__device__ __forceinline__ df df_rsqrt(df a) {
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float x = rsqrtf(a.hi);
    const df e = df_sub(df_make(1.0f), df_mul(a, two_prod(x, x)));   // 1 − a·x²
    return fast_two_sum(x, 0.5f * x * e.hi);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_from_double(double x) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

}  // namespace dash
