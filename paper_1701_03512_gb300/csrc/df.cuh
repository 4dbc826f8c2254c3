// Double-float ("FP32 pair") arithmetic for the prefix and fold steps.
//
// A value is hi + lo with |lo| <= ulp(hi)/2. The building blocks are the
// error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the
// FMA-based exact product (TwoProd); the compound operations follow the
// standard double-word algorithms (Joldes, Muller, Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 2017). Intrinsics with explicit rounding keep nvcc from contracting
// or reordering any step.
#pragma once

struct df32 {
    float hi, lo;
};

__device__ __forceinline__ df32 df_make(float hi, float lo) {
    df32 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
__device__ __forceinline__ df32 df_from2(float2 v) { return df_make(v.x, v.y); }

__device__ __forceinline__ df32 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}
__device__ __forceinline__ df32 fast_two_sum(float a, float b) {  // needs |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}
__device__ __forceinline__ df32 two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return df_make(p, e);
}
// Accurate sum of two pairs (relative error about 3 * 2^-48).
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    df32 s = two_sum(a.hi, b.hi);
    df32 t = two_sum(a.lo, b.lo);
    float c = __fadd_rn(s.lo, t.hi);
    df32 v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ df32 df_neg(df32 a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df32 df_sub(df32 a, df32 b) { return df_add(a, df_neg(b)); }
// Sum for operands of the same sign (all fold accumulators are non-negative).
__device__ __forceinline__ df32 df_add_pos(df32 a, df32 b) {
    df32 s = two_sum(a.hi, b.hi);
    float c = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, c);
}
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    df32 p = two_prod(a.hi, b.hi);
    float t = __fmul_rn(a.lo, b.lo);
    t = __fmaf_rn(a.hi, b.lo, t);
    t = __fmaf_rn(a.lo, b.hi, t);
    return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}
__device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
    df32 p = two_prod(a.hi, b);
    float t = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, t);
}
// Exact scaling by 2^e (barring under/overflow).
__device__ __forceinline__ df32 df_ldexp(df32 a, int e) {
    return df_make(ldexpf(a.hi, e), ldexpf(a.lo, e));
}
__device__ __forceinline__ bool df_gt(df32 a, df32 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ float2 split2(double x) {
    float h = (float)x;
    float l = (float)(x - (double)h);
    return make_float2(h, l);
}
