// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two float32 numbers, giving about 48 significant bits with
// float32 operations only.  Error-free transformations after Dekker (1971)
// and Knuth (TwoSum); the accurate pair addition and multiplication follow
// Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic" (ACM TOMS 2017).  Every step uses
// the __f*_rn intrinsics (or an explicit fmaf), which the compiler never
// contracts or reassociates, so the transformations stay error-free.
#pragma once

namespace unigs {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_from(float a) { return {a, 0.f}; }
__device__ __forceinline__ float ff_val(ff a) { return __fadd_rn(a.hi, a.lo); }

// a + b = s + e exactly.
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// a + b = s + e exactly, valid when |a| >= |b| (or a == 0).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// a * b = p + e exactly (barring underflow).
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    return {p, e};
}

// Accurate pair + pair (relative error below 3u^2).
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    const ff t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    ff v = fast_two_sum(s.hi, c);
    const float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

// pair * float.
__device__ __forceinline__ ff ff_mul_f(ff x, float b) {
    const ff c = two_prod(x.hi, b);
    const float cl = fmaf(x.lo, b, c.lo);
    return fast_two_sum(c.hi, cl);
}

// pair * pair.
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const ff c = two_prod(x.hi, y.hi);
    float tl = __fmul_rn(x.hi, y.lo);
    tl = fmaf(x.lo, y.hi, tl);
    const float cl = __fadd_rn(c.lo, tl);
    return fast_two_sum(c.hi, cl);
}

// x * 2^k scalings are exact.
__device__ __forceinline__ ff ff_scale(ff x, float pow2) {
    return {__fmul_rn(x.hi, pow2), __fmul_rn(x.lo, pow2)};
}

// pair / pair: one Newton-style correction of the float quotient.
__device__ __forceinline__ ff ff_div(ff x, ff y) {
    const float t = __fdiv_rn(x.hi, y.hi);
    const ff r = ff_sub(x, ff_mul_f(y, t));
    const float d = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(t, d);
}

// sqrt of a non-negative pair.
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.hi > 0.f)) return {0.f, 0.f};
    const float s = __fsqrt_rn(x.hi);
    const ff p = two_prod(s, s);
    const float r = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo),
                              __fmul_rn(2.f, s));
    return fast_two_sum(s, r);
}

}  // namespace unigs
