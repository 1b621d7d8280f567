// ff.cuh -- float-float ("double-FP32") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2,
// which carries a 48-bit significand.  The building blocks are the error-free
// transformations of Knuth (two-sum) and Dekker (fast two-sum, valid for |a| >= |b|),
// and the FMA form of the exact product a*b = p + e with e = fma(a, b, -p).  The
// compound operations below are the usual "sloppy" double-word algorithms: their error
// is a few units of 2^-48 relative to the magnitudes of the operands.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) { return ff{hi, lo}; }

__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // requires |a| >= |b|
    const float s = a + b;
    return ff{s, b - (s - a)};
}

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return ff{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = a * b;
    return ff{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

// 1 / a: FP32 seed refined by one Newton step in float-float, x1 = x0 + x0 (1 - a x0).
__device__ __forceinline__ ff ff_rcp(ff a) {
    const float x0 = 1.0f / a.hi;
    const ff ax = ff_mul_f(a, x0);
    const ff e = ff_add_f(ff_neg(ax), 1.0f);
    return ff_add_f(ff_mul_f(e, x0), x0);
}

// Conversions through binary64.
__device__ __forceinline__ ff ff_from_double(double x) {
    const float hi = __double2float_rn(x);
    return ff{hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

}  // namespace lbm
