// Float-float ("double-single") arithmetic for the ray setup.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The operations are the classical error-free
// transformations: Knuth's TwoSum and Dekker's FastTwoSum for addition, the
// FMA form of Dekker's TwoProduct for multiplication, one Newton step for the
// reciprocal and the reciprocal square root.  B300 issues FP32 arithmetic at
// dozens of times its FP64 rate, so a setup written this way runs several
// times faster than the same steps in double while its discrete decisions
// (first and last sample index) still agree with a double-precision
// computation except within ~1e-12 of a tie.
//
// Every step uses the _rn intrinsics, which the compiler never contracts or
// reorders; an FMA contraction of a - b * c would break the error terms.
#pragma once

#include <cuda_runtime.h>

namespace isaac {

struct ff {
    float hi, lo;
};

// a + b exactly, given |a| >= |b| (or a == 0).
__device__ __forceinline__ ff ff_quick(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b exactly, any magnitudes.
__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), v = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}

__device__ __forceinline__ ff ff_from(float a) { return {a, 0.0f}; }
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

// Sum with absolute error ~2^-48 (|x| + |y|).
__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = ff_two_sum(x.hi, y.hi);
    return ff_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mulf(ff x, float b)
{
    const float p = __fmul_rn(x.hi, b);
    float e = __fmaf_rn(x.hi, b, -p);
    e = __fmaf_rn(x.lo, b, e);
    return ff_quick(p, e);
}

__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return ff_quick(p, e);
}

// 1 / y: the rounded FP32 reciprocal q and one Newton correction q (1 - y q).
__device__ __forceinline__ ff ff_rcp(ff y)
{
    const float q = __frcp_rn(y.hi);
    const ff r = ff_sub(ff_from(1.0f), ff_mulf(y, q));
    return ff_quick(q, __fmul_rn(r.hi, q));
}

// x / y: quotient of the leading parts, corrected by the remainder.
__device__ __forceinline__ ff ff_div(ff x, ff y)
{
    const float ry = __frcp_rn(y.hi);
    const float q = __fmul_rn(x.hi, ry);
    const ff r = ff_sub(x, ff_mulf(y, q));
    return ff_quick(q, __fmul_rn(r.hi, ry));
}

// 1 / sqrt(x), x > 0: the FP32 estimate y and one Newton step y (1 + (1 - x y^2) / 2).
__device__ __forceinline__ ff ff_rsqrt(ff x)
{
    const float y = rsqrtf(x.hi);
    const ff e = ff_sub(ff_from(1.0f), ff_mulf(ff_mulf(x, y), y));
    return ff_quick(y, __fmul_rn(__fmul_rn(0.5f, y), e.hi));
}

__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_lt(b, a) ? b : a; }

// ceil(hi + lo) for a normalised pair.  A float that is not an integer lies at
// least one ulp from the next integer, farther than |lo| reaches.
__device__ __forceinline__ long long ff_ceil(ff u)
{
    const float c = ceilf(u.hi);
    if (c != u.hi) return (long long)c;
    return (long long)u.hi + (long long)ceilf(u.lo);
}

}  // namespace isaac
