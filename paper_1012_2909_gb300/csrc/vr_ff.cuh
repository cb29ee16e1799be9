// Float-float ("double-single") arithmetic for the few ray quantities that need
// more than FP32 precision (sample anchors o + k e far from the origin), used
// because double-precision throughput on this part is a small fraction of FP32.
// Each value is hi + lo with |lo| <= ulp(hi)/2.  The error-free transforms are
// Knuth's two-sum and the FMA-based two-product.
#pragma once

#include <cuda_runtime.h>

namespace vr {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}

__device__ __forceinline__ ff ff_quick(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = ff_two_sum(x.hi, y.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return ff_quick(s.hi, s.lo);
}

// x * f for a float f
__device__ __forceinline__ ff ff_mul_f(ff x, float f) {
    const float p = __fmul_rn(x.hi, f);
    float e = __fmaf_rn(x.hi, f, -p);
    e = __fmaf_rn(x.lo, f, e);
    return ff_quick(p, e);
}

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return ff_quick(p, e);
}

// 1 / sqrt(x) to about 44 bits: hardware estimate refined by one Newton step
// whose residual 1 - x r^2 is formed in float-float.
__device__ __forceinline__ ff ff_rsqrt(ff x) {
    const float r = rsqrtf(x.hi);
    const float r2 = __fmul_rn(r, r);
    const float r2e = __fmaf_rn(r, r, -r2);           // r^2 = r2 + r2e exactly
    ff xr2 = ff_mul(x, ff{r2, r2e});
    const ff res = ff_add(ff{1.0f, 0.0f}, ff{-xr2.hi, -xr2.lo});
    const float corr = __fmul_rn(__fmul_rn(0.5f, r), res.hi);
    return ff_quick(r, corr);
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

// x / y to about 44 bits: FP32 quotient, one correction from the float-float
// remainder x - q y.
__device__ __forceinline__ ff ff_div(ff x, ff y) {
    const float q = __fdiv_rn(x.hi, y.hi);
    const ff r = ff_add(x, ff_neg(ff_mul_f(y, q)));
    return ff_quick(q, __fdiv_rn(r.hi, y.hi));
}

__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// floor and ceiling of hi + lo as integers (|hi| < 2^62).  If hi is not an
// integer, lo cannot carry the sum across one: |lo| <= ulp(hi) / 2, and hi and
// the integers on either side of it are all multiples of ulp(hi).
__device__ __forceinline__ long long ff_ceil(ff x) {
    const float c = ceilf(x.hi);
    if (c != x.hi) return (long long)c;
    return (long long)c + (long long)ceilf(x.lo);
}

__device__ __forceinline__ long long ff_floor(ff x) {
    const float f = floorf(x.hi);
    if (f != x.hi) return (long long)f;
    return (long long)f + (long long)floorf(x.lo);
}

// An int as an exact float-float pair (|k| <= 2^31 - 128).
__device__ __forceinline__ ff ff_of_int(int k) {
    const float h = __int2float_rn(k);
    return ff{h, __int2float_rn(k - __float2int_rz(h))};
}

}  // namespace vr
