// Double-float arithmetic for the float64 parts of the mixed-precision build and true residual.
//
// A value is the unevaluated sum hi + lo of two float32 numbers with |lo| <= ulp(hi) / 2, about 48
// significant bits (relative rounding error near 2^-48 per operation, against 2^-53 for float64).
// The operations use the float32 pipe only, through error-free transformations: Knuth's two-sum
// (the exact error of a float32 addition), Dekker's fast two-sum (the same when |a| >= |b|), and the
// exact error of a float32 product from one fused multiply-add.  On this GPU the float32 pipe does
// 128 fused multiply-adds per clock and SM against 1.7 for float64, so a double-float multiply-add
// (about 15 float32 instructions) still runs several times faster than a float64 one; conversions
// between float32 and float64 run on the float64 pipe, so values stay double-float from the
// observation kernels to the per-camera and per-landmark results and convert only there.
//
// Every float32 operation here is an explicit round-to-nearest intrinsic (__fadd_rn, __fmul_rn,
// __fmaf_rn): the compiler must neither contract a product and a sum into one fused operation nor
// reorder, or the error terms would be wrong.  Addition is the cheap form (the low parts are added
// without their own two-sum): its error is bounded by about 2^-47 (|a| + |b|), which keeps sums of
// terms of mixed signs as accurate as float64 summation would be to within a factor of about 32.
// Range is float32's: magnitudes must stay within about 1e-38 .. 1e38 (BA Jacobians, residuals and
// their products do).
#pragma once

#include <cuda_runtime.h>

namespace ba {

struct df64 {
    float hi, lo;
    df64() = default;   // trivial (uninitialised), so that shared-memory arrays of df64 are allowed
    __device__ __forceinline__ df64(float h) : hi(h), lo(0.f) {}
    __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
};

// s + e = a + b exactly, s = fl(a + b); needs |a| >= |b| (or a = 0)
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df64(s, e);
}
// s + e = a + b exactly, s = fl(a + b), any a, b
__device__ __forceinline__ df64 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df64(s, e);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    const df64 s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);   // the exact error of the product a.hi b.hi
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// a * b + c
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) { return a * b + c; }

// 1 / p: the float32 reciprocal of the high part and one Newton step in double-float, r + r (1 - p r)
// (the step squares the 2^-23 error of the estimate).
__device__ __forceinline__ df64 rcp_fast(df64 p) {
    const df64 r(__frcp_rn(p.hi));
    return r + r * (df64(1.f) - p * r);
}

// 1 / sqrt(x) for x > 0 by one Newton step y + y (1 - x y^2) / 2 from the float32 estimate; 0 for
// x <= 0 or NaN (the callers report a pivot that is not positive)
__device__ __forceinline__ df64 rsqrt_fast(df64 x) {
    if (!(x.hi > 0.f)) return df64(0.f);
    const df64 y(rsqrtf(x.hi));
    const df64 t = df64(1.f) - x * (y * y);
    return y + y * df64(__fmul_rn(0.5f, t.hi), __fmul_rn(0.5f, t.lo));
}

__device__ __forceinline__ bool df_positive(df64 a) { return a.hi > 0.f; }

// float64 <-> double-float (on the float64 pipe: used per camera, per landmark or once per create)
__device__ __forceinline__ df64 df_from(double d) {
    const float h = __double2float_rn(d);
    return df64(h, __double2float_rn(d - double(h)));
}
__device__ __forceinline__ double df_to(df64 a) { return double(a.hi) + double(a.lo); }

// storage: a double-float array element is a float2 (hi, lo), 8 bytes like a double
__device__ __forceinline__ df64 df_ld(const float2* p) {
    const float2 v = *p;
    return df64(v.x, v.y);
}
__device__ __forceinline__ void df_st(float2* p, df64 a) { *p = make_float2(a.hi, a.lo); }

// shuffle of a double-float value (both halves)
__device__ __forceinline__ df64 df_shfl_xor(df64 a, int o) {
    return df64(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
}

}  // namespace ba
