// vr_df.cuh -- double-float arithmetic for the per-ray setup.
//
// A value is carried as an unevaluated sum hi + lo of two floats with
// hi = fl(hi + lo), about 48 significant bits. The building blocks are the
// error-free transformations TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|) and
// the FMA-based TwoProd; division and square root take one Newton step from the
// float approximation. On this part FP64 runs at a small fraction of the FP32 rate
// and doubles take two registers, so the ray setup uses these instead. Every
// operation is written with round-to-nearest intrinsics so that the compiler
// cannot contract or reassociate the compensated sums.
#pragma once

#include <cuda_runtime.h>

namespace vr {

struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfloat df_neg(dfloat x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    const dfloat s = df_two_sum(x.hi, y.hi);
    const dfloat t = df_two_sum(x.lo, y.lo);
    const dfloat u = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ dfloat df_add_f(dfloat x, float b) {
    const dfloat s = df_two_sum(x.hi, b);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
    const dfloat p = df_two_prod(x.hi, y.hi);
    return df_fast_two_sum(p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo)));
}

__device__ __forceinline__ dfloat df_mul_f(dfloat x, float b) {
    const dfloat p = df_two_prod(x.hi, b);
    return df_fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}

// 1 / x: y0 = 1/x.hi, then y0 + y0 (1 - x y0) with the residual formed exactly.
__device__ __forceinline__ dfloat df_recip(dfloat x) {
    const float y0 = __frcp_rn(x.hi);
    const dfloat xy = df_mul_f(x, y0);
    const float r = __fsub_rn(__fsub_rn(1.0f, xy.hi), xy.lo);  // 1 - xy.hi is exact (xy.hi ~ 1)
    return df_fast_two_sum(y0, __fmul_rn(y0, r));
}

// 1 / sqrt(x), x > 0: y0 = rsqrt(x.hi), then y0 + y0 (1 - x y0^2) / 2.
__device__ __forceinline__ dfloat df_rsqrt(dfloat x) {
    const float y0 = __frsqrt_rn(x.hi);
    const dfloat t = df_mul_f(df_mul_f(x, y0), y0);
    const float r = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
    return df_fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), r));
}

__device__ __forceinline__ bool df_lt(dfloat x, dfloat y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

// Host side: the double d split into hi = (float)d and lo = (float)(d - hi).
struct dfloat_h {
    float hi, lo;
};
inline dfloat_h df_split(double d) {
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}

}  // namespace vr
