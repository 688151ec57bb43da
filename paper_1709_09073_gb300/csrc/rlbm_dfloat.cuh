// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (about 48 significant bits), built from the error-free
// transformations TwoSum (Knuth) and TwoProduct (via FMA). GB300 executes FP64
// at 1/64 of the FP32 rate, so the mixed-precision step keeps its few
// precision-critical quantities (moment totals, Landau residual, gamma, n, eps)
// in this form on the FP32 pipe. Every operation is written with the
// round-to-nearest intrinsics, which the compiler neither reassociates nor
// contracts into an FMA with a neighbouring product: the error-free
// transformations are exact only as written, and every kernel that inlines
// them gets the same roundings.
#pragma once
#include <cuda_runtime.h>

namespace rlbm {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return df_make(s, e);
}

// s + e = a + b exactly, requires |a| >= |b|
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// p + e = a * b exactly
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df_make(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_add(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// exact scaling by a power of two
__device__ __forceinline__ df df_scale(df a, float pow2) { return df_make(__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)); }

// 1 / sqrt(a): rsqrtf seed and one Newton step evaluated in double-float
__device__ __forceinline__ df df_rsqrt(df a) {
  const float g = rsqrtf(a.hi);
  // e = 1 - a g^2 (small), g1 = g + g e / 2
  const df ag2 = df_mul(df_mul(a, g), g);
  const float e = __fsub_rn(__fsub_rn(1.0f, ag2.hi), ag2.lo);
  return quick_two_sum(g, __fmul_rn(__fmul_rn(0.5f, g), e));
}

// a / b: FP32 quotient refined once with the double-float remainder
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = df_sub(a, df_mul(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return quick_two_sum(q1, q2);
}

__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }

}  // namespace rlbm
