// Double-float arithmetic for the element kernels.  A value is the unevaluated
// sum hi + lo of two floats; products and sums are formed with error-free FP32
// transformations: Knuth's two-sum (s + e = a + b exactly) and the FMA-based
// exact product (p + e = a * b exactly, e = fma(a, b, -p)).  On GB300 the FP32
// pipes are 61 times wider than the FP64 pipe, so a contraction carried this
// way can outrun FP64 although it takes about a dozen FP32 instructions per
// multiply-add (the Q4 Jacobian action: 10.2 ms against 20.1 ms at 64^3), at
// an error of about 2^-47 of the magnitudes involved per operation (FP64:
// 2^-53).
//
// Accumulators stay unnormalised inside a contraction (|lo| may grow to a few
// ulps of hi); two-sum is exact for any pair of floats, so only the final
// conversion adds hi and lo.  Every function uses the _rn intrinsics so that
// the compiler neither contracts nor reorders the compensation terms.
#pragma once
#include <cuda_runtime.h>

#include "pff_internal.h"

namespace pff {

__device__ __forceinline__ df64 df_make(float h, float l) {
  df64 r;
  r.hi = h;
  r.lo = l;
  return r;
}

// hi + lo with hi = fl32(x), lo = fl32(x - hi): exact to 2^-48 relative.
__device__ __forceinline__ df64 df_from(double x) {
  const float h = __double2float_rn(x);
  return df_make(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth, six operations, no ordering assumption).
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a * b: exact product of the hi words plus the two cross terms.
__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_make(p, e);
}

// acc + a * b (twelve FP32 operations).
__device__ __forceinline__ df64 df_madd(df64 acc, df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, e;
  df_two_sum(acc.hi, p, s, e);
  return df_make(s, __fadd_rn(e, __fadd_rn(acc.lo, pe)));
}

// a + b
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  return df_make(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

}  // namespace pff
