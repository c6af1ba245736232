// Double-float arithmetic for the element kernels.  A value is the unevaluated
// sum hi + lo of two floats; products and sums are formed with error-free FP32
// transformations: Knuth's two-sum (s + e = a + b exactly) and the FMA-based
// exact product (p + e = a * b exactly, e = fma(a, b, -p)).  On GB300 the FP32
// pipes are 61 times wider than the FP64 pipe, so a contraction carried this
// way can outrun FP64 although it takes about a dozen FP32 instructions per
// multiply-add (the Q4 Jacobian action: 8.94 ms against 20.1 ms at 64^3), at
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
__device__ __forceinline__ df64 df_neg(df64 a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }

// Conversions between FP64 and double-float by integer operations on the bit
// patterns.  On GB300 a double <-> float conversion instruction runs at the
// FP64 rate (about 2 per clock per SM, the same as a DFMA), so code that moves
// FP64 work onto the FP32 pipes converts with these instead.
//
// df_split: hi = x with its significand truncated to 24 bits, lo = the next 23
// bits of the remainder (built as a float 2^k (1 + r 2^-23) minus 2^k, an exact
// FP32 subtraction): |x - hi - lo| < 2^-46 |x|.  |x| < 2^-103 keeps only hi,
// |x| < 2^-126 gives zero; |x| >= 2^128, inf and NaN go through the
// conversion instruction.
__device__ __forceinline__ df64 df_split(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sgn = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  const int ef = e - 896;  // float exponent of hi
  if (ef <= 0) return df_make(0.0f, 0.0f);
  if (ef >= 255) return df_make(__double2float_rn(x), 0.0f);
  const float h = __uint_as_float(sgn | ((unsigned)ef << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const int el = e - 919;  // float exponent of 2^(e - 1046), the weight of the remainder's leading bit
  float l = 0.0f;
  if (el > 0) {
    const unsigned two_k = (unsigned)el << 23;
    l = __fsub_rn(__uint_as_float(two_k | ((lw >> 6) & 0x7fffffu)), __uint_as_float(two_k));
    if (sgn) l = -l;
  }
  return df_make(h, l);
}
// The same with hi = x rounded to the nearest float (ties to even), as the
// FP32 planes of the stored words need: lo carries |x - hi| <= ulp(hi) / 2 to
// 23 bits (|x - hi - lo| < 2^-46 |x|).  Zero and FP64 subnormals give zero;
// |x| < 2^-126 and |x| >= 2^128 go through the conversion instructions.
__device__ __forceinline__ df64 df_split_rn(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sgn = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e == 0) return df_make(0.0f, 0.0f);
  const int ef = e - 896;
  if (ef <= 0 || ef >= 254) {
    const float h = __double2float_rn(x);
    return df_make(h, __double2float_rn(x - (double)h));
  }
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const unsigned rem = lw & 0x1fffffffu;  // the 29 bits below hi's significand
  const unsigned inc = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
  const float h = __uint_as_float((sgn | ((unsigned)ef << 23) | m23) + inc);  // a carry moves into the exponent
  const unsigned m = inc ? 0x20000000u - rem : rem;  // |x - hi| in units of 2^(e - 1075)
  const int el = e - 919;
  float l = 0.0f;
  if (el > 0) {
    const unsigned two_k = (unsigned)el << 23;
    l = __fsub_rn(__uint_as_float(two_k | ((m >> 6) & 0x7fffffu)), __uint_as_float(two_k));
    if ((sgn != 0u) != (inc != 0u)) l = -l;
  }
  return df_make(h, l);
}
// Exact float -> double of a normal float (zero and subnormal floats give
// zero, inf and NaN keep their class), by integer operations.
__device__ __forceinline__ double df_f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned ed = e == 255u ? 0x7ffu : e + 896u;
  const unsigned hw = e == 0u ? 0u : (b & 0x80000000u) | (ed << 20) | ((b & 0x7fffffu) >> 3);
  const unsigned lw = e == 0u ? 0u : b << 29;
  return __hiloint2double((int)hw, (int)lw);
}
// hi + lo in FP64 (one FP64 addition).
__device__ __forceinline__ double df_join(df64 a) { return df_f2d(a.hi) + df_f2d(a.lo); }

}  // namespace pff
