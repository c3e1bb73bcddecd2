// dfloat.cuh -- double-float arithmetic for the mixed-precision path.
//
// A value is held as an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, which carries a 48-bit significand (relative precision
// ~2^-48 = 3.6e-15).  On GB300 the FP64 pipe retires 1/64 of the FP32 rate,
// and conversions between double and float run on that same pipe, so the
// mixed path keeps positions, velocities and the tangential history in this
// form and updates them with FP32 instructions only.  The building blocks are
// the classic error-free transformations: Knuth's two-sum (the exact rounding
// error of a + b from six additions) and the fused multiply-add product error
// (the exact rounding error of a * b is fma(a, b, -a*b)).  They rely on
// round-to-nearest FP32 adds and products, which nvcc never reassociates.
#pragma once
#include <cuda_runtime.h>

namespace susp {

struct df {
  float hi, lo;
};

__host__ __device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

// exact: a + b = s + e
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// exact when |a| >= |b|: a + b = s + e
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// a + f
__device__ __forceinline__ df df_add_f(df a, float f) {
  float s, e;
  two_sum(a.hi, f, s, e);
  e = __fadd_rn(e, a.lo);
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// a + b
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * f
__device__ __forceinline__ df df_mul_f(df a, float f) {
  const float p = __fmul_rn(a.hi, f);
  float e = __fmaf_rn(a.hi, f, -p);
  e = __fmaf_rn(a.lo, f, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// a * b
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// (qh + ql) - (ph + pl) for two double-float values given as parts
__device__ __forceinline__ df df_diff(float qh, float ql, float ph, float pl) {
  float s, e;
  two_sum(qh, -ph, s, e);
  e = __fadd_rn(e, __fsub_rn(ql, pl));
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// a >= b
__device__ __forceinline__ bool df_ge(df a, df b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo);
}
__device__ __forceinline__ bool df_lt0(df a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f); }

__device__ __forceinline__ float df_to_f(df a) { return __fadd_rn(a.hi, a.lo); }

// Host/device split of a double into a double-float (used only where the
// FP64 value is uniform or off the hot path).
__host__ __device__ __forceinline__ df df_from_d(double x) {
  const float hi = (float)x;
  const float lo = (float)(x - (double)hi);
  return df{hi, lo};
}
__host__ __device__ __forceinline__ double df_to_d(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace susp
