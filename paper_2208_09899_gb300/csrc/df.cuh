// Double-float ("df") arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi)/2 when normalised), 48 significand bits.
// Built from the error-free transformations
//   TwoSum(a, b)      = (s, e) with s = fl(a+b), a + b = s + e exactly   (Knuth)
//   TwoProduct(a, b)  = (p, e) with p = fl(a*b), a * b = p + e exactly   (FMA form of Dekker's product)
// and compensated dot-product accumulation in the style of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005)
// (Dot2): the exact rounding errors of every product and addition are
// collected in a second FP32 accumulator.
//
// Every operation uses the _rn intrinsics so that the compiler neither
// contracts nor reorders the error-free transformations.  Conversions to and
// from FP64 run on GB300's FP64 pipe and are used only at the edges of a pass.
#pragma once
#include <cuda_runtime.h>

namespace lsba {

struct dfacc {  // running compensated sum: value = s + c (unnormalised)
  float s, c;
};

__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

// Normalise an unevaluated sum (s + c) into (hi, lo).
__device__ __forceinline__ float2 df_norm(float s, float c) { return df_two_sum(s, c); }

// acc += a * b  (a, b double-float).  The product's error term and the cross
// terms a.hi*b.lo + a.lo*b.hi go to the compensation together with the exact
// error of the addition; a.lo*b.lo (relative 2^-48) is dropped.  13 FP32 ops.
__device__ __forceinline__ void df_fma(dfacc& acc, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.x, -p);
  const float cross = __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x));
  const float t = __fadd_rn(acc.s, p);
  const float bb = __fsub_rn(t, acc.s);
  const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  acc.s = t;
  acc.c = __fadd_rn(acc.c, __fadd_rn(err, __fadd_rn(e, cross)));
}

// acc -= a * b
__device__ __forceinline__ void df_fms(dfacc& acc, float2 a, float2 b) {
  df_fma(acc, make_float2(-a.x, -a.y), b);
}

// acc += a (a double-float)
__device__ __forceinline__ void df_add_to(dfacc& acc, float2 a) {
  const float2 t = df_two_sum(acc.s, a.x);
  acc.s = t.x;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t.y, a.y));
}

// Renormalise the accumulator in place (keeps the compensation small).
__device__ __forceinline__ void df_renorm(dfacc& acc) {
  const float2 t = df_two_sum(acc.s, acc.c);
  acc.s = t.x;
  acc.c = t.y;
}

__device__ __forceinline__ float2 df_value(const dfacc& acc) { return df_norm(acc.s, acc.c); }

// Normalised product a * b.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  dfacc acc{0.f, 0.f};
  df_fma(acc, a, b);
  return df_value(acc);
}

// FP64 <-> double-float (FP64 pipe: edges of a pass only).
__device__ __forceinline__ float2 df_from_double(double d) {
  const float hi = __double2float_rn(d);
  const float lo = __double2float_rn(d - (double)hi);
  return make_float2(hi, lo);
}
__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double dfacc_to_double(const dfacc& a) { return (double)a.s + (double)a.c; }

}  // namespace lsba
