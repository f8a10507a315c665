// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
//
// GB300 executes FP64 at about 1/64 of its FP32 instruction rate, so a
// computation that needs more than FP32 accuracy but not the full FP64
// range runs several times faster on the FP32 pipes in this form than in
// native FP64. The operations are built from the classical error-free
// transformations:
//  - TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact
//    rounding error e with s + e = a + b, for any a, b;
//  - FastTwoSum (Dekker 1971): the same in three operations when
//    |a| >= |b|;
//  - TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p),
//    p + e = a b exactly.
// The file must be compiled without reassociation of floating-point sums
// (no fast-math); contraction of a * b + c into an FMA does not occur in
// these routines because every product is either explicit or an fmaf.
#pragma once

#include <cuda_runtime.h>

namespace povar {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df64 df_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df64 df_norm(df64 x) { return df_fast_two_sum(x.hi, x.lo); }

__device__ __forceinline__ df64 df_neg(df64 x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ df64 df_add(df64 x, df64 y) {
  df64 s = df_two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df64 df_sub(df64 x, df64 y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df64 df_mul(df64 x, df64 y) {
  df64 p = df_two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return df_fast_two_sum(p.hi, p.lo);
}

// Accumulator without renormalization: acc += x * y with the product and
// the sum taken exactly up to the low-order parts; acc.lo collects the
// error terms and stays small next to acc.hi. df_norm once at the end.
__device__ __forceinline__ void df_acc_mul(df64& acc, df64 x, df64 y) {
  df64 p = df_two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  const df64 s = df_two_sum(acc.hi, p.hi);
  acc.hi = s.hi;
  acc.lo += s.lo + p.lo;
}

__device__ __forceinline__ void df_acc(df64& acc, df64 x) {
  const df64 s = df_two_sum(acc.hi, x.hi);
  acc.hi = s.hi;
  acc.lo += s.lo + x.lo;
}

__device__ __forceinline__ df64 df_from_double(double a) {
  const float hi = (float)a;
  return {hi, (float)(a - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df64 x) { return (double)x.hi + (double)x.lo; }

// 1 / sqrt(a), a > 0: the FP32 reciprocal square root refined by one Newton
// step r' = r + r (1 - a r^2) / 2 with the residual 1 - a r^2 evaluated in
// double-float (the correction is of relative size 1e-7, so FP32 suffices
// for it).
__device__ __forceinline__ df64 df_rsqrt(df64 a) {
  const float r = rsqrtf(a.hi);
  const df64 e = df_sub({1.f, 0.f}, df_mul(a, df_two_prod(r, r)));
  return df_fast_two_sum(r, 0.5f * r * e.hi);
}

}  // namespace povar
