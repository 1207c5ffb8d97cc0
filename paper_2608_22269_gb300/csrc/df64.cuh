// df64.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2), about 48 significand
// bits, computed on the FP32 pipe. Built from the error-free transformations
// of Knuth (two-sum), Dekker (fast two-sum) and the FMA form of the exact
// product (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005); the
// operations are the standard double-word algorithms (Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", 2017). Every FP32 operation is an explicit
// round-to-nearest intrinsic so that the compiler neither contracts nor
// reorders them.
#pragma once
#include "common.cuh"

namespace wbsph {

struct df {
  float hi, lo;
};

// s + e = a + b exactly (no condition on the magnitudes)
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly
__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// a * b (double-word times double-word with FMA, renormalised: relative error a few u^2)
__device__ __forceinline__ df df_mul(df a, df b) {
  const df p = df_two_prod(a.hi, b.hi);
  const float t = __fmaf_rn(a.lo, b.hi, __fmul_rn(a.hi, b.lo));
  return df_fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

// a * b as (fl(a.hi b.hi), the rest): the exact product of the high parts
// plus the two cross terms, not renormalised. Neither operand needs to be
// normalised; the dropped a.lo b.lo is below u^2 |a| |b|.
__device__ __forceinline__ df df_mul_raw(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}

__device__ __forceinline__ df df_norm(df a) { return df_fast_two_sum(a.hi, a.lo); }

// acc <- acc + v, renormalised (the sloppy double-word sum: the absolute
// error is a few u^2 (|acc| + |v|), which is what a running sum needs).
__device__ __forceinline__ void df_acc(df& acc, df v) {
  const df s = df_two_sum(acc.hi, v.hi);
  acc = df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, v.lo)));
}

// a - b for two normalised values, as (fl(a.hi - b.hi), the rest), not renormalised
__device__ __forceinline__ df df_sub_raw(df a, df b) {
  const df s = df_two_sum(a.hi, -b.hi);
  return {s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo))};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// the double nearest to hi + lo (exact: both are FP32)
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// hi + lo within 2^-48 relative of x (|x| in the FP32 normal range or zero)
__device__ __forceinline__ df df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

}  // namespace wbsph
