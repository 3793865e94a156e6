// ff.cuh -- float-float ("double-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2, about 48
// significant bits.  The building blocks are the error-free transformations of
// Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum (a + b = s + e exactly), FastTwoSum
// (the same when |a| >= |b|) and TwoProd via a fused multiply-add (a*b = p + e
// exactly).  Additions use the "sloppy" double-float sum (one TwoSum of the high
// parts, the low parts added in FP32, then FastTwoSum), whose relative error is a small
// multiple of 2^-44..2^-48 -- enough for a candidate screen whose decisions are
// re-checked in FP64 whenever they are close.  Every operation is written with
// explicit round-to-nearest intrinsics so the compiler cannot contract or reorder the
// steps the transformations depend on.
#pragma once

#include <cuda_runtime.h>

namespace lagp {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_make(float h) { return ff{h, 0.0f}; }

// From a double: h = rn(x), l = rn(x - h) (the double subtraction is exact).
__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return ff{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// acc - a*b for the inner loop of a dot product (TwoProd of the high parts, cross
// terms in FP32, TwoSum into the accumulator, renormalised every term so the low part
// stays below an ulp of the high part).
__device__ __forceinline__ ff ff_sub_prod_acc(ff acc, ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const ff s = two_sum(acc.h, -p);
  return fast_two_sum(s.h, __fsub_rn(__fadd_rn(s.l, acc.l), e));
}

// Compensated dot product of float-float vectors: the running sum stays FP32 and every
// rounding error (TwoProd of the high parts with the cross terms, TwoSum of the running
// sum) is collected in a second FP32 sum (Dot2 of Ogita, Rump and Oishi, 2005, extended to
// float-float operands); the result is h + l.
struct ffacc {
  float h, l;
};

__device__ __forceinline__ void ffacc_add_prod(ffacc &acc, ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);  // a b - p to FP32 accuracy
  const float s = __fadd_rn(acc.h, p);
  const float bb = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
  acc.h = s;
}

// sqrt and reciprocal by one Newton correction of the FP32 estimate.
__device__ __forceinline__ ff ff_sqrt(ff a) {
  const float s = sqrtf(a.h);
  const float r = __fadd_rn(__fmaf_rn(-s, s, a.h), a.l);  // a - s^2
  return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

__device__ __forceinline__ ff ff_rcp(ff a) {
  const float q = __frcp_rn(a.h);
  const float e = __fsub_rn(__fmaf_rn(-a.h, q, 1.0f), __fmul_rn(a.l, q));  // 1 - a q
  return fast_two_sum(q, __fmul_rn(e, q));
}

}  // namespace lagp
