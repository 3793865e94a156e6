// ff2.cuh -- two independent float-float numbers per thread, on the packed FP32 pipes.
//
// Blackwell executes paired FP32 operations (__fadd2_rn, __fmul2_rn, __ffma2_rn on
// float2): one instruction applies the same operation to two lanes of a float2.  An ff2
// holds two float-float values (ff.cuh) side by side -- x for one candidate, y for
// another -- so every error-free transformation of the float-float arithmetic costs one
// packed instruction for both.  The formulas are those of ff.cuh, operation for
// operation.
#pragma once

#include <cuda_runtime.h>

#include "ff.cuh"

namespace lagp {

struct ff2 {
  float2 h, l;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as a packed fused multiply-add with multiplier -1: one rounding, the same result
// as a subtraction, and no separate sign flips of the packed operands.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.0f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, f2s(-1.0f)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ ff2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  const float2 e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
  return ff2{s, e};
}

__device__ __forceinline__ ff2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return ff2{s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
  const ff2 s = two_sum2(a.h, b.h);
  return fast_two_sum2(s.h, add2(s.l, add2(a.l, b.l)));
}

__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) {
  const ff2 s = two_sum2(a.h, neg2(b.h));
  return fast_two_sum2(s.h, add2(s.l, sub2(a.l, b.l)));
}

// TwoProd with the negated product formed directly: np = rn(-(a*b)) = -p, and
// fma(a, b, np) = a*b - p exactly.
__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b) {
  const float2 np = __fmul2_rn(__fmul2_rn(a.h, f2s(-1.0f)), b.h);
  float2 e = fma2(a.h, b.h, np);
  e = fma2(a.h, b.l, e);
  e = fma2(a.l, b.h, e);
  return fast_two_sum2(sub2(f2s(0.0f), np), e);
}

// acc - a*b with the same scalar multiplier a for both lanes (see ff_sub_prod_acc); the
// caller passes a and its negation (nah = -a.h) so that no sign flip is needed per term.
__device__ __forceinline__ ff2 ff2_sub_prod_acc(ff2 acc, float2 ah, float2 nah, float2 al,
                                                float2 bh, float2 bl) {
  const float2 np = mul2(nah, bh);        // -p
  float2 e = fma2(ah, bh, np);            // a.h b.h - p
  e = fma2(ah, bl, e);
  e = fma2(al, bh, e);                    // a b - p (to float precision)
  const ff2 s = two_sum2(acc.h, np);      // acc.h - p
  return fast_two_sum2(s.h, sub2(add2(s.l, acc.l), e));
}

__device__ __forceinline__ ff ff2_x(ff2 a) { return ff{a.h.x, a.l.x}; }
__device__ __forceinline__ ff ff2_y(ff2 a) { return ff{a.h.y, a.l.y}; }

// Pair layout in memory: float4 {h_x, h_y, l_x, l_y} for candidates (2q, 2q+1).
__device__ __forceinline__ ff2 ff2_load(const float4 *p) {
  const float4 v = *p;
  return ff2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void ff2_store(float4 *p, ff2 a) {
  *p = make_float4(a.h.x, a.h.y, a.l.x, a.l.y);
}
// One candidate c of a pair array.
__device__ __forceinline__ ff ff2_get(const float4 *base, int c) {
  const float4 v = base[c >> 1];
  return (c & 1) ? ff{v.y, v.w} : ff{v.x, v.z};
}

}  // namespace lagp
