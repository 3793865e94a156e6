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

// a / b: the FP32 quotient q1 = a_h / b_h (through the reciprocal), the remainder
// a - b q1 formed with TwoProd of b_h q1, and one correction q2 = remainder / b_h.
__device__ __forceinline__ ff2 ff2_div(ff2 a, ff2 b) {
  const float2 rb = f2(__frcp_rn(b.h.x), __frcp_rn(b.h.y));
  const float2 q1 = mul2(a.h, rb);
  const float2 np = mul2(neg2(b.h), q1);           // -p, p = rn(b_h q1)
  float2 e = fma2(b.h, q1, np);                    // b_h q1 - p, exact
  e = fma2(b.l, q1, e);                            // b q1 - p to FP32 accuracy
  const float2 r = add2(sub2(add2(a.h, np), e), a.l);
  return fast_two_sum2(q1, mul2(r, rb));
}

__device__ __forceinline__ ff2 ff2_bcast(ff a) { return ff2{f2s(a.h), f2s(a.l)}; }
// exact scaling by a power of two
__device__ __forceinline__ ff2 ff2_scale(ff2 a, float s) { return ff2{mul2(a.h, f2s(s)), mul2(a.l, f2s(s))}; }

// Compensated accumulation of acc - sum_i a_i b_i for float-float a_i (the same for both
// lanes) and pairs b_i: the running sum h is plain FP32; the rounding error of every
// addition (TwoSum, exact) and of every product (TwoProd with the cross terms a_h b_l and
// a_l b_h) is collected in a second FP32 sum l, and h + l is renormalised once at the end.
// This is the Dot2 scheme of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005), whose result is as accurate as the sum computed in twice
// the working precision and then rounded, extended to float-float operands.  Per term: 12
// packed instructions, and only one addition on each loop-carried chain.
// The caller passes a_h as (a_h, a_h, -a_h, -a_h) and a_l as (a_l, a_l): no sign flips or
// register moves are needed per term.
struct ff2acc {
  float2 h, l;
};

__device__ __forceinline__ void ff2acc_sub_prod(ff2acc &acc, float4 ahn, float2 al, float4 b) {
  const float2 ah = make_float2(ahn.x, ahn.y), nah = make_float2(ahn.z, ahn.w);
  const float2 bh = make_float2(b.x, b.y), bl = make_float2(b.z, b.w);
  const float2 np = mul2(nah, bh);                 // -p, p = rn(a_h b_h)
  float2 e = fma2(ah, bh, np);                     // a_h b_h - p, exact
  e = fma2(ah, bl, e);
  e = fma2(al, bh, e);                             // a b - p to FP32 accuracy
  const float2 s = add2(acc.h, np);                // TwoSum(h, -p)
  const float2 bb = sub2(s, acc.h);
  const float2 err = add2(sub2(acc.h, sub2(s, bb)), sub2(np, bb));
  acc.l = add2(acc.l, sub2(err, e));
  acc.h = s;
}

__device__ __forceinline__ ff2 ff2acc_result(ff2acc acc) { return two_sum2(acc.h, acc.l); }

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
