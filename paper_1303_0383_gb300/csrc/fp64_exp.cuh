// fp64_exp.cuh -- the library's double-precision exponential for non-positive arguments.
//
// Method: P. T. P. Tang, "Table-driven implementation of the exponential function in
// IEEE floating-point arithmetic", ACM TOMS 15(2), 1989.  With N = 64:
//   a = (k/N) ln2 + r,  k = round(a N / ln2),  |r| <= ln2/(2N) ~ 0.0054,
//   exp(a) = 2^(k >> 6) * 2^((k & 63)/64) * exp(r),
// exp(r) - 1 by its Taylor series through r^6 (the first omitted term, r^7/7!, is below
// 3e-20), the 64 values 2^(j/64) from a table computed on the host in long double and
// rounded to double, and the final power of two applied to the exponent field.
// Arguments below -707 return 0 (the true value is below 1e-307 and a correlation that
// small does not change any result in double precision).  Cost: 12 FP64 instructions
// against ~20 for the general-purpose library routine, which matters on a part whose FP64
// pipe issues 2 operations per clock per SM.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace lagp {

// 2^(j/64), j = 0..63, and the split of ln2/64 (hi has 30 significant bits so that
// k * hi is exact for |k| < 2^20).
struct ExpConsts {
  double tab[64];
  double ln2_64_hi, ln2_64_lo, inv_ln2_64;
  // float-float version: 2^(j/64) = tabf_h + tabf_l; ln2/64 = c1 + c2 + c3 with c1 of 11
  // significant bits (k * c1 exact for |k| < 2^13).
  float tabf_h[64], tabf_l[64];
  float c1, c2, c3, inv_ln2_64f;
};

// Host: the constants, computed once per process in long double (fp64_exp.cu).
const ExpConsts *exp_host_consts();

// Each translation unit that includes this header has its own constant-bank copy
// (no relocatable device code is needed) and uploads it once per CUDA context: a
// cudaDeviceReset ends the context, and the device's next one is uploaded afresh.  The
// upload must not happen during stream capture (the *_prepare calls do it beforehand).
static __constant__ ExpConsts c_exp;

static int exp_table_upload() {
  static std::mutex mu;
  static unsigned long long ctx[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= 64) return LAGP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  unsigned long long id = 0;
  int st = current_context_id(&id);
  if (st) return st;
  if (id == 0 || ctx[dev] != id) {
    e = cudaMemcpyToSymbol(c_exp, exp_host_consts(), sizeof(ExpConsts));
    if (e != cudaSuccess) return cuda_status(e);
    st = current_context_id(&id);  // the copy made the context current if there was none
    if (st) return st;
    ctx[dev] = id;
  }
  return LAGP_OK;
}

__device__ __forceinline__ double exp_nonpos(double a, const double *__restrict__ tab) {
  const double magic = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer in the low bits
  const double t = fma(a, c_exp.inv_ln2_64, magic);
  const double kd = t - magic;
  const int k = (int)(uint32_t)__double_as_longlong(t);
  double r = fma(-kd, c_exp.ln2_64_hi, a);
  r = fma(-kd, c_exp.ln2_64_lo, r);
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(r, q, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  q = fma(r, q, 1.0);
  const double p = r * q;                        // exp(r) - 1
  const double T = tab[k & 63];
  const double e = fma(T, p, T);                 // 2^((k&63)/64) exp(r), in [0.98, 2.03)
  const unsigned long long bits = (unsigned long long)__double_as_longlong(e) +
                                  ((unsigned long long)(long long)(k >> 6) << 52);
  return a < -707.0 ? 0.0 : __longlong_as_double((long long)bits);
}

}  // namespace lagp
