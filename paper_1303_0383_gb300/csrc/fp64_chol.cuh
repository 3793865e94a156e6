// fp64_chol.cuh -- block-cooperative FP64 Cholesky for one small matrix per CTA.
//
// FP64 runs at 1/64 of the FP32 rate on this GPU, so the factorisation keeps every FP64
// instruction busy on all lanes: each step's column scaling and trailing update are
// flattened over the CTA's threads.  A division by the pivot is a product with its
// reciprocal plus one correction (Markstein: with the correctly rounded reciprocal y of b
// and q = rn(a y), q + (a - b q) y is the correctly rounded a / b), and the pivot's square
// root and reciprocal are taken by the thread that finishes the pivot in the previous
// step's update, so a step costs two block barriers.  The right-looking order makes for
// every entry the same subtractions, in the same order, as the row-by-row factorisation.
#pragma once

#include <math.h>

namespace lagp {
namespace {

// Row of the lower triangle {(a, b): 0 <= b <= a} that holds flat entry e.
__device__ __forceinline__ int tri_row(int e) {
  int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (a * (a + 1) / 2 > e) a--;
  while ((a + 1) * (a + 2) / 2 <= e) a++;
  return a;
}

// In-place Cholesky A = L L^T of the n x n lower triangle of A (row-major, leading
// dimension lda), carrying naug extra columns n .. n+naug-1 along so that they end as
// L^{-1} b (forward substitution).  rl[k] receives 1 / l_kk.  Sets *fail (shared) on a
// pivot <= 0; every thread returns after the same barriers.
__device__ void chol_flat_fp64(double *A, int n, int lda, int naug, double *rl, int *fail) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __syncthreads();
  if (tid == 0) {
    const double d0 = A[0];
    if (!(d0 > 0.0)) *fail = 1;
    const double l0 = sqrt(d0);
    A[0] = l0;
    rl[0] = 1.0 / l0;
  }
  __syncthreads();
  for (int k = 0; k < n && !*fail; k++) {
    const double lkk = A[k * lda + k], r = rl[k];
    // column k and the extra columns of row k divided by the pivot
    for (int i = k + 1 + tid; i < n + naug; i += nt) {
      double *ap = (i < n) ? &A[i * lda + k] : &A[k * lda + i];
      const double a = *ap, q = a * r;
      *ap = fma(fma(-q, lkk, a), r, q);
    }
    __syncthreads();
    // a_il -= l_ik l_lk for k < l <= i, and the extra columns: b_i -= l_ik b_k
    const int rows = n - k - 1, ntr = rows * (rows + 1) / 2;
    for (int e = tid; e < ntr + naug * rows; e += nt) {
      if (e < ntr) {
        const int t = tri_row(e), c = e - t * (t + 1) / 2;
        const int i = k + 1 + t, l = k + 1 + c;
        const double v = fma(-A[i * lda + k], A[l * lda + k], A[i * lda + l]);
        if (e == 0) {  // the next pivot is final: its square root and reciprocal
          if (!(v > 0.0)) *fail = 1;
          const double lv = sqrt(v);
          A[i * lda + l] = lv;
          rl[k + 1] = 1.0 / lv;
        } else {
          A[i * lda + l] = v;
        }
      } else {
        const int i = k + 1 + (e - ntr) / naug, col = (e - ntr) % naug;
        A[i * lda + n + col] = fma(-A[i * lda + k], A[k * lda + n + col], A[i * lda + n + col]);
      }
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace lagp
