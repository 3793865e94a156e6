// predict_loc.cuh -- the FP64 predictive equations of one location on a given design:
// kernel (c)'s arithmetic (predict.cu), also run by the mixed ALC kernel on each design it
// has just selected.  Included by one translation unit each.
//
// Gramacy & Apley, Sec. 2, Eqs. predgp and preds2: with K_n = K(X_n, X_n) + g I,
// k(x) = K(X_n, x) and psi = Y^T K_n^{-1} Y,
//   mu(x) = k(x)^T K_n^{-1} Y,   s2(x) = psi (K(x, x) + g - k(x)^T K_n^{-1} k(x)) / n,
// and var = psi (K(x, x) + g - k(x)^T K_n^{-1} k(x)) / (n - 2), the variance of the
// Student-t predictive.  [K_n | k(x) | Y] is factored by a right-looking Cholesky, which
// makes for every entry the same subtractions, in the same order, as the row-by-row
// factorisation followed by forward substitution (u_x = L^{-1} k(x), y~ = L^{-1} Y):
// v_n(x) = 1 + g - |u_x|^2 is a cancellation whose rounding error is of the order of the
// tolerance, and keeping the textbook operation order keeps the rounding close to that of
// a plain sequential evaluation.  The arithmetic of every entry does not depend on the
// number of threads, so both kernels give bitwise-identical results.
#pragma once

#include <math.h>

#include "batch.cuh"
#include "fp64_chol.cuh"
#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {
namespace {

__device__ __forceinline__ double pl_corr(const double *a, const double *b, int p,
                                          double theta_inv, const double *etab) {
  double acc = 0.0;
  for (int k = 0; k < p; k++) {
    const double t = a[k] - b[k];
    acc = fma(t, t, acc);
  }
  return exp_nonpos(-acc * theta_inv, etab);
}

// Location L with design indices d[0..n) (d[0] < 0: its screen failed) and x in xl
// (shared memory).  A (n x (n + 2), leading dimension n + 2) and rl (n) are CTA-visible
// scratch, *fail a shared flag.  Every thread returns after the same barriers; thread 0
// writes mean, s2, var and status of location `loc`.
__device__ void predict_location(const LocParams &L, const int32_t *d, int n, const double *xl,
                                 double *A, double *rl, const double *etab, int *fail,
                                 int64_t loc, double *mean, double *s2, double *var,
                                 int8_t *status) {
  const int tid = threadIdx.x, nt = blockDim.x, p = L.p, lda = n + 2;
  if (tid == 0) *fail = d[0] < 0;
  __syncthreads();
  if (!*fail) {
    // K_n + g I (lower triangle), k(x) and Y
    const int ntri = n * (n + 1) / 2;
    for (int e = tid; e < ntri + 2 * n; e += nt) {
      if (e < ntri) {
        const int a = tri_row(e), b = e - a * (a + 1) / 2;
        const double *xa = L.X + (int64_t)d[a] * p;
        A[a * lda + b] = (a == b) ? L.onepg
                                  : pl_corr(xa, L.X + (int64_t)d[b] * p, p, L.theta_inv, etab);
      } else {
        const int a = (e - ntri) >> 1, col = (e - ntri) & 1;
        A[a * lda + n + col] = col == 0 ? pl_corr(L.X + (int64_t)d[a] * p, xl, p, L.theta_inv, etab)
                                        : L.Z[d[a]];
      }
    }
    chol_flat_fp64(A, n, lda, 2, rl, fail);
  }
  __syncthreads();
  if (tid == 0) {
    if (*fail) {
      mean[loc] = NAN;
      s2[loc] = NAN;
      if (var) var[loc] = NAN;
      if (status) status[loc] = (int8_t)LAGP_ERR_NOT_PD;
    } else {
      // in index order, as a sequential evaluation of the sums
      double mu = 0.0, psi = 0.0, vx = L.onepg;
      for (int i = 0; i < n; i++) {
        const double ux = A[i * lda + n], yt = A[i * lda + n + 1];
        mu = fma(ux, yt, mu);
        psi = fma(yt, yt, psi);
        vx = fma(-ux, ux, vx);
      }
      const double pv = psi * vx;
      mean[loc] = mu;
      s2[loc] = pv / n;
      if (var) var[loc] = pv / (n - 2);
      if (status) status[loc] = 0;
    }
  }
}

}  // namespace
}  // namespace lagp
