// mle.cu -- the local maximum-likelihood lengthscale of each location's design.
//
// Gramacy & Apley, Sec. 4.2 (step 3 of the stagewise scheme): given the local design
// D_n(x), the lengthscale theta maximising the log likelihood Eq. gpk of its responses,
// found by Newton's method with the analytic derivatives Eqs. dl, d2l (Sec. 3.2):
//   l'  = -tr(K^-1 Kd)/2 + (n/2) w^T Kd w / psi,
//   l'' = -tr(K^-1 [Kdd - Kd K^-1 Kd])/2 + n/(2 psi) w^T [Kdd - 2 Kd K^-1 Kd] w
//         + n/(2 psi^2) (w^T Kd w)^2,
// with K = K(X_n, X_n) + g I, w = K^-1 Y, psi = Y^T w, Kd = dK/dtheta = K o R2 / theta^2 and
// Kdd = Kd o (R2 / theta^2 - 2 / theta) off the diagonal (R2 the squared distances; the
// diagonal does not depend on theta).
//
// The iteration is safeguarded: a bracket [lo, hi] of the maximum is narrowed by the sign
// of l'; the Newton step is taken when l'' < 0 and it stays strictly inside the bracket,
// otherwise the iterate goes to the end of [tmin, tmax] uphill of theta if that end has
// not been evaluated, else to the bracket's midpoint; it stops when a step is at most
// tol * theta (the new point is returned), when l' = 0, or at an end of [tmin, tmax]
// where l' points outward.
//
// One CTA per location.  Per iteration, in FP64: K and Kd (one exp per pair), the
// Cholesky factor (fp64_chol.cuh), L^-1 by forward substitution (right-looking, one barrier
// per column), K^-1 = L^-T L^-1 and the O(n^2) vector terms; the n^3 product K^-1 Kd behind
// tr((K^-1 Kd)^2) runs in float-float on the FP32 pipes (K^-1 has large entries of both
// signs, so plain FP32 would leave l'' without a correct digit; float-float keeps about
// 48 bits per product).  The matrices live in shared memory
// when they fit, else in a per-CTA slot of the workspace.
#include <math.h>

#include "ff.cuh"
#include "fp64_chol.cuh"
#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {
namespace {

constexpr int LB = 256;                      // threads per CTA
constexpr size_t kSmemMle = 110 * 1024;      // largest per-CTA set kept in shared memory
constexpr int kSums = 7;                     // block sums per Newton iteration

struct MleParams {
  const double *X, *Z;
  int p;
  int64_t T;
  const int32_t *idx;  // T x n design indices
  int n;
  double theta0;
  const double *theta0_loc;  // may be null
  double g, tmin, tmax, tol;
  int maxit;
  double *theta_out;
  int32_t *iters;
  int8_t *status;
  unsigned char *slots;  // per-CTA buffers when not in shared memory
  size_t slot_bytes;
  int in_smem;
  int *queue;
};

// Per-CTA buffers: three n x n FP64 matrices (L then K^-1, Kd, L^-1), four FP64 vectors
// and the design's coordinates (up to kMaxP per point).  Squared distances are recomputed
// from the coordinates where needed (p operations each, in the same order every time),
// which leaves room for three CTAs per SM at n = 50: the Cholesky's pivot chain is
// sequential, and more locations in flight hide it.
size_t mle_set_bytes(int n) {
  const size_t nn = (size_t)n * n;
  return nn * 3 * sizeof(double) + (size_t)n * (4 + kMaxP) * sizeof(double);
}

// Lane 0's shuffle-tree sum of v over its warp.
__device__ __forceinline__ double warp_tree_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(LB) mle_fp64_kernel(MleParams P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nmax = P.n;
  unsigned char *base = P.in_smem ? smraw : P.slots + (size_t)blockIdx.x * P.slot_bytes;
  const size_t nn = (size_t)nmax * nmax;
  double *Lm = reinterpret_cast<double *>(base);  // K, its Cholesky factor L, then K^-1
  double *Kd = Lm + nn;
  double *Ki = Kd + nn;
  double *Y = Ki + nn, *w = Y + nmax, *kdw = w + nmax, *rl = kdw + nmax;
  double *xd = rl + nmax;    // nmax x p coordinates of the design
  __shared__ double etab[64];
  __shared__ double red[kSums][LB / 32];
  __shared__ double sh_th, sh_lo, sh_hi;
  __shared__ int sh_loc, sh_fail, sh_done, sh_lo_open, sh_hi_open, sh_it, sh_st;
  const int tid = threadIdx.x;
  if (tid < 64) etab[tid] = c_exp.tab[tid];
  const int n = P.n, p = P.p, lda = n;

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    if (sh_loc >= P.T) break;
    const int64_t loc = sh_loc;
    const int32_t *d = P.idx + loc * n;
    if (tid == 0) {
      sh_fail = d[0] < 0;  // no design (its screen failed)
      const double t0 = P.theta0_loc ? P.theta0_loc[loc] : P.theta0;
      sh_th = fmin(fmax(t0, P.tmin), P.tmax);
      sh_lo = P.tmin;
      sh_hi = P.tmax;
      sh_lo_open = sh_hi_open = 1;
      sh_done = 0;
      sh_it = 0;
      sh_st = LAGP_ERR_NO_CONVERGENCE;
    }
    __syncthreads();
    if (!sh_fail) {
      for (int i = tid; i < n; i += LB) Y[i] = P.Z[d[i]];
      for (int e = tid; e < n * p; e += LB) xd[e] = P.X[(int64_t)d[e / p] * p + e % p];
    }
    __syncthreads();  // the coordinates are read by other threads below
    // squared distance of design points a and b
    auto r2of = [&](int a, int b) {
      double r2 = 0.0;
      for (int k = 0; k < p; k++) {
        const double t = xd[a * p + k] - xd[b * p + k];
        r2 = fma(t, t, r2);
      }
      return r2;
    };
    while (!sh_fail && !sh_done) {
      const double th = sh_th;
      const double tinv = 1.0 / th, tinv2 = tinv * tinv;
      // K (lower triangle) and Kd (full): one exp per pair a > b, mirrored
      const int ntri = n * (n + 1) / 2;
      for (int e = tid; e < ntri; e += LB) {
        const int a = tri_row(e), b = e - a * (a + 1) / 2;
        if (a == b) {
          Lm[a * lda + a] = 1.0 + P.g;
          Kd[a * lda + a] = 0.0;
        } else {
          const double r2 = r2of(a, b);
          const double k = exp_nonpos(-r2 * tinv, etab);
          Lm[a * lda + b] = k;
          const double kd = k * r2 * tinv2;
          Kd[a * lda + b] = kd;
          Kd[b * lda + a] = kd;
        }
      }
      chol_flat_fp64(Lm, n, lda, 0, rl, &sh_fail);
      if (sh_fail) break;
      // X = L^-1 (lower triangle, in Ki's storage): x_ic = -(sum_{c<=m<i} l_im x_mc) / l_ii,
      // x_ii = 1 / l_ii.  Right-looking: at step m every entry (i > m, c <= m) takes its
      // term l_im x_mc -- the same terms in the same order as the row-by-row sums -- and
      // the thread that adds the last term of row m + 1 finishes that entry, so a step is
      // one barrier and all threads share its FP64 work.  Row m + 1 runs in a loop of its
      // own: in the shared loop its multiply by 1 / l_ii would be a predicated FP64
      // instruction issued by every warp.
      double *Xb = Ki;
      for (int e = tid; e < ntri; e += LB) {
        const int a = tri_row(e), b = e - a * (a + 1) / 2;
        Xb[a * lda + b] = (a == b) ? rl[a] : 0.0;
      }
      __syncthreads();
      for (int m = 0; m < n - 1; m++) {
        const int w1 = m + 1, cnt = (n - 1 - m) * w1;
        {  // row m + 1: its last term, then the division by its pivot
          const int i = m + 1;
          for (int c = tid; c < w1; c += LB)
            Xb[i * lda + c] = -fma(Lm[i * lda + m], Xb[m * lda + c], Xb[i * lda + c]) * rl[i];
        }
        for (int e = w1 + tid; e < cnt; e += LB) {
          const int i = m + 1 + e / w1, c = e % w1;
          Xb[i * lda + c] = fma(Lm[i * lda + m], Xb[m * lda + c], Xb[i * lda + c]);
        }
        __syncthreads();
      }
      // K^-1 = X^T X (both triangles) into L's storage, which is no longer needed
      double *KiM = Lm;
      for (int e = tid; e < ntri; e += LB) {
        const int a = tri_row(e), b = e - a * (a + 1) / 2;
        double s = 0.0;
        for (int m = a; m < n; m++) s = fma(Xb[m * lda + a], Xb[m * lda + b], s);
        KiM[a * lda + b] = s;
        KiM[b * lda + a] = s;
      }
      __syncthreads();
      // w = K^-1 Y, then Kd w
      for (int a = tid; a < n; a += LB) {
        double s = 0.0;
        for (int b = 0; b < n; b++) s = fma(KiM[a * lda + b], Y[b], s);
        w[a] = s;
      }
      __syncthreads();
      for (int a = tid; a < n; a += LB) {
        double s = 0.0;
        for (int b = 0; b < n; b++) s = fma(Kd[a * lda + b], w[b], s);
        kdw[a] = s;
      }
      __syncthreads();
      // per-row pieces of psi, w^T Kd w, w^T Kdd w, kdw^T K^-1 kdw, tr(K^-1 Kd), tr(K^-1 Kdd)
      double psi = 0.0, q3 = 0.0, q1 = 0.0, q2 = 0.0, t1 = 0.0, t3 = 0.0;
      for (int a = tid; a < n; a += LB) {
        psi = fma(Y[a], w[a], psi);
        q3 = fma(w[a], kdw[a], q3);
        double sdd = 0.0, sq2 = 0.0, st1 = 0.0, st3 = 0.0;
        for (int b = 0; b < n; b++) {
          const double kd = Kd[a * lda + b], kdd = kd * (r2of(a, b) * tinv2 - 2.0 * tinv);
          const double ki = KiM[a * lda + b];
          sdd = fma(kdd, w[b], sdd);
          sq2 = fma(ki, kdw[b], sq2);
          st1 = fma(ki, kd, st1);
          st3 = fma(ki, kdd, st3);
        }
        q1 = fma(w[a], sdd, q1);
        q2 = fma(kdw[a], sq2, q2);
        t1 += st1;
        t3 += st3;
      }
      __syncthreads();
      // tr((K^-1 Kd)^2) = sum_ab A_ab A_ba with A = K^-1 Kd, the n^3 term: formed in
      // float-float on the FP32 pipes (compensated dots, about 2^-48 per product).  It
      // enters l'' only, which sets the Newton step, not the root l' = 0 the iteration
      // converges to.  K^-1 and Kd are converted in place (their FP64 uses are done), one
      // float-float pair per FP64 slot.
      float2 *Kif = reinterpret_cast<float2 *>(KiM), *Kdf = reinterpret_cast<float2 *>(Kd);
      for (int e = tid; e < n * n; e += LB) {
        const ff ki = ff_from_double(KiM[e]), kd = ff_from_double(Kd[e]);
        Kif[e] = make_float2(ki.h, ki.l);
        Kdf[e] = make_float2(kd.h, kd.l);
      }
      __syncthreads();
      // The pairs a <= b, all lanes busy: (a == b ? 1 : 2) A_ab into slot (a, b) and A_ba into
      // slot (b, a) of the dead L^-1 storage (for a == b both are A_aa, in one slot).
      for (int e = tid; e < ntri; e += LB) {
        const int b = tri_row(e), a = e - b * (b + 1) / 2;
        ffacc sab{0.0f, 0.0f}, sba{0.0f, 0.0f};
        for (int m = 0; m < n; m++) {
          const float2 x1 = Kif[a * lda + m], y1 = Kdf[m * lda + b];
          const float2 x2 = Kif[b * lda + m], y2 = Kdf[m * lda + a];
          ffacc_add_prod(sab, ff{x1.x, x1.y}, ff{y1.x, y1.y});
          ffacc_add_prod(sba, ff{x2.x, x2.y}, ff{y2.x, y2.y});
        }
        const double vab = (double)sab.h + (double)sab.l, vba = (double)sba.h + (double)sba.l;
        Xb[a * lda + b] = (a == b ? 1.0 : 2.0) * vab;
        if (a != b) Xb[b * lda + a] = vba;
      }
      __syncthreads();
      // each thread adds its pairs in the order of the row-major (a, b) scan
      double t2p = 0.0;
      for (int e = tid; e < n * n; e += LB) {
        const int a = e / n, b = e % n;
        if (b < a) continue;
        t2p = fma(Xb[a * lda + b], Xb[b * lda + a], t2p);
      }
      // The seven block sums: a shuffle tree per warp, then thread 0 adds the warp totals in
      // warp order.  The six row sums are exactly +0.0 in a warp none of whose threads holds
      // a row (warp * 32 >= n), whose tree would give +0.0, so such warps skip it.
      {
        const int lane = tid & 31, warp = tid >> 5;
        double v[kSums] = {psi, q3, q1, q2, t1, t3, t2p};
        if (warp * 32 < n) {
#pragma unroll
          for (int j = 0; j < kSums - 1; j++) v[j] = warp_tree_sum(v[j]);
        }
        v[kSums - 1] = warp_tree_sum(v[kSums - 1]);
        if (lane == 0) {
#pragma unroll
          for (int j = 0; j < kSums; j++) red[j][warp] = v[j];
        }
      }
      __syncthreads();
      if (tid == 0) {
        double v[kSums];
#pragma unroll
        for (int j = 0; j < kSums; j++) {
          double s = 0.0;
          for (int w = 0; w < LB / 32; w++) s += red[j][w];
          v[j] = s;
        }
        psi = v[0];
        q3 = v[1];
        q1 = v[2];
        q2 = v[3];
        t1 = v[4];
        t3 = v[5];
        const double t2 = v[6];
        const double dn = n;
        const double d1 = -0.5 * t1 + dn / 2.0 * q3 / psi;
        const double d2 = -0.5 * (t3 - t2) + dn / (2.0 * psi) * (q1 - 2.0 * q2) +
                          dn / (2.0 * psi * psi) * q3 * q3;
        sh_it++;
        bool stop = false;
        if (d1 == 0.0) {
          stop = true;
        } else if (d1 > 0.0) {
          sh_lo = th;
          sh_lo_open = 0;
          stop = th >= P.tmax;
        } else {
          sh_hi = th;
          sh_hi_open = 0;
          stop = th <= P.tmin;
        }
        if (stop) {
          sh_st = 0;
          sh_done = 1;
        } else {
          double tn = (d2 < 0.0) ? th - d1 / d2 : NAN;
          if (!(tn > sh_lo && tn < sh_hi)) {
            if (d1 > 0.0 && sh_hi_open) tn = sh_hi;  // uphill to an end not yet evaluated
            else if (d1 < 0.0 && sh_lo_open) tn = sh_lo;
            else tn = 0.5 * (sh_lo + sh_hi);
          }
          const bool small = fabs(tn - th) <= P.tol * th;
          sh_th = tn;
          if (small) {
            sh_st = 0;
            sh_done = 1;
          } else if (sh_it >= P.maxit) {
            sh_done = 1;  // sh_st stays LAGP_ERR_NO_CONVERGENCE
          }
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
      P.theta_out[loc] = sh_fail ? NAN : sh_th;
      if (P.iters) P.iters[loc] = sh_it;
      if (P.status) P.status[loc] = sh_fail ? (int8_t)LAGP_ERR_NOT_PD : (int8_t)sh_st;
    }
  }
}

int mle_grid(int64_t T, int n, const DevInfo &di, bool in_smem) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mle_fp64_kernel, LB,
                                                    in_smem ? mle_set_bytes(n) : 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t g = (int64_t)di.num_sms * per_sm;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

// At most 2048 / LB CTAs per SM: the bound used to size the per-CTA slots.
int mle_grid_bound(int64_t T, int num_sms) {
  const int64_t g = (int64_t)num_sms * (2048 / LB);
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

bool mle_in_smem(int n) { return mle_set_bytes(n) <= kSmemMle; }

}  // namespace

size_t mle_workspace_bytes(int64_t T, int32_t n, int num_sms) {
  size_t b = 256;
  if (!mle_in_smem(n)) b += align_up((size_t)mle_grid_bound(T, num_sms) * align_up(mle_set_bytes(n), 256), 256);
  return b;
}

int mle_launch(const MleArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();  // this translation unit's copy of the exp constants
  if (st) return st;
  if (ws_bytes < mle_workspace_bytes(a.T, a.n, di.num_sms)) return LAGP_ERR_INVALID_ARG;
  const bool sm = mle_in_smem(a.n);
  const size_t smem = sm ? mle_set_bytes(a.n) : 0;
  cudaError_t e = cudaFuncSetAttribute(mle_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  int G = mle_grid(a.T, a.n, di, sm);
  const int Gb = mle_grid_bound(a.T, di.num_sms);
  if (G > Gb) G = Gb;
  char *w = static_cast<char *>(ws);
  MleParams P;
  P.X = a.X; P.Z = a.Z; P.p = a.p; P.T = a.T; P.idx = a.idx; P.n = a.n;
  P.theta0 = a.theta0; P.theta0_loc = a.theta0_loc; P.g = a.g; P.tmin = a.tmin; P.tmax = a.tmax;
  P.tol = a.tol; P.maxit = a.maxit;
  P.theta_out = a.theta_out; P.iters = a.iters; P.status = a.status;
  P.queue = reinterpret_cast<int *>(w);
  P.in_smem = sm ? 1 : 0;
  P.slot_bytes = align_up(mle_set_bytes(a.n), 256);
  P.slots = sm ? nullptr : reinterpret_cast<unsigned char *>(w + 256);
  e = cudaMemsetAsync(P.queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_status(e);
  mle_fp64_kernel<<<G, LB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

int mle_prepare() { return exp_table_upload(); }

}  // namespace lagp
