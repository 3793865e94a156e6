// select_dense.cu -- kernel (b) in the paper's own form: ALC from an explicit K_j^{-1},
// FP64.  The comparison for the Cholesky-row kernels (select.cu, select_mixed.cu).
//
// Gramacy & Apley, Sec. 3.2: every location keeps K_j^{-1}; adding the point s grows it
// by the partition inverse equations (SM "Partition inverse equations"),
//     a = K_j^{-1} k_j(s),   v = v_j(s) = K(s,s) - k_j(s)^T a,
//     K_{j+1}^{-1} = [[K_j^{-1} + a a^T / v, -a / v], [-a^T / v, 1 / v]],
// in O(j^2).  Each greedy step scores every candidate c by the reduction in variance at x
// of Eq. dxy.  With a_c = K_j^{-1} k_j(c) and g_j(c) = -a_c / v_j(c), its three terms sum
// to
//     v_j(x) - v_{j+1}(x) = (K(c,x) - k_j(x)^T a_c)^2 / v_j(c),
//     v_j(c) = K(c,c) - k_j(c)^T K_j^{-1} k_j(c),
// so a candidate costs the quadratic form k_j(c)^T K_j^{-1} k_j(c) -- O(j^2), here over
// the upper triangle of the symmetric K_j^{-1}, j(j+1)/2 multiply-adds -- plus the dot
// k_j(c)^T w with w = K_j^{-1} k_j(x), formed once per step.  The Cholesky-row kernels
// need O(j) per candidate and step for the same scores.
//
// Accuracy: v_j(c) is a difference of O(1) quantities, and the explicit inverse carries
// errors of order cond(K_j) eps into the quadratic form, so at small nuggets (large
// cond(K_j)) the scores -- and the designs -- can differ from the exact greedy ones.
// The predictive equations are evaluated on the selected design by kernel (c)
// (predict.cu, FP64 Cholesky).
//
// Layout: one persistent CTA per resident location.  Per CTA, scratch holds the rows
// Kc[i][c] = K(x_{d_i}, c) of the design's correlations with every candidate (coalesced
// over c; row i is appended when design point i is added) and the candidates'
// coordinates; K_j^{-1}, K(x, c) and the used flags live in shared memory.  K_j^{-1} is
// stored in full with rows and columns beyond j held at zero, so blocks of RB rows can
// run past j without tests.
#include <math.h>

#include "check.cuh"
#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {
namespace {

constexpr int DB = 256;        // threads per CTA
constexpr int RB = 8;          // rows of K_j^{-1} per block of the quadratic form
constexpr int kDenseCtas = 2;  // resident CTAs per SM
constexpr int kDenseMaxN = 128;

struct DenseParams {
  const double *X, *Z;
  int64_t N;
  int p;
  const double *XX;
  int64_t T;
  const int32_t *cand;
  int M, Mpad, n0, n, ld;  // ld: row stride of K_j^{-1} in shared memory (n rounded up to RB)
  double theta_inv, onepg;
  int32_t *idx;            // T x n selected indices (-1 rows for a failed location)
  double *Kc;              // gridDim.x slots of n x Mpad
  double *Xc;              // gridDim.x slots of p x Mpad
  int *queue;
};

// Score comparison as fractions cov^2 / v without dividing; ties to the smaller rank.
__device__ __forceinline__ bool dense_better(double a, double da, int ra, double b, double db,
                                             int rb) {
  const double l = a * db, r = b * da;
  return l > r || (l == r && ra < rb);
}

__global__ void __launch_bounds__(DB, kDenseCtas) select_dense_kernel(DenseParams P) {
  extern __shared__ __align__(16) double sm[];
  const int Mpad = P.Mpad, n = P.n, ld = P.ld, p = P.p;
  double *Ki = sm;                  // ld x ld
  double *kxc = Ki + ld * ld;       // Mpad: K(x, c)
  double *w = kxc + Mpad;           // ld: K_j^{-1} k_j(x), zero beyond j
  double *av = w + ld;              // ld: K_j^{-1} k_j(s)
  double *ks = av + ld;             // ld: k_j(s)
  double *kxd = ks + ld;            // ld: K(x, design point i)
  unsigned char *used = reinterpret_cast<unsigned char *>(kxd + ld);  // Mpad
  __shared__ double xl[kMaxP], xs[kMaxP];
  __shared__ double red_s[DB / 32], red_d[DB / 32];
  __shared__ int red_r[DB / 32];
  __shared__ double etab[64];
  if (threadIdx.x < 64) etab[threadIdx.x] = c_exp.tab[threadIdx.x];
  __shared__ int sh_loc, sh_best, sh_fail;
  __shared__ double sh_vinv;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double *Kc = P.Kc + (size_t)blockIdx.x * n * Mpad;
  double *Xc = P.Xc + (size_t)blockIdx.x * p * Mpad;
  // checked build: the layout above ends within the launch's dynamic shared memory
  if (!LAGP_CHK(reinterpret_cast<unsigned char *>(used + Mpad) - reinterpret_cast<unsigned char *>(sm),
                dynamic_smem_bytes() + 1u, 32))
    return;

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    const int64_t loc = sh_loc;
    if (loc >= P.T) break;
    const int32_t *cnd = P.cand + loc * P.M;
    int32_t *idx = P.idx + loc * n;
    const int M = P.M;
    if (tid < p) xl[tid] = P.XX[loc * p + tid];
    if (tid == 0) sh_fail = 0;
    for (int i = tid; i < ld * ld; i += DB) Ki[i] = 0.0;
    for (int i = tid; i < ld; i += DB) w[i] = 0.0;
    __syncthreads();
    if (P.n0 == n) {  // no greedy step: the design is the n0 nearest
      for (int i = tid; i < n; i += DB) idx[i] = cnd[i];
      continue;
    }
    // candidates' coordinates and K(x, c)
    for (int c = tid; c < M; c += DB) {
      if (!LAGP_CHK(cnd[c], P.N, 31)) {  // never read, never chosen
        kxc[c] = 0.0;
        used[c] = 1;
        for (int k = 0; k < p; k++) Xc[k * Mpad + c] = 0.0;
        continue;
      }
      const double *xc = P.X + (int64_t)cnd[c] * p;
      double acc = 0.0;
      for (int k = 0; k < p; k++) {
        const double xk = xc[k];
        Xc[k * Mpad + c] = xk;
        const double t = xl[k] - xk;
        acc = fma(t, t, acc);
      }
      kxc[c] = exp_nonpos(-acc * P.theta_inv, etab);
      used[c] = 0;
    }
    __syncthreads();

    for (int j = 0; j < n; j++) {
      int s = j;  // the start design: the n0 nearest in rank order
      if (j >= P.n0) {
        // ---- score every candidate against the j-point design (Eq. dxy) ----
        // w = K_j^{-1} k_j(x), with zeros beyond j
        for (int i = tid; i < j; i += DB) {
          const double *Kr = Ki + i * ld;
          double t = 0.0;
          for (int k = 0; k < j; k++) t = fma(Kr[k], kxd[k], t);
          w[i] = t;
        }
        __syncthreads();
        double bs = -1.0, bd = 1.0;
        int br = 0x7fffffff;
        for (int c = tid; c < M; c += DB) {
          if (used[c]) continue;
          const double *kc = Kc + c;
          double q = 0.0, cw = 0.0;
          for (int I = 0; I < j; I += RB) {
            double kI[RB], r[RB];
#pragma unroll
            for (int t = 0; t < RB; t++) {
              kI[t] = (I + t < j) ? kc[(size_t)(I + t) * Mpad] : 0.0;
              r[t] = 0.0;
            }
            // rows I..I+RB against the columns past the block: K_j^{-1}[k][I..I+RB) is
            // the block's column k by symmetry
            for (int k = I + RB; k < j; k++) {
              const double kk = kc[(size_t)k * Mpad];
              const double2 *Kr = reinterpret_cast<const double2 *>(Ki + k * ld + I);
#pragma unroll
              for (int t2 = 0; t2 < RB / 2; t2++) {
                const double2 e = Kr[t2];
                r[2 * t2] = fma(e.x, kk, r[2 * t2]);
                r[2 * t2 + 1] = fma(e.y, kk, r[2 * t2 + 1]);
              }
            }
            // the block's own upper triangle: q += k_i (K_ii k_i + 2 sum_{k > i} K_ik k_k)
#pragma unroll
            for (int t = 0; t < RB; t++) {
              const double *Kr = Ki + (I + t) * ld + I;
              double s2 = r[t];
#pragma unroll
              for (int u = t + 1; u < RB; u++) s2 = fma(Kr[u], kI[u], s2);
              q = fma(kI[t], fma(Kr[t], kI[t], 2.0 * s2), q);
              cw = fma(w[I + t], kI[t], cw);
            }
          }
          const double vc = P.onepg - q;           // v_j(c)
          const double cov = kxc[c] - cw;          // K(c,x) - k_j(x)^T K_j^{-1} k_j(c)
          if (vc > 0.0) {
            const double num = cov * cov;
            if (dense_better(num, vc, c, bs, bd, br)) { bs = num; bd = vc; br = c; }
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double os = __shfl_down_sync(0xffffffffu, bs, o);
          const double od = __shfl_down_sync(0xffffffffu, bd, o);
          const int orr = __shfl_down_sync(0xffffffffu, br, o);
          if (dense_better(os, od, orr, bs, bd, br)) { bs = os; bd = od; br = orr; }
        }
        if (lane == 0) { red_s[warp] = bs; red_d[warp] = bd; red_r[warp] = br; }
        __syncthreads();
        if (warp == 0) {
          bs = (lane < DB / 32) ? red_s[lane] : -1.0;
          bd = (lane < DB / 32) ? red_d[lane] : 1.0;
          br = (lane < DB / 32) ? red_r[lane] : 0x7fffffff;
          for (int o = 16; o > 0; o >>= 1) {
            const double os = __shfl_down_sync(0xffffffffu, bs, o);
            const double od = __shfl_down_sync(0xffffffffu, bd, o);
            const int orr = __shfl_down_sync(0xffffffffu, br, o);
            if (dense_better(os, od, orr, bs, bd, br)) { bs = os; bd = od; br = orr; }
          }
          if (lane == 0) sh_best = (br == 0x7fffffff) ? -1 : br;
        }
        __syncthreads();
        s = sh_best;
        if (s < 0) {  // no candidate with a positive conditional variance
          if (tid == 0) sh_fail = 1;
          break;
        }
      }
      // ---- add s: the partition inverse equations ----
      for (int i = tid; i < j; i += DB) ks[i] = Kc[(size_t)i * Mpad + s];
      if (tid < p) xs[tid] = Xc[tid * Mpad + s];
      __syncthreads();
      for (int i = tid; i < j; i += DB) {
        const double *Kr = Ki + i * ld;
        double t = 0.0;
        for (int k = 0; k < j; k++) t = fma(Kr[k], ks[k], t);
        av[i] = t;                                  // a = K_j^{-1} k_j(s)
      }
      __syncthreads();
      if (tid == 0) {
        double v = P.onepg;
        for (int k = 0; k < j; k++) v = fma(-ks[k], av[k], v);  // v_j(s)
        // (a used pivot is a start-design candidate the checked build dropped)
        if (!(v > 0.0) || used[s]) {
          sh_fail = 1;
        } else {
          sh_vinv = 1.0 / v;
          used[s] = 1;
          kxd[j] = kxc[s];
          idx[j] = cnd[s];
        }
      }
      __syncthreads();
      if (sh_fail) break;
      const double vinv = sh_vinv;
      for (int e = tid; e < (j + 1) * (j + 1); e += DB) {
        const int i = e / (j + 1), k = e - i * (j + 1);
        double val;
        if (i < j && k < j) val = fma(av[i] * vinv, av[k], Ki[i * ld + k]);
        else if (i < j) val = -av[i] * vinv;
        else if (k < j) val = -av[k] * vinv;
        else val = vinv;
        Ki[i * ld + k] = val;
      }
      // the new design point's correlations with every candidate, for the steps to come
      if (j + 1 < n) {
        for (int c = tid; c < M; c += DB) {
          double acc = 0.0;
          for (int k = 0; k < p; k++) {
            const double t = xs[k] - Xc[k * Mpad + c];
            acc = fma(t, t, acc);
          }
          Kc[(size_t)j * Mpad + c] = exp_nonpos(-acc * P.theta_inv, etab);
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (sh_fail)  // a failed location reports no design; kernel (c) gives it NaN and NOT_PD
      for (int i = tid; i < n; i += DB) idx[i] = -1;
  }
}

int dense_mpad(int M) { return (int)align_up((size_t)M, 32); }
int dense_ld(int n) { return (int)align_up((size_t)n, RB); }

size_t dense_smem_bytes(int Mpad, int n) {
  const int ld = dense_ld(n);
  return (size_t)(ld * ld + Mpad + 4 * ld) * sizeof(double) + align_up((size_t)Mpad, 16);
}

int dense_grid(int64_t T, int num_sms) {
  const int64_t g = (int64_t)num_sms * kDenseCtas;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

struct DenseLayout {
  size_t kc, xc, idx, pred, total;
};

// [queue | Kc | Xc | design indices | kernel (c) workspace]
DenseLayout dense_layout(int64_t T, int p, int n, int M, int num_sms) {
  const size_t G = (size_t)dense_grid(T, num_sms), Mpad = (size_t)dense_mpad(M);
  DenseLayout L;
  L.kc = align_up(G * n * Mpad * sizeof(double), 256);
  L.xc = align_up(G * p * Mpad * sizeof(double), 256);
  L.idx = align_up((size_t)(T > 0 ? T : 0) * n * sizeof(int32_t), 256);
  L.pred = predict_fp64_workspace_bytes(T, n, num_sms);
  L.total = 256 + L.kc + L.xc + L.idx + L.pred;
  return L;
}

}  // namespace

int select_dense_check_take(CheckRec *out) { return check_take_here(out); }

int select_dense_max_n() { return kDenseMaxN; }

size_t select_dense_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms) {
  return dense_layout(T, p, n, ncand, num_sms).total;
}

int select_dense_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  if (a.n > kDenseMaxN) return LAGP_ERR_UNSUPPORTED;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  const DenseLayout L = dense_layout(a.T, a.p, a.n, a.M, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  const int Mpad = dense_mpad(a.M);
  const int G = dense_grid(a.T, di.num_sms);
  char *w = static_cast<char *>(ws);
  DenseParams P;
  P.X = a.X; P.Z = a.Z; P.N = a.N; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Mpad = Mpad; P.n0 = a.n0; P.n = a.n; P.ld = dense_ld(a.n);
  P.theta_inv = 1.0 / a.theta; P.onepg = 1.0 + a.g;
  P.queue = reinterpret_cast<int *>(w);
  char *o = w + 256;
  P.Kc = reinterpret_cast<double *>(o);
  o += L.kc;
  P.Xc = reinterpret_cast<double *>(o);
  o += L.xc;
  P.idx = a.idx ? a.idx : reinterpret_cast<int32_t *>(o);
  o += L.idx;
  const size_t smem = dense_smem_bytes(Mpad, a.n);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(select_dense_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(P.queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_status(e);
  select_dense_kernel<<<G, DB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  PredictArgs pa;
  pa.X = a.X; pa.Z = a.Z; pa.p = a.p; pa.XX = a.XX; pa.T = a.T; pa.n = a.n; pa.nmax = a.n;
  pa.theta = a.theta; pa.g = a.g; pa.idx = P.idx;
  pa.B = BatchView{nullptr, nullptr, nullptr, 0, nullptr, nullptr};
  pa.mean = a.mean; pa.s2 = a.s2; pa.var = a.var; pa.status = a.status;
  return predict_fp64_launch(pa, o, L.pred, stream);
}

}  // namespace lagp
