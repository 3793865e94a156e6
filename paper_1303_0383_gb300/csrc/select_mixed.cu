// select_mixed.cu -- kernels (b)+(c), mixed precision: float-float candidate screen on the
// FP32 pipes, FP64 decisions and FP64 predictive equations.
//
// Gramacy & Apley, Sec. 3: the greedy local design adds, at each step, the candidate that
// maximises the ALC reduction cov_j(x,c)^2 / v_j(c) (Eq. dxy; SM Eq. dxy2).  The screen
// carries, for every candidate, its row of the bordered Cholesky factor, v_j(c) and
// cov_j(x,c) exactly as the FP64 kernel does (select.cu), but in float-float (FP32 pairs,
// ff.cuh): on this GPU FP32 runs 58x faster than FP64, and plain FP32 cannot be used
// because v_j(c) ~ g = 1e-6 is the difference of O(1) quantities.
//
// Decisions stay FP64-exact where they are close: when the screen's second-best score is
// within DELTA (relative) of its best, the design's FP64 Cholesky factor is rebuilt from
// scratch and every candidate within DELTA is re-scored in FP64 (forward substitution,
// one warp per candidate), the FP64 best winning with ties to the nearer candidate.
// Otherwise the screen's best is taken.  DELTA = 1e-5 is about five times the largest
// screen-vs-FP64 score discrepancy measured by emulation (2e-6 of the best score).
//
// After the last step the predictive equations (Eqs. predgp, preds2) are evaluated in
// FP64 on the final design: K_n augmented with the columns k(x) and Y is factored by a
// right-looking Cholesky, which performs for every entry the same subtractions in the
// same order as the row-by-row factorisation and forward substitution, so mu, s2 and V
// carry FP64 accuracy whatever precision screened the candidates.
#include <math.h>

#include "ff.cuh"
#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {
namespace {

constexpr int MB = 256;            // threads per CTA
constexpr float DELTA = 1e-5f;     // near-tie margin for the FP64 re-score
constexpr int RESCORE_CAP = 64;    // candidates re-scored per pass

struct MixParams {
  const double *X, *Z;
  int p;
  const double *XX;
  int64_t T;
  const int32_t *cand;
  int M, Mpad, n0, n;
  double theta, theta_inv, g, onepg;
  double *mean, *s2, *var;
  int32_t *idx;
  int8_t *status;
  ff *U;         // slots of n x Mpad
  ff *Xr;        // slots of p x Mpad: candidate coordinates minus x
  double *A;     // slots of n x (n + 2): FP64 factorisation
  int *queue;
  int *rescores; // count of FP64 re-score passes (diagnostics)
};

// exp(a) for a <= 0 in float-float (Tang's table-driven method with N = 64, see
// fp64_exp.cuh): a = k ln2/64 + r, exp(r) - 1 = r + r^2/2 + r^3/6 + r^4/24 + r^5/120 with
// the first two terms in float-float and the rest in FP32 (they are below 3e-8).
__device__ __forceinline__ ff exp_ff(ff a, const float *tabh, const float *tabl) {
  if (a.h < -87.0f) return ff{0.0f, 0.0f};
  const float magic = 12582912.0f;  // 1.5 * 2^23
  const float t = __fmaf_rn(a.h, c_exp.inv_ln2_64f, magic);
  const float kf = __fsub_rn(t, magic);
  const int k = __float_as_int(t) - 0x4B400000;
  const float r1 = __fmaf_rn(-kf, c_exp.c1, a.h);  // exact
  const float p2h = __fmul_rn(kf, c_exp.c2);
  const float p2l = __fmaf_rn(kf, c_exp.c2, -p2h);
  const ff s = two_sum(r1, -p2h);
  const float rl = __fadd_rn(__fsub_rn(__fsub_rn(s.l, p2l), __fmul_rn(kf, c_exp.c3)), a.l);
  const ff r = fast_two_sum(s.h, rl);
  const float sqh = __fmul_rn(r.h, r.h);
  const float sql = __fmaf_rn(2.0f * r.h, r.l, __fmaf_rn(r.h, r.h, -sqh));
  const float P = __fmul_rn(__fmul_rn(r.h, sqh),
                            __fmaf_rn(r.h, __fmaf_rn(r.h, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f));
  const ff e = two_sum(r.h, 0.5f * sqh);
  const ff E = fast_two_sum(e.h, __fadd_rn(__fadd_rn(e.l, r.l), __fmaf_rn(0.5f, sql, P)));
  const int j = k & 63;
  const float Th = tabh[j], Tl = tabl[j];
  const float ph = __fmul_rn(Th, E.h);
  const float pl = __fmaf_rn(Th, E.h, -ph);
  const ff s2 = two_sum(Th, ph);
  const float low = __fadd_rn(__fadd_rn(s2.l, pl), __fmaf_rn(Th, E.l, __fmaf_rn(Tl, E.h, Tl)));
  const ff res = fast_two_sum(s2.h, low);
  const float sc = __int_as_float(((k >> 6) + 127) << 23);
  return ff{__fmul_rn(res.h, sc), __fmul_rn(res.l, sc)};
}

__device__ __forceinline__ bool frac_better(double a, double da, int ra, double b, double db,
                                            int rb) {
  const double l = a * db, r = b * da;
  return l > r || (l == r && ra < rb);
}

// Right-looking FP64 Cholesky of the j x j design matrix held in A (row-major, leading
// dimension lda) together with naug extra columns (forward substitution of them).  The
// matrix entries are built by the caller.  Returns false (in *fail) on a pivot <= 0.
__device__ void chol_aug_fp64(double *A, int j, int lda, int naug, int *fail) {
  const int tid = threadIdx.x;
  for (int k = 0; k < j; k++) {
    if (tid == 0) {
      const double d = A[k * lda + k];
      if (!(d > 0.0)) *fail = 1;
      A[k * lda + k] = sqrt(d);
    }
    __syncthreads();
    if (*fail) return;
    const double lkk = A[k * lda + k];
    for (int i = k + 1 + tid; i < j; i += MB) A[i * lda + k] = A[i * lda + k] / lkk;
    if (tid < naug) A[k * lda + j + tid] = A[k * lda + j + tid] / lkk;
    __syncthreads();
    const int w = j - k - 1 + naug;
    const int rows = j - k - 1;
    for (int q = tid; q < rows * w; q += MB) {
      const int ii = k + 1 + q / w;
      const int ll = q % w;
      if (ll < rows) {
        const int l = k + 1 + ll;
        if (l <= ii) A[ii * lda + l] = fma(-A[ii * lda + k], A[l * lda + k], A[ii * lda + l]);
      } else {
        const int a = ll - rows;
        A[ii * lda + j + a] = fma(-A[ii * lda + k], A[k * lda + j + a], A[ii * lda + j + a]);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double corr64(const double *a, const double *b, int p, double theta_inv,
                                         const double *etab) {
  double acc = 0.0;
  for (int k = 0; k < p; k++) {
    const double t = a[k] - b[k];
    acc = fma(t, t, acc);
  }
  return exp_nonpos(-acc * theta_inv, etab);
}

__global__ void __launch_bounds__(MB, 2) select_mixed_kernel(MixParams P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Mpad = P.Mpad, n = P.n, p = P.p, M = P.M;
  ff *vff = reinterpret_cast<ff *>(smraw);       // Mpad
  ff *cff = vff + Mpad;                          // Mpad
  ff *srow = cff + Mpad;                         // n
  int *dr = reinterpret_cast<int *>(srow + n);   // n: ranks of the design, in order
  int *rlist = dr + n;                           // RESCORE_CAP
  unsigned char *used = reinterpret_cast<unsigned char *>(rlist + RESCORE_CAP);  // Mpad
  __shared__ float tabh[64], tabl[64];
  __shared__ double etab[64];
  __shared__ double xl[kMaxP];
  __shared__ ff xs[kMaxP];
  __shared__ float red_s1[MB / 32], red_s2[MB / 32];
  __shared__ int red_r1[MB / 32];
  __shared__ double red_n[MB / 32], red_d[MB / 32];
  __shared__ int sh_loc, sh_best, sh_fail, sh_near, sh_nlist;
  __shared__ ff sh_inv, sh_uxj;
  if (threadIdx.x < 64) {
    tabh[threadIdx.x] = c_exp.tabf_h[threadIdx.x];
    tabl[threadIdx.x] = c_exp.tabf_l[threadIdx.x];
    etab[threadIdx.x] = c_exp.tab[threadIdx.x];
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  ff *U = P.U + (size_t)blockIdx.x * n * Mpad;
  ff *Xr = P.Xr + (size_t)blockIdx.x * p * Mpad;
  const int lda = n + 2;
  double *A = P.A + (size_t)blockIdx.x * n * lda;
  const ff onepg = ff_from_double(P.onepg);
  const ff thinv = ff_from_double(P.theta_inv);

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    const int64_t loc = sh_loc;
    if (loc >= P.T) break;
    const int32_t *cnd = P.cand + loc * M;
    if (tid < p) xl[tid] = P.XX[loc * p + tid];
    if (tid == 0) sh_fail = 0;
    __syncthreads();
    // coordinates relative to x (float-float), v = 1+g, cov_0(x,c) = K(x,c) in FP64
    for (int c = tid; c < M; c += MB) {
      const double *xc = P.X + (int64_t)cnd[c] * p;
      double acc = 0.0;
      for (int k = 0; k < p; k++) {
        const double dk = xc[k] - xl[k];
        Xr[k * Mpad + c] = ff_from_double(dk);
        acc = fma(dk, dk, acc);
      }
      vff[c] = onepg;
      cff[c] = ff_from_double(exp_nonpos(-acc * P.theta_inv, etab));
      used[c] = 0;
    }
    __syncthreads();

    for (int j = 0; j < n; j++) {
      const int s = (j < P.n0) ? j : sh_best;
      if (s < 0) {  // nothing admissible left (uniform across the block)
        if (tid == 0) sh_fail = 1;
        __syncthreads();
        break;
      }
      if (tid == 0) {
        const ff vs = vff[s];
        if (!(vs.h > 0.0f)) {
          sh_fail = 1;
        } else {
          dr[j] = s;
          used[s] = 1;
          const ff inv = ff_rcp(ff_sqrt(vs));
          sh_inv = inv;
          sh_uxj = ff_mul(cff[s], inv);
        }
      }
      for (int i = tid; i < j; i += MB) srow[i] = U[(size_t)i * Mpad + s];
      if (tid < p) xs[tid] = Xr[tid * Mpad + s];
      __syncthreads();
      if (sh_fail) break;
      if (j == n - 1) break;
      const ff inv = sh_inv, uxj = sh_uxj;
      const bool want = j + 1 >= P.n0;
      float b1 = -1.0f, b2 = -1.0f;
      int r1 = 0x7fffffff;
      for (int c = tid; c < M; c += MB) {
        if (used[c]) continue;
        // squared distance to the new point, from coordinates relative to x
        float dh = 0.0f, dl = 0.0f;
        for (int k = 0; k < p; k++) {
          const ff a = xs[k], b = Xr[k * Mpad + c];
          const ff df = two_sum(a.h, -b.h);
          const float dfl = __fadd_rn(df.l, __fsub_rn(a.l, b.l));
          const float ph = __fmul_rn(df.h, df.h);
          const float pl = __fmaf_rn(2.0f * df.h, dfl, __fmaf_rn(df.h, df.h, -ph));
          const ff sacc = two_sum(dh, ph);
          dh = sacc.h;
          dl = __fadd_rn(__fadd_rn(sacc.l, dl), pl);
        }
        const ff d2 = fast_two_sum(dh, dl);
        ff t = exp_ff(ff_neg(ff_mul(d2, thinv)), tabh, tabl);   // K(s, c)
        const ff *Uc = U + c;
        for (int i = 0; i < j; i++) t = ff_sub_prod_acc(t, srow[i], Uc[(size_t)i * Mpad]);
        const ff u = ff_mul(t, inv);                              // u_c[j]
        U[(size_t)j * Mpad + c] = u;
        const ff v = ff_sub(vff[c], ff_mul(u, u));
        const ff cx = ff_sub(cff[c], ff_mul(uxj, u));
        vff[c] = v;
        cff[c] = cx;
        if (want && v.h > 0.0f) {
          const float sc = __fdiv_rn(__fmul_rn(cx.h, cx.h), v.h);
          if (sc > b1 || (sc == b1 && c < r1)) {
            b2 = b1;
            b1 = sc;
            r1 = c;
          } else if (sc > b2) {
            b2 = sc;
          }
        }
      }
      if (!want) {
        __syncthreads();
        continue;
      }
      // best and second-best screen scores over the block
      for (int o = 16; o > 0; o >>= 1) {
        const float ob1 = __shfl_down_sync(0xffffffffu, b1, o);
        const float ob2 = __shfl_down_sync(0xffffffffu, b2, o);
        const int or1 = __shfl_down_sync(0xffffffffu, r1, o);
        if (ob1 > b1 || (ob1 == b1 && or1 < r1)) {
          b2 = fmaxf(b1, ob2);
          b1 = ob1;
          r1 = or1;
        } else {
          b2 = fmaxf(b2, ob1);
        }
      }
      if (lane == 0) {
        red_s1[warp] = b1;
        red_s2[warp] = b2;
        red_r1[warp] = r1;
      }
      __syncthreads();
      if (tid == 0) {
        float B1 = red_s1[0], B2 = red_s2[0];
        int R1 = red_r1[0];
        for (int w = 1; w < MB / 32; w++) {
          const float o1 = red_s1[w], o2 = red_s2[w];
          const int orr = red_r1[w];
          if (o1 > B1 || (o1 == B1 && orr < R1)) {
            B2 = fmaxf(B1, o2);
            B1 = o1;
            R1 = orr;
          } else {
            B2 = fmaxf(B2, o1);
          }
        }
        sh_best = (R1 == 0x7fffffff) ? -1 : R1;
        sh_near = (R1 != 0x7fffffff && B2 >= B1 * (1.0f - DELTA)) ? 1 : 0;
        sh_nlist = 0;
      }
      __syncthreads();
      if (!sh_near) continue;
      // ---- FP64 re-score of the near-tied candidates (rare) ----
      if (tid == 0 && P.rescores) atomicAdd(P.rescores, 1);
      const int jd = j + 1;  // design size now
      const float Bbest = [&] {
        const ff v = vff[sh_best], cx = cff[sh_best];
        return __fdiv_rn(__fmul_rn(cx.h, cx.h), v.h);
      }();
      for (int c = tid; c < M; c += MB) {
        if (used[c]) continue;
        const ff v = vff[c], cx = cff[c];
        if (!(v.h > 0.0f)) continue;
        const float sc = __fdiv_rn(__fmul_rn(cx.h, cx.h), v.h);
        if (sc >= Bbest * (1.0f - 2.0f * DELTA)) {
          const int pos = atomicAdd(&sh_nlist, 1);
          if (pos < RESCORE_CAP) rlist[pos] = c;
        }
      }
      // FP64 factor of the current design with k(x) as an extra column
      for (int q = tid; q < jd * (jd + 1); q += MB) {
        const int a = q / (jd + 1), b = q % (jd + 1);
        const double *xa = P.X + (int64_t)cnd[dr[a]] * p;
        if (b < jd && b > a) continue;  // only the lower triangle is read
        double val;
        if (b < jd) val = (a == b) ? P.onepg : corr64(xa, P.X + (int64_t)cnd[dr[b]] * p, p, P.theta_inv, etab);
        else val = corr64(xa, xl, p, P.theta_inv, etab);
        A[a * lda + b] = val;
      }
      __syncthreads();
      // chol_aug_fp64 uses columns [0, jd) and jd as the augmented one (lda = n + 2 >= jd + 1)
      chol_aug_fp64(A, jd, lda, 1, &sh_fail);
      if (sh_fail) break;
      // more near-ties than the list holds: re-score every remaining candidate
      const bool all = sh_nlist > RESCORE_CAP;
      const int nl = all ? M : sh_nlist;
      double bn = -1.0, bd = 1.0;
      int br = 0x7fffffff;
      for (int item = warp; item < nl; item += MB / 32) {
        const int c = all ? item : rlist[item];
        if (used[c]) continue;
        const double *xc = P.X + (int64_t)cnd[c] * p;
        double tv[kMaxN / 32];
#pragma unroll
        for (int r = 0; r < kMaxN / 32; r++) {
          const int i = 32 * r + lane;
          tv[r] = (i < jd) ? corr64(P.X + (int64_t)cnd[dr[i]] * p, xc, p, P.theta_inv, etab) : 0.0;
        }
        double vsum = P.onepg;
        double cov = corr64(xl, xc, p, P.theta_inv, etab);
        for (int m = 0; m < jd; m++) {
          double own = 0.0;
#pragma unroll
          for (int r = 0; r < kMaxN / 32; r++)
            if (32 * r + lane == m) own = tv[r];
          const double um_l = own / A[m * lda + m];
          const double um = __shfl_sync(0xffffffffu, um_l, m & 31);
          vsum = fma(-um, um, vsum);
          cov = fma(-A[m * lda + jd], um, cov);
#pragma unroll
          for (int r = 0; r < kMaxN / 32; r++) {
            const int i = 32 * r + lane;
            if (i > m && i < jd) tv[r] = fma(-A[i * lda + m], um, tv[r]);
          }
        }
        if (vsum > 0.0) {
          const double num = cov * cov;
          if (frac_better(num, vsum, c, bn, bd, br)) {
            bn = num;
            bd = vsum;
            br = c;
          }
        }
      }
      if (lane == 0) {
        red_n[warp] = bn;
        red_d[warp] = bd;
        red_r1[warp] = br;
      }
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < MB / 32; w++)
          if (frac_better(red_n[w], red_d[w], red_r1[w], bn, bd, br)) {
            bn = red_n[w];
            bd = red_d[w];
            br = red_r1[w];
          }
        if (br != 0x7fffffff) sh_best = br;
      }
      __syncthreads();
    }
    __syncthreads();
    if (!sh_fail) {
      // FP64 predictive equations on the final design: factor [K_n | k(x) | Y]
      for (int q = tid; q < n * (n + 2); q += MB) {
        const int a = q / (n + 2), b = q % (n + 2);
        if (b < n && b > a) continue;  // only the lower triangle is read
        const double *xa = P.X + (int64_t)cnd[dr[a]] * p;
        double val;
        if (b < n) val = (a == b) ? P.onepg : corr64(xa, P.X + (int64_t)cnd[dr[b]] * p, p, P.theta_inv, etab);
        else if (b == n) val = corr64(xa, xl, p, P.theta_inv, etab);
        else val = P.Z[cnd[dr[a]]];
        A[a * lda + b] = val;
      }
      __syncthreads();
      chol_aug_fp64(A, n, lda, 2, &sh_fail);
    }
    __syncthreads();
    if (tid == 0) {
      if (sh_fail) {
        if (P.status) P.status[loc] = (int8_t)LAGP_ERR_NOT_PD;
        P.mean[loc] = NAN;
        P.s2[loc] = NAN;
        if (P.var) P.var[loc] = NAN;
      } else {
        double mu = 0.0, psi = 0.0, vx = P.onepg;
        for (int i = 0; i < n; i++) {
          const double ux = A[i * lda + n], yt = A[i * lda + n + 1];
          mu = fma(ux, yt, mu);
          psi = fma(yt, yt, psi);
          vx = fma(-ux, ux, vx);
        }
        const double pv = psi * vx;
        P.mean[loc] = mu;
        P.s2[loc] = pv / n;
        if (P.var) P.var[loc] = pv / (n - 2);
        if (P.status) P.status[loc] = 0;
      }
    }
    if (P.idx) {
      for (int i = tid; i < n; i += MB) P.idx[loc * n + i] = sh_fail ? -1 : cnd[dr[i]];
    }
  }
}

int mix_grid(int64_t T, int num_sms) {
  int64_t g = (int64_t)num_sms * 2;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

int mix_mpad(int M) { return (int)align_up((size_t)M, 32); }

size_t mix_smem_bytes(int Mpad, int n) {
  return (size_t)Mpad * 2 * sizeof(ff) + (size_t)n * sizeof(ff) + (size_t)n * sizeof(int) +
         RESCORE_CAP * sizeof(int) + align_up((size_t)Mpad, 16);
}

struct MixLayout {
  size_t u, xr, a, total;
};

MixLayout mix_layout(int G, int p, int n, int M) {
  const size_t Mpad = (size_t)mix_mpad(M);
  MixLayout L;
  L.u = align_up((size_t)G * n * Mpad * sizeof(ff), 256);
  L.xr = align_up((size_t)G * p * Mpad * sizeof(ff), 256);
  L.a = align_up((size_t)G * n * (n + 2) * sizeof(double), 256);
  L.total = 256 + 256 + L.u + L.xr + L.a;
  return L;
}

}  // namespace

size_t select_mixed_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms) {
  return mix_layout(mix_grid(T, num_sms), p, n, ncand).total;
}

int select_mixed_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  const int G = mix_grid(a.T, di.num_sms);
  const MixLayout L = mix_layout(G, a.p, a.n, a.M);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  char *w = static_cast<char *>(ws);
  MixParams P;
  P.X = a.X; P.Z = a.Z; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Mpad = mix_mpad(a.M); P.n0 = a.n0; P.n = a.n;
  P.theta = a.theta; P.theta_inv = 1.0 / a.theta; P.g = a.g; P.onepg = 1.0 + a.g;
  P.mean = a.mean; P.s2 = a.s2; P.var = a.var; P.idx = a.idx; P.status = a.status;
  P.queue = reinterpret_cast<int *>(w);
  P.rescores = reinterpret_cast<int *>(w + 256);
  P.U = reinterpret_cast<ff *>(w + 512);
  P.Xr = reinterpret_cast<ff *>(w + 512 + L.u);
  P.A = reinterpret_cast<double *>(w + 512 + L.u + L.xr);
  const size_t smem = mix_smem_bytes(P.Mpad, a.n);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(select_mixed_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(w, 0, 512, stream);  // work counter and re-score counter
  if (e != cudaSuccess) return cuda_status(e);
  select_mixed_kernel<<<G, MB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

}  // namespace lagp
