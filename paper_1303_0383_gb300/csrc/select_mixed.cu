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
// Each thread screens a pair of candidates with packed FP32 instructions (ff2.cuh), and a
// step needs one block barrier: every thread merges the per-warp best/second-best results
// and derives the step's pivot scalars itself.
//
// The kernel returns the selected design of every location; the predictive equations
// (Eqs. predgp, preds2) are then evaluated in FP64 on that design by kernel (c) in
// predict.cu, so mu, s2 and V carry FP64 accuracy whatever precision screened the
// candidates.
#include <math.h>

#include "ff.cuh"
#include "ff2.cuh"
#include "batch.cuh"
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
  int M, Mpad, Qpad, n0, n;
  int nmax, pmax;  // slot dimensions (the largest n and p of the launch)
  double theta, theta_inv, g, onepg;
  BatchView B;     // per-location tables (B.designs == nullptr: uniform launch)
  int32_t *idx;   // selected design indices (required: the caller's or the workspace's)
  float4 *U;     // slots of n x Qpad candidate pairs: row j of every candidate's factor row
  float4 *Xr;    // slots of p x Qpad pairs: candidate coordinates minus x
  double *A;     // slots of n x (n + 2): FP64 factorisation
  int *queue;
  int *rescores; // count of FP64 re-score passes (diagnostics)
};

// exp(a) for a <= 0 on a pair, in float-float (Tang's table-driven method with N = 64, see
// fp64_exp.cuh): a = k ln2/64 + r, exp(r) - 1 = r + r^2/2 + r^3/6 + r^4/24 + r^5/120 with
// the first two terms in float-float and the rest in FP32 (they are below 3e-8).
// Arguments below -87 give 0.
__device__ __forceinline__ ff2 exp_ff2(ff2 a, const float *tabh, const float *tabl) {
  const float2 ah = make_float2(fmaxf(a.h.x, -87.0f), fmaxf(a.h.y, -87.0f));
  const float2 magic = f2s(12582912.0f);  // 1.5 * 2^23
  const float2 t = fma2(ah, f2s(c_exp.inv_ln2_64f), magic);
  const float2 kf = sub2(t, magic);
  const int kx = __float_as_int(t.x) - 0x4B400000, ky = __float_as_int(t.y) - 0x4B400000;
  const float2 r1 = fma2(neg2(kf), f2s(c_exp.c1), ah);  // exact
  const float2 p2h = mul2(kf, f2s(c_exp.c2));
  const float2 p2l = fma2(kf, f2s(c_exp.c2), neg2(p2h));
  const ff2 s = two_sum2(r1, neg2(p2h));
  const float2 rl = add2(sub2(sub2(s.l, p2l), mul2(kf, f2s(c_exp.c3))), a.l);
  const ff2 r = fast_two_sum2(s.h, rl);
  const float2 sqh = mul2(r.h, r.h);
  const float2 sql = fma2(add2(r.h, r.h), r.l, fma2(r.h, r.h, neg2(sqh)));
  const float2 P = mul2(mul2(r.h, sqh),
                        fma2(r.h, fma2(r.h, f2s(1.0f / 120.0f), f2s(1.0f / 24.0f)), f2s(1.0f / 6.0f)));
  const ff2 e = two_sum2(r.h, mul2(f2s(0.5f), sqh));
  const ff2 E = fast_two_sum2(e.h, add2(add2(e.l, r.l), fma2(f2s(0.5f), sql, P)));
  const float2 Th = f2(tabh[kx & 63], tabh[ky & 63]), Tl = f2(tabl[kx & 63], tabl[ky & 63]);
  const float2 ph = mul2(Th, E.h);
  const float2 pl = fma2(Th, E.h, neg2(ph));
  const ff2 s2 = two_sum2(Th, ph);
  const float2 low = add2(add2(s2.l, pl), fma2(Th, E.l, fma2(Tl, E.h, Tl)));
  const ff2 res = fast_two_sum2(s2.h, low);
  const float2 sc = f2(__int_as_float(((kx >> 6) + 127) << 23), __int_as_float(((ky >> 6) + 127) << 23));
  ff2 out{mul2(res.h, sc), mul2(res.l, sc)};
  if (a.h.x < -87.0f) out.h.x = out.l.x = 0.0f;
  if (a.h.y < -87.0f) out.h.y = out.l.y = 0.0f;
  return out;
}

__device__ __forceinline__ bool frac_better(double a, double da, int ra, double b, double db,
                                            int rb) {
  const double l = a * db, r = b * da;
  return l > r || (l == r && ra < rb);
}

// Screen score comparison: larger score, ties to the smaller rank.
__device__ __forceinline__ void track2(float sc, int c, float &b1, int &r1, float &b2) {
  if (sc > b1 || (sc == b1 && c < r1)) {
    b2 = b1;
    b1 = sc;
    r1 = c;
  } else if (sc > b2) {
    b2 = sc;
  }
}

__device__ __forceinline__ void merge2(float o1, int orr, float o2, float &b1, int &r1, float &b2) {
  if (o1 > b1 || (o1 == b1 && orr < r1)) {
    b2 = fmaxf(b1, o2);
    b1 = o1;
    r1 = orr;
  } else {
    b2 = fmaxf(b2, o1);
  }
}

// Right-looking FP64 Cholesky of the j x j design matrix held in A (row-major, leading
// dimension lda) together with naug extra columns (forward substitution of them).  The
// matrix entries are built by the caller.  Sets *fail on a pivot <= 0.
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

// One step of the screen for NP candidate pairs of this thread (Sec. 3.2 update, in
// float-float): K(s, c) from the squared distance, the new factor entry
// u_c[j] = (K(s, c) - u_s . u_c) / L_jj, then v_{j+1}(c) = v_j(c) - u_c[j]^2,
// cov_{j+1}(x, c) = cov_j(x, c) - u_x[j] u_c[j], and the ALC screen score cov^2 / v.
struct StepCtx {
  float4 *U;
  const float4 *Xr;
  float4 *vp, *cp;
  const float4 *srow4;
  const float2 *srow2, *sxs;
  const float *tabh, *tabl;
  ff2 inv2, uxj2, thinv2;
  int Qpad, p, j;
  bool want;
};

template <int NP>
__device__ __forceinline__ void screen_pairs(const StepCtx &C, const int (&qs)[NP],
                                             const unsigned char *used, float &b1, int &r1,
                                             float &b2) {
  ff2acc acc[NP];
#pragma unroll
  for (int h = 0; h < NP; h++) {
    const int q = qs[h];
    // squared distance of the pair to the new point
    float2 dh = f2s(0.0f), dl = f2s(0.0f);
    for (int k = 0; k < C.p; k++) {
      const ff2 b = ff2_load(C.Xr + k * C.Qpad + q);
      const float2 a = C.sxs[k];
      const ff2 df = two_sum2(f2s(a.x), neg2(b.h));
      const float2 dfl = add2(df.l, sub2(f2s(a.y), b.l));
      const float2 ph = mul2(df.h, df.h);
      const float2 pl = fma2(add2(df.h, df.h), dfl, fma2(df.h, df.h, neg2(ph)));
      const ff2 sacc = two_sum2(dh, ph);
      dh = sacc.h;
      dl = add2(add2(sacc.l, dl), pl);
    }
    const ff2 d2 = fast_two_sum2(dh, dl);
    const ff2 arg = ff2_mul(d2, C.thinv2);
    const ff2 kc = exp_ff2(ff2{neg2(arg.h), neg2(arg.l)}, C.tabh, C.tabl);   // K(s, c)
    acc[h] = ff2acc{kc.h, kc.l};
  }
  // K(s, c) - sum_i u_s[i] u_c[i]: compensated accumulation, the pairs interleaved (four
  // loads of U in flight either way)
  const float4 *Uq[NP];
#pragma unroll
  for (int h = 0; h < NP; h++) Uq[h] = C.U + qs[h];
  constexpr int UNR = 4 / NP;
#pragma unroll UNR
  for (int i = 0; i < C.j; i++) {
    const float4 a = C.srow4[i];
    const float2 al = C.srow2[i];
    float4 b[NP];
#pragma unroll
    for (int h = 0; h < NP; h++) b[h] = Uq[h][(size_t)i * C.Qpad];
#pragma unroll
    for (int h = 0; h < NP; h++) ff2acc_sub_prod(acc[h], a, al, b[h]);
  }
#pragma unroll
  for (int h = 0; h < NP; h++) {
    const int q = qs[h];
    const bool u0 = used[2 * q], u1 = used[2 * q + 1];
    const ff2 u = ff2_mul(ff2acc_result(acc[h]), C.inv2);           // u_c[j]
    ff2_store(C.U + (size_t)C.j * C.Qpad + q, u);
    const ff2 v0 = ff2_load(C.vp + q), c0 = ff2_load(C.cp + q);
    ff2 v = ff2_sub(v0, ff2_mul(u, u));
    ff2 cx = ff2_sub(c0, ff2_mul(C.uxj2, u));
    // A used lane keeps its values: the step's pivot may be the partner of a live
    // candidate, and other threads read the pivot's v and cov at the start of the step
    // without a barrier after it.
    if (u0) { v.h.x = v0.h.x; v.l.x = v0.l.x; cx.h.x = c0.h.x; cx.l.x = c0.l.x; }
    if (u1) { v.h.y = v0.h.y; v.l.y = v0.l.y; cx.h.y = c0.h.y; cx.l.y = c0.l.y; }
    ff2_store(C.vp + q, v);
    ff2_store(C.cp + q, cx);
    if (C.want) {
      if (!u0 && v.h.x > 0.0f) track2(__fdiv_rn(cx.h.x * cx.h.x, v.h.x), 2 * q, b1, r1, b2);
      if (!u1 && v.h.y > 0.0f) track2(__fdiv_rn(cx.h.y * cx.h.y, v.h.y), 2 * q + 1, b1, r1, b2);
    }
  }
}

#ifndef LAGP_MIX_MINB
#define LAGP_MIX_MINB LAGP_MIX_CTAS_PER_SM  // 3 CTAs per SM: 85 registers, no spills
#endif
__global__ void __launch_bounds__(MB, LAGP_MIX_MINB) select_mixed_kernel(MixParams P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Qpad = P.Qpad, nmax = P.nmax;
  float4 *vp = reinterpret_cast<float4 *>(smraw);            // Qpad: v_j(c) pairs
  float4 *cp = vp + Qpad;                                    // Qpad: cov_j(x, c) pairs
  // per-warp copies of the new factor row: {h, h, -h, -h} and {l, l} per entry
  const int nrow = (nmax + 1) & ~1;
  float4 *wrow4 = reinterpret_cast<float4 *>(cp + Qpad);     // (MB/32) x nrow
  float2 *wrow2 = reinterpret_cast<float2 *>(wrow4 + (MB / 32) * nrow);  // (MB/32) x nrow
  float2 *wxs = wrow2 + (MB / 32) * nrow;                    // (MB/32) x kMaxP: new point
  int *dr = reinterpret_cast<int *>(wxs + (MB / 32) * kMaxP);  // nmax
  int *rlist = dr + nmax;                                    // RESCORE_CAP
  unsigned char *used = reinterpret_cast<unsigned char *>(rlist + RESCORE_CAP);  // Mpad
  __shared__ float tabh[64], tabl[64];
  __shared__ double etab[64];
  __shared__ double xl[kMaxP];
  __shared__ float red_s1[2][MB / 32], red_s2[2][MB / 32];
  __shared__ int red_r1[2][MB / 32];
  __shared__ double red_n[MB / 32], red_d[MB / 32];
  __shared__ int red_rr[MB / 32];
  __shared__ int sh_loc, sh_fail, sh_nlist, sh_rbest;
  if (threadIdx.x < 64) {
    tabh[threadIdx.x] = c_exp.tabf_h[threadIdx.x];
    tabl[threadIdx.x] = c_exp.tabf_l[threadIdx.x];
    etab[threadIdx.x] = c_exp.tab[threadIdx.x];
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4 *U = P.U + (size_t)blockIdx.x * nmax * Qpad;
  float4 *Xr = P.Xr + (size_t)blockIdx.x * P.pmax * Qpad;
  const int lda = nmax + 2;
  double *A = P.A + (size_t)blockIdx.x * nmax * lda;
  float4 *srow4 = wrow4 + warp * nrow;  // this warp's copy of the new factor row
  float2 *srow2 = wrow2 + warp * nrow;
  float2 *sxs = wxs + warp * kMaxP;     // and of the new point's coordinates

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    if (sh_loc >= P.T) break;
    const LocParams L = resolve_loc(P.B, sh_loc, P.X, P.Z, P.XX, P.p, P.n, P.M, P.n0, P.theta,
                                    P.g, P.cand, P.idx);
    const int n = L.n, p = L.p, M = L.M;
    const int32_t *cnd = L.cand;
    const ff onepg = ff_from_double(L.onepg);
    const ff thinv = ff_from_double(L.theta_inv);
    // Without greedy steps (n0 == n) only the start design's own rows are ever read.
    const int Q = ((L.n0 == n ? n : M) + 1) >> 1;
    if (tid < p) xl[tid] = L.x[tid];
    if (tid == 0) sh_fail = 0;
    __syncthreads();
    // coordinates relative to x (float-float pairs), v = 1+g, cov_0(x,c) = K(x,c) in FP64
    for (int q = tid; q < Qpad; q += MB) {
      ff cv[2];
      for (int h = 0; h < 2; h++) {
        const int c = 2 * q + h;
        cv[h] = ff{0.0f, 0.0f};
        if (c < M) {
          const double *xc = L.X + (int64_t)cnd[c] * p;
          double acc = 0.0;
          for (int k = 0; k < p; k++) {
            const double dk = xc[k] - xl[k];
            const ff fk = ff_from_double(dk);
            float *slot = reinterpret_cast<float *>(Xr + k * Qpad + q);
            slot[h] = fk.h;
            slot[2 + h] = fk.l;
            acc = fma(dk, dk, acc);
          }
          cv[h] = ff_from_double(exp_nonpos(-acc * L.theta_inv, etab));
        } else {
          for (int k = 0; k < p; k++) {
            float *slot = reinterpret_cast<float *>(Xr + k * Qpad + q);
            slot[h] = 0.0f;
            slot[2 + h] = 0.0f;
          }
        }
        used[c] = (c < M) ? 0 : 1;
      }
      vp[q] = make_float4(onepg.h, onepg.h, onepg.l, onepg.l);
      cp[q] = make_float4(cv[0].h, cv[1].h, cv[0].l, cv[1].l);
    }
    __syncthreads();

    int best = 0;
    for (int j = 0; j < n; j++) {
      const int s = (j < L.n0) ? j : best;
      if (s < 0) {  // nothing admissible left (the same for every thread)
        if (tid == 0) sh_fail = 1;
        break;
      }
      const ff vs = ff2_get(vp, s);
      if (!(vs.h > 0.0f)) {
        if (tid == 0) sh_fail = 1;
        break;
      }
      // every thread derives the step's scalars itself: no barrier needed for them
      const ff inv = ff_rcp(ff_sqrt(vs));
      const ff uxj = ff_mul(ff2_get(cp, s), inv);
      if (tid == 0) dr[j] = s;
      if (tid == ((s >> 1) % MB)) used[s] = 1;  // the pair's owner keeps the flags
      // this warp's copy of the new factor row u_s and of x_s (relative to x)
      for (int i = lane; i < j; i += 32) {
        const ff u = ff2_get(U + (size_t)i * Qpad, s);
        srow4[i] = make_float4(u.h, u.h, -u.h, -u.h);
        srow2[i] = f2s(u.l);
      }
      if (lane < p) {
        const ff xk = ff2_get(Xr + lane * Qpad, s);
        sxs[lane] = make_float2(xk.h, xk.l);
      }
      __syncwarp();
      if (j == n - 1) break;
      const bool want = j + 1 >= L.n0;
      const ff2 inv2{f2s(inv.h), f2s(inv.l)}, uxj2{f2s(uxj.h), f2s(uxj.l)};
      const ff2 thinv2{f2s(thinv.h), f2s(thinv.l)};
      float b1 = -1.0f, b2 = -1.0f;
      int r1 = 0x7fffffff;
      const StepCtx C{U, Xr, vp, cp, srow4, srow2, sxs, tabh, tabl, inv2, uxj2, thinv2, Qpad, p, j, want};
      // one pair at a time (interleaving two pairs per thread measured slower: the extra
      // loads in flight only add L2 pressure)
      for (int q = tid; q < Q; q += MB) {
        if (used[2 * q] && used[2 * q + 1]) continue;
        const int qs[1] = {q};
        screen_pairs<1>(C, qs, used, b1, r1, b2);
      }
      // best and second-best screen scores: warp shuffles, one barrier, then every
      // thread merges the per-warp results itself (double-buffered by step parity)
      const int par = j & 1;
      for (int o = 16; o > 0; o >>= 1) {
        const float ob1 = __shfl_down_sync(0xffffffffu, b1, o);
        const float ob2 = __shfl_down_sync(0xffffffffu, b2, o);
        const int orr = __shfl_down_sync(0xffffffffu, r1, o);
        merge2(ob1, orr, ob2, b1, r1, b2);
      }
      if (lane == 0) {
        red_s1[par][warp] = b1;
        red_s2[par][warp] = b2;
        red_r1[par][warp] = r1;
      }
      __syncthreads();
      if (!want) continue;
      float B1 = red_s1[par][0], B2 = red_s2[par][0];
      int R1 = red_r1[par][0];
      for (int w = 1; w < MB / 32; w++) merge2(red_s1[par][w], red_r1[par][w], red_s2[par][w], B1, R1, B2);
      best = (R1 == 0x7fffffff) ? -1 : R1;
      const bool near = R1 != 0x7fffffff && B2 >= B1 * (1.0f - DELTA);
      if (!near) continue;
      // ---- FP64 re-score of the near-tied candidates (rare) ----
      if (tid == 0) {
        sh_nlist = 0;
        if (P.rescores) atomicAdd(P.rescores, 1);
      }
      __syncthreads();
      const int jd = j + 1;  // design size now
      for (int c = tid; c < M; c += MB) {
        if (used[c]) continue;
        const ff v = ff2_get(vp, c), cx = ff2_get(cp, c);
        if (!(v.h > 0.0f)) continue;
        const float sc = __fdiv_rn(cx.h * cx.h, v.h);
        if (sc >= B1 * (1.0f - 2.0f * DELTA)) {
          const int pos = atomicAdd(&sh_nlist, 1);
          if (pos < RESCORE_CAP) rlist[pos] = c;
        }
      }
      // FP64 factor of the current design with k(x) as an extra column (lower triangle)
      for (int qq = tid; qq < jd * (jd + 1); qq += MB) {
        const int a = qq / (jd + 1), b = qq % (jd + 1);
        if (b < jd && b > a) continue;
        const double *xa = L.X + (int64_t)cnd[dr[a]] * p;
        double val;
        if (b < jd) val = (a == b) ? L.onepg : corr64(xa, L.X + (int64_t)cnd[dr[b]] * p, p, L.theta_inv, etab);
        else val = corr64(xa, xl, p, L.theta_inv, etab);
        A[a * lda + b] = val;
      }
      __syncthreads();
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
        const double *xc = L.X + (int64_t)cnd[c] * p;
        double tv[kMaxN / 32];
#pragma unroll
        for (int r = 0; r < kMaxN / 32; r++) {
          const int i = 32 * r + lane;
          tv[r] = (i < jd) ? corr64(L.X + (int64_t)cnd[dr[i]] * p, xc, p, L.theta_inv, etab) : 0.0;
        }
        double vsum = L.onepg;
        double cov = corr64(xl, xc, p, L.theta_inv, etab);
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
        red_rr[warp] = br;
      }
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < MB / 32; w++)
          if (frac_better(red_n[w], red_d[w], red_rr[w], bn, bd, br)) {
            bn = red_n[w];
            bd = red_d[w];
            br = red_rr[w];
          }
        sh_rbest = (br != 0x7fffffff) ? br : best;
      }
      __syncthreads();
      best = sh_rbest;
    }
    __syncthreads();
    // the design (design indices), or -1 when a step failed; kernel (c) (predict.cu)
    // evaluates the predictive equations on it in FP64
    for (int i = tid; i < n; i += MB) L.idx[i] = sh_fail ? -1 : cnd[dr[i]];
  }
}

int mix_grid(int64_t T, int num_sms) {
  int64_t g = (int64_t)num_sms * LAGP_MIX_MINB;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

int mix_mpad(int M) { return (int)align_up((size_t)M, 64); }

size_t mix_smem_bytes(int Mpad, int n) {
  const size_t Qpad = (size_t)Mpad / 2;
  const size_t nrow = (size_t)((n + 1) & ~1);
  return Qpad * 2 * sizeof(float4) +
         (size_t)(MB / 32) * (nrow * (sizeof(float4) + sizeof(float2)) + kMaxP * sizeof(float2)) +
         (size_t)n * sizeof(int) + RESCORE_CAP * sizeof(int) + align_up((size_t)Mpad, 16);
}

struct MixLayout {
  size_t u, xr, a, idx, pred, total;
};

// [queue | re-score counter | U | Xr | A | design indices | kernel (c) workspace]
MixLayout mix_layout(int G, int p, int n, int M, int64_t T, int64_t idx_total, int num_sms) {
  const size_t Qpad = (size_t)mix_mpad(M) / 2;
  MixLayout L;
  L.u = align_up((size_t)G * n * Qpad * sizeof(float4), 256);
  L.xr = align_up((size_t)G * p * Qpad * sizeof(float4), 256);
  L.a = align_up((size_t)G * n * (n + 2) * sizeof(double), 256);
  L.idx = align_up((size_t)idx_total * sizeof(int32_t), 256);
  L.pred = predict_fp64_workspace_bytes(T, n, num_sms);
  L.total = 256 + 256 + L.u + L.xr + L.a + L.idx + L.pred;
  return L;
}

// The screen, then kernel (c) on the designs it selected.
int mix_run(MixParams P, const PredictArgs &pa_in, const MixLayout &L, int G, char *w,
            int32_t *user_idx, const DevInfo &di, cudaStream_t stream) {
  P.queue = reinterpret_cast<int *>(w);
  P.rescores = reinterpret_cast<int *>(w + 256);
  char *o = w + 512;
  P.U = reinterpret_cast<float4 *>(o);
  o += L.u;
  P.Xr = reinterpret_cast<float4 *>(o);
  o += L.xr;
  P.A = reinterpret_cast<double *>(o);
  o += L.a;
  // the design goes to the caller's idx, or to the workspace when the caller wants none
  P.idx = user_idx ? user_idx : reinterpret_cast<int32_t *>(o);
  o += L.idx;
  const size_t smem = mix_smem_bytes(P.Mpad, P.nmax);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(select_mixed_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(w, 0, 512, stream);  // work counter and re-score counter
  if (e != cudaSuccess) return cuda_status(e);
  select_mixed_kernel<<<G, MB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  PredictArgs pa = pa_in;
  pa.idx = P.idx;
  return predict_fp64_launch(pa, o, L.pred, stream);
}

}  // namespace

size_t select_mixed_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms) {
  return mix_layout(mix_grid(T, num_sms), p, n, ncand, T, T * n, num_sms).total;
}

int select_mixed_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  const int G = mix_grid(a.T, di.num_sms);
  const MixLayout L = mix_layout(G, a.p, a.n, a.M, a.T, a.T * a.n, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MixParams P;
  P.X = a.X; P.Z = a.Z; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Mpad = mix_mpad(a.M); P.Qpad = P.Mpad / 2; P.n0 = a.n0; P.n = a.n;
  P.theta = a.theta; P.theta_inv = 1.0 / a.theta; P.g = a.g; P.onepg = 1.0 + a.g;
  P.nmax = a.n; P.pmax = a.p;
  P.B = BatchView{nullptr, nullptr, nullptr, 0};
  PredictArgs pa;
  pa.X = a.X; pa.Z = a.Z; pa.p = a.p; pa.XX = a.XX; pa.T = a.T; pa.n = a.n; pa.nmax = a.n;
  pa.theta = a.theta; pa.g = a.g; pa.idx = nullptr; pa.B = P.B;
  pa.mean = a.mean; pa.s2 = a.s2; pa.var = a.var; pa.status = a.status;
  return mix_run(P, pa, L, G, static_cast<char *>(ws), a.idx, di, stream);
}

size_t select_mixed_batch_workspace_bytes(const BatchLaunch &b, int G) {
  DevInfo di;
  const int sms = dev_info(&di) == LAGP_OK ? di.num_sms : 152;
  return mix_layout(G, b.pmax, b.nmax, b.Mmax, b.T, b.idx_total, sms).total;
}

int select_mixed_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, int G,
                              cudaStream_t stream) {
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();  // this translation unit's copy of the exp constants
  if (st) return st;
  const MixLayout L = mix_layout(G, b.pmax, b.nmax, b.Mmax, b.T, b.idx_total, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MixParams P;
  P.X = nullptr; P.Z = nullptr; P.p = b.pmax; P.XX = b.XX; P.T = b.T; P.cand = b.cand;
  P.M = b.Mmax; P.Mpad = mix_mpad(b.Mmax); P.Qpad = P.Mpad / 2; P.n0 = 0; P.n = b.nmax;
  P.theta = 1.0; P.theta_inv = 1.0; P.g = 0.0; P.onepg = 1.0;
  P.nmax = b.nmax; P.pmax = b.pmax;
  P.B = BatchView{b.designs, b.locs, b.order, b.ldxx};
  PredictArgs pa;
  pa.X = nullptr; pa.Z = nullptr; pa.p = b.pmax; pa.XX = b.XX; pa.T = b.T; pa.n = b.nmax;
  pa.nmax = b.nmax; pa.theta = 1.0; pa.g = 0.0; pa.idx = nullptr; pa.B = P.B;
  pa.mean = b.mean; pa.s2 = b.s2; pa.var = b.var; pa.status = b.status;
  return mix_run(P, pa, L, G, static_cast<char *>(ws), b.idx, di, stream);
}

int select_mixed_prepare() {
  const int st = exp_table_upload();
  return st ? st : predict_fp64_prepare();
}

}  // namespace lagp
