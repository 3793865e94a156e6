// select_mspe_mixed.cu -- kernel (b) for the MSPE criterion, mixed precision: FP64 design
// bookkeeping, a float-float candidate screen on the FP32 pipes, FP64 decisions where the
// screen cannot separate candidates, and kernel (c) (predict.cu) for the predictive
// equations in FP64.
//
// Gramacy & Apley, Sec. 3.1 (Eq. mspe, Eqs. newv and G) with the derivatives of SM Sec. 2
// (Eqs. dKi, d2w, dl, d2l, dz, dmu, dV, Ed2la): at each step the candidate c minimising
//   J(c) = psi_j/(j-2) v_{j+1}(x) + (dmu_j(x)/dtheta)^2 / G_{j+1}(c)
// joins the design, in the quantities and the Cholesky basis of the FP64 kernel
// (select_mspe.cu): per candidate u_c = L^{-1} k_c, ud_c = L^{-1} kd_c, v_j(c), cov_j(x,c),
// kd_c^T z_c, kd_c^T w, z_c^T Kd z_c and z_c^T Kd w, each updated in O(j) per step.
//
// Split of the work:
//  * FP64, once per step for the whole CTA (O(j^2)): the pivot's row u_s = L^{-1} k_j(s)
//    from the FP64 inverse factor L^{-1}, v_j(s), the new rows of L^{-1}, Kd, Kdd, Q and R,
//    r = Q ytil, F_j (Eq. d2l), dmu_j(x) and w^T Kd w -- exactly the FP64 kernel's step,
//    except that u_s is formed from L^{-1} instead of being read from the candidate state.
//  * Float-float, per candidate (O(j), the hot loop): K(s,c) and Kd(s,c) from the
//    coordinates, the three compensated dot products u_s.u_c, u_s.ud_c and q_j.u_c over the
//    candidate's factor rows (ff2.cuh, two candidates per thread on packed FP32), the O(1)
//    updates and J(c) itself, all in float-float.
//  * FP64 re-score: when the screen's second-best J is within DELTA (relative) of its
//    best, or a candidate's G or J is a cancellation the screen cannot resolve (a negative
//    F_j, reading of Sec. 3.1 with theta held fixed), the listed candidates are re-scored
//    from scratch in FP64 -- u_c and ud_c as L^{-1} k_c and L^{-1} kd_c, q_c = u_c^T Q u_c --
//    and the FP64 minimum wins, ties to the nearer candidate.
#include <math.h>

#include "batch.cuh"
#include "mixed_screen.cuh"

namespace lagp {
namespace {

constexpr int XB = 256;  // threads per CTA
#define LAGP_MSPE_MIX_MINB LAGP_MSPE_MIX_CTAS_PER_SM
// Factor rows in flight per thread: each thread streams its own pair's rows of U and Ud
// through a ring of RING stages in shared memory with asynchronous copies (cp.async), so
// that RING - 1 rows of both arrays are on their way while one is consumed.  The arrays
// exceed L2 on the large workloads and the loop is bound by the bytes in flight per SM.
// (the asynchronous copies and their groups: mixed_screen.cuh)
// Where the ring does not fit in shared memory (the largest candidate counts) the kernel
// is instantiated without it (RG = 0) and loads the rows straight into registers.
constexpr int RING = 6;

struct MxParams {
  const double *X, *Z;
  int p;
  const double *XX;
  int64_t T;
  const int32_t *cand;
  int M, Mpad, Qpad, n0, n;
  int nmax, pmax;  // slot dimensions (the largest n and p of the launch)
  double theta, g;
  BatchView B;     // per-location tables (B.designs == nullptr: uniform launch)
  int32_t *idx;    // selected design indices (the caller's or the workspace's)
  float4 *U, *Ud;  // slots of nmax x Qpad candidate pairs: rows of u_c and ud_c
  float4 *Xr;      // slots of pmax x Qpad pairs: candidate coordinates minus x
  float4 *cs;      // slots of 4 x Qpad pairs: kd_c^T z_c, kd_c^T w, z_c^T Kd z_c, z_c^T Kd w
  double *Li, *LiT, *Kd, *Kdd, *Qf;  // slots of nmax x nmax (FP64)
  double *Wk;      // slots of (XB/32) x 4 x nmax: per-warp scratch of the FP64 re-score
  double *mean, *s2, *var;
  int8_t *status;
  int *queue;
  int *rescores;   // count of FP64 re-score passes (diagnostics)
  const int32_t *start;  // saved start designs (T x nstart design indices), or nullptr
  int nstart;
};

__device__ __forceinline__ bool j_better64(double a, int ra, double b, int rb) {
  return a < b || (a == b && ra < rb);
}

// The O(j^2) products of the FP64 step, y1[i] = sum_{m in [lo(i), hi(i))} A1[i][m] x1[m]
// (and y2 likewise with A2, x2 when A2 is given), for rows i < rows of row-major matrices
// with leading dimension nn.  Each row is split over SPLIT threads (strided entries), so
// all warps of the CTA issue FP64 work and each chain is SPLIT times shorter; the partial
// sums meet in `part` (shared memory) and are added in a fixed order, so the result does
// not depend on the schedule.  Ends with the outputs written through out(i, y1, y2) and a
// barrier.  The matrices are read at every step of the location and are kept in L2 ahead
// of the candidates' factor rows, which stream through with an evict-first policy
// (8-d workload 393 -> 374 ms, paper-2d 76.5 -> 70.1 ms).
constexpr int SPLIT = 4;
template <class Lo, class Hi, class Out>
__device__ __forceinline__ void split_rows(const double *A1, const double *x1, const double *A2,
                                           const double *x2, int nn, int rows, Lo lo, Hi hi,
                                           double *part, Out out) {
  const int tid = threadIdx.x;
  for (int base = 0; base < rows; base += XB / SPLIT) {
    const int i = base + tid / SPLIT, c = tid % SPLIT;
    if (i < rows) {
      const double *a1 = A1 + (size_t)i * nn, *a2 = A2 ? A2 + (size_t)i * nn : nullptr;
      double s1 = 0.0, s2 = 0.0;
      const int h = hi(i);
      const unsigned long long pol = l2_evict_last_policy();
      int m = lo(i) + c;
      // eight terms' loads are issued before their multiply-adds, which keep the order of
      // the one-term loop (the same sums, bit for bit): one L2 round trip per eight terms
      // instead of one per term
      for (; m + 7 * SPLIT < h; m += 8 * SPLIT) {
        double v1[8], v2[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
          v1[u] = ld_l2_hint(a1 + m + u * SPLIT, pol);
          v2[u] = a2 ? ld_l2_hint(a2 + m + u * SPLIT, pol) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
          s1 = fma(v1[u], x1[m + u * SPLIT], s1);
          if (a2) s2 = fma(v2[u], x2[m + u * SPLIT], s2);
        }
      }
      for (; m < h; m += SPLIT) {
        s1 = fma(ld_l2_hint(a1 + m, pol), x1[m], s1);
        if (a2) s2 = fma(ld_l2_hint(a2 + m, pol), x2[m], s2);
      }
      part[2 * tid] = s1;
      part[2 * tid + 1] = s2;
    }
    __syncthreads();
    if (tid < XB / SPLIT && base + tid < rows) {
      double y1 = 0.0, y2 = 0.0;
      for (int k = 0; k < SPLIT; k++) {
        y1 += part[2 * (tid * SPLIT + k)];
        y2 += part[2 * (tid * SPLIT + k) + 1];
      }
      out(base + tid, y1, y2);
    }
    __syncthreads();
  }
}

// Screen score comparison for a minimum: smaller score, ties to the smaller rank.
__device__ __forceinline__ void track_min(float sc, int c, float &b1, int &r1, float &b2) {
  if (sc < b1 || (sc == b1 && c < r1)) {
    b2 = b1;
    b1 = sc;
    r1 = c;
  } else if (sc < b2) {
    b2 = sc;
  }
}

__device__ __forceinline__ void merge_min(float o1, int orr, float o2, float &b1, int &r1, float &b2) {
  if (o1 < b1 || (o1 == b1 && orr < r1)) {
    b2 = fminf(b1, o2);
    b1 = o1;
    r1 = orr;
  } else {
    b2 = fminf(b2, o1);
  }
}

// The step's values for the screen: broadcast float-float scalars and the new rows.
struct MStep {
  float4 *U, *Ud, *cs, *vp, *cp;
  float4 *ring;           // this thread's ring: stage k holds U at [2k XB], Ud at [(2k+1) XB]
  const float4 *Xr;
  float *Jsc;             // per candidate: the screen's J (FP32), +inf when not scored
  unsigned char *flg;     // per candidate: 1 when the screen cannot resolve its J
  const float4 *sr4, *qr4;  // u_s and -q_j (rows as {h, h, -h, -h})
  const float2 *sr2, *qr2;  // their low parts {l, l}
  const float2 *sxs;        // x_s - x (float-float)
  const float *tabh, *tabl;
  ff2 inv, uxj, ytj, rj, qjj, thinv;  // 1/L_jj, u_x[j], ytil[j], r[j], Q[j][j], 1/theta
  ff2 a, vx, wd, F, dmux2;            // psi/(j-2), v_{j+1}(x), w^T Kd w/(j-2), F_j, dmu_x^2
  float Ff;
  int Qpad, p, j;
  bool want;
};

// One step for one pair of candidates (2q, 2q+1).
template <int RG>
__device__ __forceinline__ void mspe_pair(const MStep &C, int q, const unsigned char *used,
                                          float &b1, int &r1, float &b2, int &nf) {
  // the first RING - 1 rows start on their way (one copy group per row, empty past row j)
  const unsigned long long pol = l2_evict_first_policy();
#pragma unroll
  for (int st = 0; st < RG - 1; st++) {
    if (st < C.j) {
      cp_async16_l2_hint(C.ring + (2 * st) * XB, C.U + (size_t)st * C.Qpad + q, pol);
      cp_async16_l2_hint(C.ring + (2 * st + 1) * XB, C.Ud + (size_t)st * C.Qpad + q, pol);
    }
    cp_async_commit();
  }
  // squared distance of the pair to the new point, in float-float
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
  const ff2 arg = ff2_mul(d2, C.thinv);
  const ff2 kc = exp_ff2(ff2{neg2(arg.h), neg2(arg.l)}, C.tabh, C.tabl);  // K(s, c)
  const ff2 kdc = ff2_mul(ff2_mul(kc, arg), C.thinv);                     // Kd(s, c)
  // K(s,c) - u_s.u_c, Kd(s,c) - u_s.ud_c and q_j.u_c (compensated, Dot2)
  ff2acc a1{kc.h, kc.l}, a2{kdc.h, kdc.l}, a3{f2s(0.0f), f2s(0.0f)};
  int sc = 0, sp = RG - 1;  // ring stages of rows i and i + RG - 1
#pragma unroll (RG ? 1 : 2)
  for (int i = 0; i < C.j; i++) {
    float4 bu, bd;
    if constexpr (RG > 0) {
      const int ip = i + RG - 1;
      if (ip < C.j) {  // refill the stage consumed at row i - 1
        cp_async16_l2_hint(C.ring + (2 * sp) * XB, C.U + (size_t)ip * C.Qpad + q, pol);
        cp_async16_l2_hint(C.ring + (2 * sp + 1) * XB, C.Ud + (size_t)ip * C.Qpad + q, pol);
      }
      cp_async_commit();
      cp_async_wait<RG - 1>();  // row i has landed
      bu = C.ring[(2 * sc) * XB];
      bd = C.ring[(2 * sc + 1) * XB];
      sc = (sc == RG - 1) ? 0 : sc + 1;
      sp = (sp == RG - 1) ? 0 : sp + 1;
    } else {
      bu = ld_l2_hint(C.U + (size_t)i * C.Qpad + q, pol);
      bd = ld_l2_hint(C.Ud + (size_t)i * C.Qpad + q, pol);
    }
    const float4 sa = C.sr4[i], qa = C.qr4[i];
    const float2 sl = C.sr2[i], ql = C.qr2[i];
    ff2acc_sub_prod(a1, sa, sl, bu);
    ff2acc_sub_prod(a2, sa, sl, bd);
    ff2acc_sub_prod(a3, qa, ql, bu);
  }
  const ff2 u = ff2_mul(ff2acc_result(a1), C.inv);   // u_c[j]
  const ff2 ud = ff2_mul(ff2acc_result(a2), C.inv);  // ud_c[j]
  const ff2 d3 = ff2acc_result(a3);                  // sum_i Q[j][i] u_c[i]
  ff2_store(C.U + (size_t)C.j * C.Qpad + q, u);
  ff2_store(C.Ud + (size_t)C.j * C.Qpad + q, ud);
  const ff2 vc = ff2_sub(ff2_load(C.vp + q), ff2_mul(u, u));
  const ff2 cx = ff2_sub(ff2_load(C.cp + q), ff2_mul(C.uxj, u));
  ff2_store(C.vp + q, vc);
  ff2_store(C.cp + q, cx);
  float4 *cs = C.cs + q;
  const ff2 kz = ff2_add(ff2_load(cs), ff2_mul(ud, u));
  const ff2 pc = ff2_add(ff2_load(cs + C.Qpad), ff2_mul(ud, C.ytj));
  const ff2 qn = ff2_add(ff2_load(cs + 2 * C.Qpad),
                         ff2_mul(u, ff2_add(ff2_scale(d3, 2.0f), ff2_mul(C.qjj, u))));
  const ff2 mn = ff2_add(ff2_load(cs + 3 * C.Qpad), ff2_add(ff2_mul(u, C.rj), ff2_mul(C.ytj, d3)));
  ff2_store(cs, kz);
  ff2_store(cs + C.Qpad, pc);
  ff2_store(cs + 2 * C.Qpad, qn);
  ff2_store(cs + 3 * C.Qpad, mn);
  if (!C.want) return;
  // J(c) = a (v_x - cov^2 / v_c) + dmu_x^2 / G,  G = F + (dV/V)^2 / 2 + dmu_c^2 / V,
  // V = a v_c, -dV = wd v_c + a (2 kz - q), dmu_c = pc - mn
  const ff2 A = ff2_sub(C.vx, ff2_div(ff2_mul(cx, cx), vc));
  const ff2 V = ff2_mul(C.a, vc);
  const ff2 ndV = ff2_add(ff2_mul(C.wd, vc), ff2_mul(C.a, ff2_sub(ff2_scale(kz, 2.0f), qn)));
  const ff2 rV = ff2_div(ndV, V);
  const ff2 T1 = ff2_scale(ff2_mul(rV, rV), 0.5f);
  const ff2 dmu = ff2_sub(pc, mn);
  const ff2 T2 = ff2_div(ff2_mul(dmu, dmu), V);
  const ff2 G = ff2_add(ff2_add(C.F, T1), T2);
  const ff2 J2 = ff2_div(C.dmux2, G);
  const ff2 J = ff2_add(ff2_mul(C.a, A), J2);
  const float tiny = 9.3132257e-10f;  // 2^-30: cancellation beyond the screen's resolution
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int c = 2 * q + h;
    if (used[c]) continue;
    const float vh = h ? vc.h.y : vc.h.x, Jh = h ? J.h.y : J.h.x, Gh = h ? G.h.y : G.h.x;
    float sc = INFINITY;
    bool flag = false;
    if (vh > 0.0f) {
      if (!isfinite(Jh)) {
        flag = true;  // overflow or 0/0 in FP32 range: decide in FP64
      } else {
        if (C.Ff < 0.0f) {
          const float t1 = h ? T1.h.y : T1.h.x, t2 = h ? T2.h.y : T2.h.x;
          const float aA = h ? C.a.h.x * A.h.y : C.a.h.x * A.h.x, j2 = h ? J2.h.y : J2.h.x;
          flag = fabsf(Gh) <= tiny * (fabsf(C.Ff) + t1 + t2) ||
                 (Gh < 0.0f && fabsf(Jh) <= tiny * (aA + fabsf(j2)));
        }
        sc = Jh;
        track_min(sc, c, b1, r1, b2);
      }
    }
    C.Jsc[c] = sc;
    C.flg[c] = flag;
    nf |= flag;
  }
}

// ---- FP64 re-score (Sec. 3.1 decisions in FP64) ----
struct MRescore {
  const double *X;
  const int32_t *cnd;
  const double *xl, *etab;
  const unsigned char *used, *flg;
  const float *Jsc;
  const int *dg;                    // design indices in X
  const double *LiT, *Qf;           // FP64 inverse factor (transposed) and Q (full)
  const double *ux, *yt, *r;        // u_x, ytil and Q ytil of the design
  double *wk;                       // this warp's scratch: k, kd, u, ud (nn each)
  int *rlist, *nlist;
  double *red_s;
  int *red_r;
  int p, M, jd, nn;
  double theta_inv, ith2, onepg, psi, vx, F, dmux, wKdw;
};

// One candidate's J(c) in FP64 from scratch (one warp; RR rows of the design per lane):
// u = L^{-1} k_c, ud = L^{-1} kd_c, Q u, then the sums of the FP64 kernel.  NaN when
// v_j(c) <= 0.
template <int RR>
__device__ double rescore_one(const MRescore &R, int c, double dj) {
  const int lane = threadIdx.x & 31;
  const int jd = R.jd, nn = R.nn, p = R.p;
  double *wkk = R.wk, *wkd = R.wk + nn, *wu = R.wk + 2 * nn, *wud = R.wk + 3 * nn;
  const double *xc = R.X + (int64_t)R.cnd[c] * p;
  for (int i = lane; i < jd; i += 32) {
    const double *xi = R.X + (int64_t)R.dg[i] * p;
    double acc = 0.0;
    for (int k = 0; k < p; k++) {
      const double t = xi[k] - xc[k];
      acc = fma(t, t, acc);
    }
    const double kk = exp_nonpos(-acc * R.theta_inv, R.etab);
    wkk[i] = kk;
    wkd[i] = kk * acc * R.ith2;
  }
  __syncwarp();
  // u = L^{-1} k_c and ud = L^{-1} kd_c: lane-owned rows i, L^{-1}[i][m] = LiT[m][i]
  double au[RR], ad[RR];
#pragma unroll
  for (int rr = 0; rr < RR; rr++) au[rr] = ad[rr] = 0.0;
  for (int m = 0; m < jd; m++) {
    const double km = wkk[m], kdm = wkd[m];
    const double *lt = R.LiT + (size_t)m * nn;
#pragma unroll
    for (int rr = 0; rr < RR; rr++) {
      const int i = 32 * rr + lane;
      if (i >= m && i < jd) {
        const double l = lt[i];
        au[rr] = fma(l, km, au[rr]);
        ad[rr] = fma(l, kdm, ad[rr]);
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < RR; rr++) {
    const int i = 32 * rr + lane;
    if (i < jd) {
      wu[i] = au[rr];
      wud[i] = ad[rr];
    }
  }
  __syncwarp();
  // Q u (Q symmetric, stored in full)
  double aq[RR];
#pragma unroll
  for (int rr = 0; rr < RR; rr++) aq[rr] = 0.0;
  for (int a = 0; a < jd; a++) {
    const double ua = wu[a];
    const double *qa = R.Qf + (size_t)a * nn;
#pragma unroll
    for (int rr = 0; rr < RR; rr++) {
      const int b = 32 * rr + lane;
      if (b < jd) aq[rr] = fma(qa[b], ua, aq[rr]);
    }
  }
  double s_uu = 0.0, s_ux = 0.0, s_kz = 0.0, s_pc = 0.0, s_mn = 0.0, s_qn = 0.0;
#pragma unroll
  for (int rr = 0; rr < RR; rr++) {
    const int i = 32 * rr + lane;
    if (i < jd) {
      const double u = au[rr], ud = ad[rr];
      s_uu = fma(u, u, s_uu);
      s_ux = fma(R.ux[i], u, s_ux);
      s_kz = fma(ud, u, s_kz);
      s_pc = fma(ud, R.yt[i], s_pc);
      s_mn = fma(u, R.r[i], s_mn);
      s_qn = fma(u, aq[rr], s_qn);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s_uu += __shfl_xor_sync(0xffffffffu, s_uu, o);
    s_ux += __shfl_xor_sync(0xffffffffu, s_ux, o);
    s_kz += __shfl_xor_sync(0xffffffffu, s_kz, o);
    s_pc += __shfl_xor_sync(0xffffffffu, s_pc, o);
    s_mn += __shfl_xor_sync(0xffffffffu, s_mn, o);
    s_qn += __shfl_xor_sync(0xffffffffu, s_qn, o);
  }
  const double vc = R.onepg - s_uu;
  if (!(vc > 0.0)) return NAN;
  const double cx = corr64(R.xl, xc, p, R.theta_inv, R.etab) - s_ux;
  const double Vc = R.psi * vc / dj;
  const double dmuc = s_pc - s_mn;
  const double dVc = (-R.wKdw * vc - R.psi * (2.0 * s_kz - s_qn)) / dj;
  const double G = R.F + dVc * dVc / (2.0 * Vc * Vc) + dmuc * dmuc / Vc;
  return R.psi / dj * (R.vx - cx * cx / vc) + R.dmux * R.dmux / G;
}

// Candidates within 2 DELTA of the screen's best (or flagged) are re-scored; returns (to
// every thread, after a barrier) the rank of the FP64 minimum, or -1 when none is valid.
__device__ int mspe_rescore(const MRescore &R, float B1) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jd = R.jd;
  if (tid == 0) *R.nlist = 0;
  __syncthreads();
  const float lim = B1 + 2.0f * DELTA * fabsf(B1);
  for (int c = tid; c < R.M; c += XB) {
    if (R.used[c]) continue;
    if (R.flg[c] || R.Jsc[c] <= lim) {
      const int pos = atomicAdd(R.nlist, 1);
      if (pos < RESCORE_CAP) R.rlist[pos] = c;
    }
  }
  __syncthreads();
  const bool all = *R.nlist > RESCORE_CAP;
  const int nl = all ? R.M : *R.nlist;
  const double dj = (double)(jd - 2);
  double bs = INFINITY;
  int br = 0x7fffffff;
  for (int item = warp; item < nl; item += XB / 32) {
    const int c = all ? item : R.rlist[item];
    if (R.used[c]) continue;
    // rows per lane sized to the design, so no FP64 instruction runs for absent rows
    const double Jc = jd <= 64 ? rescore_one<2>(R, c, dj) : rescore_one<kMaxN / 32>(R, c, dj);
    if (Jc == Jc && j_better64(Jc, c, bs, br)) {
      bs = Jc;
      br = c;
    }
    __syncwarp();  // the scratch is rewritten for the next candidate
  }
  if (lane == 0) {
    R.red_s[warp] = bs;
    R.red_r[warp] = br;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < XB / 32; w++)
      if (j_better64(R.red_s[w], R.red_r[w], bs, br)) {
        bs = R.red_s[w];
        br = R.red_r[w];
      }
    R.red_r[0] = br;
  }
  __syncthreads();
  const int b = R.red_r[0];
  return b == 0x7fffffff ? -1 : b;
}

template <int RG>
__global__ void __launch_bounds__(XB, LAGP_MSPE_MIX_MINB) select_mspe_mixed_kernel(MxParams P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Qpad = P.Qpad, Mpad = P.Mpad, nn = P.nmax;
  const int nrow = (nn + 1) & ~1;
  float4 *vp = reinterpret_cast<float4 *>(smraw);   // Qpad: v_j(c) pairs
  float4 *cp = vp + Qpad;                            // Qpad: cov_j(x, c) pairs
  float4 *sr4 = cp + Qpad;                           // nrow: u_s as {h, h, -h, -h}
  float4 *qr4 = sr4 + nrow;                          // nrow: -q_j likewise
  float2 *sr2 = reinterpret_cast<float2 *>(qr4 + nrow);  // nrow: {l, l}
  float2 *qr2 = sr2 + nrow;
  double *srow = reinterpret_cast<double *>(qr2 + nrow);  // nn: u_s (FP64)
  double *qrow = srow + nn;     // nn: row j of Q
  double *rrow = qrow + nn;     // nn: row j of R
  double *ux = rrow + nn;       // nn: L^{-1} k(x)
  double *udx = ux + nn;        // nn: L^{-1} kd(x)
  double *yt = udx + nn;        // nn: L^{-1} Y
  double *r = yt + nn;          // nn: Q ytil
  double *t1 = r + nn;          // nn: Kd Li[j]^T
  double *t2 = t1 + nn;         // nn: Kdd Li[j]^T
  double *ks = t2 + nn;         // nn: k_j(s)
  float *Jsc = reinterpret_cast<float *>(ks + nn);  // Mpad
  int *dr = reinterpret_cast<int *>(Jsc + Mpad);    // nn (padded to 4): ranks of the design
  int *dg = dr + ((nn + 3) & ~3);                   // nn (padded to 4): design indices in X
  int *rlist = dg + ((nn + 3) & ~3);                // RESCORE_CAP
  unsigned char *used = reinterpret_cast<unsigned char *>(rlist + RESCORE_CAP);  // Mpad
  unsigned char *flg = used + Mpad;                                             // Mpad
  float4 *ring = reinterpret_cast<float4 *>(flg + Mpad) + threadIdx.x;  // RG x 2 x XB
  // the FP64 step's partial sums (2 x XB doubles) reuse the ring, idle outside the screen
  double *part = reinterpret_cast<double *>(flg + Mpad);
  __shared__ float tabh[64], tabl[64];
  __shared__ double etab[64];
  __shared__ double xs[kMaxP], xl[kMaxP];
  __shared__ float2 sxs[kMaxP];
  __shared__ float red_s1[2][XB / 32], red_s2[2][XB / 32];
  __shared__ int red_r1[2][XB / 32];
  __shared__ double red_s[XB / 32];
  __shared__ int red_r[XB / 32];
  __shared__ double sh_d[8];  // 0 inv, 1 uxj, 2 ytj, 3 rj, 4 F, 5 dmux, 6 wKdw
  __shared__ double sh_dot[4];
  __shared__ int sh_loc, sh_fail, sh_nlist;
  __shared__ double sh_psi, sh_vx, sh_trR, sh_nQ2, sh_yRy, sh_zs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 64) {
    tabh[tid] = c_exp.tabf_h[tid];
    tabl[tid] = c_exp.tabf_l[tid];
    etab[tid] = c_exp.tab[tid];
  }
  float4 *U = P.U + (size_t)blockIdx.x * nn * Qpad;
  float4 *Ud = P.Ud + (size_t)blockIdx.x * nn * Qpad;
  float4 *Xr = P.Xr + (size_t)blockIdx.x * P.pmax * Qpad;
  float4 *cs = P.cs + (size_t)blockIdx.x * 4 * Qpad;
  double *Li = P.Li + (size_t)blockIdx.x * nn * nn;
  double *LiT = P.LiT + (size_t)blockIdx.x * nn * nn;
  double *Kd = P.Kd + (size_t)blockIdx.x * nn * nn;
  double *Kdd = P.Kdd + (size_t)blockIdx.x * nn * nn;
  double *Qf = P.Qf + (size_t)blockIdx.x * nn * nn;
  double *wk = P.Wk + ((size_t)blockIdx.x * (XB / 32) + warp) * 4 * nn;

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    if (sh_loc >= P.T) break;
    const LocParams L = resolve_loc(P.B, sh_loc, P.X, P.Z, P.XX, P.p, P.n, P.M, P.n0, P.theta,
                                    P.g, P.cand, P.idx);
    const int n = L.n, p = L.p, M = L.M;
    const int32_t *cnd = L.cand;
    const double th = L.theta, th2 = th * th, th3 = th2 * th, th4 = th2 * th2;
    const double ith2 = 1.0 / th2, ith3 = 1.0 / th3, ith4 = 1.0 / th4;
    const ff thinv = ff_from_double(L.theta_inv);
    const ff onepg = ff_from_double(L.onepg);
    // the start design: the n0 nearest, or a saved design (augmentation)
    const int n0e = P.start ? P.nstart : L.n0;
    // Without greedy steps (n0 == n) only the start design's own rows are ever read.
    const int Q = ((n0e == n && !P.start ? n : M) + 1) >> 1;
    if (tid < p) xl[tid] = L.x[tid];
    if (tid == 0) {
      sh_fail = 0;
      sh_psi = 0.0; sh_vx = L.onepg; sh_trR = 0.0; sh_nQ2 = 0.0; sh_yRy = 0.0;
    }
    __syncthreads();
    // coordinates relative to x, v = 1+g, cov_0(x,c) = K(x,c), the four sums at 0
    for (int q = tid; q < Qpad; q += XB) {
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
        flg[c] = 0;
        Jsc[c] = INFINITY;
      }
      vp[q] = make_float4(onepg.h, onepg.h, onepg.l, onepg.l);
      cp[q] = make_float4(cv[0].h, cv[1].h, cv[0].l, cv[1].l);
      for (int e = 0; e < 4; e++) cs[e * Qpad + q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    if (P.start) start_ranks(P.start + L.loc * P.nstart, P.nstart, cnd, M, dr);

    int best = 0;
    for (int j = 0; j < n; j++) {
      const int s = (j < n0e) ? (P.start ? dr[j] : j) : best;
      if (s < 0) {  // nothing admissible left (the same for every thread)
        if (tid == 0) sh_fail = 1;
        break;
      }
      // ---- FP64 phase A: the pivot's coordinates, k_j(s), Kd and Kdd rows, u_s = L^{-1} k_j(s)
      // the pivot's coordinates and response in one round of loads
      if (tid <= p) {
        const int64_t gs = cnd[s];
        if (tid < p) xs[tid] = L.X[gs * p + tid];
        else sh_zs = L.Z[gs];
      }
      __syncthreads();
      for (int i = tid; i <= j; i += XB) {
        double kk = 0.0, kd = 0.0, kdd = 0.0;
        if (i < j) {
          const double *xi = L.X + (int64_t)dg[i] * p;
          double acc = 0.0;
          for (int k = 0; k < p; k++) {
            const double t = xs[k] - xi[k];
            acc = fma(t, t, acc);
          }
          kk = exp_nonpos(-acc * L.theta_inv, etab);
          kd = kk * acc * ith2;
          kdd = kk * (acc * acc * ith4 - 2.0 * acc * ith3);
          ks[i] = kk;
        }
        // Kd and Kdd are kept symmetric in full, so that every product reads rows
        Kd[(size_t)j * nn + i] = kd;
        Kdd[(size_t)j * nn + i] = kdd;
        Kd[(size_t)i * nn + j] = kd;
        Kdd[(size_t)i * nn + j] = kdd;
      }
      __syncthreads();
      // u_s[i] = sum_{m <= i} L^{-1}[i][m] k_j(s)[m]
      split_rows(Li, ks, nullptr, nullptr, nn, j, [](int) { return 0; },
                 [](int i) { return i + 1; }, part, [&](int i, double v, double) {
                   srow[i] = v;
                   const ff f = ff_from_double(v);
                   sr4[i] = make_float4(f.h, f.h, -f.h, -f.h);
                   sr2[i] = f2s(f.l);
                 });
      // u_s.u_s, u_s.u_x, u_s.ytil, u_s.udx: one warp each
      if (warp < 4) {
        double acc = 0.0;
        const double *vec = warp == 0 ? srow : warp == 1 ? ux : warp == 2 ? yt : udx;
        for (int i = lane; i < j; i += 32) acc = fma(srow[i], vec[i], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) sh_dot[warp] = acc;
      }
      __syncthreads();
      if (tid == 0) {
        const double vs = L.onepg - sh_dot[0];  // v_j(s)
        if (!(vs > 0.0)) {
          sh_fail = 1;
        } else {
          const double sq = sqrt(vs);
          const double inv = 1.0 / sq;
          double acc = 0.0;
          for (int k = 0; k < p; k++) {
            const double t = xl[k] - xs[k];
            acc = fma(t, t, acc);
          }
          const double kxs = exp_nonpos(-acc * L.theta_inv, etab);
          const double kdxs = kxs * acc * ith2;
          const double uxj = (kxs - sh_dot[1]) * inv;
          const double ytj = (sh_zs - sh_dot[2]) * inv;
          ux[j] = uxj;
          udx[j] = (kdxs - sh_dot[3]) * inv;
          yt[j] = ytj;
          sh_d[0] = inv;
          sh_d[1] = uxj;
          sh_d[2] = ytj;
          sh_psi = fma(ytj, ytj, sh_psi);
          sh_vx = fma(-uxj, uxj, sh_vx);
          dr[j] = s;
          dg[j] = cnd[s];
          used[s] = 1;
        }
      }
      __syncthreads();
      if (sh_fail) break;
      const double inv = sh_d[0];
      // ---- FP64 phase B: row j of L^{-1} (and column j of its transpose):
      // L^{-1}[j][i] = -inv sum_{i <= m < j} u_s[m] L^{-1}[m][i], a row of the transpose
      double *lrow = ks;  // k_j(s) is no longer needed
      split_rows(LiT, srow, nullptr, nullptr, nn, j, [](int i) { return i; },
                 [j](int) { return j; }, part, [&](int i, double v, double) {
                   const double li = -v * inv;
                   lrow[i] = li;
                   Li[(size_t)j * nn + i] = li;
                   LiT[(size_t)i * nn + j] = li;
                 });
      if (tid == 0) {
        lrow[j] = inv;
        Li[(size_t)j * nn + j] = inv;
        LiT[(size_t)j * nn + j] = inv;
      }
      __syncthreads();
      // t1 = Kd Li[j]^T, t2 = Kdd Li[j]^T over rows a <= j
      split_rows(Kd, lrow, Kdd, lrow, nn, j + 1, [](int) { return 0; }, [j](int) { return j + 1; },
                 part, [&](int a, double v1, double v2) {
                   t1[a] = v1;
                   t2[a] = v2;
                 });
      // row j of Q and R: (Li t)[b] = sum_{a <= b} Li[b][a] t[a]; Q is kept in full
      split_rows(Li, t1, Li, t2, nn, j + 1, [](int) { return 0; }, [](int b) { return b + 1; },
                 part, [&](int b, double v1, double v2) {
                   Qf[(size_t)j * nn + b] = v1;
                   Qf[(size_t)b * nn + j] = v1;
                   qrow[b] = v1;
                   rrow[b] = v2;
                 });
      // r = Q ytil: old entries gain Q[j][i] ytil_j; entry j is row j of Q dotted with ytil
      const double ytj = sh_d[2];
      for (int i = tid; i < j; i += XB) {
        r[i] = fma(qrow[i], ytj, r[i]);
        const ff f = ff_from_double(-qrow[i]);
        qr4[i] = make_float4(f.h, f.h, -f.h, -f.h);
        qr2[i] = f2s(f.l);
      }
      if (warp == XB / 32 - 1 && lane < p) {
        const ff f = ff_from_double(xs[lane] - xl[lane]);
        sxs[lane] = make_float2(f.h, f.l);
      }
      if (warp == 0) {
        double a = 0.0, nq = 0.0, yr = 0.0;
        for (int i = lane; i <= j; i += 32) {
          a = fma(qrow[i], yt[i], a);
          if (i < j) {
            nq = fma(qrow[i], qrow[i], nq);
            yr = fma(rrow[i], yt[i], yr);
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_down_sync(0xffffffffu, a, o);
          nq += __shfl_down_sync(0xffffffffu, nq, o);
          yr += __shfl_down_sync(0xffffffffu, yr, o);
        }
        if (lane == 0) {
          r[j] = a;
          sh_d[3] = a;
          sh_trR += rrow[j];
          sh_nQ2 += 2.0 * nq + qrow[j] * qrow[j];
          sh_yRy += 2.0 * ytj * yr + rrow[j] * ytj * ytj;
        }
      }
      __syncthreads();
      if (warp == 0) {
        // w^T Kd w = ytil . r, ||r||^2 and dmu_x = udx . ytil - ux . r over the new design
        double wkd = 0.0, nr = 0.0, dm = 0.0;
        for (int i = lane; i <= j; i += 32) {
          wkd = fma(yt[i], r[i], wkd);
          nr = fma(r[i], r[i], nr);
          dm = fma(udx[i], yt[i], dm);
          dm = fma(-ux[i], r[i], dm);
        }
        for (int o = 16; o > 0; o >>= 1) {
          wkd += __shfl_down_sync(0xffffffffu, wkd, o);
          nr += __shfl_down_sync(0xffffffffu, nr, o);
          dm += __shfl_down_sync(0xffffffffu, dm, o);
        }
        if (lane == 0) {
          const double jd = (double)(j + 1), psi = sh_psi;
          // Eq. d2l: l'' = -1/2 (tr R - ||Q||^2) + j/(2 psi)(ytil^T R ytil - 2 ||r||^2)
          //                + j/(2 psi^2) (ytil . r)^2
          const double l2 = -0.5 * (sh_trR - sh_nQ2) + jd / (2.0 * psi) * (sh_yRy - 2.0 * nr) +
                            jd / (2.0 * psi * psi) * wkd * wkd;
          sh_d[4] = -l2;
          sh_d[5] = dm;
          sh_d[6] = wkd;
        }
      }
      __syncthreads();
      if (j == n - 1) break;
      // ---- float-float screen of every remaining candidate, O(j)
      const int jn = j + 1;  // design size after this step
      const bool want = (jn >= n0e) && (jn >= 3);
      const double dj = (double)(jn - 2);
      const double psi = sh_psi, F = sh_d[4], dmux = sh_d[5], wKdw = sh_d[6];
      MStep C;
      C.U = U; C.Ud = Ud; C.cs = cs; C.vp = vp; C.cp = cp; C.ring = ring; C.Xr = Xr; C.Jsc = Jsc;
      C.flg = flg;
      C.sr4 = sr4; C.qr4 = qr4; C.sr2 = sr2; C.qr2 = qr2; C.sxs = sxs; C.tabh = tabh; C.tabl = tabl;
      C.inv = ff2_bcast(ff_from_double(inv));
      C.uxj = ff2_bcast(ff_from_double(sh_d[1]));
      C.ytj = ff2_bcast(ff_from_double(ytj));
      C.rj = ff2_bcast(ff_from_double(sh_d[3]));
      C.qjj = ff2_bcast(ff_from_double(qrow[j]));
      C.thinv = ff2_bcast(thinv);
      C.a = ff2_bcast(ff_from_double(want ? psi / dj : 0.0));
      C.vx = ff2_bcast(ff_from_double(sh_vx));
      C.wd = ff2_bcast(ff_from_double(want ? wKdw / dj : 0.0));
      C.F = ff2_bcast(ff_from_double(F));
      C.dmux2 = ff2_bcast(ff_from_double(dmux * dmux));
      C.Ff = (float)F;
      C.Qpad = Qpad; C.p = p; C.j = j; C.want = want;
      float b1 = INFINITY, b2 = INFINITY;
      int r1 = 0x7fffffff, nf = 0;
      for (int q = tid; q < Q; q += XB) {
        if (used[2 * q] && used[2 * q + 1]) continue;
        mspe_pair<RG>(C, q, used, b1, r1, b2, nf);
      }
      // best and second-best screen scores (double-buffered by step parity)
      const int par = j & 1;
      for (int o = 16; o > 0; o >>= 1) {
        const float ob1 = __shfl_down_sync(0xffffffffu, b1, o);
        const float ob2 = __shfl_down_sync(0xffffffffu, b2, o);
        const int orr = __shfl_down_sync(0xffffffffu, r1, o);
        merge_min(ob1, orr, ob2, b1, r1, b2);
      }
      if (lane == 0) {
        red_s1[par][warp] = b1;
        red_s2[par][warp] = b2;
        red_r1[par][warp] = r1;
      }
      const int fl = __syncthreads_or(nf);  // a candidate the screen cannot resolve
      if (!want) continue;
      float B1 = red_s1[par][0], B2 = red_s2[par][0];
      int R1 = red_r1[par][0];
      for (int w = 1; w < XB / 32; w++) merge_min(red_s1[par][w], red_r1[par][w], red_s2[par][w], B1, R1, B2);
      best = (R1 == 0x7fffffff) ? -1 : R1;
      const bool near = R1 != 0x7fffffff && B2 - B1 <= DELTA * fabsf(B1);
      if (!near && !fl) continue;
      // ---- FP64 re-score of the near-tied or unresolved candidates (rare) ----
      if (tid == 0 && P.rescores) atomicAdd(P.rescores, 1);
      MRescore R;
      R.X = L.X; R.cnd = cnd; R.xl = xl; R.etab = etab; R.used = used; R.flg = flg; R.Jsc = Jsc;
      R.dg = dg; R.LiT = LiT; R.Qf = Qf; R.ux = ux; R.yt = yt; R.r = r; R.wk = wk;
      R.rlist = rlist; R.nlist = &sh_nlist; R.red_s = red_s; R.red_r = red_r;
      R.p = p; R.M = Q * 2 < M ? Q * 2 : M; R.jd = jn; R.nn = nn;
      R.theta_inv = L.theta_inv; R.ith2 = ith2; R.onepg = L.onepg; R.psi = psi; R.vx = sh_vx;
      R.F = F; R.dmux = dmux; R.wKdw = wKdw;
      const int b = mspe_rescore(R, R1 == 0x7fffffff ? INFINITY : B1);
      best = b;
    }
    __syncthreads();
    // the design (design indices), or -1 when a step failed; kernel (c) evaluates the
    // predictive equations on it in FP64
    for (int i = tid; i < n; i += XB) L.idx[i] = sh_fail ? -1 : dg[i];
  }
}

int mxm_mpad(int M) { return (int)align_up((size_t)M, 64); }

// Dynamic shared memory with a ring of RG stages (RG = 0: no ring, only the FP64 step's
// partial sums, which otherwise live in the ring).
size_t mxm_smem_bytes(int Mpad, int n, int RG) {
  const size_t Qpad = (size_t)Mpad / 2;
  const size_t nrow = (size_t)((n + 1) & ~1);
  const size_t tail = RG ? (size_t)RG * 2 * XB * sizeof(float4) : (size_t)2 * XB * sizeof(double);
  return Qpad * 2 * sizeof(float4) + nrow * 2 * (sizeof(float4) + sizeof(float2)) +
         (size_t)n * 10 * sizeof(double) + (size_t)Mpad * sizeof(float) +
         2 * (size_t)((n + 3) & ~3) * sizeof(int) + RESCORE_CAP * sizeof(int) + 2 * (size_t)Mpad +
         tail;
}

int mxm_grid(int64_t T, int num_sms) {
  const int64_t g = (int64_t)num_sms * LAGP_MSPE_MIX_MINB;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

struct MxLayout {
  size_t u, xr, cs, nn, wk, idx, pred, total;
};

// [queue | re-score counter | U | Ud | Xr | cs | Li, LiT, Kd, Kdd, Qf | Wk | design indices |
//  kernel (c) workspace]
MxLayout mxm_layout(int G, int p, int n, int M, int64_t T, int64_t idx_total, int num_sms) {
  const size_t Qpad = (size_t)mxm_mpad(M) / 2;
  MxLayout L;
  L.u = align_up((size_t)G * n * Qpad * sizeof(float4), 256);
  L.xr = align_up((size_t)G * p * Qpad * sizeof(float4), 256);
  L.cs = align_up((size_t)G * 4 * Qpad * sizeof(float4), 256);
  L.nn = align_up((size_t)G * n * n * sizeof(double), 256);
  L.wk = align_up((size_t)G * (XB / 32) * 4 * n * sizeof(double), 256);
  L.idx = align_up((size_t)idx_total * sizeof(int32_t), 256);
  L.pred = predict_fp64_workspace_bytes(T, n, num_sms);
  L.total = 512 + 2 * L.u + L.xr + L.cs + 5 * L.nn + L.wk + L.idx + L.pred;
  return L;
}

// The design kernel, then kernel (c) (predict.cu) on the designs it selected.
int mxm_run(MxParams P, const MxLayout &L, int G, char *w, int32_t *user_idx, const DevInfo &di,
            cudaStream_t stream) {
  P.queue = reinterpret_cast<int *>(w);
  P.rescores = reinterpret_cast<int *>(w + 256);
  size_t off = 512;
  P.U = reinterpret_cast<float4 *>(w + off); off += L.u;
  P.Ud = reinterpret_cast<float4 *>(w + off); off += L.u;
  P.Xr = reinterpret_cast<float4 *>(w + off); off += L.xr;
  P.cs = reinterpret_cast<float4 *>(w + off); off += L.cs;
  P.Li = reinterpret_cast<double *>(w + off); off += L.nn;
  P.LiT = reinterpret_cast<double *>(w + off); off += L.nn;
  P.Kd = reinterpret_cast<double *>(w + off); off += L.nn;
  P.Kdd = reinterpret_cast<double *>(w + off); off += L.nn;
  P.Qf = reinterpret_cast<double *>(w + off); off += L.nn;
  P.Wk = reinterpret_cast<double *>(w + off); off += L.wk;
  P.idx = user_idx ? user_idx : reinterpret_cast<int32_t *>(w + off);
  off += L.idx;
  const bool ring = mxm_smem_bytes(P.Mpad, P.nmax, RING) <= di.smem_optin;
  const size_t smem = mxm_smem_bytes(P.Mpad, P.nmax, ring ? RING : 0);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = ring ? cudaFuncSetAttribute(select_mspe_mixed_kernel<RING>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(select_mspe_mixed_kernel<0>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(w, 0, 512, stream);  // work counter and re-score counter
  if (e != cudaSuccess) return cuda_status(e);
  if (ring)
    select_mspe_mixed_kernel<RING><<<G, XB, smem, stream>>>(P);
  else
    select_mspe_mixed_kernel<0><<<G, XB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  PredictArgs pa;
  pa.X = P.X; pa.Z = P.Z; pa.p = P.pmax; pa.XX = P.XX; pa.T = P.T; pa.n = P.n; pa.nmax = P.nmax;
  pa.theta = P.theta; pa.g = P.g; pa.idx = P.idx; pa.B = P.B;
  pa.mean = P.mean; pa.s2 = P.s2; pa.var = P.var; pa.status = P.status;
  return predict_fp64_launch(pa, w + off, L.pred, stream);
}

}  // namespace

size_t select_mspe_mixed_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms) {
  return mxm_layout(mxm_grid(T, num_sms), p, n, ncand, T, T * n, num_sms).total;
}

int select_mspe_mixed_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  const int G = mxm_grid(a.T, di.num_sms);
  const MxLayout L = mxm_layout(G, a.p, a.n, a.M, a.T, a.T * a.n, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MxParams P;
  P.X = a.X; P.Z = a.Z; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Mpad = mxm_mpad(a.M); P.Qpad = P.Mpad / 2; P.n0 = a.n0; P.n = a.n;
  P.theta = a.theta; P.g = a.g;
  P.nmax = a.n; P.pmax = a.p;
  P.B = BatchView{nullptr, nullptr, nullptr, 0, a.theta_loc, nullptr};
  P.start = a.start; P.nstart = a.nstart;
  P.mean = a.mean; P.s2 = a.s2; P.var = a.var; P.status = a.status;
  return mxm_run(P, L, G, static_cast<char *>(ws), a.idx, di, stream);
}

size_t select_mspe_mixed_batch_workspace_bytes(const BatchLaunch &b, int G) {
  DevInfo di;
  const int sms = dev_info(&di) == LAGP_OK ? di.num_sms : 152;
  return mxm_layout(G, b.pmax, b.nmax, b.Mmax, b.T, b.idx_total, sms).total;
}

int select_mspe_mixed_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, int G,
                                   cudaStream_t stream) {
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();  // this translation unit's copy of the exp constants
  if (st) return st;
  const MxLayout L = mxm_layout(G, b.pmax, b.nmax, b.Mmax, b.T, b.idx_total, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MxParams P;
  P.X = nullptr; P.Z = nullptr; P.p = b.pmax; P.XX = b.XX; P.T = b.T; P.cand = b.cand;
  P.M = b.Mmax; P.Mpad = mxm_mpad(b.Mmax); P.Qpad = P.Mpad / 2; P.n0 = 0; P.n = b.nmax;
  P.theta = 1.0; P.g = 0.0;
  P.nmax = b.nmax; P.pmax = b.pmax;
  P.B = BatchView{b.designs, b.locs, b.order, b.ldxx, nullptr, nullptr};
  P.start = nullptr; P.nstart = 0;
  P.mean = b.mean; P.s2 = b.s2; P.var = b.var; P.status = b.status;
  return mxm_run(P, L, G, static_cast<char *>(ws), b.idx, di, stream);
}

int select_mspe_mixed_prepare() {
  const int st = exp_table_upload();
  return st ? st : predict_fp64_prepare();
}

}  // namespace lagp
