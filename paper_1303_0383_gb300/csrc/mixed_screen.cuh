// mixed_screen.cuh -- device code of the mixed-precision screens: the float-float exp, the
// asynchronous row copies and L2 policies, the ALC per-pair step, score tracking and the
// ALC FP64 re-score (select_mixed.cu; the MSPE kernel, select_mspe_mixed.cu, uses the
// first parts).
//
// Gramacy & Apley, Sec. 3: the greedy local design adds the candidate that maximises the
// ALC reduction cov_j(x,c)^2 / v_j(c) (Eq. dxy; SM Eq. dxy2); Sec. 3.2 gives the O(j)
// update of every candidate's quantities when the design grows by one point.
// Included by one translation unit each: c_exp is that unit's copy of the exp constants.
#pragma once

#include <math.h>

#include "check.cuh"
#include "ff.cuh"
#include "ff2.cuh"
#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {
namespace {

constexpr float DELTA = 1e-5f;     // near-tie margin for the FP64 re-score


constexpr int RESCORE_CAP = 64;    // candidates re-scored per pass

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

// The screen's ALC score cov^2 / v from the leading FP32 words, with the approximate FP32
// quotient (a reciprocal and a product, within 2 ulp): the screen only ranks, and any pair
// of scores whose order that error could swap lies well inside the near-tie band DELTA,
// whose candidates are re-scored in FP64.  The same expression forms every screen score, so
// the tracked best and the near-tie list agree.  (An IEEE quotient here: 0.8 % slower.)
__device__ __forceinline__ float screen_score(float c, float v) { return __fdividef(c * c, v); }

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
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < j; k++) {
    if (tid == 0) {
      const double d = A[k * lda + k];
      if (!(d > 0.0)) *fail = 1;
      A[k * lda + k] = sqrt(d);
    }
    __syncthreads();
    if (*fail) return;
    const double lkk = A[k * lda + k];
    for (int i = k + 1 + tid; i < j; i += nt) A[i * lda + k] = A[i * lda + k] / lkk;
    if (tid < naug) A[k * lda + j + tid] = A[k * lda + j + tid] / lkk;
    __syncthreads();
    const int w = j - k - 1 + naug;
    const int rows = j - k - 1;
    for (int q = tid; q < rows * w; q += nt) {
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

// Asynchronous 16-byte copies global -> shared (cp.async, L2 only) and their groups: a
// thread's factor rows in global memory reach its own slots of a ring in shared memory a
// few rows ahead of their use, so that the loads of the next rows are in flight while a
// row is consumed.  Each thread waits only for its own copies (no barrier).
constexpr int RING_A = 4;  // stages per thread, where the ring is used

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Factor-row loads with an L2 evict-last policy: a row is read again at every later step of
// the location, so on the workloads whose live rows fit in L2 they are kept there ahead of
// data read once (candidate lists, coordinates).  paper-2d: 14.85 -> 14.38 ms.
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double ld_l2_hint(const double *a, unsigned long long pol) {
  double v;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void cp_async16_l2_hint(float4 *smem_dst, const float4 *gmem_src,
                                                   unsigned long long pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s),
               "l"(gmem_src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ float4 ld_l2_hint(const float4 *a, unsigned long long pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(pol));
  return v;
}

// Tensor memory as a second on-chip store for factor rows (no tensor-core work): a CTA
// allocates 128 columns of its SM's tensor memory; warp w may address only the 32 lanes of
// its sub-partition, 32 (w & 3) .. 32 (w & 3) + 31, and takes columns 64 (w >> 2) .. + 63 of
// them, so every thread owns 64 32-bit words of its own lane.  Loads and stores are
// warp-collective (every lane of the warp executes them with the same address).  The load's
// wait is tied to the registers it delivers, so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t ta, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(ta));
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t (&v)[16]) {
  tmem_ld16_issue(ta, v);
  tmem_wait16(v);
}
__device__ __forceinline__ void tmem_st4(uint32_t ta, float4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ta),
               "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
               "r"(__float_as_uint(v.w))
               : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
constexpr int kTmemCols = 128;  // columns per CTA: 3 or 4 resident CTAs per SM hold 384 or 512,
                                // and the host checks the residency before it launches

// One step of the screen for one candidate pair of this thread (Sec. 3.2 update, in
// float-float): K(s, c) from the squared distance, the new factor entry
// u_c[j] = (K(s, c) - u_s . u_c) / L_jj, then v_{j+1}(c) = v_j(c) - u_c[j]^2,
// cov_{j+1}(x, c) = cov_j(x, c) - u_x[j] u_c[j], and the ALC screen score cov^2 / v.
struct StepCtx {
  float4 *U;     // factor rows in global memory (rows R .. n-1 are used)
  float4 *Us;    // the first R rows, in shared memory
  int R;
  float4 *ring;  // this thread's ring slots: stage k at ring[k * blockDim.x]
  const float4 *Xr;
  float4 *vp, *cp;
  const float4 *srow4;
  const float2 *srow2, *sxs;
  const float *tabh, *tabl;
  ff2 inv2, uxj2;
  int Qpad, p, j;
  int c0;        // global rank of the first candidate held here
  bool want;
  uint32_t tb;   // tensor-memory instance: this thread's first column (lane and column fields)
  int RT;        // rows R .. R + RT - 1 also held there (a read copy), RT words x 4 per pair
};

// RA = 0: the global rows are loaded straight into registers (four in flight); RA > 0:
// they stream through a ring of RA stages.  The ring pays where the rows come from DRAM
// (large n x M); where they mostly hit L2 its bookkeeping costs more than it hides.
// u0, u1: the pair's used flags (read once by the caller).
// TM: rows R .. R + RT - 1 are read from this thread's tensor-memory words instead of L2 or
// the ring (they are still written to global memory, where the step's pivot row is
// gathered from); the caller keeps every warp convergent.
// ps: the pair's slot among this thread's pairs (q = threadIdx.x + ps * blockDim.x), given
// by the caller's loop so that no division is needed here.
template <int RA, bool TM = false>
__device__ __forceinline__ void screen_pair(const StepCtx &C, int q, bool u0, bool u1, float &b1,
                                            int &r1, float &b2, int ps = 0) {
  const int nt = blockDim.x;
  const int jr = C.j < C.R ? C.j : C.R;  // rows R .. j-1 come from global memory
  // with tensor memory: rows R .. jt-1 from there, jt .. j-1 from global memory
  const int jt = TM ? max(jr, min(C.j, C.R + C.RT)) : jr;
  const uint32_t ta = TM ? C.tb + (uint32_t)(ps * C.RT * 4) : 0u;
  // checked build: this pair's tensor-memory words end within the thread's 64 (the test is
  // the same for a whole warp, whose pairs share ps)
  if constexpr (TM)
    if (!LAGP_CHK((ps + 1) * C.RT * 4 - 1, 64, 18)) return;
  // the first RA - 1 global rows start on their way (one copy group each); streamed rows
  // do not fit in L2 anyway, so they go evict-first and leave it to the data re-read every
  // step (candidate coordinates; 8-d workload 156.2 -> 140.5 ms)
  unsigned long long polf = 0;
  if constexpr (RA > 0) {
    polf = l2_evict_first_policy();
#pragma unroll
    for (int st = 0; st < RA - 1; st++) {
      if (jt + st < C.j)
        cp_async16_l2_hint(C.ring + st * nt, C.U + (size_t)(jt + st) * C.Qpad + q, polf);
      cp_async_commit();
    }
  }
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
  const ff2 arg = d2;  // the coordinates are stored scaled by 1/sqrt(theta): arg = d^2 / theta
  const ff2 kc = exp_ff2(ff2{neg2(arg.h), neg2(arg.l)}, C.tabh, C.tabl);   // K(s, c)
  ff2acc acc{kc.h, kc.l};
  // K(s, c) - sum_i u_s[i] u_c[i]: compensated accumulation over the rows held in shared
  // memory, then over those from global memory (loaded directly, or streamed through the
  // ring).  Four rows per iteration, written out: a row pointer per stream and the four
  // loads issued before their terms are accumulated (0.8 % faster than `#pragma unroll 4`
  // of an indexed loop, with 12 % fewer integer instructions).
  {
    const float4 *us = C.Us + q;
    const int Q = C.Qpad;
    int i = 0;
    for (; i + 4 <= jr; i += 4, us += 4 * Q) {
      const float4 b0 = us[0], b1 = us[Q], b2 = us[2 * Q], b3 = us[3 * Q];
      ff2acc_sub_prod(acc, C.srow4[i], C.srow2[i], b0);
      ff2acc_sub_prod(acc, C.srow4[i + 1], C.srow2[i + 1], b1);
      ff2acc_sub_prod(acc, C.srow4[i + 2], C.srow2[i + 2], b2);
      ff2acc_sub_prod(acc, C.srow4[i + 3], C.srow2[i + 3], b3);
    }
    for (; i < jr; i++, us += Q) ff2acc_sub_prod(acc, C.srow4[i], C.srow2[i], *us);
  }
  if constexpr (TM) {
    // four rows per load, each waited for before use: issuing the first load ahead of the
    // shared-memory rows instead keeps its 16 registers live there and spills (13.56 ->
    // 13.90 ms on paper-2d)
    for (int i = jr; i < jt; i += 4) {  // rows past jt are loaded but not used
      uint32_t tw[16];
      tmem_ld16(ta + (uint32_t)(4 * (i - C.R)), tw);
      if (i + 4 <= jt) {  // a whole group (the usual case): no per-row tests
#pragma unroll
        for (int k = 0; k < 4; k++)
          ff2acc_sub_prod(acc, C.srow4[i + k], C.srow2[i + k],
                          make_float4(__uint_as_float(tw[4 * k]), __uint_as_float(tw[4 * k + 1]),
                                      __uint_as_float(tw[4 * k + 2]), __uint_as_float(tw[4 * k + 3])));
      } else {
#pragma unroll
        for (int k = 0; k < 3; k++)
          if (i + k < jt)
            ff2acc_sub_prod(acc, C.srow4[i + k], C.srow2[i + k],
                            make_float4(__uint_as_float(tw[4 * k]), __uint_as_float(tw[4 * k + 1]),
                                        __uint_as_float(tw[4 * k + 2]), __uint_as_float(tw[4 * k + 3])));
      }
    }
  }
  if constexpr (RA == 0) {
    const unsigned long long pol = l2_evict_last_policy();
    const float4 *ug = C.U + (size_t)jt * C.Qpad + q;
    const size_t Q = C.Qpad;
    int i = jt;
    for (; i + 4 <= C.j; i += 4, ug += 4 * Q) {
      const float4 b0 = ld_l2_hint(ug, pol), b1 = ld_l2_hint(ug + Q, pol);
      const float4 b2 = ld_l2_hint(ug + 2 * Q, pol), b3 = ld_l2_hint(ug + 3 * Q, pol);
      ff2acc_sub_prod(acc, C.srow4[i], C.srow2[i], b0);
      ff2acc_sub_prod(acc, C.srow4[i + 1], C.srow2[i + 1], b1);
      ff2acc_sub_prod(acc, C.srow4[i + 2], C.srow2[i + 2], b2);
      ff2acc_sub_prod(acc, C.srow4[i + 3], C.srow2[i + 3], b3);
    }
    for (; i < C.j; i++, ug += Q) ff2acc_sub_prod(acc, C.srow4[i], C.srow2[i], ld_l2_hint(ug, pol));
  } else {
    int sc = 0, sp = RA - 1;  // ring stages of rows i and i + RA - 1
    for (int i = jt; i < C.j; i++) {
      const int ip = i + RA - 1;
      if (ip < C.j) cp_async16_l2_hint(C.ring + sp * nt, C.U + (size_t)ip * C.Qpad + q, polf);
      cp_async_commit();
      cp_async_wait<RA - 1>();  // row i has landed
      const float4 b = C.ring[sc * nt];
      sc = (sc == RA - 1) ? 0 : sc + 1;
      sp = (sp == RA - 1) ? 0 : sp + 1;
      ff2acc_sub_prod(acc, C.srow4[i], C.srow2[i], b);
    }
  }
  const ff2 u = ff2_mul(ff2acc_result(acc), C.inv2);               // u_c[j]
  if constexpr (RA == 0) {
    // the same for the whole CTA: a shared or a global store instead of a generic one
    // (paper-2d 13.93 -> 13.64 ms with the flags read once; slower with the row ring)
    if (C.j < C.R) {
      ff2_store(C.Us + C.j * C.Qpad + q, u);
    } else {
      ff2_store(C.U + (size_t)C.j * C.Qpad + q, u);
      if constexpr (TM)
        if (C.j < C.R + C.RT) tmem_st4(ta + (uint32_t)(4 * (C.j - C.R)), make_float4(u.h.x, u.h.y, u.l.x, u.l.y));
    }
  } else {
    ff2_store((C.j < C.R ? C.Us : C.U) + (size_t)C.j * C.Qpad + q, u);
    if constexpr (TM)
      if (C.j >= C.R && C.j < C.R + C.RT)
        tmem_st4(ta + (uint32_t)(4 * (C.j - C.R)), make_float4(u.h.x, u.h.y, u.l.x, u.l.y));
  }
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
    if (!u0 && v.h.x > 0.0f) track2(screen_score(cx.h.x, v.h.x), C.c0 + 2 * q, b1, r1, b2);
    if (!u1 && v.h.y > 0.0f) track2(screen_score(cx.h.y, v.h.y), C.c0 + 2 * q + 1, b1, r1, b2);
  }
}

// ---- FP64 re-score of near-tied candidates (Sec. 3.3 decisions in FP64) ----
// Scratch and inputs of one CTA's re-score pass.  The CTA holds candidates with global
// ranks c0 .. c0 + Mloc - 1 (local index c = rank - c0); the current design is dr[0..jd)
// (global ranks), its FP64 factor is formed in A (global memory, jd x (jd + 1)).
struct RescoreCtx {
  const double *X;
  const int32_t *cnd;          // the location's candidate list (global ranks -> design rows)
  const double *xl;            // x (shared memory)
  const double *etab;
  const unsigned char *used;   // local flags
  const float4 *vp, *cp;       // local screen state (pairs)
  const int *dr;
  double *A;
  int *rlist, *nlist, *fail;
  double *red_n, *red_d;
  int *red_rr;
  int p, c0, Mloc, jd, lda;
  double theta_inv, onepg;
};

// Every candidate of this CTA whose screen score is within 2 DELTA of B1 is re-scored in
// FP64: the design's FP64 Cholesky factor (with k(x) as an extra column) is formed from
// scratch, and each listed candidate's u = L^{-1} k_c is obtained by forward substitution
// (one warp per candidate), giving v_j(c) = 1 + g - |u|^2 and cov_j(x, c) = k(x, c) - u.u_x.
// On return (all threads, after a barrier): *bn / *bd is the CTA's best FP64 score as a
// fraction, *br its global rank (0x7fffffff if none), or *R.fail set (factor not PD).
__device__ void rescore_fp64(const RescoreCtx &R, float B1, double *bn_out, double *bd_out,
                             int *br_out) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int jd = R.jd, lda = R.lda, p = R.p;
  if (tid == 0) *R.nlist = 0;
  __syncthreads();
  for (int c = tid; c < R.Mloc; c += nt) {
    if (R.used[c]) continue;
    const ff v = ff2_get(R.vp, c), cx = ff2_get(R.cp, c);
    if (!(v.h > 0.0f)) continue;
    const float sc = screen_score(cx.h, v.h);
    if (sc >= B1 * (1.0f - 2.0f * DELTA)) {
      const int pos = atomicAdd(R.nlist, 1);
      if (pos < RESCORE_CAP) R.rlist[pos] = c;
    }
  }
  // FP64 factor of the current design with k(x) as an extra column (lower triangle)
  for (int qq = tid; qq < jd * (jd + 1); qq += nt) {
    const int a = qq / (jd + 1), b = qq % (jd + 1);
    if (b < jd && b > a) continue;
    const double *xa = R.X + (int64_t)R.cnd[R.dr[a]] * p;
    double val;
    if (b < jd) val = (a == b) ? R.onepg : corr64(xa, R.X + (int64_t)R.cnd[R.dr[b]] * p, p, R.theta_inv, R.etab);
    else val = corr64(xa, R.xl, p, R.theta_inv, R.etab);
    R.A[a * lda + b] = val;
  }
  __syncthreads();
  chol_aug_fp64(R.A, jd, lda, 1, R.fail);
  if (*R.fail) return;
  const double *A = R.A;
  // more near-ties than the list holds: re-score every remaining candidate
  const bool all = *R.nlist > RESCORE_CAP;
  const int nl = all ? R.Mloc : *R.nlist;
  double bn = -1.0, bd = 1.0;
  int br = 0x7fffffff;
  for (int item = warp; item < nl; item += nt / 32) {
    const int c = all ? item : R.rlist[item];
    if (R.used[c]) continue;
    const int rank = R.c0 + c;
    const double *xc = R.X + (int64_t)R.cnd[rank] * p;
    double tv[kMaxN / 32];
#pragma unroll
    for (int r = 0; r < kMaxN / 32; r++) {
      const int i = 32 * r + lane;
      tv[r] = (i < jd) ? corr64(R.X + (int64_t)R.cnd[R.dr[i]] * p, xc, p, R.theta_inv, R.etab) : 0.0;
    }
    double vsum = R.onepg;
    double cov = corr64(R.xl, xc, p, R.theta_inv, R.etab);
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
      if (frac_better(num, vsum, rank, bn, bd, br)) {
        bn = num;
        bd = vsum;
        br = rank;
      }
    }
  }
  if (lane == 0) {
    R.red_n[warp] = bn;
    R.red_d[warp] = bd;
    R.red_rr[warp] = br;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < nt / 32; w++)
      if (frac_better(R.red_n[w], R.red_d[w], R.red_rr[w], bn, bd, br)) {
        bn = R.red_n[w];
        bd = R.red_d[w];
        br = R.red_rr[w];
      }
    R.red_n[0] = bn;
    R.red_d[0] = bd;
    R.red_rr[0] = br;
  }
  __syncthreads();
  *bn_out = R.red_n[0];
  *bd_out = R.red_d[0];
  *br_out = R.red_rr[0];
}

}  // namespace
}  // namespace lagp
