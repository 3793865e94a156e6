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
// The predictive equations (Eqs. predgp, preds2) are evaluated in FP64 on each selected
// design with kernel (c)'s arithmetic (predict_loc.cuh) -- by this kernel itself right
// after the design when the matrix fits in its shared memory, else by kernel (c) in
// predict.cu afterwards -- so mu, s2 and V carry FP64 accuracy whatever precision
// screened the candidates.
#include <cooperative_groups.h>
#include <math.h>
#include <stdlib.h>

#include "batch.cuh"
#include "check.cuh"
#include "mixed_screen.cuh"
#include "predict_loc.cuh"

namespace lagp {
namespace {

namespace cg = cooperative_groups;

constexpr int MB = 256;            // threads per CTA
constexpr int kMaxCL = 8;          // CTAs per cluster in the cluster form

struct MixParams {
  const double *X, *Z;
  int64_t N;       // design rows (uniform launches; batched ones take each design's)
  int p;
  const double *XX;
  int64_t T;
  const int32_t *cand;
  int M, Mpad, Qpad, n0, n;  // Mpad = 2 Qpad: candidates (pairs) per CTA slot, padded
  int nmax, pmax;  // slot dimensions (the largest n and p of the launch)
  double theta, theta_inv, g, onepg;
  BatchView B;     // per-location tables (B.designs == nullptr: uniform launch)
  int32_t *idx;   // selected design indices (required: the caller's or the workspace's)
  float4 *U;     // slots of n x Qpad candidate pairs: row j of every candidate's factor row
  int R;         // rows 0 .. R-1 live in shared memory instead
  float4 *Xr;    // slots of p x Qpad pairs: candidate coordinates minus x
  double *A;     // slots of n x (n + 2): FP64 factorisation
  int *queue;
  int *rescores; // count of FP64 re-score passes (diagnostics)
  const int32_t *start;  // saved start designs (T x nstart design indices), or nullptr
  int nstart;
  double r_min;          // > 1: stopping rule of Sec. 6; 0: the design has n points
  int32_t *n_out;        // design sizes (T) when r_min > 1
  double *mean, *s2, *var;
  int8_t *status;
  int fuse_pred;         // 1: the predictive equations here (matrix in shared memory)
  int CL;                // CTAs per cluster (cluster form): they share one location
  int RT;                // tensor-memory instance: rows R .. R + RT - 1 also in tensor memory
};

#ifndef LAGP_MIX_MINB
#define LAGP_MIX_MINB LAGP_MIX_CTAS_PER_SM  // 3 CTAs per SM, each with its first factor rows in shared memory
#endif
// The row-ring instances (one CTA per location) run up to 4 CTAs per SM: their rows come
// from DRAM, and more warps in flight hide more of that (8-d workload, the shared-row-copy
// instance at 4 CTAs per SM: 138.7 -> 133.1 ms).  At 4 CTAs per SM the instance without
// the ring was slower (paper-2d 13.58 -> 15.25 ms: 3 rows in shared memory instead of 5).
constexpr int kRingMinB = 4;
__host__ __device__ constexpr int mix_minb(int RA, bool SR, bool CLU) {
  (void)SR;
  return (RA > 0 && !CLU) ? kRingMinB : LAGP_MIX_MINB;
}
// RA: stages of the row ring (0: none).  SR: one shared copy of the step's factor row for
// the whole CTA (one more block barrier per step) instead of one per warp, which frees
// (MB/32 - 1) row copies of shared memory for the ring on large designs.
// TM: rows R .. R + RT - 1 of each candidate are also kept in the CTA's tensor memory (128
// columns: RT = 16, 8 or 4 rows for 1, 2 or up to 4 pairs per thread) and the screen reads
// them from there instead of L2 (GB300, 24 warps per SM, four 16-byte loads per thread:
// about 200 cycles from tensor memory against about 580 for L2 hits).  One CTA per location
// only (not the cluster form); the ring instances run 4 CTAs per SM, which take all 512
// columns, so the allocation never waits there either.
// CLU: the cluster form.  The P.CL CTAs of a thread-block cluster share one location, CTA
// `crank` holding the candidate pairs crank*Qc .. crank*Qc + Qc - 1 (its own v, cov, flags,
// factor rows and coordinates); a step's pivot state -- v_j(s), cov_j(x,s), u_s and x_s -- is
// read from the CTA that holds s (its shared memory through the cluster, its global rows),
// and the per-warp best scores are merged over the cluster after one cluster barrier.  With
// 1/CL of the locations in flight, the live factor rows shrink by CL and more of each
// CTA's rows fit in shared memory.  Every candidate's arithmetic is the same in both forms.
template <int RA, bool SR, bool CLU, bool TM = false>
__global__ void __launch_bounds__(MB, mix_minb(RA, SR, CLU)) select_mixed_kernel(MixParams P) {
  static_assert(!TM || !CLU, "tensor-memory rows: one CTA per location");
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Qpad = P.Qpad, nmax = P.nmax;
  constexpr int NW = SR ? 1 : MB / 32;                       // copies of the factor row
  float4 *vp = reinterpret_cast<float4 *>(smraw);            // Qpad: v_j(c) pairs
  float4 *cp = vp + Qpad;                                    // Qpad: cov_j(x, c) pairs
  // copies of the new factor row: {h, h, -h, -h} and {l, l} per entry
  const int nrow = (nmax + 1) & ~1;
  float4 *wrow4 = reinterpret_cast<float4 *>(cp + Qpad);     // NW x nrow
  float2 *wrow2 = reinterpret_cast<float2 *>(wrow4 + NW * nrow);  // NW x nrow
  float2 *wxs = wrow2 + NW * nrow;                           // NW x kMaxP: new point
  int *dr = reinterpret_cast<int *>(wxs + NW * kMaxP);       // nmax (padded to 4)
  int *rlist = dr + ((nmax + 3) & ~3);                       // RESCORE_CAP
  unsigned char *used = reinterpret_cast<unsigned char *>(rlist + RESCORE_CAP);  // Mpad
  float4 *Us = reinterpret_cast<float4 *>(used + P.Mpad);    // R x Qpad: first factor rows
  const int R = P.R;
  float4 *ring = Us + (size_t)R * Qpad + threadIdx.x;        // RA x MB: row ring
  // checked build: the layout above ends within the launch's dynamic shared memory
  if (!LAGP_CHK(reinterpret_cast<unsigned char *>(Us + (size_t)R * Qpad + (size_t)RA * MB) - smraw,
                dynamic_smem_bytes() + 1u, 20))
    return;
  __shared__ float tabh[64], tabl[64];
  __shared__ double etab[64];
  __shared__ double xl[kMaxP];
  constexpr int NRED = (MB / 32) * (CLU ? kMaxCL : 1);  // per-warp results (of the cluster)
  __shared__ float red_s1[2][NRED], red_s2[2][NRED];
  __shared__ int red_r1[2][NRED];
  __shared__ double xr_n[CLU ? kMaxCL : 1], xr_d[CLU ? kMaxCL : 1];  // per-CTA FP64 re-score bests
  __shared__ int xr_r[CLU ? kMaxCL : 1];
  __shared__ double red_n[MB / 32], red_d[MB / 32];
  __shared__ int red_rr[MB / 32];
  __shared__ int sh_loc, sh_fail, sh_nlist;
  __shared__ uint32_t sh_tmem;
  if constexpr (TM) {
    // 128 columns of this SM's tensor memory (at most 3 CTAs per SM: 384 of 512, so the
    // allocation never waits), released at the end of the kernel
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&sh_tmem)),
                   "n"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (threadIdx.x < 64) {
    tabh[threadIdx.x] = c_exp.tabf_h[threadIdx.x];
    tabl[threadIdx.x] = c_exp.tabf_l[threadIdx.x];
    etab[threadIdx.x] = c_exp.tab[threadIdx.x];
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int CL = CLU ? P.CL : 1;
  int crank = 0;
  if constexpr (CLU) crank = (int)cg::this_cluster().block_rank();
  float4 *U = P.U + (size_t)blockIdx.x * nmax * Qpad;
  float4 *Xr = P.Xr + (size_t)blockIdx.x * P.pmax * Qpad;
  const int lda = nmax + 2;
  double *A = P.A + (size_t)blockIdx.x * nmax * lda;
  // this thread's tensor-memory words: its warp's lane quarter, its half of the columns
  const uint32_t tb = TM ? sh_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2))
                         : 0u;
  float4 *srow4 = wrow4 + (SR ? 0 : warp) * nrow;  // this warp's copy of the new factor row
  float2 *srow2 = wrow2 + (SR ? 0 : warp) * nrow;
  float2 *sxs = wxs + (SR ? 0 : warp) * kMaxP;     // and of the new point's coordinates

  for (;;) {
    int qloc;  // the location's queue position (one per cluster in the cluster form)
    if constexpr (CLU) {
      cg::this_cluster().sync();
      if (crank == 0 && tid == 0) sh_loc = atomicAdd(P.queue, 1);
      cg::this_cluster().sync();
      qloc = *cg::this_cluster().map_shared_rank(&sh_loc, 0);
    } else {
      __syncthreads();
      if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
      __syncthreads();
      qloc = sh_loc;
    }
    if (qloc >= P.T) break;
    const LocParams L = resolve_loc(P.B, qloc, P.X, P.Z, P.XX, P.p, P.n, P.M, P.n0, P.theta,
                                    P.g, P.cand, P.idx, P.N);
    const int n = L.n, p = L.p, M = L.M;
    // checked build: the location fits the slot (rows, candidates, coordinates)
    if (!(LAGP_CHK(n - 1, nmax, 13) && LAGP_CHK(M - 1, CL * P.Mpad, 14) && LAGP_CHK(p - 1, P.pmax, 15)))
      continue;
    const int32_t *cnd = L.cand;
    const ff onepg = ff_from_double(L.onepg);
    // the start design: the n0 nearest, or a saved design (augmentation)
    const int n0e = P.start ? P.nstart : L.n0;
    // Without greedy steps (n0 == n) only the start design's own rows are ever read.
    const int Q = ((n0e == n && !P.start ? n : M) + 1) >> 1;
    // this CTA's candidate pairs: q0 .. q0 + Ql - 1 of the location's (M + 1) / 2 (all of
    // them outside the cluster form), of which the first Qs are screened
    const int Qm = (M + 1) >> 1;
    const int Qc = CLU ? (Qm + CL - 1) / CL : Qm;
    const int q0 = CLU ? crank * Qc : 0;
    const int Ql = CLU ? max(0, min(Qc, Qm - q0)) : Qm;
    const int Qs = CLU ? max(0, min(Ql, Q - q0)) : Q;
    if (tid < p) xl[tid] = L.x[tid];
    if (tid == 0) sh_fail = 0;
    __syncthreads();
    // coordinates relative to x over sqrt(theta) (float-float pairs), v = 1+g,
    // cov_0(x,c) = K(x,c) in FP64
    for (int q = tid; q < Qpad; q += MB) {
      ff cv[2];
      bool flagged[2] = {false, false};  // checked build: a design index past N
      for (int h = 0; h < 2; h++) {
        const int c = 2 * q + h;             // this CTA's index
        const int cgl = 2 * (q0 + q) + h;    // the location's candidate rank
        bool live = CLU ? (q < Ql && cgl < M) : (c < M);
        if (live && !LAGP_CHK(cnd[cgl], L.N, 11)) {
          live = false;
          flagged[h] = true;
        }
        cv[h] = ff{0.0f, 0.0f};
        if (live) {
          const double *xc = L.X + (int64_t)cnd[cgl] * p;
          double acc = 0.0;
          const double sc = sqrt(L.theta_inv);  // the screen's coordinates are in units of sqrt(theta)
          for (int k = 0; k < p; k++) {
            const double dk = xc[k] - xl[k];
            const ff fk = ff_from_double(dk * sc);
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
        used[c] = live ? 0 : 1;
      }
      // (a flagged candidate gets v = 0, so that a start design holding it fails instead of
      // reading its index)
      vp[q] = make_float4(flagged[0] ? 0.0f : onepg.h, flagged[1] ? 0.0f : onepg.h,
                          flagged[0] ? 0.0f : onepg.l, flagged[1] ? 0.0f : onepg.l);
      cp[q] = make_float4(cv[0].h, cv[1].h, cv[0].l, cv[1].l);
    }
    // Cluster form: the first steps read the start pivots' v, cov and coordinates from
    // the CTA holding them, so every CTA's state must be in place before any step begins
    // (a stale value read there would let the CTAs' decisions, and barriers, diverge).
    if constexpr (CLU) cg::this_cluster().sync();
    else __syncthreads();
    if (P.start) start_ranks(P.start + L.loc * P.nstart, P.nstart, cnd, M, dr);

    int best = 0;
    int ne = n;       // the design's size (n, or where the stopping rule ends it)
    ff vx = onepg;    // v_j(x), carried by every thread for the stopping rule
    for (int j = 0; j < n; j++) {
      const int s = (j < n0e) ? (P.start ? dr[j] : j) : best;
      if (s < 0) {  // nothing admissible left (the same for every thread)
        if (tid == 0) sh_fail = 1;
        break;
      }
      // the pivot's CTA in the cluster (so) and its index there (sl), and that CTA's state
      int so = 0, sl = s;
      const float4 *vps = vp, *cps = cp, *Uss = Us, *Ugs = U, *Xrs = Xr;
      if constexpr (CLU) {
        so = (s >> 1) / Qc;
        sl = s - 2 * so * Qc;
        cg::cluster_group cl = cg::this_cluster();
        vps = cl.map_shared_rank(vp, so);
        cps = cl.map_shared_rank(cp, so);
        Uss = cl.map_shared_rank(Us, so);
        const size_t other = (size_t)((int)blockIdx.x - crank + so);
        Ugs = P.U + other * nmax * Qpad;
        Xrs = P.Xr + other * P.pmax * Qpad;
      }
      const ff vs = ff2_get(vps, sl);
      if (!(vs.h > 0.0f)) {
        if (tid == 0) sh_fail = 1;
        break;
      }
      // every thread derives the step's scalars itself: no barrier needed for them
      const ff inv = ff_rcp(ff_sqrt(vs));
      const ff uxj = ff_mul(ff2_get(cps, sl), inv);
      if (P.r_min > 0.0) {
        // Sec. 6 stopping rule: stop before a greedy point whose variance reduction ratio
        // v_j(x) / v_{j+1}(x) (psi cancels) is below r_min; every thread decides alike
        const ff vxn = ff_sub(vx, ff_mul(uxj, uxj));
        if (j >= n0e && ff_to_double(vx) / ff_to_double(vxn) < P.r_min) {
          ne = j;
          break;
        }
        vx = vxn;
      }
      if (tid == 0) dr[j] = s;
      if (crank == so && tid == ((sl >> 1) % MB)) used[sl] = 1;  // the pair's owner keeps the flags
      // this warp's (or the CTA's) copy of the new factor row u_s and of x_s (relative to x)
      {
        const int i0 = SR ? tid : lane, st = SR ? MB : 32;
        for (int i = i0; i < j; i += st) {
          const ff u = ff2_get((i < R ? Uss : Ugs) + (size_t)i * Qpad, sl);
          srow4[i] = make_float4(u.h, u.h, -u.h, -u.h);
          srow2[i] = f2s(u.l);
        }
        if (i0 < p) {
          const ff xk = ff2_get(Xrs + i0 * Qpad, sl);
          sxs[i0] = make_float2(xk.h, xk.l);
        }
      }
      if constexpr (SR) {
        __syncthreads();
      } else {
        __syncwarp();
      }
      if (j == n - 1) break;
      const bool want = j + 1 >= n0e;
      const ff2 inv2{f2s(inv.h), f2s(inv.l)}, uxj2{f2s(uxj.h), f2s(uxj.l)};
      float b1 = -1.0f, b2 = -1.0f;
      int r1 = 0x7fffffff;
      const StepCtx C{U, Us, R, ring, Xr, vp, cp, srow4, srow2, sxs, tabh, tabl, inv2, uxj2,
                      Qpad, p, j, 2 * q0, want, tb, TM ? P.RT : 0};
      if constexpr (TM) {
        // whole warps (tensor-memory accesses are warp-collective): pairs up to the next
        // multiple of 32 (all within Qpad; those past Qs only update state nobody reads),
        // a pair skipped only when the whole warp's are used
        const int Q32 = (Qs + 31) & ~31;
        for (int q = tid, ps = 0; q < Q32; q += MB, ps++) {
          const bool u0 = used[2 * q], u1 = used[2 * q + 1];
          if (__all_sync(0xffffffffu, u0 && u1)) continue;
          screen_pair<RA, true>(C, q, u0, u1, b1, r1, b2, ps);
        }
      } else {
        for (int q = tid; q < Qs; q += MB) {
          const bool u0 = used[2 * q], u1 = used[2 * q + 1];
          if (u0 && u1) continue;
          screen_pair<RA>(C, q, u0, u1, b1, r1, b2);
        }
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
        if constexpr (CLU) {  // into every CTA of the cluster
          cg::cluster_group cl = cg::this_cluster();
          const int e = crank * (MB / 32) + warp;
          for (int r = 0; r < CL; r++) {
            cl.map_shared_rank(&red_s1[par][0], r)[e] = b1;
            cl.map_shared_rank(&red_s2[par][0], r)[e] = b2;
            cl.map_shared_rank(&red_r1[par][0], r)[e] = r1;
          }
        } else {
          red_s1[par][warp] = b1;
          red_s2[par][warp] = b2;
          red_r1[par][warp] = r1;
        }
      }
      if constexpr (CLU) cg::this_cluster().sync();
      else __syncthreads();
      if (!want) continue;
      float B1 = red_s1[par][0], B2 = red_s2[par][0];
      int R1 = red_r1[par][0];
      if constexpr (CLU) {
        // the cluster's 8 CL entries: lane l merges entries l and l + 32, then a butterfly
        // over the warp (the merge is order-independent: a unique best, ties to the smaller
        // rank, and the largest other score)
        const int ne = CL * (MB / 32);
        B1 = -1.0f;
        B2 = -1.0f;
        R1 = 0x7fffffff;
        for (int w = lane; w < ne; w += 32) merge2(red_s1[par][w], red_r1[par][w], red_s2[par][w], B1, R1, B2);
        for (int o = 16; o > 0; o >>= 1) {
          const float ob1 = __shfl_xor_sync(0xffffffffu, B1, o);
          const float ob2 = __shfl_xor_sync(0xffffffffu, B2, o);
          const int orr = __shfl_xor_sync(0xffffffffu, R1, o);
          merge2(ob1, orr, ob2, B1, R1, B2);
        }
      } else {
        for (int w = 1; w < MB / 32; w++)
          merge2(red_s1[par][w], red_r1[par][w], red_s2[par][w], B1, R1, B2);
      }
      best = (R1 == 0x7fffffff) ? -1 : R1;
      const bool near = R1 != 0x7fffffff && B2 >= B1 * (1.0f - DELTA);
      if (!near) continue;
      // ---- FP64 re-score of the near-tied candidates (rare) ----
      if (tid == 0 && crank == 0 && P.rescores) atomicAdd(P.rescores, 1);
      // each CTA re-scores its own near-tied candidates (the FP64 factor of the design, the
      // same in every CTA, is formed by each)
      const RescoreCtx R{L.X, cnd, xl, etab, used, vp, cp, dr, A, rlist, &sh_nlist, &sh_fail,
                         red_n, red_d, red_rr, p, 2 * q0, CLU ? min(2 * Ql, M - 2 * q0) : M, j + 1, lda,
                         L.theta_inv, L.onepg};
      double bn, bd;
      int br;
      rescore_fp64(R, B1, &bn, &bd, &br);
      if (sh_fail) break;  // the same in every CTA of a cluster
      if constexpr (CLU) {  // the cluster's FP64 best, ties to the nearer candidate
        cg::cluster_group cl = cg::this_cluster();
        if (tid == 0)
          for (int r = 0; r < CL; r++) {
            cl.map_shared_rank(xr_n, r)[crank] = bn;
            cl.map_shared_rank(xr_d, r)[crank] = bd;
            cl.map_shared_rank(xr_r, r)[crank] = br;
          }
        cl.sync();
        bn = xr_n[0];
        bd = xr_d[0];
        br = xr_r[0];
        for (int r = 1; r < CL; r++)
          if (frac_better(xr_n[r], xr_d[r], xr_r[r], bn, bd, br)) {
            bn = xr_n[r];
            bd = xr_d[r];
            br = xr_r[r];
          }
      }
      best = (br != 0x7fffffff) ? br : best;
    }
    // (cluster form: the last step's pivot reads of the other CTAs' state are done before
    // any CTA moves on and reuses or discards it)
    if constexpr (CLU) cg::this_cluster().sync();
    else __syncthreads();
    // the design (design indices), or -1 when a step failed; kernel (c) (predict.cu)
    // evaluates the predictive equations on it in FP64
    if (crank == 0) {
      for (int i = tid; i < n; i += MB) L.idx[i] = (sh_fail || i >= ne) ? -1 : cnd[dr[i]];
      if (P.n_out && tid == 0) P.n_out[L.loc] = sh_fail ? 0 : ne;
    }
    // The predictive equations on the design (kernel (c)'s arithmetic, predict_loc.cuh),
    // here while the other resident CTAs screen -- FP64 work beside their FP32 work -- when
    // the matrix fits in the shared-memory factor rows (dead now); the reciprocal pivots go
    // to the per-warp row copies.  Otherwise kernel (c) runs after this kernel.  Only
    // the instance without the row ring carries this code (in the other it costs 2 % on
    // the 8-d workload, which has no room for the matrix anyway).
    if constexpr (RA == 0 && !CLU) {
      if (P.fuse_pred) {
        __syncthreads();  // every thread reads the design below
        predict_location(L, L.idx, sh_fail ? n : ne, xl, reinterpret_cast<double *>(Us),
                         reinterpret_cast<double *>(wrow4), etab, &sh_fail, L.loc, P.mean, P.s2,
                         P.var, P.status);
      }
    }
    // The factor rows in global memory are dead now (the next location rewrites each row
    // before reading it): drop their L2 lines without writing them back to DRAM.
    {
      char *u0 = reinterpret_cast<char *>(U + (size_t)R * Qpad);
      const int nlines = (int)(((size_t)(n > R ? n - R : 0) * Qpad * sizeof(float4)) / 128);
      for (int l = tid; l < nlines; l += MB)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(u0 + (size_t)l * 128) : "memory");
    }
  }
  // no CTA of a cluster exits while another may still read its shared memory
  if constexpr (CLU) cg::this_cluster().sync();
  if constexpr (TM) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh_tmem),
                   "n"(kTmemCols)
                   : "memory");
  }
}

// Candidate pairs of one CTA slot: M candidates over CL CTAs, padded to 32 pairs (so the
// shared-memory rows after the Mpad = 2 Qpad flag bytes start 16-byte aligned).
int mix_qpad(int M, int CL) { return (int)align_up((size_t)ceil_div(ceil_div(M, 2), CL), 32); }

// Dynamic shared memory: the per-candidate state, then the first R factor rows and the
// threads' row rings (RA stages).
size_t mix_smem_bytes(int Qpad, int n, int R, int RA, bool SR) {
  const size_t nrow = (size_t)((n + 1) & ~1);
  const size_t nw = SR ? 1 : MB / 32;
  return (size_t)Qpad * 2 * sizeof(float4) +
         nw * (nrow * (sizeof(float4) + sizeof(float2)) + kMaxP * sizeof(float2)) +
         (size_t)((n + 3) & ~3) * sizeof(int) + RESCORE_CAP * sizeof(int) + (size_t)2 * Qpad +
         (size_t)R * Qpad * sizeof(float4) + (size_t)RA * MB * sizeof(float4);
}

// The kernel instance of a launch: ring stages RA (0 or RING_A), a shared factor-row copy
// SR, and CL CTAs per location (CL > 1: the cluster form).
struct MixVariant {
  int RA;
  bool SR;
  int CL;
  bool TM = false;  // rows R .. R + RT - 1 also in tensor memory (RA == 0, CL == 1)
};

const void *mix_kernel(MixVariant v) {
  if (v.CL > 1)
    return v.RA ? reinterpret_cast<const void *>(select_mixed_kernel<RING_A, false, true>)
                : reinterpret_cast<const void *>(select_mixed_kernel<0, false, true>);
  if (!v.RA)
    return v.TM ? reinterpret_cast<const void *>(select_mixed_kernel<0, false, false, true>)
                : reinterpret_cast<const void *>(select_mixed_kernel<0, false, false>);
  if (v.SR)
    return v.TM ? reinterpret_cast<const void *>(select_mixed_kernel<RING_A, true, false, true>)
                : reinterpret_cast<const void *>(select_mixed_kernel<RING_A, true, false>);
  return v.TM ? reinterpret_cast<const void *>(select_mixed_kernel<RING_A, false, false, true>)
              : reinterpret_cast<const void *>(select_mixed_kernel<RING_A, false, false>);
}

size_t mix_static_smem(MixVariant v) {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, mix_kernel(v)) == cudaSuccess ? fa.sharedSizeBytes : 4096;
}

int mix_minb(MixVariant v) { return mix_minb(v.RA, v.SR, v.CL > 1); }

size_t mix_resident(int Qpad, int n, MixVariant v, const DevInfo &di) {
  const size_t per = mix_static_smem(v) + 1024 + mix_smem_bytes(Qpad, n, 0, v.RA, v.SR);
  const size_t k = di.smem_per_sm / per;  // 1 KB reserved per CTA
  const size_t mb = (size_t)mix_minb(v);
  return k < mb ? k : mb;
}

// Launch-shape overrides for measurements (they change no result): LAGP_MIX_CLUSTER = CTAs
// per location (1, 2, 4 or 8), LAGP_MIX_RING = 0 / 1 (row ring off / on).  -1: not set.
int mix_env(const char *name) {
  const char *e = getenv(name);
  return e && *e ? atoi(e) : -1;
}

// CTAs per location: the cluster form where a location's factor rows are large enough that
// the rows of all locations in flight overflow L2.
int mix_cluster_size(int n, int M) {
  const int e = mix_env("LAGP_MIX_CLUSTER");
  if (e == 1 || e == 2 || e == 4 || e == 8) return e;
  (void)n;
  (void)M;
  return 1;
}

// The row ring is used where a CTA's factor rows (n x M float-float entries) come mostly
// from DRAM -- 8-d workload (n = 100, M = 2000) yes, paper-2d (n = 50, M = 1000) no, both
// measured -- and only if its shared memory leaves at least as many CTAs resident per SM;
// with one shared copy of the factor row where the per-warp copies are what leave no room
// (the 8-d workload at 4 CTAs per SM, the batched workload's large n).  The cluster form has
// no shared-copy instance.
MixVariant mix_variant(int n, int M, int CL, const DevInfo &di) {
  const int Qpad = mix_qpad(M, CL);
  const MixVariant plain{0, false, CL}, ring{RING_A, false, CL}, ring_sr{RING_A, true, CL};
  const int er = mix_env("LAGP_MIX_RING");
  if (er == 0) return plain;
  if (er == 1) return ring;
  if ((int64_t)n * M < 100000 * (int64_t)CL) return plain;
  // the most resident CTAs per SM wins; at a tie, the ring with per-warp row copies (no
  // extra barrier per step)
  const size_t k0 = mix_resident(Qpad, n, plain, di);
  const size_t kr = mix_resident(Qpad, n, ring, di);
  const size_t ks = CL == 1 ? mix_resident(Qpad, n, ring_sr, di) : 0;
  if (kr >= k0 && kr >= ks) return ring;
  if (ks >= k0) return ring_sr;
  return plain;
}

// Factor rows kept in shared memory: as many as the instance's resident CTAs per SM leave
// room for (the rest stream from L2).  Row i is read at every step after step i, so the
// first rows carry the most traffic.
int mix_rows_in_smem(int Qpad, int n, MixVariant v, const DevInfo &di) {
  const size_t stat = mix_static_smem(v);
  size_t per_cta = di.smem_per_sm / mix_minb(v);
  const size_t fixed = stat + 1024 + mix_smem_bytes(Qpad, n, 0, v.RA, v.SR);  // 1 KB reserved per CTA
  if (per_cta > di.smem_optin) per_cta = di.smem_optin;
  if (per_cta <= fixed) return 0;
  const size_t row = (size_t)Qpad * sizeof(float4);
  const size_t r = (per_cta - fixed) / row;
  return (int)(r < (size_t)n ? r : (size_t)n);
}

// CTAs of a uniform launch: the instance's resident CTAs per SM (one location each), or in
// the cluster form as many clusters of CL as can be resident at once (at most one per
// location).
int mix_grid(int64_t T, int num_sms, MixVariant v) {
  int64_t g = (int64_t)num_sms * mix_minb(v);
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

int mix_cluster_grid(int64_t T, MixVariant v, size_t smem, int num_sms, int *G) {
  cudaError_t e = cudaFuncSetAttribute(mix_kernel(v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = v.CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(v.CL, 1, 1);
  cfg.blockDim = dim3(MB, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  e = cudaOccupancyMaxActiveClusters(&nc, mix_kernel(v), &cfg);
  if (e != cudaSuccess) return cuda_status(e);
  if (nc < 1) return LAGP_ERR_INVALID_ARG;
  int64_t c = nc;
  c = c < (int64_t)num_sms * LAGP_MIX_MINB / v.CL ? c : (int64_t)num_sms * LAGP_MIX_MINB / v.CL;
  c = c < (T > 0 ? T : 1) ? c : (T > 0 ? T : 1);
  *G = (int)(c * v.CL);
  return LAGP_OK;
}

struct MixLayout {
  size_t u, xr, a, idx, pred, total;
};

// [queue | re-score counter | U | Xr | A | design indices | kernel (c) workspace]
MixLayout mix_layout(int G, int p, int n, int Qpad, int64_t T, int64_t idx_total, int num_sms) {
  MixLayout L;
  L.u = align_up((size_t)G * n * Qpad * sizeof(float4), 256);
  L.xr = align_up((size_t)G * p * Qpad * sizeof(float4), 256);
  L.a = align_up((size_t)G * n * (n + 2) * sizeof(double), 256);
  L.idx = align_up((size_t)idx_total * sizeof(int32_t), 256);
  L.pred = predict_fp64_workspace_bytes(T, n, num_sms);
  L.total = 256 + 256 + L.u + L.xr + L.a + L.idx + L.pred;
  return L;
}

// The workspace of a uniform launch covers every instance and cluster size (the grid has
// at most min(resident CTAs per SM x SMs, CL x T) CTAs).
size_t mix_uniform_bytes(int64_t T, int p, int n, int M, int num_sms) {
  size_t best = 0;
  for (int CL = 1; CL <= kMaxCL; CL *= 2) {
    int64_t G = (int64_t)num_sms * (CL == 1 ? kRingMinB : LAGP_MIX_MINB);
    const int64_t cap = (int64_t)CL * (T > 0 ? T : 1);
    G = G < cap ? G : cap;
    const size_t b = mix_layout((int)G, p, n, mix_qpad(M, CL), T, T * n, num_sms).total;
    best = b > best ? b : best;
  }
  return best;
}

// The screen and, per location, the predictive equations on the design it selected: in
// the same kernel when the matrix fits in its shared memory (paper-2d: 14.43 -> 14.29 ms),
// else by kernel (c) afterwards (the 8-d workload's n = 100: 139.5 ms either way in its
// own kernel, 145.5 ms inside the screen from global memory).  The cluster form always
// leaves them to kernel (c).
int mix_run(MixParams P, MixVariant v, const MixLayout &L, int G, char *w, int32_t *user_idx,
            const DevInfo &di, cudaStream_t stream) {
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
  P.CL = v.CL;
  // tensor-memory rows (one CTA per location): 16, 8 or 4 rows per pair for 1, 2, or 3-4
  // pairs per thread, so that each thread's rows fit its 64 columns in whole loads of four
  // rows; none where n leaves no rows past shared memory.
  // LAGP_MIX_TMEM=0 turns it off (for measurements; no result changes).
  P.RT = 0;
  if (v.CL == 1 && mix_env("LAGP_MIX_TMEM") != 0) {
    const int pp = (P.Qpad + MB - 1) / MB;
    if (pp <= 4) {
      v.TM = true;
      P.RT = 4 * (4 / pp);
    }
  }
  P.R = mix_rows_in_smem(P.Qpad, P.nmax, v, di);
  if (v.TM && P.nmax <= P.R) {
    v.TM = false;
    P.RT = 0;
    P.R = mix_rows_in_smem(P.Qpad, P.nmax, v, di);
  }
  P.fuse_pred = v.RA == 0 && v.CL == 1 &&
                (size_t)P.R * P.Qpad * sizeof(float4) >= (size_t)P.nmax * (P.nmax + 2) * sizeof(double);
  const size_t smem = mix_smem_bytes(P.Qpad, P.nmax, P.R, v.RA, v.SR);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(mix_kernel(v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  if (v.TM) {
    // every resident CTA holds kTmemCols of the SM's 512 tensor-memory columns: if more
    // CTAs could be resident than that allows, an allocation would wait for a neighbour to
    // finish, so such a launch keeps its rows in global memory instead
    int k = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, mix_kernel(v), MB, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (k * kTmemCols > 512) {
      v.TM = false;
      P.RT = 0;
      e = cudaFuncSetAttribute(mix_kernel(v), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  e = cudaMemsetAsync(w, 0, 512, stream);  // work counter and re-score counter
  if (e != cudaSuccess) return cuda_status(e);
  if (v.CL > 1) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = v.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(G, 1, 1);
    cfg.blockDim = dim3(MB, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&P};
    e = cudaLaunchKernelExC(&cfg, mix_kernel(v), args);
    if (e != cudaSuccess) return cuda_status(e);
  } else if (!v.RA) {
    if (v.TM)
      select_mixed_kernel<0, false, false, true><<<G, MB, smem, stream>>>(P);
    else
      select_mixed_kernel<0, false, false><<<G, MB, smem, stream>>>(P);
  } else if (v.SR) {
    if (v.TM)
      select_mixed_kernel<RING_A, true, false, true><<<G, MB, smem, stream>>>(P);
    else
      select_mixed_kernel<RING_A, true, false><<<G, MB, smem, stream>>>(P);
  } else {
    if (v.TM)
      select_mixed_kernel<RING_A, false, false, true><<<G, MB, smem, stream>>>(P);
    else
      select_mixed_kernel<RING_A, false, false><<<G, MB, smem, stream>>>(P);
  }
  g_launches.fetch_add(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || P.fuse_pred) return cuda_status(e);
  PredictArgs pa;
  pa.X = P.X; pa.Z = P.Z; pa.p = P.pmax; pa.XX = P.XX; pa.T = P.T; pa.n = P.n; pa.nmax = P.nmax;
  pa.theta = P.theta; pa.g = P.g; pa.idx = P.idx; pa.B = P.B;
  pa.B.n_loc = P.n_out;  // adaptive designs: kernel (c) on each location's own size
  pa.mean = P.mean; pa.s2 = P.s2; pa.var = P.var; pa.status = P.status;
  return predict_fp64_launch(pa, o, L.pred, stream);
}

}  // namespace

int select_mixed_check_take(CheckRec *out) { return check_take_here(out); }

size_t select_mixed_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms) {
  return mix_uniform_bytes(T, p, n, ncand, num_sms);
}

int select_mixed_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  const MixVariant v = mix_variant(a.n, a.M, mix_cluster_size(a.n, a.M), di);
  const int Qpad = mix_qpad(a.M, v.CL);
  int G = mix_grid(a.T, di.num_sms, v);
  if (v.CL > 1) {
    const int R = mix_rows_in_smem(Qpad, a.n, v, di);
    st = mix_cluster_grid(a.T, v, mix_smem_bytes(Qpad, a.n, R, v.RA, v.SR), di.num_sms, &G);
    if (st) return st;
  }
  const MixLayout L = mix_layout(G, a.p, a.n, Qpad, a.T, a.T * a.n, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MixParams P;
  P.X = a.X; P.Z = a.Z; P.N = a.N; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Qpad = Qpad; P.Mpad = 2 * Qpad; P.n0 = a.n0; P.n = a.n;
  P.theta = a.theta; P.theta_inv = 1.0 / a.theta; P.g = a.g; P.onepg = 1.0 + a.g;
  P.nmax = a.n; P.pmax = a.p;
  P.B = BatchView{nullptr, nullptr, nullptr, 0, a.theta_loc, nullptr};
  P.start = a.start; P.nstart = a.nstart;
  P.r_min = a.r_min; P.n_out = a.n_out;
  P.mean = a.mean; P.s2 = a.s2; P.var = a.var; P.status = a.status;
  return mix_run(P, v, L, G, static_cast<char *>(ws), a.idx, di, stream);
}

size_t select_mixed_batch_workspace_bytes(const BatchLaunch &b, int G) {
  DevInfo di;
  const int sms = dev_info(&di) == LAGP_OK ? di.num_sms : 152;
  return mix_layout(G, b.pmax, b.nmax, mix_qpad(b.Mmax, 1), b.T, b.idx_total, sms).total;
}

int select_mixed_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, int G,
                              cudaStream_t stream) {
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();  // this translation unit's copy of the exp constants
  if (st) return st;
  const int Qpad = mix_qpad(b.Mmax, 1);
  const MixLayout L = mix_layout(G, b.pmax, b.nmax, Qpad, b.T, b.idx_total, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MixParams P;
  P.X = nullptr; P.Z = nullptr; P.N = 0; P.p = b.pmax; P.XX = b.XX; P.T = b.T; P.cand = b.cand;
  P.M = b.Mmax; P.Qpad = Qpad; P.Mpad = 2 * Qpad; P.n0 = 0; P.n = b.nmax;
  P.theta = 1.0; P.theta_inv = 1.0; P.g = 0.0; P.onepg = 1.0;
  P.nmax = b.nmax; P.pmax = b.pmax;
  P.B = BatchView{b.designs, b.locs, b.order, b.ldxx, nullptr, nullptr};
  P.start = nullptr; P.nstart = 0;
  P.r_min = 0.0; P.n_out = nullptr;
  P.mean = b.mean; P.s2 = b.s2; P.var = b.var; P.status = b.status;
  // batches keep one CTA per location (their tuner chooses the CTAs per SM)
  MixVariant v = mix_variant(b.nmax, b.Mmax, 1, di);
  return mix_run(P, v, L, G, static_cast<char *>(ws), b.idx, di, stream);
}

int select_mixed_prepare() {
  const int st = exp_table_upload();
  return st ? st : predict_fp64_prepare();
}

}  // namespace lagp
