// select_mspe.cu -- kernels (b)+(c) for the MSPE criterion, FP64.
//
// Gramacy & Apley, Sec. 3.1 (Eq. mspe, Eqs. newv and G) with the derivatives of SM Sec. 2
// (Eqs. dKi, d2w, dl, d2l, dz, dmu, dV, Ed2la): at each step the candidate c minimising
//   J(c) = psi_j/(j-2) v_{j+1}(x) + (dmu_j(x)/dtheta)^2 / G_{j+1}(c),
//   G_{j+1}(c) = F_j + dV_c^2 / (2 V_c^2) + dmu_c^2 / V_c,    V_c = psi_j v_j(c)/(j-2),
//   dmu_c = kd_c^T w - z_c^T Kd w,   dV_c = [-(w^T Kd w) v_j(c) - psi_j (2 kd_c^T z_c - z_c^T Kd z_c)]/(j-2),
// joins the design (theta fixed at d; Kd, Kdd are dK/dtheta, d2K/dtheta2; z_c = K_j^{-1} k_c;
// F_j = -l''(Y_j) of Eq. d2l), with v_{j+1}(x) = v_j(x) - cov_j(x,c)^2/v_j(c) as for ALC.
//
// Every quantity is carried in the basis of the bordered Cholesky factor L_j of K_j
// (K_j^{-1} = L^{-T} L^{-1}), which makes each candidate's update O(j) per step:
//   u_c = L^{-1} k_c, ud_c = L^{-1} kd_c      (one new entry each per step, as in select.cu)
//   kdz_c = kd_c^T z_c = ud_c . u_c,  pd_c = kd_c^T w = ud_c . ytil,
//   q_c = z_c^T Kd z_c = u_c^T Q u_c,  m_c = z_c^T Kd w = u_c . r,
// with Q = L^{-1} Kd L^{-T}, r = Q ytil, ytil = L^{-1} Y.  Appending a point appends a row to
// L^{-1}, Q and R = L^{-1} Kdd L^{-T} (the leading blocks do not change), so per step the
// CTA forms the new rows in O(j^2) and every candidate updates q_c and m_c with one extra
// O(j) dot against the new row of Q.  F_j follows Eq. d2l from tr R, ||Q||_F^2, ytil^T R ytil,
// ||r||^2 and (ytil . r)^2, all updated as rows are appended.
#include <math.h>

#include "batch.cuh"
#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {
namespace {

constexpr int TB = 256;  // threads per CTA

struct MspeParams {
  const double *X, *Z;
  int p;
  const double *XX;
  int64_t T;
  const int32_t *cand;
  int M, Mpad, n0, n;
  int nmax, pmax;  // slot dimensions (the largest n and p of the launch)
  double theta, theta_inv, g, onepg;
  BatchView B;     // per-location tables (B.designs == nullptr: uniform launch)
  double *mean, *s2, *var;
  int32_t *idx;
  int8_t *status;
  double *U, *Ud;     // slots of n x Mpad
  double *Xc;         // slots of p x Mpad
  double *cs;         // slots of 4 x Mpad: kdz, pd, q, m per candidate
  double *Li, *Kd, *Kdd, *Q;  // slots of n x n
  int *queue;
  const int32_t *start;  // saved start designs (T x nstart design indices), or nullptr
  int nstart;
};

__device__ __forceinline__ bool j_better(double a, int ra, double b, int rb) {
  return a < b || (a == b && ra < rb);
}

__global__ void __launch_bounds__(TB, 1) select_mspe_kernel(MspeParams P) {
  extern __shared__ __align__(16) double sm[];
  const int Mpad = P.Mpad, nn = P.nmax;  // nn: row stride of the n x n slot matrices
  double *v = sm;               // Mpad: v_j(c)
  double *cov = v + Mpad;       // Mpad: cov_j(x, c)
  double *srow = cov + Mpad;    // nn: u_s
  double *sdrow = srow + nn;    // nn: ud_s
  double *qrow = sdrow + nn;    // nn: row j of Q
  double *rrow = qrow + nn;     // nn: row j of R
  double *ux = rrow + nn;       // nn: L^{-1} k(x)
  double *udx = ux + nn;        // nn: L^{-1} kd(x)
  double *yt = udx + nn;        // nn: L^{-1} Y
  double *r = yt + nn;          // nn: Q ytil
  double *t1 = r + nn;          // nn: Kd Li[j]^T
  double *t2 = t1 + nn;         // nn: Kdd Li[j]^T
  int *dr = reinterpret_cast<int *>(t2 + nn);  // nn: ranks of the design
  unsigned char *used = reinterpret_cast<unsigned char *>(dr + nn);  // Mpad
  __shared__ double etab[64];
  __shared__ double xs[kMaxP], xl[kMaxP];
  __shared__ double red_s[TB / 32];
  __shared__ int red_r[TB / 32];
  __shared__ double sh_d[8];  // per-step scalars: 0 inv, 1 uxj, 2 ytj, 3 rj, 4 F, 5 dmux, 6 wKdw
  __shared__ double sh_dot[3];
  __shared__ int sh_loc, sh_best, sh_fail;
  __shared__ double sh_psi, sh_vx, sh_trR, sh_nQ2, sh_yRy;
  if (threadIdx.x < 64) etab[threadIdx.x] = c_exp.tab[threadIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double *U = P.U + (size_t)blockIdx.x * nn * Mpad;
  double *Ud = P.Ud + (size_t)blockIdx.x * nn * Mpad;
  double *Xc = P.Xc + (size_t)blockIdx.x * P.pmax * Mpad;
  double *cs = P.cs + (size_t)blockIdx.x * 4 * Mpad;
  double *kdz = cs, *pd = cs + Mpad, *qc = cs + 2 * Mpad, *mc = cs + 3 * Mpad;
  double *Li = P.Li + (size_t)blockIdx.x * nn * nn;
  double *Kd = P.Kd + (size_t)blockIdx.x * nn * nn;
  double *Kdd = P.Kdd + (size_t)blockIdx.x * nn * nn;
  double *Q = P.Q + (size_t)blockIdx.x * nn * nn;

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    if (sh_loc >= P.T) break;
    const LocParams L = resolve_loc(P.B, sh_loc, P.X, P.Z, P.XX, P.p, P.n, P.M, P.n0, P.theta,
                                    P.g, P.cand, P.idx);
    const int64_t loc = L.loc;
    const int n = L.n, p = L.p, M = L.M;
    const int32_t *cnd = L.cand;
    const double th = L.theta, th2 = th * th, th3 = th2 * th, th4 = th2 * th2;
    const double ith2 = 1.0 / th2;
    if (tid < p) xl[tid] = L.x[tid];
    if (tid == 0) {
      sh_fail = 0;
      sh_psi = 0.0; sh_vx = L.onepg; sh_trR = 0.0; sh_nQ2 = 0.0; sh_yRy = 0.0;
    }
    __syncthreads();
    // the start design: the n0 nearest, or a saved design (augmentation)
    const int n0e = P.start ? P.nstart : L.n0;
    const int limit = (n0e == n && !P.start) ? n : M;
    for (int c = tid; c < limit; c += TB) {
      const double *xc = L.X + (int64_t)cnd[c] * p;
      double acc = 0.0;
      for (int k = 0; k < p; k++) {
        const double xk = xc[k];
        Xc[k * Mpad + c] = xk;
        const double t = xl[k] - xk;
        acc = fma(t, t, acc);
      }
      v[c] = L.onepg;
      cov[c] = exp_nonpos(-acc * L.theta_inv, etab);
      kdz[c] = 0.0; pd[c] = 0.0; qc[c] = 0.0; mc[c] = 0.0;
      used[c] = 0;
    }
    __syncthreads();
    if (P.start) start_ranks(P.start + L.loc * P.nstart, P.nstart, cnd, M, dr);

    for (int j = 0; j < n; j++) {
      const int s = (j < n0e) ? (P.start ? dr[j] : j) : sh_best;
      if (s < 0) {
        if (tid == 0) sh_fail = 1;
        __syncthreads();
        break;
      }
      // ---- phase A: the pivot's rows, coordinates and scalars
      for (int i = tid; i < j; i += TB) {
        srow[i] = U[(size_t)i * Mpad + s];
        sdrow[i] = Ud[(size_t)i * Mpad + s];
      }
      if (tid < p) xs[tid] = Xc[tid * Mpad + s];
      __syncthreads();
      const double vs = v[s];
      if (!(vs > 0.0)) {
        if (tid == 0) sh_fail = 1;
        __syncthreads();
        break;
      }
      // three dots of length j (u_s . ytil, u_s . udx, and u_s . ux is cov[s]), one warp each
      if (warp < 2) {
        double acc = 0.0;
        const double *vec = (warp == 0) ? yt : udx;
        for (int i = lane; i < j; i += 32) acc = fma(srow[i], vec[i], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) sh_dot[warp] = acc;
      }
      __syncthreads();
      if (tid == 0) {
        const double sq = sqrt(vs);
        const double inv = 1.0 / sq;
        double acc = 0.0;
        for (int k = 0; k < p; k++) {
          const double t = xl[k] - xs[k];
          acc = fma(t, t, acc);
        }
        const double kxs = exp_nonpos(-acc * L.theta_inv, etab);
        const double kdxs = kxs * acc / th2;
        const double uxj = cov[s] / sq;
        const double ytj = (L.Z[cnd[s]] - sh_dot[0]) / sq;
        ux[j] = uxj;
        udx[j] = (kdxs - sh_dot[1]) * inv;
        yt[j] = ytj;
        sh_d[0] = inv;
        sh_d[1] = uxj;
        sh_d[2] = ytj;
        sh_psi = fma(ytj, ytj, sh_psi);
        sh_vx = fma(-uxj, uxj, sh_vx);
        dr[j] = s;
        used[s] = 1;
      }
      __syncthreads();
      const double inv = sh_d[0];
      // ---- phase B: new rows of L^{-1}, Kd, Kdd (O(j^2), parallel)
      for (int i = tid; i <= j; i += TB) {
        double li;
        if (i == j) {
          li = inv;
        } else {
          double acc = 0.0;
          for (int m = i; m < j; m++) acc = fma(srow[m], Li[(size_t)m * nn + i], acc);
          li = -acc * inv;
        }
        Li[(size_t)j * nn + i] = li;
        double kd = 0.0, kdd = 0.0;
        if (i < j) {
          const double *xi = L.X + (int64_t)cnd[dr[i]] * p;
          double acc = 0.0;
          for (int k = 0; k < p; k++) {
            const double t = xs[k] - xi[k];
            acc = fma(t, t, acc);
          }
          const double kk = exp_nonpos(-acc * L.theta_inv, etab);
          kd = kk * acc / th2;
          kdd = kk * (acc * acc / th4 - 2.0 * acc / th3);
        }
        Kd[(size_t)j * nn + i] = kd;
        Kdd[(size_t)j * nn + i] = kdd;
      }
      __syncthreads();
      // t1 = Kd Li[j]^T, t2 = Kdd Li[j]^T over rows a <= j (symmetric: entry (a,c) at row max)
      for (int a = tid; a <= j; a += TB) {
        double s1 = 0.0, s2 = 0.0;
        for (int c = 0; c <= j; c++) {
          const int hi = a > c ? a : c, lo = a > c ? c : a;
          const double lj = Li[(size_t)j * nn + c];
          s1 = fma(Kd[(size_t)hi * nn + lo], lj, s1);
          s2 = fma(Kdd[(size_t)hi * nn + lo], lj, s2);
        }
        t1[a] = s1;
        t2[a] = s2;
      }
      __syncthreads();
      // row j of Q and R: (Li t)[b] = sum_{a <= b} Li[b][a] t[a]
      for (int b = tid; b <= j; b += TB) {
        double s1 = 0.0, s2 = 0.0;
        for (int a = 0; a <= b; a++) {
          const double l = Li[(size_t)b * nn + a];
          s1 = fma(l, t1[a], s1);
          s2 = fma(l, t2[a], s2);
        }
        Q[(size_t)j * nn + b] = s1;
        qrow[b] = s1;
        rrow[b] = s2;
      }
      __syncthreads();
      // r = Q ytil: old entries gain Q[j][i] ytil_j; entry j is row j of Q dotted with ytil
      const double ytj = sh_d[2];
      for (int i = tid; i < j; i += TB) r[i] = fma(qrow[i], ytj, r[i]);
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
        double wk = 0.0, nr = 0.0, dm = 0.0;
        for (int i = lane; i <= j; i += 32) {
          wk = fma(yt[i], r[i], wk);
          nr = fma(r[i], r[i], nr);
          dm = fma(udx[i], yt[i], dm);
          dm = fma(-ux[i], r[i], dm);
        }
        for (int o = 16; o > 0; o >>= 1) {
          wk += __shfl_down_sync(0xffffffffu, wk, o);
          nr += __shfl_down_sync(0xffffffffu, nr, o);
          dm += __shfl_down_sync(0xffffffffu, dm, o);
        }
        if (lane == 0) {
          const double jd = (double)(j + 1), psi = sh_psi;
          // Eq. d2l: l'' = -1/2 (tr R - ||Q||^2) + j/(2 psi)(ytil^T R ytil - 2 ||r||^2)
          //                + j/(2 psi^2) (ytil . r)^2
          const double l2 = -0.5 * (sh_trR - sh_nQ2) + jd / (2.0 * psi) * (sh_yRy - 2.0 * nr) +
                            jd / (2.0 * psi * psi) * wk * wk;
          sh_d[4] = -l2;
          sh_d[5] = dm;
          sh_d[6] = wk;
        }
      }
      __syncthreads();
      if (j == n - 1) break;
      // ---- phase C: every remaining candidate, O(j)
      const double uxj = sh_d[1], rj = sh_d[3], F = sh_d[4], dmux = sh_d[5], wKdw = sh_d[6];
      const double psi = sh_psi, vx = sh_vx, qjj = qrow[j];
      const int jn = j + 1;  // design size after this step
      const bool want = (jn >= n0e) && (jn >= 3);
      const double dj = (double)(jn - 2);
      const double rdj = 1.0 / dj, pdj = psi / dj;
      double bs = INFINITY;
      int br = 0x7fffffff;
      for (int c = tid; c < limit; c += TB) {
        if (used[c]) continue;
        double acc = 0.0;
        for (int k = 0; k < p; k++) {
          const double t = xs[k] - Xc[k * Mpad + c];
          acc = fma(t, t, acc);
        }
        const double ksc = exp_nonpos(-acc * L.theta_inv, etab);
        const double kdsc = ksc * acc * ith2;
        double d1 = ksc, d2 = kdsc, d3 = 0.0;
        const double *Uc = U + c, *Udc = Ud + c;
        for (int i = 0; i < j; i++, Uc += Mpad, Udc += Mpad) {
          const double uci = *Uc;
          d1 = fma(-srow[i], uci, d1);
          d2 = fma(-srow[i], *Udc, d2);
          d3 = fma(qrow[i], uci, d3);
        }
        const double u = d1 * inv, ud = d2 * inv;
        U[(size_t)j * Mpad + c] = u;
        Ud[(size_t)j * Mpad + c] = ud;
        const double vc = fma(-u, u, v[c]);
        const double cx = fma(-uxj, u, cov[c]);
        v[c] = vc;
        cov[c] = cx;
        const double kz = fma(ud, u, kdz[c]);
        const double pc = fma(ud, ytj, pd[c]);
        const double qn = fma(qjj * u, u, fma(2.0 * u, d3, qc[c]));
        const double mn = fma(u, rj, fma(ytj, d3, mc[c]));
        kdz[c] = kz;
        pd[c] = pc;
        qc[c] = qn;
        mc[c] = mn;
        if (want && vc > 0.0) {
          // two divisions, 1 / V_c and 1 / G: dVc^2 / (2 V_c^2) = (dVc / V_c)^2 / 2 and
          // 1 / v_c = (psi / (j - 2)) / V_c
          const double Vc = pdj * vc;
          const double rV = 1.0 / Vc;
          const double dmuc = pc - mn;
          const double dVc = (-wKdw * vc - psi * (2.0 * kz - qn)) * rdj;
          const double dr = dVc * rV;
          const double G = F + 0.5 * dr * dr + dmuc * dmuc * rV;
          const double Jc = pdj * (vx - cx * cx * (pdj * rV)) + dmux * dmux / G;
          if (Jc == Jc && j_better(Jc, c, bs, br)) { bs = Jc; br = c; }
        }
      }
      if (want) {
        for (int o = 16; o > 0; o >>= 1) {
          const double os = __shfl_down_sync(0xffffffffu, bs, o);
          const int orr = __shfl_down_sync(0xffffffffu, br, o);
          if (j_better(os, orr, bs, br)) { bs = os; br = orr; }
        }
        if (lane == 0) { red_s[warp] = bs; red_r[warp] = br; }
        __syncthreads();
        if (warp == 0) {
          bs = (lane < TB / 32) ? red_s[lane] : INFINITY;
          br = (lane < TB / 32) ? red_r[lane] : 0x7fffffff;
          for (int o = 16; o > 0; o >>= 1) {
            const double os = __shfl_down_sync(0xffffffffu, bs, o);
            const int orr = __shfl_down_sync(0xffffffffu, br, o);
            if (j_better(os, orr, bs, br)) { bs = os; br = orr; }
          }
          if (lane == 0) sh_best = (br == 0x7fffffff) ? -1 : br;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
      if (sh_fail) {
        if (P.status) P.status[loc] = (int8_t)LAGP_ERR_NOT_PD;
        P.mean[loc] = NAN;
        P.s2[loc] = NAN;
        if (P.var) P.var[loc] = NAN;
      } else {
        double mu = 0.0;
        for (int i = 0; i < n; i++) mu = fma(ux[i], yt[i], mu);
        const double pv = sh_psi * sh_vx;
        P.mean[loc] = mu;
        P.s2[loc] = pv / n;
        if (P.var) P.var[loc] = pv / (n - 2);
        if (P.status) P.status[loc] = 0;
      }
    }
    if (L.idx)
      for (int i = tid; i < n; i += TB) L.idx[i] = sh_fail ? -1 : cnd[dr[i]];
  }
}

int mspe_grid(int64_t T, int num_sms) {
  const int64_t g = num_sms;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

struct MspeLayout {
  size_t u, ud, xc, cs, nn, idx, pred, total;
};

// [queue | U | Ud | Xc | cs | Li, Kd, Kdd, Q | design indices | kernel (c) workspace]
MspeLayout mspe_layout(int G, int p, int n, int M, int64_t T, int64_t idx_total, int num_sms) {
  const size_t Mpad = align_up((size_t)M, 32);
  MspeLayout L;
  L.u = align_up((size_t)G * n * Mpad * sizeof(double), 256);
  L.ud = L.u;
  L.xc = align_up((size_t)G * p * Mpad * sizeof(double), 256);
  L.cs = align_up((size_t)G * 4 * Mpad * sizeof(double), 256);
  L.nn = align_up((size_t)G * n * n * sizeof(double), 256);
  L.idx = align_up((size_t)idx_total * sizeof(int32_t), 256);
  L.pred = predict_fp64_workspace_bytes(T, n, num_sms);
  L.total = 256 + L.u + L.ud + L.xc + L.cs + 4 * L.nn + L.idx + L.pred;
  return L;
}

size_t mspe_smem_bytes(int Mpad, int n) {
  return (size_t)(2 * Mpad + 10 * n) * sizeof(double) + (size_t)n * sizeof(int) +
         align_up((size_t)Mpad, 16);
}

// The design kernel, then kernel (c) (predict.cu) on the designs it selected: the
// predictive equations are re-evaluated from a fresh FP64 factorisation in the textbook
// operation order, which tracks a sequential evaluation more closely in the strongly
// cancelling cases than the step-by-step updates do.
int mspe_run(MspeParams P, const MspeLayout &L, int G, char *w, int32_t *user_idx,
             const DevInfo &di, cudaStream_t stream) {
  P.queue = reinterpret_cast<int *>(w);
  size_t off = 256;
  P.U = reinterpret_cast<double *>(w + off); off += L.u;
  P.Ud = reinterpret_cast<double *>(w + off); off += L.ud;
  P.Xc = reinterpret_cast<double *>(w + off); off += L.xc;
  P.cs = reinterpret_cast<double *>(w + off); off += L.cs;
  P.Li = reinterpret_cast<double *>(w + off); off += L.nn;
  P.Kd = reinterpret_cast<double *>(w + off); off += L.nn;
  P.Kdd = reinterpret_cast<double *>(w + off); off += L.nn;
  P.Q = reinterpret_cast<double *>(w + off); off += L.nn;
  P.idx = user_idx ? user_idx : reinterpret_cast<int32_t *>(w + off);
  off += L.idx;
  const size_t smem = mspe_smem_bytes(P.Mpad, P.nmax);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(select_mspe_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(P.queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_status(e);
  select_mspe_kernel<<<G, TB, smem, stream>>>(P);
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

size_t select_mspe_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms) {
  return mspe_layout(mspe_grid(T, num_sms), p, n, ncand, T, T * n, num_sms).total;
}

int select_mspe_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  const int G = mspe_grid(a.T, di.num_sms);
  const MspeLayout L = mspe_layout(G, a.p, a.n, a.M, a.T, a.T * a.n, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MspeParams P;
  P.X = a.X; P.Z = a.Z; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Mpad = (int)align_up((size_t)a.M, 32); P.n0 = a.n0; P.n = a.n;
  P.theta = a.theta; P.theta_inv = 1.0 / a.theta; P.g = a.g; P.onepg = 1.0 + a.g;
  P.nmax = a.n; P.pmax = a.p;
  P.B = BatchView{nullptr, nullptr, nullptr, 0, a.theta_loc, nullptr};
  P.start = a.start; P.nstart = a.nstart;
  P.mean = a.mean; P.s2 = a.s2; P.var = a.var; P.status = a.status;
  return mspe_run(P, L, G, static_cast<char *>(ws), a.idx, di, stream);
}

size_t select_mspe_batch_workspace_bytes(const BatchLaunch &b, int G) {
  DevInfo di;
  const int sms = dev_info(&di) == LAGP_OK ? di.num_sms : 152;
  return mspe_layout(G, b.pmax, b.nmax, b.Mmax, b.T, b.idx_total, sms).total;
}

int select_mspe_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, int G,
                             cudaStream_t stream) {
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();  // this translation unit's copy of the exp constants
  if (st) return st;
  const MspeLayout L = mspe_layout(G, b.pmax, b.nmax, b.Mmax, b.T, b.idx_total, di.num_sms);
  if (ws_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  MspeParams P;
  P.X = nullptr; P.Z = nullptr; P.p = b.pmax; P.XX = b.XX; P.T = b.T; P.cand = b.cand;
  P.M = b.Mmax; P.Mpad = (int)align_up((size_t)b.Mmax, 32); P.n0 = 0; P.n = b.nmax;
  P.theta = 1.0; P.theta_inv = 1.0; P.g = 0.0; P.onepg = 1.0;
  P.nmax = b.nmax; P.pmax = b.pmax;
  P.B = BatchView{b.designs, b.locs, b.order, b.ldxx, nullptr, nullptr};
  P.start = nullptr; P.nstart = 0;
  P.mean = b.mean; P.s2 = b.s2; P.var = b.var; P.status = b.status;
  return mspe_run(P, L, G, static_cast<char *>(ws), b.idx, di, stream);
}

int select_mspe_prepare() {
  const int st = exp_table_upload();
  return st ? st : predict_fp64_prepare();
}

}  // namespace lagp
