// select.cu -- kernels (b)+(c): greedy local design and predictive equations, FP64.
//
// Gramacy & Apley, Sec. 3: starting from the n0 nearest neighbours, the local design
// grows one point at a time; each step adds the candidate c that maximises the ALC
// reduction in variance at x (Eq. dxy; SM "partial correlations", Eq. dxy2):
//     score(c) = cov_j(x,c)^2 / v_j(c),
//     cov_j(a,b) = K(a,b) - k_j(a)^T K_j^{-1} k_j(b),  v_j(c) = cov_j(c,c),
// or, for NN, simply the next nearest.  Sec. 3.2 requires every step to cost O(j^2)
// per candidate at most; this kernel costs O(j) per candidate per step by carrying,
// for every candidate, the row u_c = L_j^{-1} k_j(c) of the bordered Cholesky factor
// L_j of K_j together with v_j(c) and cov_j(x,c).  Adding point s appends
//     L_{j+1} = [[L_j, 0], [u_s^T, sqrt(v_j(s))]]
// (the Cholesky counterpart of the partitioned inverse of SM Sec. 1, with the same
// Schur-complement scalar v_j(s)), and every candidate updates in O(j):
//     u_c[j]     = (K(s,c) - u_s . u_c) / sqrt(v_j(s))      (= cov_j(s,c)/sqrt(v_j(s)))
//     v_{j+1}(c) = v_j(c) - u_c[j]^2                         (Eq. dxy applied at c)
//     cov_{j+1}(x,c) = cov_j(x,c) - u_x[j] u_c[j].
// The same recursion gives u_x = L^{-1} k(x) and ytil = L^{-1} Y, hence
//     psi_{j+1} = psi_j + ytil_j^2   with ytil_j = (y_s - mu_j(s)) / sqrt(v_j(s))
// (Eq. psiup in the form the SM derives for E{psi_{j+1}}), and at the end
// mu = u_x . ytil, v_n(x) = K(x,x) - ||u_x||^2, s2 = psi v_n(x)/n, V = psi v_n(x)/(n-2)
// (Eqs. predgp, preds2).  The start design is built by the same recursion with the
// pivot forced to ranks 0..n0-1.
//
// Correlations use the library's table-driven FP64 exponential (fp64_exp.cuh); ALC scores
// are compared as fractions, without a division per candidate.
//
// Layout: one persistent CTA per resident location (a work counter hands out
// locations).  Per CTA, scratch holds U[j][c] (row j of every candidate, coalesced
// over c) and the candidates' coordinates Xc[k][c]; v, cov(x,.) and the used flags
// live in shared memory.
#include <math.h>

#include "batch.cuh"
#include "check.cuh"
#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {
namespace {

constexpr int SB = 256;  // threads per CTA

struct SelParams {
  const double *X, *Z;
  int64_t N;       // design rows (uniform launches; batched ones take each design's)
  int p;
  const double *XX;
  int64_t T;
  const int32_t *cand;
  int M, Mpad, n0, n, method;
  int nmax, pmax;  // slot dimensions (the largest n and p of the launch)
  double theta, g;
  double *mean, *s2, *var;
  int32_t *idx;
  int8_t *status;
  double *U;      // gridDim.x slots of nmax x Mpad
  double *Xc;     // gridDim.x slots of pmax x Mpad
  int *queue;
  BatchView B;    // per-location tables (B.designs == nullptr: uniform launch)
  const int32_t *start;  // saved start designs (T x nstart design indices), or nullptr
  int nstart;
  double r_min;          // > 1: stopping rule of Sec. 6 (ALC); 0: the design has n points
  int32_t *n_out;        // design sizes (T) when r_min > 1
};

// ALC scores are compared as fractions cov^2 / v without dividing: a/da beats b/db when
// a*db > b*da (both denominators are positive), ties going to the smaller rank.
__device__ __forceinline__ bool score_better(double a, double da, int ra, double b, double db,
                                             int rb) {
  const double l = a * db, r = b * da;
  return l > r || (l == r && ra < rb);
}

__global__ void __launch_bounds__(SB, 2) select_fp64_kernel(SelParams P) {
  extern __shared__ __align__(16) double sm[];
  const int Mpad = P.Mpad, nmax = P.nmax;
  double *v = sm;                       // Mpad
  double *covx = v + Mpad;              // Mpad
  double *srow = covx + Mpad;           // nmax  (u_s, the new row of L)
  double *ux = srow + nmax;             // nmax  (u_x = L^{-1} k(x))
  double *yt = ux + nmax;               // nmax  (ytil = L^{-1} Y)
  unsigned char *used = reinterpret_cast<unsigned char *>(yt + nmax);  // Mpad
  int *sr = reinterpret_cast<int *>(used + Mpad);                     // nmax: start ranks
  __shared__ double xs[kMaxP], xl[kMaxP];
  __shared__ double red_s[SB / 32], red_d[SB / 32];
  __shared__ int red_r[SB / 32];
  __shared__ double etab[64];
  if (threadIdx.x < 64) etab[threadIdx.x] = c_exp.tab[threadIdx.x];
  __shared__ int sh_loc, sh_best, sh_fail, sh_n;
  __shared__ double sh_inv, sh_uxj, sh_vx, sh_psi;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double *U = P.U + (size_t)blockIdx.x * nmax * Mpad;
  double *Xc = P.Xc + (size_t)blockIdx.x * P.pmax * Mpad;
  // checked build: the layout above ends within the launch's dynamic shared memory
  if (!LAGP_CHK(reinterpret_cast<unsigned char *>(sr + nmax) - reinterpret_cast<unsigned char *>(sm),
                dynamic_smem_bytes() + 1u, 25))
    return;

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    if (sh_loc >= P.T) break;
    const LocParams L = resolve_loc(P.B, sh_loc, P.X, P.Z, P.XX, P.p, P.n, P.M, P.n0, P.theta,
                                    P.g, P.cand, P.idx, P.N);
    const int64_t loc = L.loc;
    const int n = L.n, p = L.p, M = L.M;
    // checked build: the location fits the slot (rows, candidates, coordinates)
    if (!(LAGP_CHK(n - 1, nmax, 21) && LAGP_CHK(M - 1, Mpad, 22) && LAGP_CHK(p - 1, P.pmax, 23)))
      continue;
    const int32_t *cnd = L.cand;
    if (tid < p) xl[tid] = L.x[tid];
    if (tid == 0) { sh_fail = 0; sh_vx = L.onepg; sh_psi = 0.0; sh_n = n; }
    __syncthreads();
    // the start design: the n0 nearest, or a saved design (augmentation)
    const int n0e = P.start ? P.nstart : L.n0;
    if (P.start) start_ranks(P.start + loc * P.nstart, P.nstart, cnd, M, sr);
    // Stage candidate coordinates; v = K(c,c) = 1+g, cov_0(x,c) = K(x,c).
    // NN, and ALC without greedy steps (n0 == n), never look past rank n-1
    const int limit = ((P.method == LAGP_NN || n0e == n) && !P.start) ? n : M;
    for (int c = tid; c < limit; c += SB) {
      if (!LAGP_CHK(cnd[c], L.N, 24)) {  // never read, never chosen
        v[c] = 0.0;
        covx[c] = 0.0;
        used[c] = 1;
        continue;
      }
      const double *xc = L.X + (int64_t)cnd[c] * p;
      double acc = 0.0;
      for (int k = 0; k < p; k++) {
        double xk = xc[k];
        Xc[k * Mpad + c] = xk;
        double t = xl[k] - xk;
        acc = fma(t, t, acc);
      }
      v[c] = L.onepg;
      covx[c] = exp_nonpos(-acc * L.theta_inv, etab);
      used[c] = 0;
    }
    __syncthreads();

    int s = 0;
    for (int j = 0; j < n; j++) {
      if (j >= n0e && P.method == LAGP_ALC) s = sh_best;
      else s = (P.start && j < n0e) ? sr[j] : j;
      if (s < 0) {  // nothing admissible left
        if (tid == 0) sh_fail = 1;
        __syncthreads();
        break;
      }
      for (int i = tid; i < j; i += SB) srow[i] = U[(size_t)i * Mpad + s];
      if (tid < p) xs[tid] = Xc[tid * Mpad + s];
      __syncthreads();
      if (tid == 0) {
        const double vs = v[s];
        if (!(vs > 0.0)) {
          sh_fail = 1;
        } else {
          const double sq = sqrt(vs);
          const double uxj = covx[s] / sq;                 // u_x[j]
          const double vxn = fma(-uxj, uxj, sh_vx);       // v_{j+1}(x)
          if (P.r_min > 0.0 && j >= n0e && sh_vx / vxn < P.r_min) {
            // Sec. 6 stopping rule: the design stops before a greedy point whose variance
            // reduction ratio v_j(x) / v_{j+1}(x) (psi cancels) is below r_min
            sh_n = j;
          } else {
            double t = L.Z[cnd[s]];
            for (int i = 0; i < j; i++) t = fma(-srow[i], yt[i], t);
            const double ytj = t / sq;                     // ytil[j]
            ux[j] = uxj;
            yt[j] = ytj;
            sh_vx = vxn;
            sh_psi = fma(ytj, ytj, sh_psi);
            sh_inv = 1.0 / sq;
            sh_uxj = uxj;
            used[s] = 1;
            if (L.idx) L.idx[j] = cnd[s];
          }
        }
      }
      __syncthreads();
      if (sh_n == j) break;
      if (sh_fail) break;
      if (j == n - 1) break;
      const double inv = sh_inv, uxj = sh_uxj;
      const bool want_score = (P.method == LAGP_ALC) && (j + 1 >= n0e);
      double bs = -1.0, bd = 1.0;   // best score as a fraction bs/bd (none yet: -1)
      int br = 0x7fffffff;
      for (int c = tid; c < limit; c += SB) {
        if (used[c]) continue;
        double acc = 0.0;
        for (int k = 0; k < p; k++) {
          double t = xs[k] - Xc[k * Mpad + c];
          acc = fma(t, t, acc);
        }
        double t = exp_nonpos(-acc * L.theta_inv, etab);  // K(s, c)
        const double *Uc = U + c;
        for (int i = 0; i < j; i++, Uc += Mpad) t = fma(-srow[i], *Uc, t);
        const double u = t * inv;                          // u_c[j]
        U[(size_t)j * Mpad + c] = u;
        const double vc = fma(-u, u, v[c]);
        const double cx = fma(-uxj, u, covx[c]);
        v[c] = vc;
        covx[c] = cx;
        if (want_score && vc > 0.0) {
          const double num = cx * cx;                      // ALC reduction num/vc, Eq. dxy
          if (score_better(num, vc, c, bs, bd, br)) { bs = num; bd = vc; br = c; }
        }
      }
      if (want_score) {
        for (int o = 16; o > 0; o >>= 1) {
          double os = __shfl_down_sync(0xffffffffu, bs, o);
          double od = __shfl_down_sync(0xffffffffu, bd, o);
          int orr = __shfl_down_sync(0xffffffffu, br, o);
          if (score_better(os, od, orr, bs, bd, br)) { bs = os; bd = od; br = orr; }
        }
        if (lane == 0) { red_s[warp] = bs; red_d[warp] = bd; red_r[warp] = br; }
        __syncthreads();
        if (warp == 0) {
          bs = (lane < SB / 32) ? red_s[lane] : -1.0;
          bd = (lane < SB / 32) ? red_d[lane] : 1.0;
          br = (lane < SB / 32) ? red_r[lane] : 0x7fffffff;
          for (int o = 16; o > 0; o >>= 1) {
            double os = __shfl_down_sync(0xffffffffu, bs, o);
            double od = __shfl_down_sync(0xffffffffu, bd, o);
            int orr = __shfl_down_sync(0xffffffffu, br, o);
            if (score_better(os, od, orr, bs, bd, br)) { bs = os; bd = od; br = orr; }
          }
          if (lane == 0) sh_best = (br == 0x7fffffff) ? -1 : br;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    const int ne = sh_n;  // the design's size (n, or where the stopping rule ended it)
    if (tid == 0) {
      if (P.n_out) P.n_out[loc] = sh_fail ? 0 : ne;
      if (sh_fail) {
        if (P.status) P.status[loc] = (int8_t)LAGP_ERR_NOT_PD;
        P.mean[loc] = NAN;
        P.s2[loc] = NAN;
        if (P.var) P.var[loc] = NAN;
      } else {
        double mu = 0.0;
        for (int i = 0; i < ne; i++) mu = fma(ux[i], yt[i], mu);
        const double pv = sh_psi * sh_vx;
        P.mean[loc] = mu;
        P.s2[loc] = pv / ne;
        if (P.var) P.var[loc] = pv / (ne - 2);
        if (P.status) P.status[loc] = 0;
      }
    }
    if (L.idx) {
      // A failed location reports no design: every index is -1; an adaptive design's
      // unused slots are -1 too.
      for (int i = tid; i < n; i += SB)
        if (sh_fail || i >= ne) L.idx[i] = -1;
    }
  }
}

int sel_grid(int64_t T, int num_sms) {
  int64_t g = (int64_t)num_sms * 2;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

int mpad_of(int M) { return (int)align_up((size_t)M, 32); }

size_t sel_smem_bytes(int Mpad, int n) {
  return (size_t)(2 * Mpad + 3 * n) * sizeof(double) + align_up((size_t)Mpad, 16) +
         align_up((size_t)n * sizeof(int), 16);
}

}  // namespace

int select_check_take(CheckRec *out) { return check_take_here(out); }

size_t select_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int32_t method,
                              int32_t precision, int num_sms) {
  if (method == LAGP_MSPE)
    return precision == LAGP_MIXED ? select_mspe_mixed_workspace_bytes(T, p, n, ncand, num_sms)
                                   : select_mspe_workspace_bytes(T, p, n, ncand, num_sms);
  if (precision == LAGP_MIXED && method == LAGP_ALC)
    return select_mixed_workspace_bytes(T, p, n, ncand, num_sms);
  const size_t Mpad = (size_t)mpad_of(ncand);
  const size_t G = (size_t)sel_grid(T, num_sms);
  return 256 + align_up(G * (size_t)n * Mpad * sizeof(double), 256) +
         align_up(G * (size_t)p * Mpad * sizeof(double), 256);
}

int select_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  if (a.method == LAGP_MSPE)
    return a.precision == LAGP_MIXED ? select_mspe_mixed_launch(a, ws, ws_bytes, stream)
                                     : select_mspe_launch(a, ws, ws_bytes, stream);
  if (a.precision == LAGP_MIXED && a.method == LAGP_ALC)
    return select_mixed_launch(a, ws, ws_bytes, stream);
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  if (ws_bytes < select_workspace_bytes(a.T, a.p, a.n, a.M, a.method, a.precision, di.num_sms))
    return LAGP_ERR_INVALID_ARG;
  const int Mpad = mpad_of(a.M);
  const int G = sel_grid(a.T, di.num_sms);
  char *w = static_cast<char *>(ws);
  SelParams P;
  P.X = a.X; P.Z = a.Z; P.N = a.N; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Mpad = Mpad; P.n0 = a.n0; P.n = a.n; P.method = a.method;
  P.theta = a.theta;
  P.g = a.g;
  P.nmax = a.n;
  P.pmax = a.p;
  P.B = BatchView{nullptr, nullptr, nullptr, 0, a.theta_loc, nullptr};
  P.start = a.start; P.nstart = a.nstart;
  P.r_min = a.r_min; P.n_out = a.n_out;
  P.mean = a.mean; P.s2 = a.s2; P.var = a.var; P.idx = a.idx; P.status = a.status;
  P.queue = reinterpret_cast<int *>(w);
  P.U = reinterpret_cast<double *>(w + 256);
  P.Xc = reinterpret_cast<double *>(w + 256 + align_up((size_t)G * a.n * Mpad * sizeof(double), 256));
  const size_t smem = sel_smem_bytes(Mpad, a.n);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(select_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(P.queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_status(e);
  select_fp64_kernel<<<G, SB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

int select_default_grid(int64_t T, int num_sms) { return sel_grid(T, num_sms); }

size_t select_scratch_bytes_for_grid(int G, int32_t p, int32_t n, int32_t ncand) {
  const size_t Mpad = (size_t)mpad_of(ncand);
  return 256 + align_up((size_t)G * (size_t)n * Mpad * sizeof(double), 256) +
         align_up((size_t)G * (size_t)p * Mpad * sizeof(double), 256);
}

int select_launch_on_grid(const SelectArgs &a, void *ws, size_t ws_bytes, int G,
                          cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  if (G < 1) return LAGP_ERR_INVALID_ARG;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  if (ws_bytes < select_scratch_bytes_for_grid(G, a.p, a.n, a.M)) return LAGP_ERR_INVALID_ARG;
  const int Mpad = mpad_of(a.M);
  char *w = static_cast<char *>(ws);
  SelParams P;
  P.X = a.X; P.Z = a.Z; P.N = a.N; P.p = a.p; P.XX = a.XX; P.T = a.T; P.cand = a.cand;
  P.M = a.M; P.Mpad = Mpad; P.n0 = a.n0; P.n = a.n; P.method = a.method;
  P.theta = a.theta;
  P.g = a.g;
  P.nmax = a.n;
  P.pmax = a.p;
  P.B = BatchView{nullptr, nullptr, nullptr, 0, a.theta_loc, nullptr};
  P.start = a.start; P.nstart = a.nstart;
  P.r_min = a.r_min; P.n_out = a.n_out;
  P.mean = a.mean; P.s2 = a.s2; P.var = a.var; P.idx = a.idx; P.status = a.status;
  P.queue = reinterpret_cast<int *>(w);
  P.U = reinterpret_cast<double *>(w + 256);
  P.Xc = reinterpret_cast<double *>(w + 256 + align_up((size_t)G * a.n * Mpad * sizeof(double), 256));
  const size_t smem = sel_smem_bytes(Mpad, a.n);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(select_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(P.queue, 0, sizeof(int), stream);   // the work counter starts at zero
  if (e != cudaSuccess) return cuda_status(e);
  select_fp64_kernel<<<G, SB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

int select_max_ctas(int32_t method, int32_t precision) {
  if (method == LAGP_MSPE) return precision == LAGP_MIXED ? LAGP_MSPE_MIX_CTAS_PER_SM : 1;
  if (precision == LAGP_MIXED && method == LAGP_ALC) return LAGP_MIX_CTAS_PER_SM;
  return 2;
}

static int batch_grid(const BatchLaunch &b, int num_sms) {
  int c = b.ctas_per_sm;
  const int cmax = select_max_ctas(b.method, b.precision);
  if (c < 1 || c > cmax) c = cmax;
  const int64_t g = (int64_t)num_sms * c;
  return (int)(b.T < g ? (b.T > 0 ? b.T : 1) : g);
}

size_t select_batch_workspace_bytes(const BatchLaunch &b, int num_sms) {
  const int G = batch_grid(b, num_sms);
  if (b.method == LAGP_MSPE)
    return b.precision == LAGP_MIXED ? select_mspe_mixed_batch_workspace_bytes(b, G)
                                     : select_mspe_batch_workspace_bytes(b, G);
  if (b.precision == LAGP_MIXED && b.method == LAGP_ALC) return select_mixed_batch_workspace_bytes(b, G);
  return select_scratch_bytes_for_grid(G, b.pmax, b.nmax, b.Mmax);
}

int select_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (b.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();
  if (st) return st;
  const int G = batch_grid(b, di.num_sms);
  if (b.method == LAGP_MSPE)
    return b.precision == LAGP_MIXED ? select_mspe_mixed_batch_launch(b, ws, ws_bytes, G, stream)
                                     : select_mspe_batch_launch(b, ws, ws_bytes, G, stream);
  if (b.precision == LAGP_MIXED && b.method == LAGP_ALC)
    return select_mixed_batch_launch(b, ws, ws_bytes, G, stream);
  if (ws_bytes < select_scratch_bytes_for_grid(G, b.pmax, b.nmax, b.Mmax)) return LAGP_ERR_INVALID_ARG;
  const int Mpad = mpad_of(b.Mmax);
  char *w = static_cast<char *>(ws);
  SelParams P;
  P.X = nullptr; P.Z = nullptr; P.N = 0; P.p = b.pmax; P.XX = b.XX; P.T = b.T; P.cand = b.cand;
  P.M = b.Mmax; P.Mpad = Mpad; P.n0 = 0; P.n = b.nmax; P.method = b.method;
  P.theta = 1.0; P.g = 0.0; P.nmax = b.nmax; P.pmax = b.pmax;
  P.B = BatchView{b.designs, b.locs, b.order, b.ldxx, nullptr, nullptr};
  P.start = nullptr; P.nstart = 0;
  P.r_min = 0.0; P.n_out = nullptr;
  P.mean = b.mean; P.s2 = b.s2; P.var = b.var; P.idx = b.idx; P.status = b.status;
  P.queue = reinterpret_cast<int *>(w);
  P.U = reinterpret_cast<double *>(w + 256);
  P.Xc = reinterpret_cast<double *>(w + 256 + align_up((size_t)G * b.nmax * Mpad * sizeof(double), 256));
  const size_t smem = sel_smem_bytes(Mpad, b.nmax);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(select_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemsetAsync(P.queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_status(e);
  select_fp64_kernel<<<G, SB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

int select_prepare() { return exp_table_upload(); }

}  // namespace lagp
