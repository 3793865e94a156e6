// predict.cu -- kernel (c) for a screen that returns only the local design: the FP64
// predictive equations (Sec. 2, Eqs. predgp and preds2) on the selected design of every
// location, with the per-location arithmetic of predict_loc.cuh.
//
// One CTA owns one location at a time (persistent CTAs over a work queue); the matrix
// lives in shared memory when it fits, else in a per-CTA slot of the workspace.
#include <math.h>

#include "predict_loc.cuh"

namespace lagp {
namespace {

constexpr int PB = 128;              // threads per CTA
constexpr size_t kSmemA = 48 * 1024; // largest matrix kept in shared memory

struct PredParams {
  const double *X, *Z;
  int p;
  const double *XX;
  int64_t T;
  int n, nmax;
  double theta, g;
  const int32_t *idx;     // selected design indices (location t's n at its offset)
  BatchView B;
  double *mean, *s2, *var;
  int8_t *status;
  double *Ag;             // per-CTA matrix slots when the matrix is not in shared memory
  int a_in_smem;
  int *queue;
};

__global__ void __launch_bounds__(PB) predict_fp64_kernel(PredParams P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nmax = P.nmax;
  double *rl = reinterpret_cast<double *>(smraw);     // nmax: 1 / l_kk
  double *A = P.a_in_smem ? rl + nmax : P.Ag + (size_t)blockIdx.x * nmax * (nmax + 2);
  __shared__ double etab[64];
  __shared__ double xl[kMaxP];
  __shared__ int sh_loc, sh_fail;
  const int tid = threadIdx.x;
  if (tid < 64) etab[tid] = c_exp.tab[tid];

  for (;;) {
    __syncthreads();
    if (tid == 0) sh_loc = atomicAdd(P.queue, 1);
    __syncthreads();
    if (sh_loc >= P.T) break;
    const LocParams L = resolve_loc(P.B, sh_loc, P.X, P.Z, P.XX, P.p, P.n, 0, 0, P.theta, P.g,
                                    P.idx, const_cast<int32_t *>(P.idx));
    if (tid < L.p) xl[tid] = L.x[tid];
    predict_location(L, L.idx, L.n, xl, A, rl, etab, &sh_fail, L.loc, P.mean, P.s2, P.var,
                     P.status);
  }
}

bool a_fits_smem(int nmax) { return (size_t)nmax * (nmax + 2) * sizeof(double) <= kSmemA; }

size_t pred_smem_bytes(int nmax) {
  return (size_t)nmax * sizeof(double) +
         (a_fits_smem(nmax) ? (size_t)nmax * (nmax + 2) * sizeof(double) : 0);
}

int pred_grid(int64_t T, int nmax, const DevInfo &di) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, predict_fp64_kernel, PB,
                                                    pred_smem_bytes(nmax)) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t g = (int64_t)di.num_sms * per_sm;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

// Worst-case grid for sizing the workspace before the occupancy is known: the smem limit
// alone allows at most this many CTAs of 128 threads per SM (2048 threads per SM).
int pred_grid_bound(int64_t T, int num_sms) {
  const int64_t g = (int64_t)num_sms * 16;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

}  // namespace

size_t predict_fp64_workspace_bytes(int64_t T, int32_t nmax, int num_sms) {
  size_t b = 256;
  if (!a_fits_smem(nmax))
    b += align_up((size_t)pred_grid_bound(T, num_sms) * nmax * (nmax + 2) * sizeof(double), 256);
  return b;
}

int predict_fp64_launch(const PredictArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (a.T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  st = exp_table_upload();  // this translation unit's copy of the exp constants
  if (st) return st;
  if (ws_bytes < predict_fp64_workspace_bytes(a.T, a.nmax, di.num_sms)) return LAGP_ERR_INVALID_ARG;
  const size_t smem = pred_smem_bytes(a.nmax);
  cudaError_t e = cudaFuncSetAttribute(predict_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  int G = pred_grid(a.T, a.nmax, di);
  const int Gb = pred_grid_bound(a.T, di.num_sms);
  if (G > Gb) G = Gb;
  char *w = static_cast<char *>(ws);
  PredParams P;
  P.X = a.X; P.Z = a.Z; P.p = a.p; P.XX = a.XX; P.T = a.T; P.n = a.n; P.nmax = a.nmax;
  P.theta = a.theta; P.g = a.g; P.idx = a.idx;
  P.B = a.B;
  P.mean = a.mean; P.s2 = a.s2; P.var = a.var; P.status = a.status;
  P.queue = reinterpret_cast<int *>(w);
  P.a_in_smem = a_fits_smem(a.nmax) ? 1 : 0;
  P.Ag = P.a_in_smem ? nullptr : reinterpret_cast<double *>(w + 256);
  e = cudaMemsetAsync(P.queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_status(e);
  predict_fp64_kernel<<<G, PB, smem, stream>>>(P);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

int predict_fp64_prepare() { return exp_table_upload(); }

}  // namespace lagp
