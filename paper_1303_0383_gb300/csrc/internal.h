// internal.h -- declarations shared by the translation units of liblagp (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "lagp.h"
#include "batch.cuh"

namespace lagp {

// Upper limits checked by the entry points (see the argument rules in lagp.h).
constexpr int kMaxP = 8;
constexpr int kMaxN = 256;       // local design size n
constexpr int kMaxCand = 8192;   // candidate count
#define LAGP_MIX_CTAS_PER_SM 3     // resident CTAs per SM of the mixed kernel

extern std::atomic<int64_t> g_launches;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device properties of the current device, cached per device ordinal.
struct DevInfo {
  int device;
  int num_sms;
  size_t smem_optin;
  size_t smem_per_sm;
};
int dev_info(DevInfo *out);

// Kernel (a): candidate sets.
size_t knn_workspace_bytes(int64_t N, int64_t T, int32_t ncand, int num_sms);
int knn_launch(const double *X, int64_t N, int32_t p, const double *XX, int64_t T, int32_t ncand,
               int32_t *cand, void *ws, size_t ws_bytes, cudaStream_t stream);
int knn_launch_list(const double *X, int64_t N, int32_t p, const double *XX, int64_t nloc,
                    int32_t M, int32_t *cand, void *ws, size_t ws_bytes, cudaStream_t stream,
                    const int32_t *list, const LocDesc *locs, int ldxx, int ctas_per_sm);

// Kernels (b)+(c): greedy design and predictive equations.
struct SelectArgs {
  const double *X, *Z;
  int64_t N;
  int32_t p;
  const double *XX;
  int64_t T;
  const int32_t *cand;
  int32_t M, n0, n;
  double theta, g;
  const double *theta_loc;  // per-location lengthscale (device, T), or nullptr: theta
  const int32_t *start;     // saved start designs (device, T x nstart), or nullptr: n0 nearest
  int32_t nstart;
  double r_min;             // > 1: stopping rule of Sec. 6 (ALC), 0: fixed n
  int32_t *n_out;           // adaptive designs' sizes (device, T), with r_min
  int32_t method, precision;
  double *mean, *s2, *var;
  int32_t *idx;
  int8_t *status;
};
size_t select_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int32_t method,
                              int32_t precision, int num_sms);
int select_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream);
// The same launch on a caller-chosen grid of G CTAs (G >= 1), and the scratch it needs.
int select_default_grid(int64_t T, int num_sms);
size_t select_scratch_bytes_for_grid(int G, int32_t p, int32_t n, int32_t ncand);
int select_launch_on_grid(const SelectArgs &a, void *ws, size_t ws_bytes, int G,
                          cudaStream_t stream);

// Mixed-precision variant of kernels (b)+(c) (ALC): float-float screen, FP64 decisions.
size_t select_mixed_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms);
int select_mixed_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream);

// ALC in the paper's own form (explicit K_j^{-1}, partition inverse updates), FP64:
// kernel (b) then kernel (c) on the selected design (select_dense.cu).
int select_dense_max_n();
size_t select_dense_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms);
int select_dense_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream);

// Kernel (c) on a selected design: FP64 predictive equations for every location from its
// design indices (idx < 0 marks a location whose screen failed).
struct PredictArgs {
  const double *X, *Z;
  int32_t p;
  const double *XX;
  int64_t T;
  int32_t n, nmax;
  double theta, g;
  const int32_t *idx;
  BatchView B;  // per-location tables, or designs == nullptr for a uniform launch
  double *mean, *s2, *var;
  int8_t *status;
};
size_t predict_fp64_workspace_bytes(int64_t T, int32_t nmax, int num_sms);
int predict_fp64_launch(const PredictArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream);
int predict_fp64_prepare();

// Local maximum-likelihood lengthscale of each location's design (mle.cu).
struct MleArgs {
  const double *X, *Z;
  int32_t p;
  int64_t T;
  const int32_t *idx;
  int32_t n;
  double theta0;
  const double *theta0_loc;
  double g, tmin, tmax, tol;
  int32_t maxit;
  double *theta_out;
  int32_t *iters;
  int8_t *status;
};
size_t mle_workspace_bytes(int64_t T, int32_t n, int num_sms);
int mle_launch(const MleArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream);
int mle_prepare();

// MSPE variant of kernels (b)+(c), FP64.
size_t select_mspe_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms);
int select_mspe_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream);
// MSPE, mixed precision: float-float screen, FP64 bookkeeping and decisions.
size_t select_mspe_mixed_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int num_sms);
int select_mspe_mixed_launch(const SelectArgs &a, void *ws, size_t ws_bytes, cudaStream_t stream);
#define LAGP_MSPE_MIX_CTAS_PER_SM 2  // resident CTAs per SM of the mixed MSPE kernel

// Batched launch of kernels (b)+(c): per-location tables in device memory (batch.cuh),
// one persistent launch of G = ctas_per_sm x SMs CTAs over the cost-ordered queue.
struct BatchDesign;
struct BatchLaunch {
  int32_t method, precision;
  int64_t T;
  const BatchDesign *designs;  // device
  const LocDesc *locs;         // device, T entries
  const int32_t *order;        // device, queue position -> location
  const double *XX;
  int32_t ldxx;
  const int32_t *cand;         // device; location t's list at locs[t].cand_off
  int32_t nmax, pmax, Mmax;
  double *mean, *s2, *var;
  int32_t *idx;                // location t's indices at locs[t].idx_off
  int64_t idx_total;           // sum of the locations' n (the length of idx)
  int8_t *status;
  int32_t ctas_per_sm;         // 1 .. select_max_ctas()
};
int select_max_ctas(int32_t method, int32_t precision);
// Per-translation-unit set-up that must not happen during stream capture (constant uploads).
int select_prepare();
int select_mixed_prepare();
int select_mspe_prepare();
int select_mspe_mixed_prepare();
size_t select_batch_workspace_bytes(const BatchLaunch &b, int num_sms);
int select_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t select_mixed_batch_workspace_bytes(const BatchLaunch &b, int G);
int select_mixed_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, int G, cudaStream_t stream);
size_t select_mspe_batch_workspace_bytes(const BatchLaunch &b, int G);
int select_mspe_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, int G, cudaStream_t stream);
size_t select_mspe_mixed_batch_workspace_bytes(const BatchLaunch &b, int G);
int select_mspe_mixed_batch_launch(const BatchLaunch &b, void *ws, size_t ws_bytes, int G,
                                   cudaStream_t stream);

// Argument checks shared by the entry points (api.cu).
int check_common(int64_t N, int32_t p, int64_t T, int32_t n0, int32_t n, int32_t ncand,
                 double theta, double g, int32_t method, int32_t precision);
int check_supported(int32_t method, int32_t precision);

// Unique id of the calling thread's current CUDA context, 0 if none (api.cu).
int current_context_id(unsigned long long *id);

// Bounds-check records of the checked build (check.cuh): one per instrumented translation
// unit, read and cleared by these (all zero in normal builds).
struct CheckRec {
  unsigned long long count;  // violations since the last take
  long long site, index, bound;
};
int knn_check_take(CheckRec *out);
int select_check_take(CheckRec *out);
int select_mixed_check_take(CheckRec *out);
int select_dense_check_take(CheckRec *out);

// Map the last CUDA error to a library code.
int cuda_status(cudaError_t e);

}  // namespace lagp
