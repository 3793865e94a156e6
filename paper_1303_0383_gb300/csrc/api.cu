// api.cu -- the C ABI of liblagp (declared in include/lagp.h): argument checks, the
// resident design handle, scratch sizing and the host-buffer wrapper around the device
// path.  All arithmetic of the method runs in the kernels of knn.cu and select.cu.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>

#include "internal.h"

namespace lagp {

std::atomic<int64_t> g_launches{0};

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LAGP_OK;
  if (e == cudaErrorMemoryAllocation) return LAGP_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return LAGP_ERR_NO_DEVICE;
  return LAGP_ERR_CUDA;
}

int dev_info(DevInfo *out) {
  static std::mutex mu;
  static DevInfo cache[64];
  static bool have[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= 64) return LAGP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  if (!have[dev]) {
    DevInfo d;
    d.device = dev;
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    d.num_sms = v;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_status(e);
    d.smem_optin = (size_t)v;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return cuda_status(e);
    d.smem_per_sm = (size_t)v;
    cache[dev] = d;
    have[dev] = true;
  }
  *out = cache[dev];
  return LAGP_OK;
}

// The unique id of the calling thread's current CUDA context (0 if it has none yet).  The
// per-device caches of device addresses and constant uploads are keyed on it: after a
// cudaDeviceReset the device's next context is a new one, whose constant banks are not
// uploaded and whose symbol addresses may differ.  The driver functions are reached
// through the runtime, so the library does not link the driver library itself.
int current_context_id(unsigned long long *id) {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static std::once_flag once;
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  *id = 0;
  if (!get_current || !get_id) return LAGP_ERR_CUDA;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS) return LAGP_ERR_CUDA;
  if (!c) return LAGP_OK;
  return get_id(c, id) == CUDA_SUCCESS ? LAGP_OK : LAGP_ERR_CUDA;
}

int check_common(int64_t N, int32_t p, int64_t T, int32_t n0, int32_t n, int32_t ncand,
                 double theta, double g, int32_t method, int32_t precision) {
  if (N < 1 || p < 1 || p > kMaxP || T < 0) return LAGP_ERR_INVALID_ARG;
  if (N > INT32_MAX || T > INT32_MAX) return LAGP_ERR_INVALID_ARG;
  if (n0 < 1 || n < n0 || n < 3 || n > kMaxN) return LAGP_ERR_INVALID_ARG;
  if (ncand < n || (int64_t)ncand > N || ncand > kMaxCand) return LAGP_ERR_INVALID_ARG;
  if (!(theta > 0.0) || !isfinite(theta) || !(g >= 0.0) || !isfinite(g)) return LAGP_ERR_INVALID_ARG;
  if (method != LAGP_ALC && method != LAGP_MSPE && method != LAGP_NN) return LAGP_ERR_INVALID_ARG;
  if (precision != LAGP_FP64 && precision != LAGP_MIXED) return LAGP_ERR_INVALID_ARG;
  if (method == LAGP_MSPE && n0 < 3) return LAGP_ERR_INVALID_ARG;
  return LAGP_OK;
}

int check_supported(int32_t method, int32_t precision) {
  (void)method;
  (void)precision;
  return LAGP_OK;
}

}  // namespace lagp

using namespace lagp;

struct lagp_design {
  double *X;
  double *Z;
  int64_t N;
  int32_t p;
  int device;
};

extern "C" {

const char *lagp_strerror(int code) {
  switch (code) {
    case LAGP_OK: return "ok";
    case LAGP_ERR_INVALID_ARG: return "invalid argument";
    case LAGP_ERR_OOM: return "out of device memory";
    case LAGP_ERR_CUDA: return "CUDA error";
    case LAGP_ERR_TIMEOUT: return "timed out";
    case LAGP_ERR_NOT_PD: return "conditional variance not positive (matrix not positive definite in FP64)";
    case LAGP_ERR_NO_DEVICE: return "no usable CUDA device";
    case LAGP_ERR_UNSUPPORTED: return "method/precision combination not supported by this build";
    case LAGP_ERR_SCRATCH_LIMIT: return "problem too large for the static scratch of the no-allocation entry point";
    case LAGP_ERR_NO_CONVERGENCE: return "iteration limit reached before the stopping rule was met";
    case LAGP_ERR_CANCELLED: return "request cancelled";
    default: return "unknown error code";
  }
}

int lagp_version(void) { return 100; }

int64_t lagp_launch_count(void) { return g_launches.load(); }

int lagp_design_create(const double *X, const double *Z, int64_t N, int32_t p, lagp_design **out) {
  if (!X || !Z || !out || N < 1 || N > INT32_MAX || p < 1 || p > kMaxP) return LAGP_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  lagp_design *d = new (std::nothrow) lagp_design();
  if (!d) return LAGP_ERR_OOM;
  d->N = N;
  d->p = p;
  d->device = dev;
  e = cudaMalloc(&d->X, (size_t)N * p * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d->Z, (size_t)N * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(d->X, X, (size_t)N * p * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d->Z, Z, (size_t)N * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d->X);
    cudaFree(d->Z);
    delete d;
    return cuda_status(e);
  }
  *out = d;
  return LAGP_OK;
}

int lagp_design_destroy(lagp_design *d) {
  if (!d) return LAGP_ERR_INVALID_ARG;
  cudaError_t e1 = cudaFree(d->X);
  cudaError_t e2 = cudaFree(d->Z);
  delete d;
  return cuda_status(e1 != cudaSuccess ? e1 : e2);
}

size_t lagp_knn_workspace_bytes(int64_t N, int64_t T, int32_t ncand) {
  DevInfo di;
  if (dev_info(&di)) return 0;
  return knn_workspace_bytes(N, T, ncand, di.num_sms);
}

int lagp_knn_dev(const double *X, int64_t N, int32_t p, const double *XX, int64_t T,
                 int32_t ncand, int32_t *cand, void *workspace, size_t workspace_bytes,
                 void *stream) {
  if (N < 1 || N > INT32_MAX || p < 1 || p > kMaxP || T < 0 || T > INT32_MAX || ncand < 1 ||
      (int64_t)ncand > N || ncand > kMaxCand)
    return LAGP_ERR_INVALID_ARG;
  if (T > 0 && (!X || !XX || !cand || !workspace)) return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  return knn_launch(X, N, p, XX, T, ncand, cand, workspace, workspace_bytes,
                    static_cast<cudaStream_t>(stream));
}

size_t lagp_select_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand, int32_t method,
                                   int32_t precision) {
  DevInfo di;
  if (dev_info(&di)) return 0;
  return select_workspace_bytes(T, p, n, ncand, method, precision, di.num_sms);
}

int lagp_select_dev(const double *X, const double *Z, int64_t N, int32_t p, const double *XX,
                    int64_t T, const int32_t *cand, int32_t ncand, int32_t n0, int32_t n,
                    double theta, double g, int32_t method, int32_t precision, double *mean,
                    double *s2, double *var, int32_t *idx, int8_t *status, void *workspace,
                    size_t workspace_bytes, void *stream) {
  int st = check_common(N, p, T, n0, n, ncand, theta, g, method, precision);
  if (st) return st;
  st = check_supported(method, precision);
  if (st) return st;
  if (T > 0 && (!X || !Z || !XX || !cand || !mean || !s2 || !workspace)) return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  SelectArgs a;
  a.X = X; a.Z = Z; a.N = N; a.p = p; a.XX = XX; a.T = T; a.cand = cand;
  a.M = ncand; a.n0 = n0; a.n = n; a.theta = theta; a.g = g; a.theta_loc = nullptr;
  a.start = nullptr; a.nstart = 0; a.r_min = 0.0; a.n_out = nullptr;
  a.method = method; a.precision = precision;
  a.mean = mean; a.s2 = s2; a.var = var; a.idx = idx; a.status = status;
  return select_launch(a, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

size_t lagp_select_dense_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand) {
  DevInfo di;
  if (dev_info(&di)) return 0;
  return select_dense_workspace_bytes(T, p, n, ncand, di.num_sms);
}

int lagp_select_dense_dev(const double *X, const double *Z, int64_t N, int32_t p,
                          const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                          int32_t n0, int32_t n, double theta, double g, double *mean, double *s2,
                          double *var, int32_t *idx, int8_t *status, void *workspace,
                          size_t workspace_bytes, void *stream) {
  int st = check_common(N, p, T, n0, n, ncand, theta, g, LAGP_ALC, LAGP_FP64);
  if (st) return st;
  if (n > select_dense_max_n()) return LAGP_ERR_UNSUPPORTED;
  if (T > 0 && (!X || !Z || !XX || !cand || !mean || !s2 || !workspace)) return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  SelectArgs a;
  a.X = X; a.Z = Z; a.N = N; a.p = p; a.XX = XX; a.T = T; a.cand = cand;
  a.M = ncand; a.n0 = n0; a.n = n; a.theta = theta; a.g = g; a.theta_loc = nullptr;
  a.start = nullptr; a.nstart = 0; a.r_min = 0.0; a.n_out = nullptr;
  a.method = LAGP_ALC; a.precision = LAGP_FP64;
  a.mean = mean; a.s2 = s2; a.var = var; a.idx = idx; a.status = status;
  return select_dense_launch(a, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

int lagp_check_take(int32_t *checked, int64_t *count, int32_t *site, int64_t *index,
                    int64_t *bound) {
#ifdef LAGP_CHECKED
  if (checked) *checked = 1;
#else
  if (checked) *checked = 0;
#endif
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  int (*const takes[])(CheckRec *) = {knn_check_take, select_check_take, select_mixed_check_take,
                                      select_dense_check_take};
  CheckRec first = {0ull, 0, 0, 0};
  unsigned long long total = 0ull;
  for (auto take : takes) {
    CheckRec r;
    const int st = take(&r);
    if (st) return st;
    if (r.count && !first.count) first = r;
    total += r.count;
  }
  if (count) *count = (int64_t)total;
  if (site) *site = (int32_t)first.site;
  if (index) *index = first.index;
  if (bound) *bound = first.bound;
  return LAGP_OK;
}

int lagp_select_rescore_count(const void *workspace, size_t workspace_bytes, int32_t method,
                              int32_t precision, int64_t *count, void *stream) {
  if (!count) return LAGP_ERR_INVALID_ARG;
  if (method != LAGP_ALC && method != LAGP_MSPE && method != LAGP_NN) return LAGP_ERR_INVALID_ARG;
  if (precision != LAGP_FP64 && precision != LAGP_MIXED) return LAGP_ERR_INVALID_ARG;
  *count = 0;
  if (precision != LAGP_MIXED || method == LAGP_NN) return LAGP_OK;
  if (!workspace || workspace_bytes < 512 || ((uintptr_t)workspace & 255) != 0)
    return LAGP_ERR_INVALID_ARG;
  // the mixed screens keep the count at byte 256 of their workspace (cleared at launch)
  int32_t v = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&v, static_cast<const char *>(workspace) + 256, sizeof(v),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  *count = v;
  return LAGP_OK;
}

size_t lagp_predict_workspace_bytes(int64_t N, int64_t T, int32_t p, int32_t n, int32_t ncand,
                                    int32_t method, int32_t precision) {
  DevInfo di;
  if (dev_info(&di)) return 0;
  size_t cand = align_up((size_t)(T > 0 ? T : 0) * (size_t)ncand * sizeof(int32_t), 256);
  size_t a = knn_workspace_bytes(N, T, ncand, di.num_sms);
  size_t b = select_workspace_bytes(T, p, n, ncand, method, precision, di.num_sms);
  return cand + (a > b ? a : b);
}

int lagp_predict_dev(const double *X, const double *Z, int64_t N, int32_t p, const double *XX,
                     int64_t T, int32_t n0, int32_t n, int32_t ncand, double theta, double g,
                     int32_t method, int32_t precision, double *mean, double *s2, double *var,
                     int32_t *idx, int8_t *status, void *workspace, size_t workspace_bytes,
                     void *stream) {
  int st = check_common(N, p, T, n0, n, ncand, theta, g, method, precision);
  if (st) return st;
  st = check_supported(method, precision);
  if (st) return st;
  if (T == 0) return LAGP_OK;
  if (!X || !Z || !XX || !mean || !s2 || !workspace) return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  if (workspace_bytes < lagp_predict_workspace_bytes(N, T, p, n, ncand, method, precision))
    return LAGP_ERR_INVALID_ARG;
  char *w = static_cast<char *>(workspace);
  size_t cand_bytes = align_up((size_t)T * (size_t)ncand * sizeof(int32_t), 256);
  int32_t *cand = reinterpret_cast<int32_t *>(w);
  void *rest = w + cand_bytes;
  size_t rest_bytes = workspace_bytes - cand_bytes;
  st = lagp_knn_dev(X, N, p, XX, T, ncand, cand, rest, rest_bytes, stream);
  if (st) return st;
  return lagp_select_dev(X, Z, N, p, XX, T, cand, ncand, n0, n, theta, g, method, precision, mean,
                         s2, var, idx, status, rest, rest_bytes, stream);
}

namespace {

// The host entry point's device blocks come from a pool of the library's own per device,
// which keeps up to kPoolKeep bytes of freed memory mapped for the next call (the default
// pool returns everything at each synchronisation, and re-mapping a few hundred MB of
// workspace costs about a millisecond per call).
constexpr uint64_t kPoolKeep = 4ull << 30;
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

int lib_pool(int device, cudaMemPool_t *out) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(device);
  if (it != g_pools.end()) {
    *out = it->second;
    return LAGP_OK;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  cudaMemPool_t pool;
  cudaError_t e = cudaMemPoolCreate(&pool, &props);
  if (e != cudaSuccess) return cuda_status(e);
  uint64_t keep = kPoolKeep;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) {
    cudaMemPoolDestroy(pool);
    return cuda_status(e);
  }
  g_pools[device] = pool;
  *out = pool;
  return LAGP_OK;
}

}  // namespace

int lagp_predict(const lagp_design *d, const double *XX, int64_t T, int32_t n0, int32_t n,
                 int32_t ncand, double theta, double g, int32_t method, int32_t precision,
                 double *mean, double *s2, double *var, int32_t *idx, int8_t *status) {
  if (!d) return LAGP_ERR_INVALID_ARG;
  int st = check_common(d->N, d->p, T, n0, n, ncand, theta, g, method, precision);
  if (st) return st;
  st = check_supported(method, precision);
  if (st) return st;
  if (T == 0) return LAGP_OK;
  if (!XX || !mean || !s2) return LAGP_ERR_INVALID_ARG;
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_status(e);
  if (cur != d->device) {
    e = cudaSetDevice(d->device);
    if (e != cudaSuccess) return cuda_status(e);
  }
  cudaStream_t s = cudaStreamPerThread;
  const size_t nT = (size_t)T, p = (size_t)d->p;
  const size_t ws_bytes = lagp_predict_workspace_bytes(d->N, T, d->p, n, ncand, method, precision);
  // One device block: XX | mean | s2 | var | idx | status | workspace
  size_t off_xx = 0;
  size_t off_mean = align_up(off_xx + nT * p * sizeof(double), 256);
  size_t off_s2 = align_up(off_mean + nT * sizeof(double), 256);
  size_t off_var = align_up(off_s2 + nT * sizeof(double), 256);
  size_t off_idx = align_up(off_var + nT * sizeof(double), 256);
  size_t off_st = align_up(off_idx + nT * (size_t)n * sizeof(int32_t), 256);
  size_t off_ws = align_up(off_st + nT, 256);
  size_t total = off_ws + ws_bytes;
  char *buf = nullptr;
  cudaMemPool_t pool;
  st = lib_pool(d->device, &pool);
  if (st) return st;
  e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&buf), total, pool, s);
  if (e != cudaSuccess) return cuda_status(e);
  double *dXX = reinterpret_cast<double *>(buf + off_xx);
  double *dmean = reinterpret_cast<double *>(buf + off_mean);
  double *ds2 = reinterpret_cast<double *>(buf + off_s2);
  double *dvar = reinterpret_cast<double *>(buf + off_var);
  int32_t *didx = reinterpret_cast<int32_t *>(buf + off_idx);
  int8_t *dst = reinterpret_cast<int8_t *>(buf + off_st);
  e = cudaMemcpyAsync(dXX, XX, nT * p * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    st = lagp_predict_dev(d->X, d->Z, d->N, d->p, dXX, T, n0, n, ncand, theta, g, method,
                          precision, dmean, ds2, dvar, didx, dst, buf + off_ws, ws_bytes, s);
    if (st == LAGP_OK) {
      e = cudaMemcpyAsync(mean, dmean, nT * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(s2, ds2, nT * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess && var)
        e = cudaMemcpyAsync(var, dvar, nT * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess && idx)
        e = cudaMemcpyAsync(idx, didx, nT * (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess && status)
        e = cudaMemcpyAsync(status, dst, nT, cudaMemcpyDeviceToHost, s);
    }
  }
  cudaError_t ef = cudaFreeAsync(buf, s);
  cudaError_t es = cudaStreamSynchronize(s);
  if (cur != d->device) cudaSetDevice(cur);
  if (st) return st;
  if (e != cudaSuccess) return cuda_status(e);
  if (ef != cudaSuccess) return cuda_status(ef);
  return cuda_status(es);
}

// ---- stagewise scheme (Sec. 4.2) ----

int lagp_select_augment_dev(const double *X, const double *Z, int64_t N, int32_t p,
                            const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                            const int32_t *start, int32_t n1, int32_t n, double theta, double g,
                            int32_t method, int32_t precision, double *mean, double *s2,
                            double *var, int32_t *idx, int8_t *status, void *workspace,
                            size_t workspace_bytes, void *stream) {
  int st = check_common(N, p, T, n1, n, ncand, theta, g, method, precision);
  if (st) return st;
  st = check_supported(method, precision);
  if (st) return st;
  if (method == LAGP_NN) return LAGP_ERR_UNSUPPORTED;
  if (T > 0 && (!X || !Z || !XX || !cand || !start || !mean || !s2 || !workspace))
    return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  SelectArgs a;
  a.X = X; a.Z = Z; a.N = N; a.p = p; a.XX = XX; a.T = T; a.cand = cand;
  a.M = ncand; a.n0 = n1; a.n = n; a.theta = theta; a.g = g; a.theta_loc = nullptr;
  a.start = start; a.nstart = n1; a.r_min = 0.0; a.n_out = nullptr;
  a.method = method; a.precision = precision;
  a.mean = mean; a.s2 = s2; a.var = var; a.idx = idx; a.status = status;
  return select_launch(a, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

int lagp_select_adaptive_dev(const double *X, const double *Z, int64_t N, int32_t p,
                             const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                             int32_t n0, int32_t n, double theta, double g, int32_t precision,
                             double r_min, double *mean, double *s2, double *var, int32_t *idx,
                             int32_t *n_out, int8_t *status, void *workspace,
                             size_t workspace_bytes, void *stream) {
  int st = check_common(N, p, T, n0, n, ncand, theta, g, LAGP_ALC, precision);
  if (st) return st;
  if (n0 < 3 || !(r_min > 1.0) || !isfinite(r_min)) return LAGP_ERR_INVALID_ARG;
  if (T > 0 && (!X || !Z || !XX || !cand || !mean || !s2 || !n_out || !workspace))
    return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  SelectArgs a;
  a.X = X; a.Z = Z; a.N = N; a.p = p; a.XX = XX; a.T = T; a.cand = cand;
  a.M = ncand; a.n0 = n0; a.n = n; a.theta = theta; a.g = g; a.theta_loc = nullptr;
  a.start = nullptr; a.nstart = 0; a.r_min = r_min; a.n_out = n_out;
  a.method = LAGP_ALC; a.precision = precision;
  a.mean = mean; a.s2 = s2; a.var = var; a.idx = idx; a.status = status;
  return select_launch(a, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

int lagp_select_theta_dev(const double *X, const double *Z, int64_t N, int32_t p, const double *XX,
                          int64_t T, const int32_t *cand, int32_t ncand, int32_t n0, int32_t n,
                          const double *theta, double g, int32_t method, int32_t precision,
                          double *mean, double *s2, double *var, int32_t *idx, int8_t *status,
                          void *workspace, size_t workspace_bytes, void *stream) {
  int st = check_common(N, p, T, n0, n, ncand, 1.0, g, method, precision);
  if (st) return st;
  st = check_supported(method, precision);
  if (st) return st;
  if (T > 0 && (!X || !Z || !XX || !cand || !theta || !mean || !s2 || !workspace))
    return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  SelectArgs a;
  a.X = X; a.Z = Z; a.N = N; a.p = p; a.XX = XX; a.T = T; a.cand = cand;
  a.M = ncand; a.n0 = n0; a.n = n; a.theta = 1.0; a.g = g; a.theta_loc = theta;
  a.start = nullptr; a.nstart = 0; a.r_min = 0.0; a.n_out = nullptr;
  a.method = method; a.precision = precision;
  a.mean = mean; a.s2 = s2; a.var = var; a.idx = idx; a.status = status;
  return select_launch(a, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

size_t lagp_mle_workspace_bytes(int64_t T, int32_t n) {
  DevInfo di;
  if (dev_info(&di) || T < 0 || n < 2 || n > kMaxN) return 0;
  return mle_workspace_bytes(T, n, di.num_sms);
}

int lagp_mle_dev(const double *X, const double *Z, int64_t N, int32_t p, int64_t T,
                 const int32_t *idx, int32_t n, double theta0, const double *theta0_loc,
                 double g, double tmin, double tmax, int32_t maxit, double tol,
                 double *theta_out, int32_t *iters, int8_t *status, void *workspace,
                 size_t workspace_bytes, void *stream) {
  if (N < 1 || p < 1 || p > kMaxP || T < 0 || n < 2 || n > kMaxN || !(tmin > 0) ||
      !(tmax > tmin) || maxit < 1 || !(tol > 0) || !(g >= 0) || !(theta0 > 0))
    return LAGP_ERR_INVALID_ARG;
  if (T == 0) return LAGP_OK;
  if (!X || !Z || !idx || !theta_out || !workspace) return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  MleArgs a;
  a.X = X; a.Z = Z; a.p = p; a.T = T; a.idx = idx; a.n = n; a.theta0 = theta0;
  a.theta0_loc = theta0_loc; a.g = g; a.tmin = tmin; a.tmax = tmax; a.tol = tol; a.maxit = maxit;
  a.theta_out = theta_out; a.iters = iters; a.status = status;
  return mle_launch(a, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

size_t lagp_design_predict_workspace_bytes(int64_t T, int32_t n) {
  DevInfo di;
  if (dev_info(&di) || T < 0 || n < 3 || n > kMaxN) return 0;
  return predict_fp64_workspace_bytes(T, n, di.num_sms);
}

int lagp_design_predict_dev(const double *X, const double *Z, int64_t N, int32_t p,
                            const double *XX, int64_t T, const int32_t *idx, int32_t n,
                            double theta, const double *theta_loc, double g, double *mean,
                            double *s2, double *var, int8_t *status, void *workspace,
                            size_t workspace_bytes, void *stream) {
  if (N < 1 || p < 1 || p > kMaxP || T < 0 || n < 3 || n > kMaxN || n > N || !(theta > 0) ||
      !(g >= 0))
    return LAGP_ERR_INVALID_ARG;
  if (T == 0) return LAGP_OK;
  if (!X || !Z || !XX || !idx || !mean || !s2 || !workspace) return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  PredictArgs a;
  a.X = X; a.Z = Z; a.p = p; a.XX = XX; a.T = T; a.n = n; a.nmax = n; a.theta = theta; a.g = g;
  a.idx = idx; a.B = BatchView{nullptr, nullptr, nullptr, 0, theta_loc, nullptr};
  a.mean = mean; a.s2 = s2; a.var = var; a.status = status;
  return predict_fp64_launch(a, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

