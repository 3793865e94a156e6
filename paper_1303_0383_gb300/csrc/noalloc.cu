// noalloc.cu -- lagp_select_dev_noalloc: the greedy-design kernels (b)+(c) with their
// scratch in a static device array, for callers that must not allocate device memory.
//
// The array below is defined once per process and exists on every device that loads
// the library until the process exits.  Host code cannot use its name as a device
// address, so the first call in each CUDA context looks the address up with
// cudaGetSymbolAddress while that device is current, checks the result, and caches it
// for that context (after a cudaDeviceReset the device's next context looks it up again).
// Every call reuses the same bytes: the launcher clears the work counter it needs at
// zero, and two calls whose kernels overlap on the GPU would corrupt each other.
#include <mutex>

#include "internal.h"

namespace lagp {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LAGP_NOALLOC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void *g_scratch_ptr[64];
unsigned long long g_scratch_ctx[64];  // the context the cached address belongs to

// Device address of g_noalloc_scratch on the current device (looked up once per context).
int noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= 64) return LAGP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  unsigned long long id = 0;
  int st = current_context_id(&id);
  if (st) return st;
  if (id == 0 || g_scratch_ctx[dev] != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_status(e != cudaSuccess ? e : cudaErrorUnknown);
    st = current_context_id(&id);  // the lookup made the context current if there was none
    if (st) return st;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = id;
  }
  *out = g_scratch_ptr[dev];
  return LAGP_OK;
}

}  // namespace
}  // namespace lagp

using namespace lagp;

extern "C" int lagp_select_dev_noalloc(const double *X, const double *Z, int64_t N, int32_t p,
                                       const double *XX, int64_t T, const int32_t *cand,
                                       int32_t ncand, int32_t n0, int32_t n, double theta,
                                       double g, int32_t method, int32_t precision, double *mean,
                                       double *s2, double *var, int32_t *idx, int8_t *status,
                                       void *stream) {
  int st = check_common(N, p, T, n0, n, ncand, theta, g, method, precision);
  if (st) return st;
  st = check_supported(method, precision);
  if (st) return st;
  if (method == LAGP_MSPE || (precision != LAGP_FP64 && method != LAGP_NN)) return LAGP_ERR_UNSUPPORTED;
  if (T == 0) return LAGP_OK;
  if (!X || !Z || !XX || !cand || !mean || !s2) return LAGP_ERR_INVALID_ARG;
  const size_t cap = LAGP_NOALLOC_SCRATCH_BYTES;
  if (select_scratch_bytes_for_grid(1, p, n, ncand) > cap) return LAGP_ERR_SCRATCH_LIMIT;
  DevInfo di;
  st = dev_info(&di);
  if (st) return st;
  // As many CTAs as fit in the array, at most the grid the workspace entry point uses.
  int G = select_default_grid(T, di.num_sms);
  while (G > 1 && select_scratch_bytes_for_grid(G, p, n, ncand) > cap) G--;
  void *scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st) return st;
  SelectArgs a;
  a.X = X; a.Z = Z; a.N = N; a.p = p; a.XX = XX; a.T = T; a.cand = cand;
  a.M = ncand; a.n0 = n0; a.n = n; a.theta = theta; a.g = g; a.theta_loc = nullptr;
  a.start = nullptr; a.nstart = 0; a.r_min = 0.0; a.n_out = nullptr;
  a.method = method; a.precision = precision;
  a.mean = mean; a.s2 = s2; a.var = var; a.idx = idx; a.status = status;
  return select_launch_on_grid(a, scratch, cap, G, static_cast<cudaStream_t>(stream));
}
