// fp64_exp.cu -- constants of the table-driven exponential (see fp64_exp.cuh) and a
// device-buffer entry point that evaluates it, so it can be checked against CUDA's exp.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fp64_exp.cuh"
#include "internal.h"

namespace lagp {

namespace {

void compute_host_consts(ExpConsts *c) {
  const long double ln2 = logl(2.0L);
  for (int j = 0; j < 64; j++) c->tab[j] = (double)exp2l((long double)j / 64.0L);
  const long double c64 = ln2 / 64.0L;
  double hi = (double)c64;
  uint64_t b;
  memcpy(&b, &hi, sizeof b);
  b &= ~((1ull << 23) - 1);  // keep 30 significant bits
  memcpy(&hi, &b, sizeof b);
  c->ln2_64_hi = hi;
  c->ln2_64_lo = (double)(c64 - (long double)hi);
  c->inv_ln2_64 = (double)(64.0L / ln2);
  for (int j = 0; j < 64; j++) {
    const long double v = exp2l((long double)j / 64.0L);
    const float h = (float)v;
    c->tabf_h[j] = h;
    c->tabf_l[j] = (float)(v - (long double)h);
  }
  float c1 = (float)c64;
  uint32_t u;
  memcpy(&u, &c1, sizeof u);
  u &= ~((1u << 13) - 1);  // 11 significant bits
  memcpy(&c1, &u, sizeof u);
  const float c2 = (float)(c64 - (long double)c1);
  const float c3 = (float)(c64 - (long double)c1 - (long double)c2);
  c->c1 = c1;
  c->c2 = c2;
  c->c3 = c3;
  c->inv_ln2_64f = (float)(64.0L / ln2);
}

__global__ void exp_eval_kernel(const double *__restrict__ x, double *__restrict__ y, int64_t n) {
  __shared__ double tab[64];
  if (threadIdx.x < 64) tab[threadIdx.x] = c_exp.tab[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = exp_nonpos(x[i], tab);
}

}  // namespace

const ExpConsts *exp_host_consts() {
  static std::once_flag once;
  static ExpConsts consts;
  std::call_once(once, [] { compute_host_consts(&consts); });
  return &consts;
}

}  // namespace lagp

extern "C" int lagp_exp_dev(const double *x, double *y, int64_t n, void *stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return LAGP_ERR_INVALID_ARG;
  if (n == 0) return LAGP_OK;
  int st = lagp::exp_table_upload();
  if (st) return st;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  lagp::exp_eval_kernel<<<(int)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  lagp::g_launches.fetch_add(1);
  return lagp::cuda_status(cudaGetLastError());
}
