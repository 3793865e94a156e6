// knn.cu -- kernel (a): candidate sets of the ncand nearest design points.
//
// Gramacy & Apley, Sec. 3 (the nearest-neighbour sub-design, also the start design
// D_{n0}) and Sec. 6 (every search is restricted to the N' nearest candidates).  For
// each predictive location x the kernel returns the ncand design indices with the
// smallest exact FP64 squared distance, ordered by (d2, index).
//
// One CTA owns one location at a time (grid-stride over locations):
//   pass 1  exact d2 for every design point (fixed dimension order, no FMA), written
//           to the CTA's scratch row, and a 4096-bin histogram of the top 12 bits of
//           float(d2).  Rounding to float is monotone, so bins order the points
//           correctly across bins;
//   select  a block scan of the histogram finds the bin b* holding the ncand-th point;
//   pass 2  points of bins < b* are certainly selected and go to shared memory; the
//           points of b* are resolved exactly: copied too when they fit, otherwise by
//           radix refinement on the 96-bit key (d2 bits, index);
//   sort    bitonic sort of the shared-memory keys by (d2 bits, index); the first
//           ncand indices are written out.
// Non-negative doubles order like their bit patterns, so every exact comparison is an
// integer comparison of (bits, index) and the result is bit-identical to a full sort.
#include <float.h>

#include "internal.h"

namespace lagp {
namespace {

constexpr int KB = 256;               // threads per CTA
constexpr int HBITS = 12;
constexpr int HBINS = 1 << HBITS;     // 4096 histogram bins

__device__ __forceinline__ double sqdist_exact(const double *x, const double *xi, int p) {
  double acc = 0.0;
  for (int k = 0; k < p; k++) {
    double t = __dsub_rn(x[k], xi[k]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

__device__ __forceinline__ uint32_t coarse_bin(double d2) {
  return __float_as_uint(__double2float_rn(d2)) >> (31 - HBITS);
}

__device__ __forceinline__ bool key_less(uint64_t ka, int32_t ia, uint64_t kb, int32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Digit d (0..11, most significant first) of the 96-bit key (bits:64 | index:32).
__device__ __forceinline__ uint32_t key_digit(uint64_t bits, uint32_t idx, int d) {
  return d < 8 ? (uint32_t)(bits >> (56 - 8 * d)) & 0xFFu : (idx >> (24 - 8 * (d - 8))) & 0xFFu;
}

// True if the top 8*nd bits of the key equal the recorded prefix digits.
__device__ __forceinline__ bool key_prefix_eq(uint64_t bits, uint32_t idx, int nd,
                                              const uint32_t *pref) {
  for (int d = 0; d < nd; d++)
    if (key_digit(bits, idx, d) != pref[d]) return false;
  return true;
}

// Exclusive block scan of one value per thread; returns the prefix, *total gets the sum.
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *warp_tmp, uint32_t *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tmp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t s = (lane < KB / 32) ? warp_tmp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < KB / 32) warp_tmp[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  uint32_t base = (w > 0) ? warp_tmp[w - 1] : 0;
  *total = warp_tmp[KB / 32 - 1];
  __syncthreads();
  return base + inc - v;
}

// Find, over hist[0..nbins), the bin where the cumulative count first reaches `rank`
// (1-based); returns the bin and the count strictly below it.  nbins == HBINS or 256.
__device__ void find_rank_bin(const uint32_t *hist, int nbins, uint32_t rank, uint32_t *warp_tmp,
                              int *bin_out, uint32_t *below_out) {
  const int per = nbins / KB > 0 ? nbins / KB : 1;
  const int first = threadIdx.x * per;
  uint32_t part = 0;
  if (first < nbins)
    for (int b = 0; b < per; b++) part += hist[first + b];
  uint32_t total;
  uint32_t pre = block_excl_scan(part, warp_tmp, &total);
  if (first < nbins && pre < rank && rank <= pre + part) {
    uint32_t cum = pre;
    for (int b = 0; b < per; b++) {
      uint32_t h = hist[first + b];
      if (cum + h >= rank) {
        *bin_out = first + b;
        *below_out = cum;
        break;
      }
      cum += h;
    }
  }
  __syncthreads();
}

__device__ void bitonic_sort(uint64_t *key, int32_t *idx, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += KB) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint64_t a = key[i], b = key[ixj];
          int32_t ia = idx[i], ib = idx[ixj];
          bool up = (i & k) == 0;
          bool sw = up ? key_less(b, ib, a, ia) : key_less(a, ia, b, ib);
          if (sw) {
            key[i] = b; key[ixj] = a;
            idx[i] = ib; idx[ixj] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(KB) knn_kernel(const double *__restrict__ X, int64_t N, int p,
                                                 const double *__restrict__ XX, int64_t T, int M,
                                                 int32_t *__restrict__ cand, double *__restrict__ ws,
                                                 int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *skey = reinterpret_cast<uint64_t *>(smem);                 // cap
  int32_t *sidx = reinterpret_cast<int32_t *>(skey + cap);             // cap
  uint32_t *hist = reinterpret_cast<uint32_t *>(sidx + cap);           // HBINS
  __shared__ double xs[kMaxP];
  __shared__ uint32_t warp_tmp[32];
  __shared__ int sh_bin;
  __shared__ uint32_t sh_below, sh_count;
  __shared__ uint32_t pref[12];

  double *D = ws + (size_t)blockIdx.x * (size_t)N;
  for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
    if (threadIdx.x < p) xs[threadIdx.x] = XX[t * p + threadIdx.x];
    for (int b = threadIdx.x; b < HBINS; b += KB) hist[b] = 0;
    if (threadIdx.x == 0) sh_count = 0;
    __syncthreads();
    // pass 1: exact distances and coarse histogram
    for (int64_t i = threadIdx.x; i < N; i += KB) {
      double d2 = sqdist_exact(xs, X + i * p, p);
      D[i] = d2;
      atomicAdd(&hist[coarse_bin(d2)], 1u);
    }
    __syncthreads();
    find_rank_bin(hist, HBINS, (uint32_t)M, warp_tmp, &sh_bin, &sh_below);
    const uint32_t bstar = (uint32_t)sh_bin;
    const uint32_t below = sh_below;
    const uint32_t nb = hist[bstar];
    const bool fits = below + nb <= (uint32_t)cap;
    // pass 2: certain members (and the boundary bin when it fits) into shared memory
    for (int64_t i = threadIdx.x; i < N; i += KB) {
      double d2 = D[i];
      uint32_t b = coarse_bin(d2);
      if (b < bstar || (fits && b == bstar)) {
        uint32_t pos = atomicAdd(&sh_count, 1u);
        skey[pos] = (uint64_t)__double_as_longlong(d2);
        sidx[pos] = (int32_t)i;
      }
    }
    __syncthreads();
    if (!fits) {
      // Boundary bin too large: radix refinement over its members, 8 bits at a time on
      // the 96-bit key.  Members below the selected digit are certain; the loop ends
      // once the remaining tie group fits.  Rare (many equal distances).
      uint32_t need = (uint32_t)M - below;
      uint32_t *h256 = hist;  // reuse
      for (int d = 0; d < 12; d++) {
        for (int b = threadIdx.x; b < 256; b += KB) h256[b] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < N; i += KB) {
          double d2 = D[i];
          if (coarse_bin(d2) != bstar) continue;
          uint64_t bits = (uint64_t)__double_as_longlong(d2);
          if (!key_prefix_eq(bits, (uint32_t)i, d, pref)) continue;
          atomicAdd(&h256[key_digit(bits, (uint32_t)i, d)], 1u);
        }
        __syncthreads();
        const uint32_t cnt0 = sh_count;  // stable here: no thread appends until after the scan
        find_rank_bin(h256, 256, need, warp_tmp, &sh_bin, &sh_below);
        const uint32_t dd = (uint32_t)sh_bin, dbelow = sh_below, deq = h256[dd];
        const bool last = cnt0 + dbelow + deq <= (uint32_t)cap;
        for (int64_t i = threadIdx.x; i < N; i += KB) {
          double d2 = D[i];
          if (coarse_bin(d2) != bstar) continue;
          uint64_t bits = (uint64_t)__double_as_longlong(d2);
          if (!key_prefix_eq(bits, (uint32_t)i, d, pref)) continue;
          uint32_t dg = key_digit(bits, (uint32_t)i, d);
          if (dg < dd || (last && dg == dd)) {
            uint32_t pos = atomicAdd(&sh_count, 1u);
            skey[pos] = bits;
            sidx[pos] = (int32_t)i;
          }
        }
        __syncthreads();
        if (last) break;
        need -= dbelow;
        if (threadIdx.x == 0) pref[d] = dd;
        __syncthreads();
      }
    }
    const int cnt = (int)sh_count;
    int n2 = 1;
    while (n2 < cnt) n2 <<= 1;
    for (int i = cnt + threadIdx.x; i < n2; i += KB) {
      skey[i] = ~0ull;
      sidx[i] = 0x7fffffff;
    }
    __syncthreads();
    bitonic_sort(skey, sidx, n2);
    for (int r = threadIdx.x; r < M; r += KB) cand[t * M + r] = sidx[r];
    __syncthreads();
  }
}

int knn_cap(int M) {
  int cap = 2048;
  while (cap < 2 * M && cap < 16384) cap <<= 1;
  return cap;
}

size_t knn_smem_bytes(int cap) { return (size_t)cap * (8 + 4) + HBINS * 4; }

int knn_grid(int64_t T, int num_sms) {
  int64_t g = (int64_t)num_sms * 2;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

}  // namespace

size_t knn_workspace_bytes(int64_t N, int64_t T, int32_t ncand, int num_sms) {
  (void)ncand;
  return align_up((size_t)knn_grid(T, num_sms) * (size_t)N * sizeof(double), 256);
}

int knn_launch(const double *X, int64_t N, int32_t p, const double *XX, int64_t T, int32_t ncand,
               int32_t *cand, void *ws, size_t ws_bytes, cudaStream_t stream) {
  if (T == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  if (ws_bytes < knn_workspace_bytes(N, T, ncand, di.num_sms)) return LAGP_ERR_INVALID_ARG;
  const int cap = knn_cap(ncand);
  const size_t smem = knn_smem_bytes(cap);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  cudaError_t e = cudaFuncSetAttribute(knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  const int grid = knn_grid(T, di.num_sms);
  knn_kernel<<<grid, KB, smem, stream>>>(X, N, p, XX, T, ncand, cand, static_cast<double *>(ws),
                                         cap);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

}  // namespace lagp
