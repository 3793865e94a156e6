// knn.cu -- kernel (a): candidate sets of the ncand nearest design points.
//
// Gramacy & Apley, Sec. 3 (the nearest-neighbour sub-design, also the start design
// D_{n0}) and Sec. 6 (every search is restricted to the N' nearest candidates).  For
// each predictive location x the kernel returns the ncand design indices with the
// smallest exact FP64 squared distance, ordered by (d2, index).
//
// FP64 is 1/58 of FP32 throughput on this GPU, so exact distances are computed only for
// the few points that can be members.  One CTA owns one location at a time:
//   prep    (once per call) an FP32 copy of X, dimension-major (a warp's load of one
//           coordinate of 32 consecutive points is one 128-byte line), and
//           B = max |coordinate|;
//   pass 1  FP32 squared distance d2f of every design point and a 4096-bin histogram of
//           the top 12 bits of d2f (non-negative floats order like their bit patterns);
//   select  a block scan finds the bin b* holding the ncand-th smallest d2f; tau is the
//           upper edge of b*;
//   pass 2  d2f recomputed (bit-identical); every point with d2f <= tau + 2E survives, where
//           E bounds |d2f - d2| (FP32 rounding of the coordinates, the differences and the
//           fused sum; see fp32_err_bound) -- all true members survive; the survivors are
//           listed in shared memory and then get their exact FP64 d2 from that list, so
//           the FP64 work runs on full warps;
//   sort    the survivors in (d2, index) order: a bucket sort on d2 with insertion in the
//           buckets, or a bitonic sort on (d2 bits, index) where buckets overflow; the
//           first ncand indices are written out.
// If the survivors do not fit in shared memory (many points tied at the boundary), the
// CTA redoes that location exactly in FP64: a 4096-bin histogram of float(d2) over exact
// d2 (recomputed in every pass: no scratch), and radix refinement on the 96-bit key (d2 bits, index) for an
// oversized boundary bin.  Either way the result is bit-identical to a full sort.
#include <float.h>

#include "batch.cuh"
#include "check.cuh"
#include "internal.h"

namespace lagp {
namespace {

constexpr int KB = 256;               // threads per CTA
constexpr int HBITS = 12;
constexpr int KS = 16;                // the sample that bounds the M-th distance: one block of
                                      // 32 consecutive design points in every KS blocks
constexpr int HBINS = 1 << HBITS;     // 4096 histogram bins
// The bucket sort's permutation gets cap entries of its own where they fit in shared
// memory next to the keys (cap <= 8192); otherwise it uses the histogram's second half
// (HBINS / 2 entries) and larger survivor sets take the bitonic sort.
__host__ __device__ constexpr bool knn_own_perm(int cap) { return cap > HBINS / 2 && cap <= 8192; }


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

// Keys are (d2 bits, index) compared as three 32-bit words (hi, lo, index): non-negative
// doubles order like their bit patterns.
__device__ __forceinline__ bool key_less3(uint32_t ah, uint32_t al, int32_t ai, uint32_t bh,
                                          uint32_t bl, int32_t bi) {
  return ah < bh || (ah == bh && (al < bl || (al == bl && ai < bi)));
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
  const int per = nbins / KB > 0 ? nbins / KB : 1;  // a power of two
  const int first = threadIdx.x * per;
  uint32_t part = 0;
  // each thread's range starts at its own rotation: the lanes of a warp read different
  // banks instead of all `per` apart (a per-way bank conflict)
  if (first < nbins)
    for (int b = 0; b < per; b++) part += hist[first + ((b + threadIdx.x) & (per - 1))];
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

// Bitonic sort of n2 (a power of two) keys held as (hi, lo, index) words in shared memory;
// each stage visits exactly its n2/2 compare-exchange pairs.
__device__ void bitonic_sort(uint32_t *kh, uint32_t *kl, int32_t *idx, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int lj = __ffs(j) - 1;
      for (int pp = threadIdx.x; pp < (n2 >> 1); pp += KB) {
        const int i = ((pp >> lj) << (lj + 1)) | (pp & (j - 1));
        const int ixj = i + j;
        const uint32_t ah = kh[i], al = kl[i], bh = kh[ixj], bl = kl[ixj];
        const int32_t ai = idx[i], bi = idx[ixj];
        const bool up = (i & k) == 0;
        const bool sw = up ? key_less3(bh, bl, bi, ah, al, ai) : key_less3(ah, al, ai, bh, bl, bi);
        if (sw) {
          kh[i] = bh; kl[i] = bl; idx[i] = bi;
          kh[ixj] = ah; kl[ixj] = al; idx[ixj] = ai;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void put_key(uint32_t *kh, uint32_t *kl, int32_t *sidx, uint32_t pos,
                                        double d2, int32_t i) {
  const uint64_t b = (uint64_t)__double_as_longlong(d2);
  kh[pos] = (uint32_t)(b >> 32);
  kl[pos] = (uint32_t)b;
  sidx[pos] = i;
}

// Bound on |d2f - d2| for a squared distance d2 <= d computed in FP32 from coordinates
// of magnitude <= B (u = 2^-24): rounding the coordinates and each difference gives
// |diff_f - diff| <= 2uB + u|diff|, squaring and the p fused additions add (2+p)u d2;
// summed over k with sum |diff_k| <= sqrt(p d2).  Constants doubled for safety.
__device__ __forceinline__ double fp32_err_bound(double d, double B, int p) {
  const double u = 5.9604644775390625e-08;  // 2^-24
  return 8.0 * u * B * sqrt((double)p * d) + (4.0 + 2.0 * p) * u * d + 16.0 * p * u * u * B * B;
}

// Exact path for one location (the fallback when many points tie at the boundary):
// exact FP64 d2 of every point (recomputed in each pass, no scratch), coarse histogram of
// float(d2), boundary resolution by radix refinement; keys into shared memory; returns
// the count.
__device__ int knn_exact_location(const double *__restrict__ X, int N, int p, int M,
                                  const double *xs, uint32_t *kh, uint32_t *kl, int32_t *sidx,
                                  uint32_t *hist, int cap, uint32_t *warp_tmp, int *sh_bin,
                                  uint32_t *sh_below, uint32_t *sh_count, uint32_t *pref) {
  for (int b = threadIdx.x; b < HBINS; b += KB) hist[b] = 0;
  if (threadIdx.x == 0) *sh_count = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += KB)
    atomicAdd(&hist[coarse_bin(sqdist_exact(xs, X + (size_t)i * p, p))], 1u);
  __syncthreads();
  find_rank_bin(hist, HBINS, (uint32_t)M, warp_tmp, sh_bin, sh_below);
  const uint32_t bstar = (uint32_t)*sh_bin;
  const uint32_t below = *sh_below;
  const uint32_t nb = hist[bstar];
  const bool fits = below + nb <= (uint32_t)cap;
  for (int i = threadIdx.x; i < N; i += KB) {
    const double d2 = sqdist_exact(xs, X + (size_t)i * p, p);
    const uint32_t b = coarse_bin(d2);
    if (b < bstar || (fits && b == bstar)) put_key(kh, kl, sidx, atomicAdd(sh_count, 1u), d2, i);
  }
  __syncthreads();
  if (!fits) {
    uint32_t need = (uint32_t)M - below;
    uint32_t *h256 = hist;
    for (int d = 0; d < 12; d++) {
      for (int b = threadIdx.x; b < 256; b += KB) h256[b] = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += KB) {
        const double d2 = sqdist_exact(xs, X + (size_t)i * p, p);
        if (coarse_bin(d2) != bstar) continue;
        const uint64_t bits = (uint64_t)__double_as_longlong(d2);
        if (!key_prefix_eq(bits, (uint32_t)i, d, pref)) continue;
        atomicAdd(&h256[key_digit(bits, (uint32_t)i, d)], 1u);
      }
      __syncthreads();
      const uint32_t cnt0 = *sh_count;  // stable here: no thread appends until after the scan
      find_rank_bin(h256, 256, need, warp_tmp, sh_bin, sh_below);
      const uint32_t dd = (uint32_t)*sh_bin, dbelow = *sh_below, deq = h256[dd];
      const bool last = cnt0 + dbelow + deq <= (uint32_t)cap;
      for (int i = threadIdx.x; i < N; i += KB) {
        const double d2 = sqdist_exact(xs, X + (size_t)i * p, p);
        if (coarse_bin(d2) != bstar) continue;
        const uint64_t bits = (uint64_t)__double_as_longlong(d2);
        if (!key_prefix_eq(bits, (uint32_t)i, d, pref)) continue;
        const uint32_t dg = key_digit(bits, (uint32_t)i, d);
        if (dg < dd || (last && dg == dd)) put_key(kh, kl, sidx, atomicAdd(sh_count, 1u), d2, i);
      }
      __syncthreads();
      if (last) break;
      need -= dbelow;
      if (threadIdx.x == 0) pref[d] = dd;
      __syncthreads();
    }
  }
  return (int)*sh_count;
}

// The FP32 copy of X (N x p, row-major) in dimension-major order, and B = max |coordinate|.
__global__ void knn_prep_kernel(const double *__restrict__ X, int64_t N, int p,
                                float *__restrict__ Xf, unsigned int *__restrict__ bmax) {
  __shared__ unsigned int wmax[KB / 32];
  unsigned int m = 0;
  const int64_t n = N * p;
  for (int64_t i = blockIdx.x * (int64_t)KB + threadIdx.x; i < n; i += (int64_t)gridDim.x * KB) {
    const double x = X[i];
    Xf[(i % p) * N + i / p] = __double2float_rn(x);
    const float a = __double2float_ru(fabs(x));
    m = max(m, __float_as_uint(a));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < KB / 32; w++) m = max(m, wmax[w]);
    atomicMax(bmax, m);
  }
}

// FP32 d2 of point i; Xf is dimension-major (coordinate k of point i at Xf[k N + i]), so a
// warp's load of one coordinate is one contiguous 128-byte line.
template <int P>
__device__ __forceinline__ float sqdist_f32(const float *xf, const float *__restrict__ Xf, int i,
                                            int N, int p) {
  float acc = 0.0f;
  if (P > 0) {
#pragma unroll
    for (int k = 0; k < P; k++) {
      const float dk = __fsub_rn(xf[k], Xf[(size_t)k * N + i]);
      acc = __fmaf_rn(dk, dk, acc);
    }
  } else {
    for (int k = 0; k < p; k++) {
      const float dk = __fsub_rn(xf[k], Xf[(size_t)k * N + i]);
      acc = __fmaf_rn(dk, dk, acc);
    }
  }
  return acc;
}

// Visits the points i = first, first + stride, ... < N: the FP32 distances of KU points are
// formed -- their loads in flight together -- before f(d2f, i) uses any of them (one point
// at a time, each pass was bound by the L2 latency of its dependent loads).
constexpr int KU = 4;
template <int P, typename F>
__device__ __forceinline__ void each_point(const float *xf, const float *__restrict__ Xf, int N,
                                           int p, int first, int stride, F f) {
  int i = first;
  for (; i + (KU - 1) * stride < N; i += KU * stride) {
    float d[KU];
#pragma unroll
    for (int u = 0; u < KU; u++) d[u] = sqdist_f32<P>(xf, Xf, i + u * stride, N, p);
#pragma unroll
    for (int u = 0; u < KU; u++) f(d[u], i + u * stride);
  }
  for (; i < N; i += stride) f(sqdist_f32<P>(xf, Xf, i, N, p), i);
}

constexpr int BUCKET_CAP = 32; // largest bucket sorted in place; beyond, the bitonic sort

// Rank order of the cnt survivors (keys (d2 hi, d2 lo, index) in kh/kl/sidx) by a bucket
// sort: floor(d2 (nb - 1) / max d2) is monotone in d2, so buckets in index order hold
// increasing distances; each bucket is then put in exact key order by insertion (buckets
// hold a few survivors on average).  Writes the first M indices to out and returns true;
// returns false (nothing written) when a bucket holds more than BUCKET_CAP survivors
// (many equal distances), leaving the keys for the bitonic sort.  The bucket bounds use
// hist[0, nb); the permutation goes to perm (cnt entries), which may be hist + nb.
// Every thread returns after the same barriers.
__device__ bool bucket_order(const uint32_t *kh, const uint32_t *kl, const int32_t *sidx, int cnt,
                             int M, uint32_t *hist, int nb, uint32_t *perm, uint32_t *warp_tmp,
                             uint32_t *sh_flag, unsigned long long *sh_dmax, int32_t *out) {
  uint32_t *bound = hist;
  if (threadIdx.x == 0) {
    *sh_dmax = 0ull;
    *sh_flag = 0u;
  }
  for (int b = threadIdx.x; b < nb; b += KB) bound[b] = 0;
  // the largest key (non-negative doubles order like their bits): a warp maximum, then one
  // shared atomic per warp
  unsigned long long wmax = 0ull;
  for (int r = threadIdx.x; r < cnt; r += KB) {
    const unsigned long long k = ((unsigned long long)kh[r] << 32) | kl[r];
    wmax = k > wmax ? k : wmax;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, wmax, o);
    wmax = w > wmax ? w : wmax;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && wmax) atomicMax(sh_dmax, wmax);
  __syncthreads();
  // buckets from FP32: float(d2) is non-decreasing in d2 and so is its product with a
  // positive scale and the truncation, so bucket order is distance order (equal floats
  // share a bucket, which the insertion below orders by the exact key)
  const float dmax = __double2float_ru(__longlong_as_double((long long)*sh_dmax));
  if (!(dmax > 0.0f)) return false;
  const float scale = (float)(nb - 1) / dmax;
  auto bucket_of = [&](int r) {
    const float d2 = __double2float_rn(
        __longlong_as_double((long long)(((unsigned long long)kh[r] << 32) | kl[r])));
    const int b = (int)(d2 * scale);
    return b < nb - 1 ? b : nb - 1;
  };
  for (int r = threadIdx.x; r < cnt; r += KB) atomicAdd(&bound[bucket_of(r)], 1u);
  __syncthreads();
  // exclusive scan of the counts (nb / KB buckets per thread), flagging an oversized bucket
  const int per = nb / KB;  // a power of two
  uint32_t part = 0;
  for (int k = 0; k < per; k++) {  // rotated start per thread: no bank conflicts
    const uint32_t c = bound[threadIdx.x * per + ((k + threadIdx.x) & (per - 1))];
    part += c;
    if (c > BUCKET_CAP) *sh_flag = 1u;
  }
  uint32_t total;
  uint32_t run = block_excl_scan(part, warp_tmp, &total);
  for (int k = 0; k < per; k++) {
    const uint32_t c = bound[threadIdx.x * per + k];
    bound[threadIdx.x * per + k] = run;
    run += c;
  }
  __syncthreads();
  if (*sh_flag) return false;
  // scatter: afterwards bound[b] is the end of bucket b (= the start of bucket b + 1)
  for (int r = threadIdx.x; r < cnt; r += KB) {
    const uint32_t at = atomicAdd(&bound[bucket_of(r)], 1u);
    if (LAGP_CHK(at, cnt, 3)) perm[at] = r;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += KB) {
    const uint32_t lo = b ? bound[b - 1] : 0u, hi = bound[b];
    for (uint32_t i = lo + 1; i < hi; i++) {  // insertion by the exact key
      const uint32_t v = perm[i];
      uint32_t k = i;
      while (k > lo) {
        const uint32_t u = perm[k - 1];
        if (!key_less3(kh[v], kl[v], sidx[v], kh[u], kl[u], sidx[u])) break;
        perm[k] = u;
        k--;
      }
      perm[k] = v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < M; r += KB) {
    const uint32_t pr = perm[r];
    out[r] = LAGP_CHK(pr, cnt, 4) ? sidx[pr] : -1;
  }
  return true;
}

// P > 0: the dimension is a compile-time constant; P == 0: runtime p.
// Batched launches pass `list` (launch position -> location), `locs` (each location's
// candidate count and output offset) and the row stride of XX; uniform launches pass
// nullptr and use M, t*M and t*p.
template <int P>
__global__ void __launch_bounds__(KB, 4) knn_kernel(const double *__restrict__ X, int N, int p,
                                                 const double *__restrict__ XX, int64_t T, int M,
                                                 int32_t *__restrict__ cand,
                                                 const float *__restrict__ Xf,
                                                 const unsigned int *__restrict__ bmax, int cap,
                                                 const int32_t *__restrict__ list,
                                                 const LocDesc *__restrict__ locs, int ldxx) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *kh = reinterpret_cast<uint32_t *>(smem);   // cap
  uint32_t *kl = kh + cap;                              // cap
  int32_t *sidx = reinterpret_cast<int32_t *>(kl + cap);  // cap
  uint32_t *hist = reinterpret_cast<uint32_t *>(sidx + cap);  // HBINS
  // the bucket sort's permutation: the histogram's second half, or its own cap entries
  const bool own_perm = knn_own_perm(cap);
  uint32_t *perm = own_perm ? hist + HBINS : hist + HBINS / 2;
  const int nb = own_perm ? HBINS : HBINS / 2;
  const int perm_cap = own_perm ? cap : HBINS / 2;
  __shared__ double xs[kMaxP];
  __shared__ float xf[kMaxP];
  __shared__ uint32_t warp_tmp[32];
  __shared__ int sh_bin;
  __shared__ uint32_t sh_below, sh_count;
  __shared__ uint32_t pref[12];
  __shared__ float sh_thr;
  __shared__ unsigned long long sh_dmax;
  if (P > 0) p = P;

  const double Bx = (double)__uint_as_float(*bmax);
  const int Mu = M;
  for (int64_t tt = blockIdx.x; tt < T; tt += gridDim.x) {
    const int64_t t = list ? list[tt] : tt;
    int32_t *out = cand + (locs ? locs[t].cand_off : t * Mu);
    M = locs ? locs[t].M : Mu;
    if (threadIdx.x < p) {
      xs[threadIdx.x] = XX[t * (locs ? ldxx : p) + threadIdx.x];
      xf[threadIdx.x] = __double2float_rn(xs[threadIdx.x]);
    }
    for (int b = threadIdx.x; b < HBINS; b += KB) hist[b] = 0;
    if (threadIdx.x == 0) sh_count = 0;
    __syncthreads();
    // The screen's threshold thr = tau + 2E: tau the upper edge of the bin holding the M-th
    // smallest d2f in `hist` (complete up to that bin), E the FP32 error bound.
    auto set_threshold = [&]() {
      find_rank_bin(hist, HBINS, (uint32_t)M, warp_tmp, &sh_bin, &sh_below);
      if (threadIdx.x == 0) {
        double B = Bx;
        for (int k = 0; k < p; k++) B = fmax(B, fabs(xs[k]));
        const double tau = (double)__uint_as_float(((uint32_t)sh_bin + 1u) << (31 - HBITS));
        const double E0 = fp32_err_bound(tau, B, p);
        const double E = fp32_err_bound(tau + 2.0 * E0, B, p);
        sh_thr = __double2float_ru(tau + 2.0 * E);
      }
      __syncthreads();
    };
    int cnt = 0;
    bool listed = false;
    // pass 0: a sample of the design -- 32 consecutive points (one coalesced warp load per
    // coordinate) out of every 32 KS, spread over any ordering of X -- bounds the M-th
    // smallest d2f from above: bound = the upper edge of the bin holding the sample's
    // ceil(1.5 M ns / N)-th smallest, about 1.5 M points of the whole design
    const int ns = (N / (32 * KS)) * 32 + min(32, N % (32 * KS));
    const int ks = (int)(((int64_t)3 * M * ns + 2 * (int64_t)N - 1) / (2 * (int64_t)N));
    if (ks < ns) {
      each_point<P>(xf, Xf, N, p, (threadIdx.x >> 5) * 32 * KS + (threadIdx.x & 31),
                    (KB / 32) * 32 * KS, [&](float d2f, int) {
        atomicAdd(&hist[__float_as_uint(d2f) >> (31 - HBITS)], 1u);
      });
      __syncthreads();
      find_rank_bin(hist, HBINS, (uint32_t)ks, warp_tmp, &sh_bin, &sh_below);
      const float bound = __uint_as_float(((uint32_t)sh_bin + 1u) << (31 - HBITS));
      for (int b = threadIdx.x; b < HBINS; b += KB) hist[b] = 0;
      __syncthreads();
      // pass 1: the points with d2f <= bound are listed (d2f bits, index) and histogrammed;
      // the list's histogram is the whole design's in every bin up to the M-th's
      each_point<P>(xf, Xf, N, p, threadIdx.x, KB, [&](float d2f, int i) {
        if (d2f <= bound) {
          const uint32_t pos = atomicAdd(&sh_count, 1u);
          if (pos < (uint32_t)cap) {
            kh[pos] = __float_as_uint(d2f);
            kl[pos] = (uint32_t)i;
          }
          atomicAdd(&hist[__float_as_uint(d2f) >> (31 - HBITS)], 1u);
        }
      });
      __syncthreads();
      const uint32_t nl = sh_count;
      if (nl >= (uint32_t)M && nl <= (uint32_t)cap) {
        set_threshold();
        const float thr = sh_thr;
        if (thr <= bound) {  // every point with d2f <= thr is in the list: keep those
          listed = true;
          __syncthreads();
          if (threadIdx.x == 0) sh_count = 0;
          __syncthreads();
          // warp-aggregated appends: one shared atomic per warp and pass
          for (int r0 = threadIdx.x & ~31; r0 < (int)nl; r0 += KB) {
            const int r = r0 + (threadIdx.x & 31);
            const bool keep = r < (int)nl && __uint_as_float(kh[r]) <= thr;
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            uint32_t base = 0;
            if ((threadIdx.x & 31) == 0 && ball) base = atomicAdd(&sh_count, (uint32_t)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            const uint32_t at = base + __popc(ball & ((1u << (threadIdx.x & 31)) - 1u));
            if (keep && LAGP_CHK(at, cap, 1)) sidx[at] = (int32_t)kl[r];
          }
          __syncthreads();
          cnt = (int)sh_count;
        }
      }
      if (!listed) {  // the sample's bound missed (rare): the two full passes below
        __syncthreads();
        for (int b = threadIdx.x; b < HBINS; b += KB) hist[b] = 0;
        if (threadIdx.x == 0) sh_count = 0;
        __syncthreads();
      }
    }
    if (!listed) {
      // pass 1: histogram of the FP32 distances of every point
      each_point<P>(xf, Xf, N, p, threadIdx.x, KB, [&](float d2f, int) {
        atomicAdd(&hist[__float_as_uint(d2f) >> (31 - HBITS)], 1u);
      });
      __syncthreads();
      set_threshold();
      const float thr = sh_thr;
      // pass 2: the same FP32 distances again (bit for bit); survivors are listed first
      each_point<P>(xf, Xf, N, p, threadIdx.x, KB, [&](float d2f, int i) {
        if (d2f <= thr) {
          const uint32_t pos = atomicAdd(&sh_count, 1u);
          if (pos < (uint32_t)cap) sidx[pos] = i;
        }
      });
      __syncthreads();
      cnt = (int)sh_count;
    }
    // then get their exact FP64 distances from the compacted list: a warp instruction of
    // the FP64 pipe serves 32 survivors instead of the few a strided pass would hold
    if (cnt <= cap)
      for (int r = threadIdx.x; r < cnt; r += KB) {
        const int32_t i = sidx[r];
        if (LAGP_CHK(i, N, 2)) put_key(kh, kl, sidx, (uint32_t)r, sqdist_exact(xs, X + (size_t)i * p, p), i);
      }
    __syncthreads();
    if (cnt > cap || cnt < M)  // too many ties at the boundary (or, defensively, too few)
      cnt = knn_exact_location(X, N, p, M, xs, kh, kl, sidx, hist, cap, warp_tmp, &sh_bin,
                               &sh_below, &sh_count, pref);
    if (cnt > cap || cnt > perm_cap ||
        !bucket_order(kh, kl, sidx, cnt, M, hist, nb, perm, warp_tmp, &sh_count,
                                   &sh_dmax, out)) {
      int n2 = 1;
      while (n2 < cnt) n2 <<= 1;
      for (int i = cnt + threadIdx.x; i < n2; i += KB) {
        kh[i] = 0xffffffffu;
        kl[i] = 0xffffffffu;
        sidx[i] = 0x7fffffff;
      }
      __syncthreads();
      bitonic_sort(kh, kl, sidx, n2);
      for (int r = threadIdx.x; r < M; r += KB) {
        const int32_t v = sidx[r];
        out[r] = LAGP_CHK(v, N, 5) ? v : -1;
      }
    }
    __syncthreads();
  }
}

int knn_cap(int M) {
  int cap = 2048;
  while (cap < 2 * M && cap < 16384) cap <<= 1;
  return cap;
}

size_t knn_smem_bytes(int cap) {
  return (size_t)cap * (4 + 4 + 4) + HBINS * 4 + (knn_own_perm(cap) ? (size_t)cap * 4 : 0);
}

int knn_grid(int64_t T, int num_sms, size_t smem) {
  int per_sm = (int)(200000 / (smem + 1024));  // leave room, at most 8 CTAs of 256 threads
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  const int64_t g = (int64_t)num_sms * per_sm;
  return (int)(T < g ? (T > 0 ? T : 1) : g);
}

}  // namespace

int knn_check_take(CheckRec *out) { return check_take_here(out); }

// Scratch layout: [bmax (256 B)] [Xf: p x N floats, dimension-major]
size_t knn_workspace_bytes(int64_t N, int64_t T, int32_t ncand, int num_sms) {
  (void)T;
  (void)ncand;
  (void)num_sms;
  return 256 + align_up((size_t)N * kMaxP * sizeof(float), 256);
}

// Launch kernel (a) over nloc locations of one design.  Uniform launches: list == nullptr,
// locs == nullptr, candidate count M.  Batched: the design's locations in list, their
// counts and offsets in locs (M is then the largest count, which sizes shared memory).
int knn_launch_list(const double *X, int64_t N, int32_t p, const double *XX, int64_t nloc,
                    int32_t M, int32_t *cand, void *ws, size_t ws_bytes, cudaStream_t stream,
                    const int32_t *list, const LocDesc *locs, int ldxx, int ctas_per_sm) {
  if (nloc == 0) return LAGP_OK;
  DevInfo di;
  int st = dev_info(&di);
  if (st) return st;
  if (ws_bytes < knn_workspace_bytes(N, nloc, M, di.num_sms)) return LAGP_ERR_INVALID_ARG;
  const int cap = knn_cap(M);
  const size_t smem = knn_smem_bytes(cap);
  if (smem > di.smem_optin) return LAGP_ERR_INVALID_ARG;
  const void *fn;
  switch (p) {
    case 1: fn = (const void *)knn_kernel<1>; break;
    case 2: fn = (const void *)knn_kernel<2>; break;
    case 3: fn = (const void *)knn_kernel<3>; break;
    case 4: fn = (const void *)knn_kernel<4>; break;
    case 8: fn = (const void *)knn_kernel<8>; break;
    default: fn = (const void *)knn_kernel<0>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);
  int grid = knn_grid(nloc, di.num_sms, smem);
  if (ctas_per_sm > 0) {
    const int64_t g2 = (int64_t)di.num_sms * ctas_per_sm;
    grid = (int)(nloc < g2 ? nloc : g2);
  }
  char *w = static_cast<char *>(ws);
  unsigned int *bmax = reinterpret_cast<unsigned int *>(w);
  float *Xf = reinterpret_cast<float *>(w + 256);
  e = cudaMemsetAsync(bmax, 0, sizeof(unsigned int), stream);
  if (e != cudaSuccess) return cuda_status(e);
  const int64_t n = N * p;
  int pblocks = (int)((n + KB - 1) / KB);
  if (pblocks > 4 * di.num_sms) pblocks = 4 * di.num_sms;
  knn_prep_kernel<<<pblocks, KB, 0, stream>>>(X, N, p, Xf, bmax);
  g_launches.fetch_add(1);
  const int Ni = (int)N;
  void *args[] = {(void *)&X, (void *)&Ni, (void *)&p, (void *)&XX, (void *)&nloc, (void *)&M,
                  (void *)&cand, (void *)&Xf, (void *)&bmax, (void *)&cap, (void *)&list,
                  (void *)&locs, (void *)&ldxx};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(KB), args, smem, stream);
  if (e != cudaSuccess) return cuda_status(e);
  g_launches.fetch_add(1);
  return cuda_status(cudaGetLastError());
}

int knn_launch(const double *X, int64_t N, int32_t p, const double *XX, int64_t T, int32_t ncand,
               int32_t *cand, void *ws, size_t ws_bytes, cudaStream_t stream) {
  return knn_launch_list(X, N, p, XX, T, ncand, cand, ws, ws_bytes, stream, nullptr, nullptr, p, 0);
}

}  // namespace lagp
