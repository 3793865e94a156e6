// check.cuh -- device-side bounds checks of the checked build (-DLAGP_CHECKED).
//
// A stand-in for a memory sanitizer: in a checked build every guarded index is compared
// with the extent of the array it addresses; a violation is recorded (the first one's site,
// index and extent, and a count) and the access is skipped, and the kernel reports the
// location as failed, so an out-of-range index becomes a status the host reads through
// lagp_check_take() instead of a memory fault.  In normal builds LAGP_CHK is the constant
// true and the records stay zero.
//
// Each translation unit that includes this header has its own record; it exposes it to the
// host through a function of its own (declared in internal.h), which api.cu combines.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lagp {

static __device__ CheckRec g_check;

__device__ __forceinline__ bool check_in(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_check.count, 1ull) == 0ull) {
    g_check.site = site;
    g_check.index = i;
    g_check.bound = n;
  }
  return false;
}

// Bytes of dynamic shared memory this launch was given.
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned v;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

#ifdef LAGP_CHECKED
#define LAGP_CHK(i, n, site) ::lagp::check_in((long long)(i), (long long)(n), (site))
#else
#define LAGP_CHK(i, n, site) true
#endif

// Host: read this translation unit's record and clear it (the current device).
static int check_take_here(CheckRec *out) {
  CheckRec zero = {0ull, 0, 0, 0};
  cudaError_t e = cudaMemcpyFromSymbol(out, g_check, sizeof(CheckRec));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check, &zero, sizeof(CheckRec));
  return e == cudaSuccess ? LAGP_OK : LAGP_ERR_CUDA;
}

}  // namespace lagp
