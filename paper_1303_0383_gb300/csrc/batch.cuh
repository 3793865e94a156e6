// batch.cuh -- per-location parameters for batched launches with uneven local problems.
//
// A batch holds locations against several resident designs, each location with its own
// design size n and candidate count M (the paper's "knobs" n and N', Sec. 6, chosen per
// location).  Kernels read a location's parameters from these tables after popping it
// from the work queue; without tables (uniform launches) they use the launch-wide values.
#pragma once

#include <stdint.h>

namespace lagp {

struct BatchDesign {
  const double *X;  // N x p, device
  const double *Z;  // N, device
  int64_t N;
  int32_t p, n0;
  double theta, g;
};

struct LocDesc {
  int32_t design, n, M, pad;
  int64_t cand_off;  // offset of this location's candidate list
  int64_t idx_off;   // offset of this location's selected indices (in the idx output)
};

// Launch-wide view of the tables (device pointers) plus the uniform fallback values.
struct BatchView {
  const BatchDesign *designs;  // nullptr: uniform launch
  const LocDesc *locs;         // T descriptors
  const int32_t *order;        // queue position -> location (cost-sorted), may be nullptr
  int ldxx;                    // row stride of XX in doubles
  const double *theta_loc;     // per-location lengthscale (T), or nullptr
  const int32_t *n_loc;        // per-location design size (T, adaptive designs), or nullptr
};

// A location's parameters, resolved from the tables or the uniform values.
struct LocParams {
  int64_t loc;
  int64_t N;        // design rows (the extent design indices are checked against)
  const double *X, *Z, *x;
  int p, n, M, n0;
  double theta, theta_inv, onepg;
  const int32_t *cand;
  int32_t *idx;
};

__device__ __forceinline__ LocParams resolve_loc(const BatchView &B, int64_t q, const double *X,
                                                 const double *Z, const double *XX, int p, int n,
                                                 int M, int n0, double theta, double g,
                                                 const int32_t *cand, int32_t *idx,
                                                 int64_t N = INT64_MAX) {
  LocParams L;
  if (B.designs) {
    L.loc = B.order ? B.order[q] : q;
    const LocDesc d = B.locs[L.loc];
    const BatchDesign D = B.designs[d.design];
    L.N = D.N;
    L.X = D.X; L.Z = D.Z; L.p = D.p; L.n = d.n; L.M = d.M; L.n0 = D.n0;
    L.theta = D.theta; L.theta_inv = 1.0 / D.theta; L.onepg = 1.0 + D.g;
    L.x = XX + L.loc * B.ldxx;
    L.cand = cand + d.cand_off;
    L.idx = idx ? idx + d.idx_off : nullptr;
  } else {
    L.loc = q;
    L.N = N;
    L.X = X; L.Z = Z; L.p = p; L.n = n; L.M = M; L.n0 = n0;
    L.theta = theta; L.theta_inv = 1.0 / theta; L.onepg = 1.0 + g;
    L.x = XX + q * p;
    L.cand = cand + q * M;
    L.idx = idx ? idx + q * n : nullptr;
  }
  if (B.theta_loc) {  // a lengthscale per location (stage 2 of the stagewise scheme)
    L.theta = B.theta_loc[L.loc];
    L.theta_inv = 1.0 / L.theta;
  }
  if (B.n_loc) L.n = B.n_loc[L.loc];  // an adaptive design's size (idx keeps the launch stride)
  return L;
}

// A saved start design (design augmentation): sr[i] = the rank of start[i] in the
// location's candidate list cnd (M entries), or -1 when it is not a candidate.  Block-
// cooperative; every thread returns after the same two barriers.
__device__ __forceinline__ void start_ranks(const int32_t *start, int nstart, const int32_t *cnd,
                                            int M, int *sr) {
  for (int i = threadIdx.x; i < nstart; i += blockDim.x) sr[i] = -1;
  __syncthreads();
  for (int c = threadIdx.x; c < M; c += blockDim.x) {
    const int32_t v = cnd[c];
    for (int i = 0; i < nstart; i++)
      if (start[i] == v) sr[i] = c;
  }
  __syncthreads();
}

}  // namespace lagp
