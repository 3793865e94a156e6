// batch.cu -- lagp_predict_batch_dev: many locations, several resident designs, per-location
// n and candidate count, in one persistent launch of kernels (b)+(c).
//
// The host builds the per-location tables (batch.cuh), orders the work queue by estimated
// cost (n^2 M, longest first, so the persistent CTAs finish together), launches kernel (a)
// once per design over that design's locations, then kernels (b)+(c) once over the whole
// batch.  Two options:
//   LAGP_BATCH_TUNE   the launch shape (resident CTAs per SM of both kernels) is chosen by
//                     timing the candidates on the first batch of each signature (method,
//                     precision, dimensions present, n and M buckets, T bucket); the choice
//                     is cached for the process;
//   LAGP_BATCH_GRAPH  the launches are captured into a CUDA graph the first time a batch
//                     signature and buffer set is seen, and the graph is replayed afterwards
//                     (the tables are copied in before each replay).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "batch.cuh"
#include "internal.h"

namespace lagp {
namespace {

struct Layout {
  size_t designs, locs, order, lists, cand, scratch, total;
  size_t knn_ws, sel_ws;
};

struct Plan {
  std::vector<BatchDesign> designs;
  std::vector<LocDesc> locs;
  std::vector<int32_t> order, lists, list_off, list_cnt;
  int32_t nmax = 0, pmax = 0, Mmax = 0;
  std::vector<int32_t> Mmax_d;
  int64_t cand_total = 0, idx_total = 0, Nmax = 0;
};

int validate_and_plan(const lagp_design_desc *designs, int32_t nd, int64_t T, const int32_t *design_of,
                      const int32_t *n, const int32_t *ncand, int32_t method, int32_t precision,
                      Plan *P) {
  if (nd < 1 || T < 0 || (T > 0 && (!design_of || !n || !ncand)) || !designs) return LAGP_ERR_INVALID_ARG;
  if (method != LAGP_ALC && method != LAGP_MSPE && method != LAGP_NN) return LAGP_ERR_INVALID_ARG;
  if (precision != LAGP_FP64 && precision != LAGP_MIXED) return LAGP_ERR_INVALID_ARG;
  int st = check_supported(method, precision);
  if (st) return st;
  P->designs.resize(nd);
  P->Mmax_d.assign(nd, 0);
  for (int d = 0; d < nd; d++) {
    const lagp_design_desc &D = designs[d];
    if (!D.X || !D.Z || D.N < 1 || D.N > INT32_MAX || D.p < 1 || D.p > kMaxP || D.n0 < 1) return LAGP_ERR_INVALID_ARG;
    if (!(D.theta > 0.0) || !isfinite(D.theta) || !(D.g >= 0.0) || !isfinite(D.g)) return LAGP_ERR_INVALID_ARG;
    if (method == LAGP_MSPE && D.n0 < 3) return LAGP_ERR_INVALID_ARG;
    P->designs[d] = BatchDesign{D.X, D.Z, D.N, D.p, D.n0, D.theta, D.g};
    P->Nmax = std::max(P->Nmax, D.N);
  }
  P->locs.resize(T);
  P->list_cnt.assign(nd, 0);
  for (int64_t t = 0; t < T; t++) {
    const int d = design_of[t];
    if (d < 0 || d >= nd) return LAGP_ERR_INVALID_ARG;
    const lagp_design_desc &D = designs[d];
    const int nt = n[t], mt = ncand[t];
    if (nt < 3 || nt < D.n0 || nt > kMaxN) return LAGP_ERR_INVALID_ARG;
    if (mt < nt || (int64_t)mt > D.N || mt > kMaxCand) return LAGP_ERR_INVALID_ARG;
    P->locs[t] = LocDesc{d, nt, mt, 0, P->cand_total, P->idx_total};
    P->cand_total += mt;
    P->idx_total += nt;
    P->nmax = std::max(P->nmax, nt);
    P->pmax = std::max(P->pmax, D.p);
    P->Mmax = std::max(P->Mmax, mt);
    P->Mmax_d[d] = std::max(P->Mmax_d[d], mt);
    P->list_cnt[d]++;
  }
  // queue order: estimated cost n^2 M, longest first (ties by index, deterministic)
  P->order.resize(T);
  std::iota(P->order.begin(), P->order.end(), 0);
  const double mspe = (method == LAGP_MSPE) ? 3.0 : 1.0;
  std::vector<double> cost(T);
  for (int64_t t = 0; t < T; t++)
    cost[t] = mspe * (double)P->locs[t].n * P->locs[t].n * P->locs[t].M;
  std::stable_sort(P->order.begin(), P->order.end(),
                   [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  // per-design location lists for kernel (a)
  P->list_off.assign(nd + 1, 0);
  for (int d = 0; d < nd; d++) P->list_off[d + 1] = P->list_off[d] + P->list_cnt[d];
  P->lists.resize(T);
  std::vector<int32_t> fill(P->list_off.begin(), P->list_off.end() - 1);
  for (int64_t t = 0; t < T; t++) P->lists[fill[P->locs[t].design]++] = (int32_t)t;
  return LAGP_OK;
}

BatchLaunch make_launch(const Plan &P, int32_t method, int32_t precision, int64_t T,
                        const double *XX, int32_t ldxx, double *mean, double *s2, double *var,
                        int32_t *idx, int8_t *status, int ctas) {
  BatchLaunch b;
  b.method = method;
  b.precision = precision;
  b.T = T;
  b.designs = nullptr;
  b.locs = nullptr;
  b.order = nullptr;
  b.XX = XX;
  b.ldxx = ldxx;
  b.cand = nullptr;
  b.nmax = P.nmax;
  b.pmax = P.pmax;
  b.Mmax = P.Mmax;
  b.mean = mean; b.s2 = s2; b.var = var; b.idx = idx; b.status = status;
  b.idx_total = P.idx_total;
  b.ctas_per_sm = ctas;
  return b;
}

Layout layout_of(const Plan &P, int32_t method, int32_t precision, int64_t T, int num_sms) {
  Layout L;
  L.designs = 0;
  L.locs = align_up(L.designs + P.designs.size() * sizeof(BatchDesign), 256);
  L.order = align_up(L.locs + (size_t)T * sizeof(LocDesc), 256);
  L.lists = align_up(L.order + (size_t)T * sizeof(int32_t), 256);
  L.cand = align_up(L.lists + (size_t)T * sizeof(int32_t), 256);
  L.scratch = align_up(L.cand + (size_t)P.cand_total * sizeof(int32_t), 256);
  L.knn_ws = knn_workspace_bytes(P.Nmax, T, P.Mmax, num_sms);
  BatchLaunch b = make_launch(P, method, precision, T, nullptr, 0, nullptr, nullptr, nullptr,
                              nullptr, nullptr, select_max_ctas(method, precision));
  L.sel_ws = select_batch_workspace_bytes(b, num_sms);
  L.total = L.scratch + std::max(L.knn_ws, L.sel_ws);
  return L;
}

// ---- autotuner: resident CTAs per SM of kernels (a) and (b)+(c), per batch signature
struct TuneChoice {
  int knn_ctas, sel_ctas;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;

std::string signature(const Plan &P, int32_t method, int32_t precision, int64_t T) {
  std::string k = std::to_string(method) + "/" + std::to_string(precision) + "/p";
  bool seen[kMaxP + 1] = {false};
  for (const auto &d : P.designs) seen[d.p] = true;
  for (int p = 1; p <= kMaxP; p++)
    if (seen[p]) k += std::to_string(p);
  int tb = 0;
  while ((int64_t(1) << tb) < T) tb++;
  k += "/n" + std::to_string((P.nmax + 31) / 32) + "/M" + std::to_string((P.Mmax + 511) / 512) +
       "/T" + std::to_string(tb);
  return k;
}

// ---- graph cache: one instantiated graph per (signature, buffers, launch shape)
std::mutex g_graph_mu;
// An instantiated graph and the number of kernels it launches (counted at capture, where
// the launches are recorded but do not run; added to the launch counter at each replay).
struct GraphEntry {
  cudaGraphExec_t exec;
  int64_t kernels;
};
std::map<std::string, GraphEntry> g_graphs;

// One non-blocking stream per device for graph capture (created on first use).
cudaStream_t capture_stream(int device) {
  static std::mutex mu;
  static cudaStream_t streams[64];
  if (device < 0 || device >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[device] && cudaStreamCreateWithFlags(&streams[device], cudaStreamNonBlocking) != cudaSuccess)
    streams[device] = nullptr;
  return streams[device];
}

}  // namespace

// The launches of one batch (kernel (a) per design, then kernels (b)+(c)).
static int launch_all(const Plan &P, const Layout &L, char *w, const double *XX, int32_t ldxx,
                      int64_t T, int32_t method, int32_t precision, double *mean, double *s2,
                      double *var, int32_t *idx, int8_t *status, int knn_ctas, int sel_ctas,
                      cudaStream_t stream) {
  const BatchDesign *ddev = reinterpret_cast<const BatchDesign *>(w + L.designs);
  const LocDesc *ldev = reinterpret_cast<const LocDesc *>(w + L.locs);
  const int32_t *odev = reinterpret_cast<const int32_t *>(w + L.order);
  const int32_t *lsdev = reinterpret_cast<const int32_t *>(w + L.lists);
  int32_t *cand = reinterpret_cast<int32_t *>(w + L.cand);
  void *scratch = w + L.scratch;
  const size_t sbytes = std::max(L.knn_ws, L.sel_ws);
  for (size_t d = 0; d < P.designs.size(); d++) {
    const int cnt = P.list_cnt[d];
    if (!cnt) continue;
    const BatchDesign &D = P.designs[d];
    int st = knn_launch_list(D.X, D.N, D.p, XX, cnt, P.Mmax_d[d], cand, scratch, sbytes, stream,
                             lsdev + P.list_off[d], ldev, ldxx, knn_ctas);
    if (st) return st;
  }
  BatchLaunch b = make_launch(P, method, precision, T, XX, ldxx, mean, s2, var, idx, status, sel_ctas);
  b.designs = ddev;
  b.locs = ldev;
  b.order = odev;
  b.cand = cand;
  return select_batch_launch(b, scratch, sbytes, stream);
}

}  // namespace lagp

using namespace lagp;

extern "C" size_t lagp_predict_batch_workspace_bytes(const lagp_design_desc *designs, int32_t ndesigns,
                                                     int64_t T, const int32_t *design_of,
                                                     const int32_t *n, const int32_t *ncand,
                                                     int32_t method, int32_t precision) {
  Plan P;
  if (validate_and_plan(designs, ndesigns, T, design_of, n, ncand, method, precision, &P)) return 0;
  DevInfo di;
  if (dev_info(&di)) return 0;
  return layout_of(P, method, precision, T, di.num_sms).total;
}

extern "C" int lagp_predict_batch_dev(const lagp_design_desc *designs, int32_t ndesigns,
                                      const double *XX, int32_t ldxx, int64_t T,
                                      const int32_t *design_of, const int32_t *n,
                                      const int32_t *ncand, int32_t method, int32_t precision,
                                      double *mean, double *s2, double *var, int32_t *idx,
                                      int8_t *status, uint32_t flags, void *workspace,
                                      size_t workspace_bytes, void *stream_) {
  Plan P;
  int st = validate_and_plan(designs, ndesigns, T, design_of, n, ncand, method, precision, &P);
  if (st) return st;
  if (T == 0) return LAGP_OK;
  if (!XX || ldxx < P.pmax || !mean || !s2 || !workspace) return LAGP_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return LAGP_ERR_INVALID_ARG;
  DevInfo di;
  st = dev_info(&di);
  if (st) return st;
  const Layout L = layout_of(P, method, precision, T, di.num_sms);
  if (workspace_bytes < L.total) return LAGP_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  char *w = static_cast<char *>(workspace);
  // tables to the device (outside any graph: the host vectors are pageable)
  cudaError_t e = cudaMemcpyAsync(w + L.designs, P.designs.data(), P.designs.size() * sizeof(BatchDesign),
                                  cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + L.locs, P.locs.data(), (size_t)T * sizeof(LocDesc), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + L.order, P.order.data(), (size_t)T * sizeof(int32_t), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + L.lists, P.lists.data(), (size_t)T * sizeof(int32_t), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_status(e);

  // launch shape: tuned per signature, or the defaults
  const std::string sig = signature(P, method, precision, T);
  int knn_ctas = 0, sel_ctas = select_max_ctas(method, precision);
  bool have = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(sig);
    if (it != g_tune.end()) {
      knn_ctas = it->second.knn_ctas;
      sel_ctas = it->second.sel_ctas;
      have = true;
    }
  }
  if ((flags & LAGP_BATCH_TUNE) && !have) {
    // time every candidate shape on this batch (results are the same whatever the shape)
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LAGP_ERR_CUDA;
    float best = 1e30f;
    const int kn_opts[2] = {2, 4};
    const int smax = select_max_ctas(method, precision);
    for (int ko = 0; ko < 2; ko++)
      for (int so = 1; so <= smax; so++) {
        cudaEventRecord(e0, stream);
        st = launch_all(P, L, w, XX, ldxx, T, method, precision, mean, s2, var, idx, status,
                        kn_opts[ko], so, stream);
        cudaEventRecord(e1, stream);
        if (st) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = LAGP_ERR_CUDA; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          knn_ctas = kn_opts[ko];
          sel_ctas = so;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[sig] = TuneChoice{knn_ctas, sel_ctas};
    return LAGP_OK;  // every timed run produced the outputs; they do not depend on the shape
  }
  if (flags & LAGP_BATCH_GRAPH) {
    char key[512];
    snprintf(key, sizeof key, "%s|%p|%p|%d|%p|%p|%p|%p|%p|%d|%d|%zu", sig.c_str(), (void *)w,
             (const void *)XX, ldxx, (void *)mean, (void *)s2, (void *)var, (void *)idx,
             (void *)status, knn_ctas, sel_ctas, (size_t)T);
    std::string k(key);
    for (const auto &d : P.designs) {
      char dk[96];
      snprintf(dk, sizeof dk, "|%p,%p,%lld", (const void *)d.X, (const void *)d.Z, (long long)d.N);
      k += dk;
    }
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    {
      std::lock_guard<std::mutex> lk(g_graph_mu);
      auto it = g_graphs.find(k);
      if (it != g_graphs.end()) {
        exec = it->second.exec;
        kernels = it->second.kernels;
      }
    }
    if (!exec) {
      // Capture on a library-owned stream (the legacy default stream cannot be captured);
      // the graph is then launched on the caller's stream, after the table copies.
      st = select_prepare();
      if (!st) st = select_mixed_prepare();
      if (!st) st = select_mspe_prepare();
      if (!st) st = select_mspe_mixed_prepare();
      if (st) return st;
      cudaStream_t cap = capture_stream(di.device);
      if (!cap) return LAGP_ERR_CUDA;
      cudaGraph_t graph;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_status(e);
      const int64_t before = g_launches.load();
      st = launch_all(P, L, w, XX, ldxx, T, method, precision, mean, s2, var, idx, status,
                      knn_ctas, sel_ctas, cap);
      kernels = g_launches.load() - before;
      g_launches.fetch_sub(kernels);  // recorded, not run
      e = cudaStreamEndCapture(cap, &graph);
      if (st) return st;
      if (e != cudaSuccess) return cuda_status(e);
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_status(e);
      std::lock_guard<std::mutex> lk(g_graph_mu);
      g_graphs[k] = GraphEntry{exec, kernels};
    }
    e = cudaGraphLaunch(exec, stream);
    if (e == cudaSuccess) g_launches.fetch_add(kernels);
    return cuda_status(e);
  }
  return launch_all(P, L, w, XX, ldxx, T, method, precision, mean, s2, var, idx, status, knn_ctas,
                    sel_ctas, stream);
}
