// server.cu -- lagp_server_*: a continuous-batching serving loop over resident designs.
//
// Requests (a block of predictive locations against one resident design, with their n and
// candidate count) are queued on submit.  A scheduler thread coalesces queued requests
// into batches and runs each batch with the batched path (batch.cu) on one of a few
// in-flight slots, each with its own CUDA stream, device buffers and pinned staging
// buffers.  A request that arrives while other batches are on the GPU is admitted into the
// next batch as soon as a slot is free, so batches overlap on the device.  Admission is
// bounded by device memory: the number of slots is the memory budget divided by the
// bytes one slot needs for its largest batch.  Every location's arithmetic depends only on
// its own inputs, so a request's results are the same alone and in any mix.
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace lagp {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  int32_t design, n, ncand;
  int64_t L;
  std::vector<double> XX;  // L x p
  std::vector<double> mean, s2, var;
  std::vector<int32_t> idx;
  std::vector<int8_t> status;
  Clock::time_point t_submit, t_done;
  int code = 0;
  bool done = false;
  bool cancelled = false;  // cancelled while its batch was on the GPU: outputs dropped
  int inject = 0;          // test hook: the batch holding it fails with this code, on the host
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  char *dev = nullptr;      // device block: XX | mean | s2 | var | idx | status | workspace
  char *host = nullptr;     // pinned: XX staging | outputs
  size_t dev_bytes = 0, host_bytes = 0, ws_bytes = 0;
  bool busy = false;
  std::vector<std::shared_ptr<Request>> reqs;
  int64_t T = 0, idx_total = 0;
};

}  // namespace
}  // namespace lagp

using namespace lagp;

struct lagp_server {
  std::vector<lagp_design_desc> designs;
  int32_t precision = LAGP_MIXED, method = LAGP_ALC;
  int64_t max_batch = 0;
  int32_t nmax = 0, Mmax = 0;
  int device = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::atomic<uint64_t> next_id{1};
  std::atomic<bool> stop{false};
  std::thread worker;
  int64_t batches = 0, locations = 0, max_inflight_seen = 0;
  int last_error = 0;
};

namespace {

size_t off_mean(int64_t T) { return align_up((size_t)T * kMaxP * sizeof(double), 256); }

// Pinned output layout after the XX staging area: mean | s2 | var | status | idx.
size_t idx_host_offset(int64_t max_batch) { return align_up((size_t)max_batch * 25, 256); }

struct Offsets {
  size_t xx, mean, s2, var, idx, status, ws, total;
};

Offsets dev_offsets(int64_t T, int32_t nmax) {
  Offsets o;
  o.xx = 0;
  o.mean = off_mean(T);
  o.s2 = align_up(o.mean + (size_t)T * 8, 256);
  o.var = align_up(o.s2 + (size_t)T * 8, 256);
  o.idx = align_up(o.var + (size_t)T * 8, 256);
  o.status = align_up(o.idx + (size_t)T * nmax * 4, 256);
  o.ws = align_up(o.status + (size_t)T, 256);
  o.total = o.ws;
  return o;
}

// Workspace of the worst batch a slot accepts: max_batch locations, all with nmax and Mmax,
// spread over every design (the largest N and p).
size_t worst_workspace(const lagp_design_desc *designs, int nd, int32_t method, int32_t precision,
                       int32_t nmax, int32_t Mmax, int64_t max_batch) {
  std::vector<int32_t> dof(max_batch), n(max_batch, nmax), m(max_batch);
  for (int64_t t = 0; t < max_batch; t++) {
    dof[t] = (int32_t)(t % nd);
    m[t] = (int32_t)std::min<int64_t>(Mmax, designs[dof[t]].N);
  }
  return lagp_predict_batch_workspace_bytes(designs, nd, max_batch, dof.data(), n.data(), m.data(),
                                            method, precision);
}

// Device bytes of one in-flight slot (its buffers and the worst batch's workspace), 0 if the
// arguments are invalid.
size_t slot_device_bytes(const lagp_design_desc *designs, int nd, int32_t method,
                         int32_t precision, int32_t nmax, int32_t Mmax, int64_t max_batch) {
  const size_t ws = worst_workspace(designs, nd, method, precision, nmax, Mmax, max_batch);
  if (ws == 0) return 0;
  return dev_offsets(max_batch, nmax).total + ws;
}

// A batch that fails before reaching the GPU: its requests complete with the code at once.
void fail_batch_now(lagp_server *S, std::vector<std::shared_ptr<Request>> &reqs, int code) {
  std::lock_guard<std::mutex> lk(S->mu);
  const auto now = Clock::now();
  for (auto &r : reqs) {
    r->code = r->cancelled ? LAGP_ERR_CANCELLED : code;
    r->done = true;
    r->t_done = now;
  }
  S->last_error = code;
  S->cv_done.notify_all();
}

void run_batch(lagp_server *S, Slot &sl, std::vector<std::shared_ptr<Request>> &&reqs) {
  for (auto &r : reqs)
    if (r->inject) {  // a request marked by lagp_server_inject_error runs in a batch alone
      fail_batch_now(S, reqs, r->inject);
      return;
    }
  sl.reqs = std::move(reqs);
  int64_t T = 0, itot = 0;
  for (auto &r : sl.reqs) { T += r->L; itot += r->L * r->n; }
  sl.T = T;
  sl.idx_total = itot;
  const Offsets o = dev_offsets(S->max_batch, S->nmax);
  double *hXX = reinterpret_cast<double *>(sl.host);
  std::vector<int32_t> dof(T), n(T), m(T);
  int64_t t = 0;
  for (auto &r : sl.reqs) {
    const int p = S->designs[r->design].p;
    for (int64_t l = 0; l < r->L; l++, t++) {
      dof[t] = r->design;
      n[t] = r->n;
      m[t] = r->ncand;
      memset(hXX + t * kMaxP, 0, sizeof(double) * kMaxP);
      memcpy(hXX + t * kMaxP, r->XX.data() + l * p, sizeof(double) * p);
    }
  }
  double *dXX = reinterpret_cast<double *>(sl.dev + o.xx);
  double *dmean = reinterpret_cast<double *>(sl.dev + o.mean);
  double *ds2 = reinterpret_cast<double *>(sl.dev + o.s2);
  double *dvar = reinterpret_cast<double *>(sl.dev + o.var);
  int32_t *didx = reinterpret_cast<int32_t *>(sl.dev + o.idx);
  int8_t *dst = reinterpret_cast<int8_t *>(sl.dev + o.status);
  int code = cuda_status(cudaMemcpyAsync(dXX, hXX, (size_t)T * kMaxP * sizeof(double),
                                         cudaMemcpyHostToDevice, sl.stream));
  if (!code)
    code = lagp_predict_batch_dev(S->designs.data(), (int32_t)S->designs.size(), dXX, kMaxP, T,
                                  dof.data(), n.data(), m.data(), S->method, S->precision, dmean,
                                  ds2, dvar, didx, dst, 0, sl.dev + o.ws, sl.ws_bytes, sl.stream);
  // outputs back into the slot's pinned buffer: mean | s2 | var | status | idx
  char *hout = sl.host + align_up((size_t)S->max_batch * kMaxP * sizeof(double), 256);
  if (!code) {
    cudaError_t e = cudaMemcpyAsync(hout, dmean, (size_t)T * 8, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout + (size_t)S->max_batch * 8, ds2, (size_t)T * 8, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout + (size_t)S->max_batch * 16, dvar, (size_t)T * 8, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout + (size_t)S->max_batch * 24, dst, (size_t)T, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout + idx_host_offset(S->max_batch), didx, (size_t)itot * 4, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done_ev, sl.stream);
    code = cuda_status(e);
  }
  if (code) {
    for (auto &r : sl.reqs) { r->code = code; }
    S->last_error = code;
  }
  sl.busy = true;
}

void finish_batch(lagp_server *S, Slot &sl) {
  const char *hout = sl.host + align_up((size_t)S->max_batch * kMaxP * sizeof(double), 256);
  const double *hm = reinterpret_cast<const double *>(hout);
  const double *hs = reinterpret_cast<const double *>(hout + (size_t)S->max_batch * 8);
  const double *hv = reinterpret_cast<const double *>(hout + (size_t)S->max_batch * 16);
  const int8_t *hst = reinterpret_cast<const int8_t *>(hout + (size_t)S->max_batch * 24);
  const int32_t *hi = reinterpret_cast<const int32_t *>(hout + idx_host_offset(S->max_batch));
  const auto now = Clock::now();
  int64_t t = 0, io = 0;
  std::lock_guard<std::mutex> lk(S->mu);
  int64_t served = 0;
  for (auto &r : sl.reqs) {
    if (r->cancelled) r->code = LAGP_ERR_CANCELLED;
    if (r->code) {
      t += r->L;
      io += r->L * r->n;
      r->t_done = now;
      r->done = true;
      continue;
    }
    served += r->L;
    r->mean.assign(hm + t, hm + t + r->L);
    r->s2.assign(hs + t, hs + t + r->L);
    r->var.assign(hv + t, hv + t + r->L);
    r->status.assign(hst + t, hst + t + r->L);
    r->idx.assign(hi + io, hi + io + r->L * r->n);
    t += r->L;
    io += r->L * r->n;
    r->t_done = now;
    r->done = true;
  }
  S->batches++;
  S->locations += served;
  sl.reqs.clear();
  sl.busy = false;
  S->cv_done.notify_all();
}

void scheduler(lagp_server *S) {
  cudaSetDevice(S->device);
  while (!S->stop.load()) {
    // retire finished batches
    int inflight = 0;
    for (auto &sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done_ev);
      if (q == cudaSuccess) finish_batch(S, sl);
      else if (q != cudaErrorNotReady) {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &r : sl.reqs) {
          r->code = r->cancelled ? LAGP_ERR_CANCELLED : LAGP_ERR_CUDA;
          r->done = true;
          r->t_done = Clock::now();
        }
        sl.reqs.clear();
        sl.busy = false;
        S->last_error = LAGP_ERR_CUDA;
        S->cv_done.notify_all();
      } else {
        inflight++;
      }
    }
    // admit queued requests into a free slot
    Slot *free_slot = nullptr;
    for (auto &sl : S->slots)
      if (!sl.busy) { free_slot = &sl; break; }
    std::vector<std::shared_ptr<Request>> take;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (free_slot) {
        int64_t T = 0;
        while (!S->pending.empty() && T + S->pending.front()->L <= S->max_batch) {
          const bool alone = S->pending.front()->inject != 0;
          if (alone && !take.empty()) break;
          T += S->pending.front()->L;
          take.push_back(S->pending.front());
          S->pending.pop_front();
          if (alone) break;
        }
      }
      if (take.empty()) {
        if (inflight == 0 && S->pending.empty())
          S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        else
          lk.unlock(), std::this_thread::sleep_for(std::chrono::microseconds(50));
        continue;
      }
    }
    run_batch(S, *free_slot, std::move(take));
    int busy = 0;
    for (auto &sl : S->slots) busy += sl.busy;
    std::lock_guard<std::mutex> lk(S->mu);
    if (busy > S->max_inflight_seen) S->max_inflight_seen = busy;
  }
}

}  // namespace

extern "C" {

int lagp_server_create(const lagp_design_desc *designs, int32_t ndesigns, int32_t method,
                       int32_t precision, int32_t nmax, int32_t ncand_max, int64_t max_batch,
                       size_t memory_budget, int32_t max_slots, lagp_server **out) {
  if (!out || !designs || ndesigns < 1 || nmax < 3 || nmax > kMaxN || ncand_max < nmax ||
      ncand_max > kMaxCand || max_batch < 1 || max_slots < 1)
    return LAGP_ERR_INVALID_ARG;
  *out = nullptr;
  int st = check_supported(method, precision);
  if (st) return st;
  lagp_server *S = new (std::nothrow) lagp_server();
  if (!S) return LAGP_ERR_OOM;
  S->designs.assign(designs, designs + ndesigns);
  S->method = method;
  S->precision = precision;
  S->nmax = nmax;
  S->Mmax = ncand_max;
  S->max_batch = max_batch;
  cudaGetDevice(&S->device);
  const size_t slot_dev = slot_device_bytes(designs, ndesigns, method, precision, nmax, ncand_max,
                                            max_batch);
  if (slot_dev == 0) { delete S; return LAGP_ERR_INVALID_ARG; }
  const size_t ws = slot_dev - dev_offsets(max_batch, nmax).total;
  int nslots = (int)std::min<size_t>((size_t)max_slots, memory_budget / slot_dev);
  if (nslots < 1) { delete S; return LAGP_ERR_OOM; }
  S->slots.resize(nslots);
  const size_t host_bytes = align_up((size_t)max_batch * kMaxP * sizeof(double), 256) +
                            idx_host_offset(max_batch) + (size_t)max_batch * 4 * (size_t)nmax;
  for (auto &sl : S->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dev, slot_dev);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.host, host_bytes);
    if (e != cudaSuccess) {
      lagp_server_destroy(S);
      return cuda_status(e);
    }
    sl.dev_bytes = slot_dev;
    sl.host_bytes = host_bytes;
    sl.ws_bytes = ws;
  }
  S->worker = std::thread(scheduler, S);
  *out = S;
  return LAGP_OK;
}

int lagp_server_submit(lagp_server *S, int32_t design, const double *XX, int64_t L, int32_t n,
                       int32_t ncand, uint64_t *request_id) {
  if (!S || !XX || !request_id || design < 0 || design >= (int32_t)S->designs.size() || L < 1 ||
      L > S->max_batch || n < 3 || n > S->nmax || n < S->designs[design].n0 || ncand < n ||
      ncand > S->Mmax || (int64_t)ncand > S->designs[design].N)
    return LAGP_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->id = S->next_id.fetch_add(1);
  r->design = design;
  r->n = n;
  r->ncand = ncand;
  r->L = L;
  const int p = S->designs[design].p;
  r->XX.assign(XX, XX + L * p);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->pending.push_back(r);
    S->all[r->id] = r;
  }
  S->cv_work.notify_one();
  *request_id = r->id;
  return LAGP_OK;
}

int lagp_server_wait(lagp_server *S, uint64_t id, int32_t timeout_ms, int32_t *done) {
  if (!S || !done) return LAGP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return LAGP_ERR_INVALID_ARG;
  auto r = it->second;
  if (timeout_ms != 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 3600000 : timeout_ms),
                        [&] { return r->done; });
  *done = r->done ? 1 : 0;
  return LAGP_OK;
}

int lagp_server_results(lagp_server *S, uint64_t id, double *mean, double *s2, double *var,
                        int32_t *idx, int8_t *status, double *latency_ms) {
  if (!S) return LAGP_ERR_INVALID_ARG;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end() || !it->second->done) return LAGP_ERR_INVALID_ARG;
    r = it->second;
    S->all.erase(it);
  }
  if (r->code) return r->code;
  if (mean) memcpy(mean, r->mean.data(), r->L * sizeof(double));
  if (s2) memcpy(s2, r->s2.data(), r->L * sizeof(double));
  if (var) memcpy(var, r->var.data(), r->L * sizeof(double));
  if (idx) memcpy(idx, r->idx.data(), r->L * r->n * sizeof(int32_t));
  if (status) memcpy(status, r->status.data(), r->L);
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  return LAGP_OK;
}

size_t lagp_server_slot_bytes(const lagp_design_desc *designs, int32_t ndesigns, int32_t method,
                              int32_t precision, int32_t nmax, int32_t ncand_max,
                              int64_t max_batch) {
  if (!designs || ndesigns < 1 || nmax < 3 || nmax > kMaxN || ncand_max < nmax ||
      ncand_max > kMaxCand || max_batch < 1)
    return 0;
  return slot_device_bytes(designs, ndesigns, method, precision, nmax, ncand_max, max_batch);
}

int lagp_server_cancel(lagp_server *S, uint64_t id) {
  if (!S) return LAGP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end() || it->second->done) return LAGP_ERR_INVALID_ARG;
  auto r = it->second;
  for (auto q = S->pending.begin(); q != S->pending.end(); ++q)
    if (*q == r) {  // still queued: it never reaches the GPU
      S->pending.erase(q);
      r->code = LAGP_ERR_CANCELLED;
      r->done = true;
      r->t_done = Clock::now();
      S->cv_done.notify_all();
      return LAGP_OK;
    }
  r->cancelled = true;  // in a batch on the GPU: the batch finishes, this request's outputs are dropped
  return LAGP_OK;
}

int lagp_server_inject_error(lagp_server *S, uint64_t id, int32_t code) {
  if (!S || code >= 0) return LAGP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return LAGP_ERR_INVALID_ARG;
  for (auto &q : S->pending)
    if (q == it->second) {
      q->inject = code;
      return LAGP_OK;
    }
  return LAGP_ERR_INVALID_ARG;  // already in a batch or finished
}

int lagp_server_stats(lagp_server *S, int64_t *batches, int64_t *locations, int32_t *slots,
                      int32_t *max_inflight) {
  if (!S) return LAGP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (batches) *batches = S->batches;
  if (locations) *locations = S->locations;
  if (slots) *slots = (int32_t)S->slots.size();
  if (max_inflight) *max_inflight = (int32_t)S->max_inflight_seen;
  return S->last_error;
}

int lagp_server_destroy(lagp_server *S) {
  if (!S) return LAGP_ERR_INVALID_ARG;
  S->stop.store(true);
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto &sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.dev) cudaFree(sl.dev);
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete S;
  return LAGP_OK;
}

}  // extern "C"
