/*
 * lagp.h -- C ABI of liblagp: local approximate Gaussian-process prediction on one GPU.
 *
 * Method: R. B. Gramacy and D. W. Apley, "Local Gaussian process approximation for large
 * computer experiments" (arXiv:1303.0383).  Each predictive location x is an independent
 * problem (Sec. 4, "Parallelization"):
 *   (a) the M nearest design points of x form its candidate set, the first n0 of them the
 *       start design D_{n0} (Sec. 3 intro; Sec. 6 restricts the search to the N' nearest);
 *   (b) the design grows greedily to n points, each step adding the candidate that
 *       maximises the ALC reduction in variance (Eq. dxy, Sec. 3.3), minimises the MSPE
 *       (Eq. mspe, Sec. 3.1), or is simply the next nearest (NN), with the fast
 *       sequential updates of Sec. 3.2;
 *   (c) the Student-t predictive equations are evaluated on D_n (Eqs. predgp, preds2).
 *
 * Conventions shared by every entry point
 *   - Arrays are row-major, C order.  X is N x p (float64), Z is N (float64), XX is T x p.
 *   - Correlation K(a,b) = exp(-||a-b||^2 / theta) for distinct design indices;
 *     K(a,a) = 1 + g, and K(x,x) = 1 + g for the predictive location (Sec. 2).
 *   - Squared distances are summed over k = 0..p-1 in that order without fused
 *     multiply-add, so neighbour sets are reproducible bit for bit; ties in distance go
 *     to the smaller design index.  Ties in the design criterion go to the nearer
 *     candidate (smaller neighbour rank).
 *   - Indices are 0-based int32 design rows; selected indices are in selection order
 *     (the first n0 are the start design in distance order).
 *   - Outputs per location: mean = mu_n(x) (Eq. predgp); s2 = psi_n v_n(x) / n, the
 *     Student-t scale with n degrees of freedom (Eq. preds2); var = s2 n/(n-2), the
 *     predictive variance.
 *   - status[t] = 0 on success, or LAGP_ERR_NOT_PD when a chosen point's conditional
 *     variance is not positive in FP64; that location's outputs are NaN and the rest of
 *     the batch is unaffected.
 *
 * Argument rules (violations return LAGP_ERR_INVALID_ARG before any GPU work):
 *   N >= 1, p in [1, 8], T >= 0, 1 <= n0 <= n, 3 <= n <= 256, n <= ncand <= min(N, 8192),
 *   theta > 0, g >= 0, method in lagp_method, precision in lagp_precision,
 *   MSPE needs n0 >= 3 (its variance uses psi_j/(j-2)).
 *
 * Errors: every call returns LAGP_OK (0) or a negative code; nothing is thrown across
 * the ABI.  lagp_strerror() names a code.  A CUDA failure returns LAGP_ERR_CUDA and
 * leaves the outputs undefined.
 *
 * Threads and streams: calls are thread-safe for distinct output buffers.  The *_dev
 * entry points enqueue work on the given stream (NULL = legacy default stream) and
 * return without synchronising; the host entry points synchronise before returning.
 */
#ifndef LAGP_H
#define LAGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LAGP_OK 0
#define LAGP_ERR_INVALID_ARG (-1)
#define LAGP_ERR_OOM (-2)
#define LAGP_ERR_CUDA (-3)
#define LAGP_ERR_TIMEOUT (-4)
#define LAGP_ERR_NOT_PD (-5)
#define LAGP_ERR_NO_DEVICE (-6)
#define LAGP_ERR_UNSUPPORTED (-7)
#define LAGP_ERR_SCRATCH_LIMIT (-8)
#define LAGP_ERR_NO_CONVERGENCE (-9)
#define LAGP_ERR_CANCELLED (-10)

typedef enum { LAGP_ALC = 0, LAGP_MSPE = 1, LAGP_NN = 2 } lagp_method;

/* LAGP_FP64: every step in FP64.
 * LAGP_MIXED: the candidate screen (ALC or MSPE) runs in float-float (pairs of FP32,
 * about 48 significant bits) on the FP32 pipes; near-tied decisions, and MSPE scores whose
 * G or J is a cancellation beyond the screen's resolution, are re-scored in FP64.  The MSPE
 * design bookkeeping (inverse factor, F_j, dmu_j(x)) stays FP64, and the predictive
 * equations are evaluated in FP64 on the final design.  NN has no screen. */
typedef enum { LAGP_FP64 = 0, LAGP_MIXED = 1 } lagp_precision;

/* Human-readable name of a return code; never NULL, static storage. */
const char *lagp_strerror(int code);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int lagp_version(void);

/* ------------------------------------------------------------------ host-buffer API */

/* Opaque resident design: the library's device copies of X (N x p) and Z (N).
 * lagp_design_create copies both from host memory (the caller keeps ownership of its
 * buffers) onto the current CUDA device; the handle owns the device memory until
 * lagp_design_destroy.  A design is immutable; concurrent predictions on it are allowed. */
typedef struct lagp_design lagp_design;

int lagp_design_create(const double *X, const double *Z, int64_t N, int32_t p,
                       lagp_design **out);
int lagp_design_destroy(lagp_design *d);

/* Local approximate GP prediction at T host locations XX (T x p) against a resident
 * design (Secs. 3-4): candidate sets of the ncand nearest, greedy design from n0 to n
 * by `method`, predictive equations.  Host outputs (caller-owned): mean[T], s2[T];
 * var[T], idx[T x n] and status[T] may be NULL.  The call copies XX to the device,
 * runs kernels (a)-(c), copies the results back and synchronises.  Device memory for
 * inputs, outputs and scratch is taken from and returned to a memory pool of the
 * library's own (one per device), which keeps up to 4 GiB of freed memory for the next
 * call until the process exits. */
int lagp_predict(const lagp_design *d, const double *XX, int64_t T, int32_t n0, int32_t n,
                 int32_t ncand, double theta, double g, int32_t method, int32_t precision,
                 double *mean, double *s2, double *var, int32_t *idx, int8_t *status);

/* ------------------------------------------------------------------ device-buffer API */
/* Every pointer below is a device pointer the caller allocated (for example a PyTorch
 * tensor's storage) and keeps owning.  `workspace` is caller-owned device scratch of at
 * least the size the matching *_workspace_bytes call returns (contents need not be
 * initialised; 256-byte alignment required); concurrent calls need distinct workspaces.
 * `stream` is a cudaStream_t passed as void*. */

/* Scratch bytes lagp_knn_dev needs for T locations against N design points. */
size_t lagp_knn_workspace_bytes(int64_t N, int64_t T, int32_t ncand);

/* Kernel (a): for each location t, the ncand nearest design points in (d2, index)
 * order (Sec. 3 intro; Sec. 6, candidate restriction).  X: N x p, XX: T x p;
 * cand: T x ncand int32 output. */
int lagp_knn_dev(const double *X, int64_t N, int32_t p, const double *XX, int64_t T,
                 int32_t ncand, int32_t *cand, void *workspace, size_t workspace_bytes,
                 void *stream);

/* Scratch bytes lagp_select_dev needs. */
size_t lagp_select_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand,
                                   int32_t method, int32_t precision);

/* Kernels (b)+(c): greedy local design and predictive equations for T locations whose
 * candidate lists `cand` (T x ncand, rank order, e.g. from lagp_knn_dev) are given
 * (Sec. 3.1-3.3 greedy design with the Sec. 3.2 updates; Eqs. predgp, preds2).
 * Outputs: mean[T], s2[T] required; var[T], idx[T x n], status[T] (int8) may be NULL. */
int lagp_select_dev(const double *X, const double *Z, int64_t N, int32_t p, const double *XX,
                    int64_t T, const int32_t *cand, int32_t ncand, int32_t n0, int32_t n,
                    double theta, double g, int32_t method, int32_t precision, double *mean,
                    double *s2, double *var, int32_t *idx, int8_t *status, void *workspace,
                    size_t workspace_bytes, void *stream);

/* Scratch bytes lagp_select_dense_dev needs. */
size_t lagp_select_dense_workspace_bytes(int64_t T, int32_t p, int32_t n, int32_t ncand);

/* ALC in the paper's own form, the comparison for lagp_select_dev (Sec. 3.2; SM "Partition
 * inverse equations"): each location keeps K_j^{-1} explicitly and grows it by the
 * partition inverse equations; each step scores every candidate by Eq. dxy from K_j^{-1},
 * O(j^2) per candidate (the quadratic form k_j(c)^T K_j^{-1} k_j(c)) where lagp_select_dev
 * takes O(j).  FP64 throughout.  The explicit inverse carries errors of order
 * cond(K_j) eps into v_j(c) = K(c,c) - k_j(c)^T K_j^{-1} k_j(c), so with small nuggets
 * the choices can differ from the exact greedy design that lagp_select_dev returns; the
 * outputs are the predictive equations on the design this call chose (FP64 Cholesky, as
 * lagp_design_predict_dev).  Arguments and outputs as lagp_select_dev with method ALC and
 * precision FP64; n > 128 returns LAGP_ERR_UNSUPPORTED (K_j^{-1} lives in shared memory).
 * A location where no candidate keeps a positive v_j(c) gets NaN outputs, idx -1 and
 * status LAGP_ERR_NOT_PD. */
int lagp_select_dense_dev(const double *X, const double *Z, int64_t N, int32_t p,
                          const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                          int32_t n0, int32_t n, double theta, double g, double *mean, double *s2,
                          double *var, int32_t *idx, int8_t *status, void *workspace,
                          size_t workspace_bytes, void *stream);

/* Diagnostics of the mixed-precision screens (Sec. 3.3 decisions; no counterpart in the
 * paper): the number of FP64 re-score passes -- steps of some location at which the screen's
 * best scores were near-tied (or, for MSPE, G or J was a cancellation beyond the screen's
 * resolution), so the decision was re-scored in FP64 -- made by the last lagp_select_dev,
 * lagp_select_theta_dev, lagp_select_augment_dev or lagp_select_adaptive_dev call that ran
 * on `workspace` with this method and precision.  Waits for the work on `stream`, then reads
 * the count (a 4-byte device-to-host copy).  *count = 0 for LAGP_FP64 and for NN.
 * workspace: that call's workspace (device, 256-byte aligned, at least 512 bytes). */
int lagp_select_rescore_count(const void *workspace, size_t workspace_bytes, int32_t method,
                              int32_t precision, int64_t *count, void *stream);

/* Scratch bytes lagp_predict_dev needs (candidate lists plus both kernels' scratch). */
size_t lagp_predict_workspace_bytes(int64_t N, int64_t T, int32_t p, int32_t n,
                                    int32_t ncand, int32_t method, int32_t precision);

/* The whole path on device buffers: lagp_knn_dev then lagp_select_dev (the candidate
 * lists live in the workspace). */
int lagp_predict_dev(const double *X, const double *Z, int64_t N, int32_t p, const double *XX,
                     int64_t T, int32_t n0, int32_t n, int32_t ncand, double theta, double g,
                     int32_t method, int32_t precision, double *mean, double *s2, double *var,
                     int32_t *idx, int8_t *status, void *workspace, size_t workspace_bytes,
                     void *stream);

/* ------------------------------------------------------------------ batched uneven problems */
/* A batch mixes locations against several resident designs, each location with its own
 * local design size n[t] and candidate count ncand[t] (the paper's knobs n and N', Secs.
 * 3 and 6, chosen per location; Sec. 6 discusses spending effort unevenly).  Kernel (a)
 * runs once per design over that design's locations and kernels (b)+(c) once over the
 * whole batch, as one persistent launch over a queue ordered by estimated cost n^2 ncand
 * (longest first).  Every location's results are bitwise the same as in a uniform call. */
typedef struct {
  const double *X;  /* N x p, device */
  const double *Z;  /* N, device */
  int64_t N;
  int32_t p;        /* 1 .. 8 */
  int32_t n0;       /* start-design size of every location on this design */
  double theta;     /* lengthscale d */
  double g;         /* nugget */
} lagp_design_desc;

/* flags of lagp_predict_batch_dev */
#define LAGP_BATCH_TUNE 1u  /* first batch of a signature: time the launch shapes, keep the best */
#define LAGP_BATCH_GRAPH 2u /* capture the launches in a CUDA graph once, replay afterwards */

/* Scratch bytes lagp_predict_batch_dev needs (0 if the arguments are invalid).  The
 * per-location arrays are host arrays of T entries. */
size_t lagp_predict_batch_workspace_bytes(const lagp_design_desc *designs, int32_t ndesigns,
                                          int64_t T, const int32_t *design_of, const int32_t *n,
                                          const int32_t *ncand, int32_t method,
                                          int32_t precision);

/* The whole path for a batch (Secs. 3-4).  designs: host array of ndesigns descriptors
 * (device X, Z).  XX: device, T rows of ldxx doubles (row t holds the location's p
 * coordinates first).  design_of, n, ncand: host arrays (T each).  Rules per location:
 * 3 <= n[t] <= 256, n[t] >= n0 of its design, n[t] <= ncand[t] <= min(N, 8192).
 * Outputs (device): mean[T], s2[T] required; var[T], status[T] optional; idx, optional,
 * holds sum(n) indices, location t's n[t] at offset n[0] + ... + n[t-1].
 * flags: LAGP_BATCH_TUNE and/or LAGP_BATCH_GRAPH (see above; graphs are cached per
 * signature and buffer set, and the per-location tables are copied in before each replay).
 * The call enqueues on `stream`; with LAGP_BATCH_TUNE on a new signature it synchronises. */
int lagp_predict_batch_dev(const lagp_design_desc *designs, int32_t ndesigns, const double *XX,
                           int32_t ldxx, int64_t T, const int32_t *design_of, const int32_t *n,
                           const int32_t *ncand, int32_t method, int32_t precision, double *mean,
                           double *s2, double *var, int32_t *idx, int8_t *status, uint32_t flags,
                           void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ serving loop */
/* A continuous-batching server over resident designs (the paper's global emulation of
 * Sec. 4, served request by request).  A request is a block of L locations against one
 * design with its n and candidate count.  A scheduler thread coalesces queued requests
 * into batches (lagp_predict_batch_dev) and runs each on one of a few in-flight slots
 * (own stream, device buffers and pinned staging), so requests arriving while other
 * batches run are admitted as soon as a slot frees and their work overlaps on the device.
 * Admission is bounded by device memory: slots = min(max_slots, memory_budget / bytes of
 * one slot sized for max_batch locations with nmax and ncand_max).  Results of a request
 * do not depend on what else was batched with it (bitwise).
 * lagp_server_create copies the design descriptors (the designs' device X, Z must stay
 * valid until destroy) and allocates every slot up front (LAGP_ERR_OOM if not even one
 * fits the budget).  submit copies XX (host, L x p) and returns at once; wait blocks up
 * to timeout_ms (negative: no limit) for a request; results copies a finished request's
 * outputs to host buffers (mean, s2, var: L; idx: L x n; status: L; any may be NULL),
 * gives its latency from submit to completion in ms, and forgets the request; for a request
 * whose batch failed (or that was cancelled) it returns that code instead and forgets it. */
typedef struct lagp_server lagp_server;
int lagp_server_create(const lagp_design_desc *designs, int32_t ndesigns, int32_t method,
                       int32_t precision, int32_t nmax, int32_t ncand_max, int64_t max_batch,
                       size_t memory_budget, int32_t max_slots, lagp_server **out);
int lagp_server_submit(lagp_server *s, int32_t design, const double *XX, int64_t L, int32_t n,
                       int32_t ncand, uint64_t *request_id);
int lagp_server_wait(lagp_server *s, uint64_t request_id, int32_t timeout_ms, int32_t *done);
int lagp_server_results(lagp_server *s, uint64_t request_id, double *mean, double *s2,
                        double *var, int32_t *idx, int8_t *status, double *latency_ms);
/* Batches and locations completed, slots, the most batches seen in flight at once; the
 * return value is the last error a batch met (LAGP_OK if none). */
int lagp_server_stats(lagp_server *s, int64_t *batches, int64_t *locations, int32_t *slots,
                      int32_t *max_inflight);
int lagp_server_destroy(lagp_server *s);

/* Device bytes of one in-flight slot of a server created with these arguments (its buffers
 * and the workspace of the largest batch it accepts); 0 if the arguments are invalid.  A
 * memory_budget of k times this gives min(k, max_slots) slots; below it, create returns
 * LAGP_ERR_OOM (admission refused).  The paper has no counterpart. */
size_t lagp_server_slot_bytes(const lagp_design_desc *designs, int32_t ndesigns, int32_t method,
                              int32_t precision, int32_t nmax, int32_t ncand_max,
                              int64_t max_batch);

/* Cancels a request that has not completed.  A request still queued leaves the queue and
 * never reaches the GPU; a request whose batch is already on the GPU lets that batch run to
 * completion (the other requests in it are unaffected) and drops its own outputs.  Either
 * way the request completes at once or with its batch, and lagp_server_results then returns
 * LAGP_ERR_CANCELLED (and forgets it).  Returns LAGP_ERR_INVALID_ARG for an unknown or
 * already completed request.  The paper has no counterpart. */
int lagp_server_cancel(lagp_server *s, uint64_t request_id);

/* Test hook for the server's failure path (the paper has no counterpart): marks a request
 * that is still queued so that the batch holding it -- the scheduler gives it a batch of
 * its own -- fails on the host with `code` (< 0) in place of the batched call's return code,
 * before any GPU work.  The request completes with that code (lagp_server_results returns
 * it), lagp_server_stats reports it as the last error, and every other request is served as
 * usual.  Returns LAGP_ERR_INVALID_ARG if the request is unknown or no longer queued, or if
 * code >= 0. */
int lagp_server_inject_error(lagp_server *s, uint64_t request_id, int32_t code);

/* ------------------------------------------------------------------ no-allocation variant */
/* Kernels (b)+(c) as lagp_select_dev, for callers that cannot allocate device memory: a
 * plugin running inside a host application that owns every device allocation and forbids
 * others once it has started, a real-time loop that cannot afford cudaMalloc's device-wide
 * synchronisation and unbounded latency, or a process whose allocation budget is spent.
 * The paper has no counterpart; it is a deployment convenience.
 *
 * There is no workspace argument.  The scratch is one static device array of
 * LAGP_NOALLOC_SCRATCH_BYTES (16 MiB) defined by the library; every device that loads
 * the library holds it until the process exits.  The call itself allocates nothing (no
 * cudaMalloc, no cudaFree, no allocating library routine); inputs and outputs are the
 * caller's device buffers, with the meaning, layout and rules of lagp_select_dev.
 *   - The first call on a device looks up the array's device address with that device
 *     current; make that first call before any stream capture.  The address is cached
 *     for that CUDA context: after a cudaDeviceReset the first call in the device's new
 *     context looks it up again (so it, too, should come before any capture).
 *   - All calls share the array, which keeps the previous call's contents; the call
 *     clears the part that must start at zero.  Calls whose kernels overlap on the GPU
 *     (for example on two streams) race on the array: serialise them.
 *   - The grid is limited to the CTA slots that fit in the array, so a large batch may
 *     use fewer SMs (and take longer) than lagp_select_dev; results are identical.
 *   - A problem whose single CTA slot, 256 + (n + p) x ceil32(ncand) x 8 bytes (each
 *     part rounded up to 256), exceeds the array returns LAGP_ERR_SCRATCH_LIMIT.
 *   - Only the FP64 ALC and NN forms run here: precision LAGP_MIXED with ALC, and the
 *     MSPE method, return LAGP_ERR_UNSUPPORTED. */
#define LAGP_NOALLOC_SCRATCH_BYTES (16u << 20)

int lagp_select_dev_noalloc(const double *X, const double *Z, int64_t N, int32_t p,
                            const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                            int32_t n0, int32_t n, double theta, double g, int32_t method,
                            int32_t precision, double *mean, double *s2, double *var,
                            int32_t *idx, int8_t *status, void *stream);

/* The library's FP64 exponential (Tang's table-driven method, the one kernels (b)+(c) use
 * for correlations), evaluated elementwise on device buffers: y[i] = exp(x[i]) for
 * x[i] in [-707, 0]; arguments below -707 give 0.  For verification against a reference
 * exponential.  x, y: n doubles (device).  No counterpart in the paper. */
int lagp_exp_dev(const double *x, double *y, int64_t n, void *stream);

/* Bounds checks of the checked build (the library built with -DLAGP_CHECKED,
 * liblagp_checked.so): a stand-in for a memory sanitizer.  Its kernels compare every
 * data-dependent index and every size taken from the launch (design indices against N,
 * a location's n, candidate count and dimension against its scratch slot, the shared-memory
 * layout against the launch's dynamic shared memory, tensor-memory columns against a
 * thread's words) with its extent; a violation is recorded and the access skipped, and the
 * location is abandoned.  Waits for the device, then returns in *count the violations since
 * the last call and in *site, *index, *bound the first one (site codes: 1-5 kernel (a):
 * survivor list, survivor design index, bucket scatter, bucket permutation, output index;
 * 11, 13-15, 18, 20 the mixed ALC screen: candidate design index, n, candidate count,
 * dimension, tensor-memory column, shared-memory layout; 21-25 the FP64 ALC kernel: n,
 * candidate count, dimension, candidate design index, shared-memory layout; 31-32 the
 * paper-form kernel: candidate design index, shared-memory layout), and clears the records.
 * *checked = 1 in the checked build, 0 otherwise (where every count is 0).  Any output may
 * be NULL. */
int lagp_check_take(int32_t *checked, int64_t *count, int32_t *site, int64_t *index,
                    int64_t *bound);

/* Number of kernel launches this library has issued in this process (all entry
 * points, all threads).  Used to report how many of the library's kernels a timed
 * region launched. */
int64_t lagp_launch_count(void);

/* Design augmentation (Sec. 6: once the indices of the local designs are saved, a design
 * can later be extended from where its construction stopped): kernels (b)+(c) where location t's
 * design starts from the n1 saved points start[t*n1 .. t*n1+n1) (design indices in
 * selection order, e.g. a previous call's idx) instead of its n0 nearest neighbours, and
 * grows greedily to n points.  The greedy choice depends only on the current design, so
 * augmenting the first n1 points of a design of size n reproduces that design.  Every
 * saved point must be among the location's ncand candidates (the same X, x and ncand as
 * the call that chose it); a location where one is not gets NaN outputs and status
 * LAGP_ERR_NOT_PD.  method ALC or MSPE (n1 >= 3 for MSPE); NN returns
 * LAGP_ERR_UNSUPPORTED (its design does not depend on the start).  Rules otherwise as
 * lagp_select_dev with n0 := n1 (1 <= n1 <= n); the workspace is sized by
 * lagp_select_workspace_bytes. */
int lagp_select_augment_dev(const double *X, const double *Z, int64_t N, int32_t p,
                            const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                            const int32_t *start, int32_t n1, int32_t n, double theta, double g,
                            int32_t method, int32_t precision, double *mean, double *s2,
                            double *var, int32_t *idx, int8_t *status, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Adaptive local design size (Sec. 6: a stopping criterion tracking the ratio of the
 * predictive variance before and after each added point, V_j(x) / V_{j+1}(x), in which
 * psi_j cancels): ALC designs grow from the n0 nearest as in lagp_select_dev, but stop
 * before the first greedy point whose ratio v_j(x) / v_{j+1}(x) is below r_min (> 1), or
 * at n points.  Outputs as lagp_select_dev, computed on each location's own design;
 * n_out[t] (device, int32, required) gets its size n0 <= n_out[t] <= n (0 for a failed
 * location); idx rows keep stride n, with -1 after n_out[t].  Rules as lagp_select_dev
 * with n0 >= 3 (var needs n_out - 2 > 0), r_min > 1; the workspace is sized by
 * lagp_select_workspace_bytes for LAGP_ALC. */
int lagp_select_adaptive_dev(const double *X, const double *Z, int64_t N, int32_t p,
                             const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                             int32_t n0, int32_t n, double theta, double g, int32_t precision,
                             double r_min, double *mean, double *s2, double *var, int32_t *idx,
                             int32_t *n_out, int8_t *status, void *workspace,
                             size_t workspace_bytes, void *stream);

/* ---- Local lengthscale estimates and the stagewise scheme (Sec. 4.2) ----
 * Sec. 4.2: (1) start from a global theta_0; (2) build each location's design with
 * theta_x; (3) estimate theta_x by maximum likelihood on that design; (4) set theta_x to
 * the estimate and repeat (2)-(3) as desired; predict on the last design with the last
 * estimate.  lagp_select_dev performs (2) with theta_0, lagp_mle_dev (3),
 * lagp_select_theta_dev (2) with per-location theta_x, lagp_design_predict_dev the output.
 * No spatial smoothing of the estimates is applied (the paper's borehole runs used the
 * unsmoothed first-stage estimates). */

/* Kernels (b)+(c) with a lengthscale per location: lagp_select_dev, except that location
 * t uses theta[t] (device array of T values, each > 0; the caller guarantees this) for
 * its candidate scores and predictive equations.  The workspace is sized by
 * lagp_select_workspace_bytes. */
int lagp_select_theta_dev(const double *X, const double *Z, int64_t N, int32_t p,
                          const double *XX, int64_t T, const int32_t *cand, int32_t ncand,
                          int32_t n0, int32_t n, const double *theta, double g, int32_t method,
                          int32_t precision, double *mean, double *s2, double *var, int32_t *idx,
                          int8_t *status, void *workspace, size_t workspace_bytes, void *stream);

/* Scratch bytes lagp_mle_dev needs for T designs of size n. */
size_t lagp_mle_workspace_bytes(int64_t T, int32_t n);

/* Local maximum-likelihood lengthscale, step (3): for each location t, the theta in
 * [tmin, tmax] maximising the log likelihood of Eq. gpk for the design
 * idx[t*n .. t*n+n) (design rows of X and Z), by Newton's method on the analytic
 * derivatives Eqs. dl, d2l (Sec. 3.2), started from theta0_loc[t] (device, T values) or,
 * when theta0_loc is NULL, from theta0.  Safeguards: a bracket of the maximum is narrowed
 * by the sign of l'; the Newton step is taken when l'' < 0 and it stays inside the
 * bracket, otherwise the iterate goes to the end of [tmin, tmax] uphill of theta if that
 * end has not been evaluated, else to the bracket's midpoint; the iteration stops when a
 * step is at most tol * theta (the new point is returned), when l' = 0, or at an end of
 * [tmin, tmax] where l' points outward (a boundary maximum).  All arithmetic is FP64.
 * Arguments: N >= 1, p in [1, 8], T >= 0, 2 <= n <= 256, 0 < tmin < tmax, maxit >= 1,
 * tol > 0, g >= 0; idx device, T x n (a row whose first entry is negative, a location
 * whose screen failed, gives NaN and LAGP_ERR_NOT_PD).
 * Outputs (device): theta_out[T]; iters[T] (int32, optional): derivative evaluations;
 * status[T] (int8, optional): 0, LAGP_ERR_NOT_PD (K_n not positive definite in FP64) or
 * LAGP_ERR_NO_CONVERGENCE (maxit evaluations; theta_out holds the last iterate). */
int lagp_mle_dev(const double *X, const double *Z, int64_t N, int32_t p, int64_t T,
                 const int32_t *idx, int32_t n, double theta0, const double *theta0_loc,
                 double g, double tmin, double tmax, int32_t maxit, double tol,
                 double *theta_out, int32_t *iters, int8_t *status, void *workspace,
                 size_t workspace_bytes, void *stream);

/* Scratch bytes lagp_design_predict_dev needs. */
size_t lagp_design_predict_workspace_bytes(int64_t T, int32_t n);

/* Kernel (c) alone, the output step: the predictive equations (Eqs. predgp, preds2) at
 * XX[t] on the given design idx[t*n .. t*n+n) with lengthscale theta_loc[t] (device) or,
 * when theta_loc is NULL, theta; FP64.  Argument rules as lagp_select_dev (n >= 3,
 * theta > 0 is checked for the scalar only).  A row of idx whose first entry is negative
 * gives NaN outputs and status LAGP_ERR_NOT_PD, as does a K_n that is not positive
 * definite.  Outputs (device): mean[T], s2[T] required; var[T], status[T] optional. */
int lagp_design_predict_dev(const double *X, const double *Z, int64_t N, int32_t p,
                            const double *XX, int64_t T, const int32_t *idx, int32_t n,
                            double theta, const double *theta_loc, double g, double *mean,
                            double *s2, double *var, int8_t *status, void *workspace,
                            size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LAGP_H */
