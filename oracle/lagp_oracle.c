/*
 * lagp_oracle.c -- CPU oracle for local approximate Gaussian-process prediction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path and the CUDA path never calls it.
 *
 * Method: R. B. Gramacy and D. W. Apley, "Local Gaussian process approximation for
 * large computer experiments" (arXiv:1303.0383).  Citations below name the paper's
 * sections and equations; "SM" is its supplementary material.
 *
 * What it computes, deliberately slowly and directly:
 *   - the M nearest design points of a predictive location x by a full sort of the
 *     exact squared distances, ties broken by index (Sec. 3 intro; Sec. 6 on the
 *     restriction to the N' nearest candidates);
 *   - the greedy local design D_{n0} -> D_n by ALC (Eq. dxy, read through SM "partial
 *     correlations", Eq. dxy2), by MSPE (Eq. mspe with Eqs. newv, G and the SM
 *     derivatives) or by nearest neighbours;
 *   - the Student-t predictive equations on D_n (Eqs. predgp, preds2);
 *   - the local maximum-likelihood lengthscale of a design (Sec. 4.2, step 3) by
 *     Newton's method on the analytic derivatives Eqs. dl, d2l (Sec. 3.2).
 * Every greedy step rebuilds K_j from its definition and refactors it from scratch
 * (hand-written Cholesky, K_j = L L^T); no quantity is carried from one step to the
 * next except the list of chosen points.  For ALC and for the predictive equations
 * the quadratic forms a^T K_j^{-1} b are evaluated as (L^{-1} a) . (L^{-1} b), the
 * same number in exact arithmetic without forming the ill-conditioned inverse; the
 * MSPE derivative terms use the explicit direct inverse K_j^{-1} = L^{-T} L^{-1}.
 * The paper's partitioned-inverse update (orc_pinv_update) is provided only for
 * the identities the tests pin.
 *
 * Conventions (readings of the paper):
 *   - K(a,b) = exp(-||a-b||^2/theta) for distinct design indices, K(a,a) = 1+g, and
 *     K(x,x) = 1+g for the predictive location; coincident values with distinct
 *     indices get no nugget (Sec. 2).
 *   - squared distances are summed over dimensions k = 0..p-1 in that order, each
 *     term the product of one rounded difference with itself, with no fused
 *     multiply-add (build with -ffp-contract=off), so neighbour sets are
 *     reproducible bit for bit.
 *   - the first n0 of the M nearest form D_{n0}; the other M-n0 are the search
 *     pool; the final design has exactly n points (n-n0 greedy steps).
 *   - ALC ties go to the smaller neighbour rank; MSPE ties likewise.
 *   - a pool member with v_j(c) <= 0, or whose criterion evaluates to NaN (possible for
 *     MSPE when the expected information is zero), is skipped by the criterion; if the
 *     chosen point has v <= 0 the location fails with status LAGP_ORC_NOT_PD.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared.  Built a
 * second time with -DLAGP_ORACLE_LONG the same source computes in long double, an
 * adjudicating reference for rounding questions (inputs and outputs stay double).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef LAGP_ORACLE_LONG
typedef long double real;
#define R_EXP expl
#define R_SQRT sqrtl
#define R_LOG logl
#else
typedef double real;
#define R_EXP exp
#define R_SQRT sqrt
#define R_LOG log
#endif

#define LAGP_ORC_OK 0
#define LAGP_ORC_INVALID (-1)
#define LAGP_ORC_OOM (-2)
#define LAGP_ORC_NOT_PD (-5)
#define LAGP_ORC_NO_CONV (-9)

enum { ORC_ALC = 0, ORC_MSPE = 1, ORC_NN = 2, ORC_MSPE_NODERIV = 3 };

/* Per greedy step, the trace holds these doubles (TRACE_W of them). */
#define TRACE_W 7
/* [0] best rank by the oracle's own criterion, [1] its score,
 * [2] chosen rank (== best unless a path is forced), [3] the chosen rank's score,
 * [4] second-best score, [5] v_j(x) before the step. */

int orc_real_bytes(void) { return (int)sizeof(real); }

/* ---------------------------------------------------------------- distances */

/* Squared distance in double, fixed order, no contraction (reading above). */
static double sqdist_d(const double *a, const double *b, int p) {
  double acc = 0.0;
  for (int k = 0; k < p; k++) {
    double t = a[k] - b[k];
    double t2 = t * t;
    acc = acc + t2;
  }
  return acc;
}

static real sqdist_r(const double *a, const double *b, int p) {
  real acc = 0;
  for (int k = 0; k < p; k++) {
    real t = (real)a[k] - (real)b[k];
    real t2 = t * t;
    acc = acc + t2;
  }
  return acc;
}

/* Isotropic Gaussian correlation of two distinct points (Sec. 2). */
static real corr_r(const double *a, const double *b, int p, real theta) {
  return R_EXP(-sqdist_r(a, b, p) / theta);
}

double orc_corr(const double *a, const double *b, int32_t p, double theta) {
  return (double)corr_r(a, b, p, (real)theta);
}

/* ---------------------------------------------------------------- kNN */

typedef struct { double d2; int32_t idx; } dkey;

static int cmp_dkey(const void *pa, const void *pb) {
  const dkey *a = (const dkey *)pa, *b = (const dkey *)pb;
  if (a->d2 < b->d2) return -1;
  if (a->d2 > b->d2) return 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

/* M nearest design points of each predictive location, in (d2, index) order
 * (Sec. 3 intro: NN sub-design; Sec. 6: search restricted to the nearest N').
 * cand: T x M int32 (0-based design indices).  d2out: T x M or NULL. */
int orc_knn(const double *X, int64_t N, int32_t p, const double *XX, int64_t T,
            int32_t M, int32_t *cand, double *d2out, int32_t nthreads) {
  if (N < 1 || p < 1 || T < 0 || M < 1 || M > N) return LAGP_ORC_INVALID;
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    dkey *keys = (dkey *)malloc((size_t)N * sizeof(dkey));
    if (!keys) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < T; t++) {
      if (!keys) continue;
      const double *x = XX + t * p;
      for (int64_t i = 0; i < N; i++) {
        keys[i].d2 = sqdist_d(x, X + i * p, p);
        keys[i].idx = (int32_t)i;
      }
      qsort(keys, (size_t)N, sizeof(dkey), cmp_dkey);
      for (int32_t m = 0; m < M; m++) {
        cand[t * M + m] = keys[m].idx;
        if (d2out) d2out[t * M + m] = keys[m].d2;
      }
    }
    free(keys);
  }
  return err ? LAGP_ORC_OOM : LAGP_ORC_OK;
}

/* ---------------------------------------------------------------- dense linear algebra */

/* Cholesky K = L L^T, row by row; L lower triangular, row-major j x j (upper part
 * zeroed).  Returns LAGP_ORC_NOT_PD if a pivot is <= 0. */
static int chol_r(const real *K, int j, real *L) {
  for (int i = 0; i < j * j; i++) L[i] = 0;
  for (int i = 0; i < j; i++) {
    for (int k = 0; k < i; k++) {
      real t = K[i * j + k];
      for (int m = 0; m < k; m++) t = t - L[i * j + m] * L[k * j + m];
      L[i * j + k] = t / L[k * j + k];
    }
    real t = K[i * j + i];
    for (int m = 0; m < i; m++) t = t - L[i * j + m] * L[i * j + m];
    if (!(t > 0)) return LAGP_ORC_NOT_PD;
    L[i * j + i] = R_SQRT(t);
  }
  return LAGP_ORC_OK;
}

/* u = L^{-1} b by forward substitution. */
static void fwd_r(const real *L, int j, const real *b, real *u) {
  for (int i = 0; i < j; i++) {
    real t = b[i];
    for (int m = 0; m < i; m++) t = t - L[i * j + m] * u[m];
    u[i] = t / L[i * j + i];
  }
}

/* z = L^{-T} u by back substitution. */
static void bwd_r(const real *L, int j, const real *u, real *z) {
  for (int i = j - 1; i >= 0; i--) {
    real t = u[i];
    for (int m = i + 1; m < j; m++) t = t - L[m * j + i] * z[m];
    z[i] = t / L[i * j + i];
  }
}

/* Direct inverse K^{-1} = L^{-T} L^{-1}, column by column. */
static int inverse_r(const real *K, int j, real *Kinv, real *L, real *e, real *u, real *z) {
  int st = chol_r(K, j, L);
  if (st) return st;
  for (int c = 0; c < j; c++) {
    for (int i = 0; i < j; i++) e[i] = (i == c) ? 1 : 0;
    fwd_r(L, j, e, u);
    bwd_r(L, j, u, z);
    for (int i = 0; i < j; i++) Kinv[i * j + c] = z[i];
  }
  return LAGP_ORC_OK;
}

int orc_chol(const double *K, int32_t j, double *Lout) {
  real *Kr = (real *)malloc(sizeof(real) * j * j), *L = (real *)malloc(sizeof(real) * j * j);
  if (!Kr || !L) { free(Kr); free(L); return LAGP_ORC_OOM; }
  for (int i = 0; i < j * j; i++) Kr[i] = K[i];
  int st = chol_r(Kr, j, L);
  for (int i = 0; i < j * j; i++) Lout[i] = (double)L[i];
  free(Kr); free(L);
  return st;
}

int orc_inverse(const double *K, int32_t j, double *Kinv) {
  size_t b = sizeof(real);
  real *Kr = malloc(b * j * j), *L = malloc(b * j * j), *Ki = malloc(b * j * j);
  real *e = malloc(b * j), *u = malloc(b * j), *z = malloc(b * j);
  int st = LAGP_ORC_OOM;
  if (Kr && L && Ki && e && u && z) {
    for (int i = 0; i < j * j; i++) Kr[i] = K[i];
    st = inverse_r(Kr, j, Ki, L, e, u, z);
    for (int i = 0; i < j * j; i++) Kinv[i] = (double)Ki[i];
  }
  free(Kr); free(L); free(Ki); free(e); free(u); free(z);
  return st;
}

/* Partitioned inverse (SM Sec. 1, Barnett): from K_j^{-1} (j x j), the new column
 * k = k_j(x_{j+1}) and kss = K(x_{j+1}, x_{j+1}), form the (j+1) x (j+1) inverse
 *   [K^{-1} + g g^T v, g; g^T, 1/v], g = -K^{-1} k / v, v = kss - k^T K^{-1} k.
 * This is the update the paper uses between greedy steps (Sec. 3.2); the oracle
 * itself never uses it, the tests compare it with the direct inverse. */
int orc_pinv_update(const double *Kinv, int32_t j, const double *k, double kss, double *out) {
  int j1 = j + 1;
  real *Kk = (real *)malloc(sizeof(real) * (j > 0 ? j : 1));
  if (!Kk) return LAGP_ORC_OOM;
  real v = kss;
  for (int a = 0; a < j; a++) {
    real t = 0;
    for (int b = 0; b < j; b++) t += (real)Kinv[a * j + b] * k[b];
    Kk[a] = t;
  }
  for (int a = 0; a < j; a++) v -= (real)k[a] * Kk[a];
  if (!(v > 0)) { free(Kk); return LAGP_ORC_NOT_PD; }
  for (int a = 0; a < j; a++) {
    real ga = -Kk[a] / v;
    for (int b = 0; b < j; b++) {
      real gb = -Kk[b] / v;
      out[a * j1 + b] = (double)((real)Kinv[a * j + b] + ga * gb * v);
    }
    out[a * j1 + j] = (double)ga;
    out[j * j1 + a] = (double)ga;
  }
  out[j * j1 + j] = (double)(1 / v);
  free(Kk);
  return LAGP_ORC_OK;
}

/* ---------------------------------------------------------------- local design */

typedef struct {
  const double *X, *Z;
  int64_t N;
  int p;
  real theta, g;
} prob_t;

/* Workspace for one location; sizes for a design of at most n points and M candidates. */
typedef struct {
  int n, M;
  real *Kc;    /* n x M: K(design member i, candidate c); row i filled when i joins */
  real *K, *L; /* n x n */
  real *Ki;    /* n x n explicit inverse (MSPE) */
  real *Kd, *Kdd; /* n x n derivative matrices (MSPE) */
  real *tmp_nn;   /* n x n */
  real *kx, *ux, *u, *b, *e, *z, *y, *yt, *w, *kdx, *kdw, *Kinv_kdw, *ud, *q, *r;
  real *kcol;
  int32_t *dr;   /* ranks of design members, in selection order */
  char *used;    /* M flags */
} work_t;

static void work_free(work_t *W) {
  free(W->Kc); free(W->K); free(W->L); free(W->Ki); free(W->Kd); free(W->Kdd); free(W->tmp_nn);
  free(W->kx); free(W->ux); free(W->u); free(W->b); free(W->e); free(W->z); free(W->y);
  free(W->yt); free(W->w); free(W->kdx); free(W->kdw); free(W->Kinv_kdw); free(W->ud);
  free(W->q); free(W->r); free(W->kcol); free(W->dr); free(W->used);
  memset(W, 0, sizeof(*W));
}

static int work_alloc(work_t *W, int n, int M) {
  memset(W, 0, sizeof(*W));
  W->n = n; W->M = M;
  size_t b = sizeof(real), nn = (size_t)n * n;
  W->Kc = malloc(b * (size_t)n * M);
  W->K = malloc(b * nn); W->L = malloc(b * nn); W->Ki = malloc(b * nn);
  W->Kd = malloc(b * nn); W->Kdd = malloc(b * nn); W->tmp_nn = malloc(b * nn);
  W->kx = malloc(b * (size_t)M);
  W->ux = malloc(b * n); W->u = malloc(b * n); W->b = malloc(b * n); W->e = malloc(b * n);
  W->z = malloc(b * n); W->y = malloc(b * n); W->yt = malloc(b * n); W->w = malloc(b * n);
  W->kdx = malloc(b * n); W->kdw = malloc(b * n); W->Kinv_kdw = malloc(b * n);
  W->ud = malloc(b * n); W->q = malloc(b * n); W->r = malloc(b * n); W->kcol = malloc(b * n);
  W->dr = malloc(sizeof(int32_t) * n); W->used = malloc((size_t)M);
  if (!W->Kc || !W->K || !W->L || !W->Ki || !W->Kd || !W->Kdd || !W->tmp_nn || !W->kx ||
      !W->ux || !W->u || !W->b || !W->e || !W->z || !W->y || !W->yt || !W->w || !W->kdx ||
      !W->kdw || !W->Kinv_kdw || !W->ud || !W->q || !W->r || !W->kcol || !W->dr || !W->used) {
    work_free(W);
    return LAGP_ORC_OOM;
  }
  return LAGP_ORC_OK;
}

static const double *cand_pt(const prob_t *P, const int32_t *cand, int c) {
  return P->X + (int64_t)cand[c] * P->p;
}

/* K_j from the definition: K(X_j, X_j) + g I, members given by their ranks. */
static void build_K(const prob_t *P, work_t *W, int j) {
  for (int a = 0; a < j; a++)
    for (int b = 0; b < j; b++)
      W->K[a * j + b] = (a == b) ? 1 + P->g : W->Kc[(size_t)a * W->M + W->dr[b]];
}

/* Row i of Kc: correlations of design member i (rank dr[i]) with every candidate;
 * the member's own column gets 1+g (identical index). */
static void fill_Kc_row(const prob_t *P, work_t *W, const int32_t *cand, int i) {
  const double *s = cand_pt(P, cand, W->dr[i]);
  for (int c = 0; c < W->M; c++)
    W->Kc[(size_t)i * W->M + c] =
        (c == W->dr[i]) ? 1 + P->g : corr_r(s, cand_pt(P, cand, c), P->p, P->theta);
}

/* Quantities of the MSPE criterion that do not depend on the candidate (Sec. 3.1,
 * SM Sec. 2), all at the fixed theta: K_j^{-1} (direct), w = K^{-1} Y, psi = Y^T w,
 * Kd = dK/dtheta, Kdd = d^2K/dtheta^2 (zero diagonal: identical arguments do not
 * depend on theta), F_j = -l''(Y_j) (Eq. d2l with N -> j), dmu_x (derivative of the
 * predictive mean at x), wKdw = w^T Kd w and Kinv_kdw = K^{-1} (Kd w). */
typedef struct { real psi, F, dmu_x, wKdw; } mspe_step_t;

static int mspe_prepare(const prob_t *P, work_t *W, const int32_t *cand, const double *x,
                        int j, mspe_step_t *S) {
  real th = P->theta;
  int st = inverse_r(W->K, j, W->Ki, W->tmp_nn, W->e, W->u, W->z);
  if (st) return st;
  for (int a = 0; a < j; a++) W->y[a] = P->Z[cand[W->dr[a]]];
  for (int a = 0; a < j; a++) {
    const double *xa = cand_pt(P, cand, W->dr[a]);
    for (int b = 0; b < j; b++) {
      if (a == b) { W->Kd[a * j + b] = 0; W->Kdd[a * j + b] = 0; continue; }
      const double *xb = cand_pt(P, cand, W->dr[b]);
      real r2 = sqdist_r(xa, xb, P->p);
      real kab = W->K[a * j + b];
      W->Kd[a * j + b] = kab * r2 / (th * th);
      W->Kdd[a * j + b] = kab * (r2 * r2 / (th * th * th * th) - 2 * r2 / (th * th * th));
    }
  }
  /* w, psi */
  real psi = 0;
  for (int a = 0; a < j; a++) {
    real t = 0;
    for (int b = 0; b < j; b++) t += W->Ki[a * j + b] * W->y[b];
    W->w[a] = t;
  }
  for (int a = 0; a < j; a++) psi += W->y[a] * W->w[a];
  /* kdw = Kd w ; wKdw ; Kinv_kdw */
  real wKdw = 0, wKddw = 0, q2 = 0;
  for (int a = 0; a < j; a++) {
    real t = 0, t2 = 0;
    for (int b = 0; b < j; b++) { t += W->Kd[a * j + b] * W->w[b]; t2 += W->Kdd[a * j + b] * W->w[b]; }
    W->kdw[a] = t;
    wKdw += W->w[a] * t;
    wKddw += W->w[a] * t2;
  }
  for (int a = 0; a < j; a++) {
    real t = 0;
    for (int b = 0; b < j; b++) t += W->Ki[a * j + b] * W->kdw[b];
    W->Kinv_kdw[a] = t;
  }
  for (int a = 0; a < j; a++) q2 += W->kdw[a] * W->Kinv_kdw[a];
  /* traces: tr(K^{-1} Kdd), tr(K^{-1} Kd K^{-1} Kd) via A = K^{-1} Kd */
  real tr1 = 0, tr2 = 0;
  for (int a = 0; a < j; a++)
    for (int b = 0; b < j; b++) tr1 += W->Ki[a * j + b] * W->Kdd[b * j + a];
  for (int a = 0; a < j; a++)
    for (int b = 0; b < j; b++) {
      real t = 0;
      for (int m = 0; m < j; m++) t += W->Ki[a * j + m] * W->Kd[m * j + b];
      W->tmp_nn[a * j + b] = t;
    }
  for (int a = 0; a < j; a++)
    for (int b = 0; b < j; b++) tr2 += W->tmp_nn[a * j + b] * W->tmp_nn[b * j + a];
  real dj = (real)j;
  /* Eq. d2l: l'' = -1/2 tr{K^-1 [Kdd - Kd K^-1 Kd]} + j/(2 psi) Y^T K^-1 [Kdd - 2 Kd K^-1 Kd] K^-1 Y
   *               + j/(2 psi^2) [Y^T K^-1 Kd K^-1 Y]^2 */
  real l2 = -0.5 * (tr1 - tr2) + dj / (2 * psi) * (wKddw - 2 * q2) + dj / (2 * psi * psi) * wKdw * wKdw;
  /* derivative of the predictive mean at x: kd(x)^T w - ktilde^T Kd w, ktilde = K^{-1} k(x) */
  real dmu = 0;
  for (int a = 0; a < j; a++) {
    const double *xa = cand_pt(P, cand, W->dr[a]);
    real r2 = sqdist_r(x, xa, P->p);
    real kxa = R_EXP(-r2 / th);
    W->kdx[a] = kxa * r2 / (th * th);
    W->b[a] = kxa;
  }
  for (int a = 0; a < j; a++) {
    real kt = 0;
    for (int b = 0; b < j; b++) kt += W->Ki[a * j + b] * W->b[b];
    dmu += W->kdx[a] * W->w[a] - kt * W->kdw[a];
  }
  S->psi = psi;
  S->F = -l2;
  S->dmu_x = dmu;
  S->wKdw = wKdw;
  return LAGP_ORC_OK;
}

/* One location: greedy local design and predictive equations.
 * cand: the M nearest (rank order).  forced: n design indices or NULL.
 * idx_out: n design indices.  trace: (n-n0) x TRACE_W or NULL. */
static int local_design(const prob_t *P, work_t *W, const double *x, const int32_t *cand,
                        int n0, int n, int method, const int32_t *forced, const int32_t *start,
                        real r_min, int32_t *n_out, int32_t *idx_out, double *mean, double *s2,
                        double *var, double *trace) {
  int M = W->M;
  const int n_alloc = n;  /* idx_out's length; n shrinks if the stopping rule ends early */
  real onepg = 1 + P->g;
  memset(W->used, 0, (size_t)M);
  for (int c = 0; c < M; c++) W->kx[c] = corr_r(x, cand_pt(P, cand, c), P->p, P->theta);
  /* the start design: the n0 nearest, or the saved design start[0..n0) (Sec. 6) */
  for (int i = 0; i < n0; i++) {
    int r = i;
    if (start) {
      r = -1;
      for (int c = 0; c < M; c++)
        if (cand[c] == start[i]) { r = c; break; }
      if (r < 0 || W->used[r]) return LAGP_ORC_INVALID;
    }
    W->dr[i] = r;
    W->used[r] = 1;
    fill_Kc_row(P, W, cand, i);
  }
  for (int j = n0; j < n; j++) {
    build_K(P, W, j);
    int st = chol_r(W->K, j, W->L);
    if (st) return st;
    /* u_x = L^{-1} k_j(x);  v_j(x) = K(x,x) - ||u_x||^2 */
    for (int a = 0; a < j; a++) W->b[a] = W->kx[W->dr[a]];
    fwd_r(W->L, j, W->b, W->ux);
    real vx = onepg;
    for (int a = 0; a < j; a++) vx = vx - W->ux[a] * W->ux[a];
    mspe_step_t S = {0, 0, 0, 0};
    if (method == ORC_MSPE || method == ORC_MSPE_NODERIV) {
      st = mspe_prepare(P, W, cand, x, j, &S);
      if (st) return st;
    }
    int best = -1, forced_rank = -1;
    real best_s = 0, second_s = 0, forced_s = 0;
    int have_second = 0;
    int want_min = (method == ORC_MSPE || method == ORC_MSPE_NODERIV);
    if (forced) {
      for (int c = 0; c < M; c++)
        if (cand[c] == forced[j]) { forced_rank = c; break; }
      if (forced_rank < 0 || W->used[forced_rank]) return LAGP_ORC_INVALID;
    }
    for (int c = 0; c < M; c++) {
      if (W->used[c]) continue;
      real score;
      if (method == ORC_NN) {
        score = -(real)c; /* nearest remaining rank wins */
      } else {
        for (int a = 0; a < j; a++) W->kcol[a] = W->Kc[(size_t)a * M + c];
        fwd_r(W->L, j, W->kcol, W->u);
        real vc = onepg;
        for (int a = 0; a < j; a++) vc = vc - W->u[a] * W->u[a];
        if (!(vc > 0)) continue;
        real cov = W->kx[c];
        for (int a = 0; a < j; a++) cov = cov - W->ux[a] * W->u[a];
        real alc = cov * cov / vc; /* v_j(x) - v_{j+1}(x), Eq. dxy = SM Eq. dxy2 */
        if (method == ORC_ALC) {
          score = alc;
        } else {
          /* MSPE (Eq. mspe): J = psi/(j-2) v_{j+1}(x) + dmu_x^2 / G_{j+1}(c) */
          real dj2 = (real)(j - 2);
          real Vred = S.psi / dj2 * (vx - alc);
          if (method == ORC_MSPE_NODERIV) {
            score = Vred;
          } else {
            const double *xc = cand_pt(P, cand, c);
            /* z_c = K^{-1} k_c; kd_c = dk_c/dtheta */
            for (int a = 0; a < j; a++) {
              real t = 0;
              for (int b2 = 0; b2 < j; b2++) t += W->Ki[a * j + b2] * W->kcol[b2];
              W->z[a] = t;
              const double *xa = cand_pt(P, cand, W->dr[a]);
              real r2 = sqdist_r(xc, xa, P->p);
              W->ud[a] = W->kcol[a] * r2 / (P->theta * P->theta);
            }
            /* dmu_c = kd_c^T w - z_c^T Kd w   (SM Eqs. dz, dmu) */
            real dmu_c = 0, kdz = 0, zKdz = 0;
            for (int a = 0; a < j; a++) {
              dmu_c += W->ud[a] * W->w[a] - W->z[a] * W->kdw[a];
              kdz += W->ud[a] * W->z[a];
            }
            for (int a = 0; a < j; a++) {
              real t = 0;
              for (int b2 = 0; b2 < j; b2++) t += W->Kd[a * j + b2] * W->z[b2];
              zKdz += W->z[a] * t;
            }
            real Vc = S.psi * vc / dj2;
            /* SM Eq. dV: dV = [Y^T dw v - psi (kd^T z + k^T dz)]/(j-2), Y^T dw = -w^T Kd w,
             * k^T dz = kd^T z - z^T Kd z */
            real dVc = (-S.wKdw * vc - S.psi * (2 * kdz - zKdz)) / dj2;
            /* Eq. G with SM Eq. Ed2la */
            real G = S.F + dVc * dVc / (2 * Vc * Vc) + dmu_c * dmu_c / Vc;
            score = Vred + S.dmu_x * S.dmu_x / G;
          }
        }
      }
      if (c == forced_rank) forced_s = score;
      if (score != score) continue;  /* a criterion that evaluates to NaN is not admissible */
      if (best < 0) {
        best = c; best_s = score;
      } else {
        int better = want_min ? (score < best_s) : (score > best_s);
        if (better) {
          second_s = best_s; have_second = 1;
          best = c; best_s = score;
        } else if (!have_second || (want_min ? score < second_s : score > second_s)) {
          second_s = score; have_second = 1;
        }
      }
    }
    if (best < 0) return LAGP_ORC_NOT_PD;
    int chosen = forced ? forced_rank : best;
    /* Sec. 6 stopping rule: v_j(x) / v_{j+1}(x), the chosen point's variance reduction
     * ratio (psi cancels); the design stops before a point whose ratio is below r_min */
    const real chosen_s = forced ? forced_s : best_s;
    const real ratio = (method == ORC_ALC) ? vx / (vx - chosen_s) : NAN;
    if (trace) {
      double *tr = trace + (size_t)(j - n0) * TRACE_W;
      tr[0] = best; tr[1] = (double)best_s; tr[2] = chosen;
      tr[3] = (double)chosen_s;
      tr[4] = have_second ? (double)second_s : NAN;
      tr[5] = (double)vx;
      tr[6] = (double)ratio;
    }
    if (r_min > 0 && !forced && ratio < r_min) {
      n = j;
      break;
    }
    W->dr[j] = chosen;
    W->used[chosen] = 1;
    fill_Kc_row(P, W, cand, j);
  }
  /* Predictive equations on D_n (Eqs. predgp, preds2): with K_n = L L^T,
   * mu = (L^{-1} k(x)) . (L^{-1} Y), psi = ||L^{-1} Y||^2, v = K(x,x) - ||L^{-1} k(x)||^2,
   * s2 = psi v / n, V = s2 n/(n-2). */
  build_K(P, W, n);
  int st = chol_r(W->K, n, W->L);
  if (st) return st;
  for (int a = 0; a < n; a++) {
    W->b[a] = W->kx[W->dr[a]];
    W->y[a] = P->Z[cand[W->dr[a]]];
  }
  fwd_r(W->L, n, W->b, W->ux);
  fwd_r(W->L, n, W->y, W->yt);
  real mu = 0, psi = 0, vx = onepg;
  for (int a = 0; a < n; a++) {
    mu += W->ux[a] * W->yt[a];
    psi += W->yt[a] * W->yt[a];
    vx = vx - W->ux[a] * W->ux[a];
  }
  for (int a = 0; a < n; a++) idx_out[a] = cand[W->dr[a]];
  for (int a = n; a < n_alloc; a++) idx_out[a] = -1;
  if (n_out) *n_out = n;
  *mean = (double)mu;
  *s2 = (double)(psi * vx / n);
  *var = (double)(psi * vx / (n - 2));
  return LAGP_ORC_OK;
}

static int check_args(int64_t N, int32_t p, int64_t T, int32_t n0, int32_t n, int32_t M,
                      double theta, double g, int32_t method) {
  if (N < 1 || p < 1 || T < 0) return LAGP_ORC_INVALID;
  if (n0 < 1 || n < n0 || n < 3 || M < n || (int64_t)M > N) return LAGP_ORC_INVALID;
  if (!(theta > 0) || !(g >= 0)) return LAGP_ORC_INVALID;
  if (method < 0 || method > 3) return LAGP_ORC_INVALID;
  if ((method == ORC_MSPE || method == ORC_MSPE_NODERIV) && n0 < 3) return LAGP_ORC_INVALID;
  return LAGP_ORC_OK;
}

/* One location with a given candidate list (rank order).  forced may be NULL. */
int orc_local_design(const double *X, const double *Z, int64_t N, int32_t p, const double *x,
                     const int32_t *cand, int32_t M, int32_t n0, int32_t n, double theta,
                     double g, int32_t method, const int32_t *forced, int32_t *idx,
                     double *mean, double *s2, double *var, double *trace) {
  int st = check_args(N, p, 1, n0, n, M, theta, g, method);
  if (st) return st;
  prob_t P = {X, Z, N, p, (real)theta, (real)g};
  work_t W;
  if (work_alloc(&W, n, M)) return LAGP_ORC_OOM;
  st = local_design(&P, &W, x, cand, n0, n, method, forced, NULL, 0, NULL, idx, mean, s2, var,
                    trace);
  work_free(&W);
  return st;
}

/* orc_local_design grown from a saved start design (Sec. 6, "picking up where they left
 * off"): the first n1 members are start[0..n1) (design indices, each one of the location's
 * candidates), then greedy steps to n.  LAGP_ORC_INVALID if a start index is not a
 * candidate or repeats. */
int orc_local_design_start(const double *X, const double *Z, int64_t N, int32_t p,
                           const double *x, const int32_t *cand, int32_t M, const int32_t *start,
                           int32_t n1, int32_t n, double theta, double g, int32_t method,
                           const int32_t *forced, int32_t *idx, double *mean, double *s2,
                           double *var, double *trace) {
  int st = check_args(N, p, 1, n1, n, M, theta, g, method);
  if (st) return st;
  prob_t P = {X, Z, N, p, (real)theta, (real)g};
  work_t W;
  if (work_alloc(&W, n, M)) return LAGP_ORC_OOM;
  st = local_design(&P, &W, x, cand, n1, n, method, forced, start, 0, NULL, idx, mean, s2, var,
                    trace);
  work_free(&W);
  return st;
}

/* orc_local_design with the stopping rule of Sec. 6 (ALC): the design stops growing
 * before the first greedy point whose variance-reduction ratio v_j(x) / v_{j+1}(x) is
 * below r_min (> 1), and at n at the latest; *n_out gets its size, idx the n_out indices
 * followed by -1.  With forced, the path is replayed in full and only traced (field 6
 * of each trace row is the ratio). */
int orc_local_design_adaptive(const double *X, const double *Z, int64_t N, int32_t p,
                              const double *x, const int32_t *cand, int32_t M, int32_t n0,
                              int32_t n, double theta, double g, double r_min,
                              const int32_t *forced, int32_t *idx, double *mean, double *s2,
                              double *var, double *trace, int32_t *n_out) {
  int st = check_args(N, p, 1, n0, n, M, theta, g, ORC_ALC);
  if (st) return st;
  if (n0 < 3 || !(r_min > 1)) return LAGP_ORC_INVALID;
  prob_t P = {X, Z, N, p, (real)theta, (real)g};
  work_t W;
  if (work_alloc(&W, n, M)) return LAGP_ORC_OOM;
  st = local_design(&P, &W, x, cand, n0, n, ORC_ALC, forced, NULL, (real)r_min, n_out, idx, mean,
                    s2, var, trace);
  work_free(&W);
  return st;
}

/* Whole predictive set: kNN then local design per location (Sec. 4: independent
 * problems, one parallel loop over locations).  status[t] = 0 or a negative code;
 * failed locations get NaN outputs.  cand_out (T x M) may be NULL. */
int orc_predict(const double *X, const double *Z, int64_t N, int32_t p, const double *XX,
                int64_t T, int32_t n0, int32_t n, int32_t M, double theta, double g,
                int32_t method, int32_t *idx, double *mean, double *s2, double *var,
                int32_t *status, int32_t *cand_out, int32_t nthreads) {
  int st = check_args(N, p, T, n0, n, M, theta, g, method);
  if (st) return st;
  if (T == 0) return LAGP_ORC_OK;
  int32_t *cand = cand_out ? cand_out : (int32_t *)malloc(sizeof(int32_t) * (size_t)T * M);
  if (!cand) return LAGP_ORC_OOM;
  st = orc_knn(X, N, p, XX, T, M, cand, NULL, nthreads);
  if (st) { if (!cand_out) free(cand); return st; }
  prob_t P = {X, Z, N, p, (real)theta, (real)g};
  int err = 0;
#pragma omp parallel
  {
    work_t W;
    int ok = (work_alloc(&W, n, M) == LAGP_ORC_OK);
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < T; t++) {
      if (!ok) continue;
      int s = local_design(&P, &W, XX + t * p, cand + t * M, n0, n, method, NULL, NULL, 0, NULL,
                           idx + t * n, mean + t, s2 + t, var + t, NULL);
      status[t] = s;
      if (s) { mean[t] = NAN; s2[t] = NAN; var[t] = NAN; }
    }
    if (ok) work_free(&W);
  }
  if (!cand_out) free(cand);
  return err ? LAGP_ORC_OOM : LAGP_ORC_OK;
}

/* Predictive equations (Eqs. predgp, preds2) at x on a given design (n design indices):
 * builds K_n, factors it and returns out = {mean, s2, var}.  Used, in the long-double
 * build, to adjudicate rounding differences along a fixed design. */
int orc_design_predict(const double *X, const double *Z, int64_t N, int32_t p, const double *x,
                       const int32_t *idx, int32_t n, double theta, double g, double *out) {
  if (n < 3 || N < 1) return LAGP_ORC_INVALID;
  for (int a = 0; a < n; a++)
    if (idx[a] < 0 || idx[a] >= N) return LAGP_ORC_INVALID;
  size_t b = sizeof(real);
  real *K = malloc(b * n * n), *L = malloc(b * n * n), *kx = malloc(b * n), *y = malloc(b * n);
  real *ux = malloc(b * n), *yt = malloc(b * n);
  int st = LAGP_ORC_OOM;
  if (K && L && kx && y && ux && yt) {
    for (int a = 0; a < n; a++) {
      const double *xa = X + (int64_t)idx[a] * p;
      for (int c = 0; c < n; c++)
        K[a * n + c] = (a == c) ? 1 + (real)g : corr_r(xa, X + (int64_t)idx[c] * p, p, theta);
      kx[a] = corr_r(x, xa, p, theta);
      y[a] = Z[idx[a]];
    }
    st = chol_r(K, n, L);
    if (!st) {
      fwd_r(L, n, kx, ux);
      fwd_r(L, n, y, yt);
      real mu = 0, psi = 0, v = 1 + (real)g;
      for (int a = 0; a < n; a++) {
        mu += ux[a] * yt[a];
        psi += yt[a] * yt[a];
        v = v - ux[a] * ux[a];
      }
      out[0] = (double)mu;
      out[1] = (double)(psi * v / n);
      out[2] = (double)(psi * v / (n - 2));
    }
  }
  free(K); free(L); free(kx); free(y); free(ux); free(yt);
  return st;
}

/* Full GP at x on the whole design (Eqs. predgp, preds2 with all N points): the
 * special case the local predictor reaches when n = N. */
int orc_full_gp(const double *X, const double *Z, int64_t N, int32_t p, const double *x,
                double theta, double g, double *mean, double *s2) {
  if (N < 1 || N > 20000) return LAGP_ORC_INVALID;
  int n = (int)N;
  size_t b = sizeof(real);
  real *K = malloc(b * n * n), *L = malloc(b * n * n), *kx = malloc(b * n), *y = malloc(b * n);
  real *ux = malloc(b * n), *yt = malloc(b * n);
  int st = LAGP_ORC_OOM;
  if (K && L && kx && y && ux && yt) {
    for (int a = 0; a < n; a++) {
      for (int c = 0; c < n; c++)
        K[a * n + c] = (a == c) ? 1 + (real)g : corr_r(X + (int64_t)a * p, X + (int64_t)c * p, p, theta);
      kx[a] = corr_r(x, X + (int64_t)a * p, p, theta);
      y[a] = Z[a];
    }
    st = chol_r(K, n, L);
    if (!st) {
      fwd_r(L, n, kx, ux);
      fwd_r(L, n, y, yt);
      real mu = 0, psi = 0, v = 1 + (real)g;
      for (int a = 0; a < n; a++) { mu += ux[a] * yt[a]; psi += yt[a] * yt[a]; v = v - ux[a] * ux[a]; }
      *mean = (double)mu;
      *s2 = (double)(psi * v / n);
    }
  }
  free(K); free(L); free(kx); free(y); free(ux); free(yt);
  return st;
}

/* ---------------------------------------------------------------- pieces for the pins */

/* Log marginal likelihood and its theta derivatives on a design (Eqs. gpk, dl, d2l):
 * out[0] = log p(Y|K) without the Gamma/(2 pi) constant, i.e. -1/2 log|K| - N/2 log(psi/2),
 * out[1] = l'(theta), out[2] = l''(theta). */
int orc_loglik(const double *Xd, const double *Y, int32_t j, int32_t p, double theta, double g,
               double *out) {
  if (j < 1) return LAGP_ORC_INVALID;
  size_t b = sizeof(real);
  real th = theta;
  real *K = malloc(b * j * j), *L = malloc(b * j * j), *Ki = malloc(b * j * j);
  real *Kd = malloc(b * j * j), *Kdd = malloc(b * j * j), *A = malloc(b * j * j);
  real *e = malloc(b * j), *u = malloc(b * j), *z = malloc(b * j), *w = malloc(b * j);
  real *kdw = malloc(b * j), *kikdw = malloc(b * j);
  int st = LAGP_ORC_OOM;
  if (K && L && Ki && Kd && Kdd && A && e && u && z && w && kdw && kikdw) {
    for (int a = 0; a < j; a++)
      for (int c = 0; c < j; c++) {
        if (a == c) { K[a * j + c] = 1 + (real)g; Kd[a * j + c] = 0; Kdd[a * j + c] = 0; continue; }
        real r2 = sqdist_r(Xd + (int64_t)a * p, Xd + (int64_t)c * p, p);
        real k = R_EXP(-r2 / th);
        K[a * j + c] = k;
        Kd[a * j + c] = k * r2 / (th * th);
        Kdd[a * j + c] = k * (r2 * r2 / (th * th * th * th) - 2 * r2 / (th * th * th));
      }
    st = inverse_r(K, j, Ki, L, e, u, z);
    if (!st) {
      real logdet = 0, psi = 0, q3 = 0, q1 = 0, q2 = 0, tr1 = 0, tr2 = 0, tr0 = 0;
      for (int a = 0; a < j; a++) logdet += 2 * R_LOG(L[a * j + a]);
      for (int a = 0; a < j; a++) {
        real t = 0;
        for (int c = 0; c < j; c++) t += Ki[a * j + c] * Y[c];
        w[a] = t;
      }
      for (int a = 0; a < j; a++) psi += Y[a] * w[a];
      for (int a = 0; a < j; a++) {
        real t = 0, t2 = 0;
        for (int c = 0; c < j; c++) { t += Kd[a * j + c] * w[c]; t2 += Kdd[a * j + c] * w[c]; }
        kdw[a] = t; q3 += w[a] * t; q1 += w[a] * t2;
      }
      for (int a = 0; a < j; a++) {
        real t = 0;
        for (int c = 0; c < j; c++) t += Ki[a * j + c] * kdw[c];
        kikdw[a] = t;
      }
      for (int a = 0; a < j; a++) q2 += kdw[a] * kikdw[a];
      for (int a = 0; a < j; a++)
        for (int c = 0; c < j; c++) {
          tr0 += Ki[a * j + c] * Kd[c * j + a];
          tr1 += Ki[a * j + c] * Kdd[c * j + a];
          real t = 0;
          for (int m = 0; m < j; m++) t += Ki[a * j + m] * Kd[m * j + c];
          A[a * j + c] = t;
        }
      for (int a = 0; a < j; a++)
        for (int c = 0; c < j; c++) tr2 += A[a * j + c] * A[c * j + a];
      real dj = j;
      out[0] = (double)(-0.5 * logdet - dj / 2 * R_LOG(psi / 2));
      out[1] = (double)(-0.5 * tr0 + dj / 2 * q3 / psi);
      out[2] = (double)(-0.5 * (tr1 - tr2) + dj / (2 * psi) * (q1 - 2 * q2) + dj / (2 * psi * psi) * q3 * q3);
    }
  }
  free(K); free(L); free(Ki); free(Kd); free(Kdd); free(A); free(e); free(u); free(z); free(w);
  free(kdw); free(kikdw);
  return st;
}

/* Local maximum-likelihood lengthscale (Sec. 4.2, step 3): the theta in [tmin, tmax]
 * maximising the log likelihood Eq. gpk of the design given by idx (n rows of X and Z),
 * by Newton's method on l'(theta) = 0 with the analytic derivatives Eqs. dl, d2l
 * (Sec. 3.2 names Newton-like methods; the safeguards are this oracle's reading):
 *   - a bracket [a, b] is kept in which the maximum lies: l' > 0 at a (the likelihood
 *     still increases there), l' < 0 at b; each iterate narrows it by the sign of l';
 *   - the Newton step theta - l'/l'' is taken when l'' < 0 and it lands strictly inside
 *     (a, b); otherwise the next iterate is the end of [tmin, tmax] uphill of theta (the
 *     side l' points to) if that end has not been evaluated yet, else the bracket's
 *     midpoint;
 *   - it stops when a step is at most tol * theta (returning the new point), when l' = 0,
 *     or at an end of [tmin, tmax] where l' points outward (the maximum on the boundary).
 * *theta_out gets the estimate, *iters_out the number of derivative evaluations.
 * Returns LAGP_ORC_OK, LAGP_ORC_NOT_PD (K_n not positive definite), LAGP_ORC_NO_CONV
 * (maxit evaluations without meeting the stopping rule; the last iterate is returned)
 * or LAGP_ORC_INVALID. */
int orc_mle(const double *X, const double *Z, int64_t N, int32_t p, const int32_t *idx, int32_t n,
            double theta0, double g, double tmin, double tmax, int32_t maxit, double tol,
            double *theta_out, int32_t *iters_out) {
  if (n < 2 || p < 1 || !(tmin > 0) || !(tmax > tmin) || maxit < 1 || !(tol > 0))
    return LAGP_ORC_INVALID;
  for (int a = 0; a < n; a++)
    if (idx[a] < 0 || idx[a] >= N) return LAGP_ORC_INVALID;
  double *Xd = malloc(sizeof(double) * (size_t)n * p), *Y = malloc(sizeof(double) * n);
  if (!Xd || !Y) { free(Xd); free(Y); return LAGP_ORC_OOM; }
  for (int a = 0; a < n; a++) {
    for (int k = 0; k < p; k++) Xd[a * p + k] = X[(int64_t)idx[a] * p + k];
    Y[a] = Z[idx[a]];
  }
  double lo = tmin, hi = tmax;
  double th = theta0 < tmin ? tmin : (theta0 > tmax ? tmax : theta0);
  int lo_open = 1, hi_open = 1;  /* the ends of [tmin, tmax] not yet evaluated */
  int st = LAGP_ORC_NO_CONV, it = 0;
  double l[3];
  while (it < maxit) {
    it++;
    int e = orc_loglik(Xd, Y, n, p, th, g, l);
    if (e) { st = e; break; }
    const double d1 = l[1], d2 = l[2];
    if (d1 == 0) { st = LAGP_ORC_OK; break; }
    if (d1 > 0) {
      lo = th; lo_open = 0;
      if (th >= tmax) { st = LAGP_ORC_OK; break; }
    } else {
      hi = th; hi_open = 0;
      if (th <= tmin) { st = LAGP_ORC_OK; break; }
    }
    double tn = (d2 < 0) ? th - d1 / d2 : NAN;
    if (!(tn > lo && tn < hi)) {
      if (d1 > 0 && hi_open) tn = hi;         /* uphill to an end not yet evaluated */
      else if (d1 < 0 && lo_open) tn = lo;
      else tn = 0.5 * (lo + hi);
    }
    const int done = fabs(tn - th) <= tol * th;
    th = tn;
    if (done) { st = LAGP_ORC_OK; break; }
  }
  *theta_out = th;
  *iters_out = it;
  free(Xd); free(Y);
  return st;
}

/* orc_mle for T designs (idx: T x n), starting values theta0[t]; OpenMP over designs.
 * status[t] is orc_mle's return value for design t. */
int orc_mle_batch(const double *X, const double *Z, int64_t N, int32_t p, int64_t T,
                  const int32_t *idx, int32_t n, const double *theta0, double g, double tmin,
                  double tmax, int32_t maxit, double tol, double *theta_out, int32_t *iters_out,
                  int32_t *status, int32_t nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < T; t++)
    status[t] = orc_mle(X, Z, N, p, idx + t * n, n, theta0[t], g, tmin, tmax, maxit, tol,
                        theta_out + t, iters_out + t);
  return LAGP_ORC_OK;
}

/* Predictive quantities at a point xs given design (Xd, Y) of size j, and their theta
 * derivatives (SM Sec. 2: Eqs. dKi, d2w, dz, d2z, dmu, dV, d2V):
 * out[0..5] = mu, dmu, d2mu, V, dV, d2V with V = psi v/(j-2);
 * out[6] = v (ALC-scale variance), out[7] = psi. xs must not be a design point. */
int orc_pred_derivs(const double *Xd, const double *Y, int32_t j, int32_t p, const double *xs,
                    double theta, double g, double *out) {
  if (j < 3) return LAGP_ORC_INVALID;
  size_t b = sizeof(real);
  real th = theta;
  real *K = malloc(b * j * j), *L = malloc(b * j * j), *Ki = malloc(b * j * j);
  real *Kd = malloc(b * j * j), *Kdd = malloc(b * j * j);
  real *e = malloc(b * j), *u = malloc(b * j), *zz = malloc(b * j);
  real *k = malloc(b * j), *kd = malloc(b * j), *kdd = malloc(b * j);
  real *z = malloc(b * j), *dz = malloc(b * j), *d2z = malloc(b * j);
  real *w = malloc(b * j), *dw = malloc(b * j), *d2w = malloc(b * j), *t1 = malloc(b * j);
  int st = LAGP_ORC_OOM;
  if (K && L && Ki && Kd && Kdd && e && u && zz && k && kd && kdd && z && dz && d2z && w && dw &&
      d2w && t1) {
    for (int a = 0; a < j; a++) {
      for (int c = 0; c < j; c++) {
        if (a == c) { K[a * j + c] = 1 + (real)g; Kd[a * j + c] = 0; Kdd[a * j + c] = 0; continue; }
        real r2 = sqdist_r(Xd + (int64_t)a * p, Xd + (int64_t)c * p, p);
        real kk = R_EXP(-r2 / th);
        K[a * j + c] = kk;
        Kd[a * j + c] = kk * r2 / (th * th);
        Kdd[a * j + c] = kk * (r2 * r2 / (th * th * th * th) - 2 * r2 / (th * th * th));
      }
      real r2 = sqdist_r(xs, Xd + (int64_t)a * p, p);
      real kk = R_EXP(-r2 / th);
      k[a] = kk;
      kd[a] = kk * r2 / (th * th);
      kdd[a] = kk * (r2 * r2 / (th * th * th * th) - 2 * r2 / (th * th * th));
    }
    st = inverse_r(K, j, Ki, L, e, u, zz);
    if (!st) {
#define MATVEC(M_, v_, o_) for (int a = 0; a < j; a++) { real s_ = 0; for (int c = 0; c < j; c++) s_ += M_[a * j + c] * v_[c]; o_[a] = s_; }
      MATVEC(Ki, k, z);                                   /* z = K^-1 k */
      MATVEC(Kd, z, t1);                                  /* Kd z */
      for (int a = 0; a < j; a++) t1[a] = kd[a] - t1[a];
      MATVEC(Ki, t1, dz);                                 /* dz = K^-1 (kd - Kd z)  Eq. dz */
      {
        real *a1 = e, *a2 = u;
        MATVEC(Kdd, z, a1);
        MATVEC(Kd, dz, a2);
        for (int a = 0; a < j; a++) t1[a] = kdd[a] - a1[a] - 2 * a2[a];
        MATVEC(Ki, t1, d2z);                              /* Eq. d2z */
      }
      for (int a = 0; a < j; a++) e[a] = Y[a];
      MATVEC(Ki, e, w);                                   /* w = K^-1 Y */
      MATVEC(Kd, w, t1);
      MATVEC(Ki, t1, dw);
      for (int a = 0; a < j; a++) dw[a] = -dw[a];         /* dw = -K^-1 Kd w  Eq. d2w */
      {
        real *a1 = u, *a2 = zz;
        MATVEC(Kdd, w, a1);
        MATVEC(Kd, dw, a2);
        for (int a = 0; a < j; a++) t1[a] = a1[a] + 2 * a2[a];
        MATVEC(Ki, t1, d2w);
        for (int a = 0; a < j; a++) d2w[a] = -d2w[a];     /* Eq. d2w */
      }
#undef MATVEC
      real mu = 0, dmu = 0, d2mu = 0, psi = 0, dpsi = 0, d2psi = 0, kz = 0, dv1 = 0, d2v1 = 0;
      for (int a = 0; a < j; a++) {
        mu += z[a] * Y[a];
        dmu += dz[a] * Y[a];                              /* Eq. dmu */
        d2mu += d2z[a] * Y[a];
        psi += Y[a] * w[a];
        dpsi += Y[a] * dw[a];
        d2psi += Y[a] * d2w[a];
        kz += k[a] * z[a];
        dv1 += kd[a] * z[a] + k[a] * dz[a];
        d2v1 += kdd[a] * z[a] + 2 * kd[a] * dz[a] + k[a] * d2z[a];
      }
      real v = 1 + (real)g - kz, dv = -dv1, d2v = -d2v1;
      real dj2 = (real)(j - 2);
      out[0] = (double)mu; out[1] = (double)dmu; out[2] = (double)d2mu;
      out[3] = (double)(psi * v / dj2);
      out[4] = (double)((dpsi * v + psi * dv) / dj2);               /* Eq. dV */
      out[5] = (double)((d2psi * v + 2 * dpsi * dv + psi * d2v) / dj2); /* Eq. d2V */
      out[6] = (double)v; out[7] = (double)psi;
    }
  }
  free(K); free(L); free(Ki); free(Kd); free(Kdd); free(e); free(u); free(zz); free(k); free(kd);
  free(kdd); free(z); free(dz); free(d2z); free(w); free(dw); free(d2w); free(t1);
  return st;
}

/* Second theta-derivative of the conditional log-likelihood of y_{j+1} given Y_j
 * (SM Eq. d2lx, one parameter), from the predictive quantities at x_{j+1}:
 * pd = {mu, dmu, d2mu, V, dV, d2V} as returned by orc_pred_derivs. */
double orc_d2l_conditional(const double *pd, double y, int32_t j) {
  real mu = pd[0], dmu = pd[1], d2mu = pd[2], V = pd[3], dV = pd[4], d2V = pd[5];
  real e = (real)y - mu;
  real D = (real)(j - 2) + e * e / V;
  real a = 2 * e * dmu / V + e * e * dV / (V * V);
  real da = -2 * dmu * dmu / V - (2 * e / (V * V)) * (2 * dmu * dV) + (2 * e / V) * d2mu
            - (2 * e * e / (V * V * V)) * dV * dV + (e * e / (V * V)) * d2V;
  real h = (real)(j + 1) / 2;
  return (double)(-d2V / (2 * V) + dV * dV / (2 * V * V) + h * a * a / (D * D) + h * da / D);
}

/* The three forms of the ALC reduction at x for adding candidate xc to design Xd
 * (size j):  out[0] = cov_j(x,c)^2 / v_j(c)  (SM Eq. dxy2 via partial correlations),
 * out[1] = Eq. dxy expanded with g = -K^{-1} k_j(c) / v_j(c) (the sign of SM Sec. 1),
 * out[2] = v_j(x) - v_{j+1}(x) with K_{j+1} inverted directly. */
int orc_alc_forms(const double *Xd, int32_t j, int32_t p, const double *x, const double *xc,
                  double theta, double g, double *out) {
  if (j < 1) return LAGP_ORC_INVALID;
  int j1 = j + 1;
  size_t b = sizeof(real);
  real *K = malloc(b * j1 * j1), *L = malloc(b * j1 * j1), *Ki = malloc(b * j1 * j1);
  real *e = malloc(b * j1), *u = malloc(b * j1), *z = malloc(b * j1);
  real *kx = malloc(b * j1), *kc = malloc(b * j1), *gv = malloc(b * j1);
  int st = LAGP_ORC_OOM;
  if (K && L && Ki && e && u && z && kx && kc && gv) {
    for (int a = 0; a < j; a++) {
      kx[a] = corr_r(x, Xd + (int64_t)a * p, p, theta);
      kc[a] = corr_r(xc, Xd + (int64_t)a * p, p, theta);
    }
    real kxc = corr_r(x, xc, p, theta);
    /* K_j and its direct inverse */
    for (int a = 0; a < j; a++)
      for (int c = 0; c < j; c++)
        K[a * j + c] = (a == c) ? 1 + (real)g : corr_r(Xd + (int64_t)a * p, Xd + (int64_t)c * p, p, theta);
    st = inverse_r(K, j, Ki, L, e, u, z);
    if (!st) {
      real vx = 1 + (real)g, vc = 1 + (real)g, cxc = kxc;
      for (int a = 0; a < j; a++) {
        real sx = 0, sc = 0;
        for (int c = 0; c < j; c++) { sx += Ki[a * j + c] * kx[c]; sc += Ki[a * j + c] * kc[c]; }
        vx -= kx[a] * sx;
        vc -= kc[a] * sc;
        cxc -= kx[a] * sc;
        gv[a] = -sc; /* will divide by vc below */
      }
      for (int a = 0; a < j; a++) gv[a] /= vc;
      out[0] = (double)(cxc * cxc / vc);
      /* Eq. dxy: k^T G v k + 2 k^T g K(x_{j+1},x) + K(x_{j+1},x)^2 / v, G = g g^T */
      real kg = 0;
      for (int a = 0; a < j; a++) kg += kx[a] * gv[a];
      out[1] = (double)(kg * kg * vc + 2 * kg * kxc + kxc * kxc / vc);
      /* brute force: invert K_{j+1} directly */
      for (int a = 0; a < j1; a++)
        for (int c = 0; c < j1; c++) {
          const double *pa = (a < j) ? Xd + (int64_t)a * p : xc;
          const double *pc = (c < j) ? Xd + (int64_t)c * p : xc;
          K[a * j1 + c] = (a == c) ? 1 + (real)g : corr_r(pa, pc, p, theta);
        }
      st = inverse_r(K, j1, Ki, L, u, z, gv);
      if (!st) {
        kx[j] = kxc;
        real v1 = 1 + (real)g;
        for (int a = 0; a < j1; a++) {
          real s = 0;
          for (int c = 0; c < j1; c++) s += Ki[a * j1 + c] * kx[c];
          v1 -= kx[a] * s;
        }
        out[2] = (double)(vx - v1);
      }
    }
  }
  free(K); free(L); free(Ki); free(e); free(u); free(z); free(kx); free(kc); free(gv);
  return st;
}
