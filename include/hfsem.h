/*
 * hfsem -- H-matrix-preconditioned Krylov solver for the spectral element
 * (SEM) system of the 1D two-sided Riemann-Liouville fractional diffusion
 * equation, for NVIDIA GB300 (sm_103a).
 *
 *   -D^2( theta aI_x^{2-alpha} u + (1-theta) xI_b^{2-alpha} u ) + rho u = f
 *   on (a, b),  u(a) = c1,  u(b) = c2,  1 < alpha < 2,  0 <= theta <= 1
 *                                                  (Sec. 1, eq. (Model))
 *
 * Discretisation (Sec. 2.2): N elements, degree P on every element, hats plus
 * bubbles psi_p = L_{p-1} - L_{p+1}; N_d = N P - 1 unknowns; the linear
 * system A X = (rho M + S) X = G, S = theta S_l + (1 - theta) S_l^T
 * (eq. (lsys)).  The boundary values enter by lifting with the two boundary
 * hats (the paper's basis spans H^1_0 only).
 *
 * Vector layout at this boundary: X's ordering of Sec. 2.2, i.e. all bubbles
 * element by element (element-major, p = 1..P-1), then the N-1 interior hats
 * in node order.  Several vectors of one instance are stored column-major
 * (N_d x nrhs, leading dimension N_d); instances are concatenated in the
 * order they were assembled.
 *
 * Pointers: every vector argument may be host memory or device memory of the
 * current device; the library finds out with cudaPointerGetAttributes.
 * Host arrays inside the parameter structs are read during the call only.
 * Handles are owned by the library and released with the *_free calls.
 * All work is issued on the stream given to hfsem_assemble; calls return
 * after that work completes unless stated otherwise.
 *
 * Errors: every int-returning call returns an HFSEM_* status and never
 * throws across this boundary.  On error nothing is written to the outputs
 * unless stated.
 */
#ifndef HFSEM_H
#define HFSEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HFSEM_OK                 0
#define HFSEM_ERR_INVALID_ARG    1  /* bad size, parameter range, pointer   */
#define HFSEM_ERR_OOM            2  /* device allocation failed             */
#define HFSEM_ERR_NOT_CONVERGED  3  /* Krylov hit max_iter; X = last iterate */
#define HFSEM_ERR_BREAKDOWN      4  /* BiCGSTAB breakdown (rho or omega = 0) */
#define HFSEM_ERR_TIMEOUT        5  /* a device-side wait reached its limit
                                       (a tensor-core product or a bulk copy
                                       that did not complete); the kernel
                                       gave up and returned, the context is
                                       still usable                       */
#define HFSEM_ERR_DEVICE         6  /* CUDA error                           */
#define HFSEM_ERR_UNSUPPORTED    7  /* valid request the library cannot do  */

/* ---- enumerations ------------------------------------------------------ */
#define HFSEM_MATVEC_AUTO      0  /* Toeplitz when the mesh is uniform or
                                     geometric with a mild ratio, else dense */
#define HFSEM_MATVEC_DENSE     1  /* O(N_d^2) dense operator (Sec. 4.2)      */
#define HFSEM_MATVEC_TOEPLITZ  2  /* block-Toeplitz FFT operator (Sec. 4.3);
                                     needs h_{i+1}/h_i constant               */
#define HFSEM_MATVEC_HMATRIX   3  /* FP64 H-matrix operator (Sec. 3 at high
                                     rank): exact near-field pairs, Taylor
                                     rank 24, min-diameter admissibility with
                                     lambda = 1 (bound (1/3)^24, below FP64
                                     rounding); O(N_d log N) storage and
                                     product instead of O(N_d^2).  An H-LU
                                     factor of such a system must use
                                     HFSEM_ADM_MIN with lambda >= 1 and
                                     automatic leaves (its near field must
                                     lie in the operator's); otherwise
                                     hfsem_hlu_factor returns UNSUPPORTED    */

#define HFSEM_PREC_FP64   0       /* H-matrix, H-LU and H-solves in FP64     */
#define HFSEM_PREC_MIXED  1       /* H-matrix, H-LU and H-solves in FP32;
                                     Krylov loop and operator stay FP64.  A
                                     batch holding a mesh whose element sizes
                                     span more than 1e45 is factored in FP64 */
#define HFSEM_PREC_MIXED_TC 2     /* as HFSEM_PREC_MIXED, with the dense leaf
                                     products of the H-LU (128-row GEMMs and
                                     the multiplies by inverted diagonal
                                     leaves) on the tensor cores: each FP32
                                     operand split into BF16 head and tail,
                                     three MMAs per K step, FP32 accumulation
                                     (Sec. 4.1 H-LU); products to ~2^-16
                                     relative, the preconditioner as strong
                                     as HFSEM_PREC_MIXED's                   */

#define HFSEM_RHS_LOAD_VECTOR  0  /* G given directly                        */
#define HFSEM_RHS_FRAC_POWERS  1  /* f = sum c_k (x-a)^mu_k + sum d_k (b-x)^nu_k */
#define HFSEM_RHS_LEGENDRE_AB  2  /* f = sum g_k L_k(xi_[a,b](x))           */

/* ---- one problem instance (Sec. 1 eq. (Model), Sec. 2.2 eq. (Partition)) */
typedef struct {
  int32_t     n_elem;   /* N >= 1                                            */
  int32_t     P;        /* polynomial degree on every element, 1 <= P <= 32 */
  double      a, b;     /* interval, a < b                                   */
  const double *h;      /* host, N element lengths h_i > 0 with
                           sum h_i = b - a to 1e-12 relative; copied         */
  double      alpha;    /* 1 < alpha < 2                                     */
  double      theta;    /* 0 <= theta <= 1                                   */
  double      rho;      /* reaction coefficient, >= 0                        */
  double      c1, c2;   /* boundary values u(a), u(b)                        */
  int32_t     matvec;   /* HFSEM_MATVEC_*                                    */
} hfsem_problem;

/* ---- H-matrix / H-LU options (Sec. 3 and Sec. 4.1) ---------------------- */
typedef struct {
  int32_t R;          /* Taylor rank of eq. (eqn:Lexpan), 1 <= R <= 32       */
  double  lambda;     /* admissibility parameter of eq. (admis), > 0 (1.0)  */
  double  tol_hlu;    /* Tol_HLU: singular values below tol_hlu * sigma_1
                         are dropped when blocks are recompressed (pivots of
                         a rank-revealing QR of the core); 0 keeps every
                         nonzero one (up to kmax).  In the FP32 modes the
                         factors' own directions below ~1e-6 of their
                         largest singular value (their rounding level) are
                         dropped as well. 1e-3 in Sec. 5                     */
  int32_t precision;  /* HFSEM_PREC_*                                        */
  int32_t leaf_elems; /* elements per leaf cluster; 0 = automatic           */
  int32_t kmax;       /* rank cap after recompression; 0 = automatic        */
  int32_t build_only; /* 1: build the H-matrix, do not factor (inspection)  */
  int32_t admissibility; /* HFSEM_ADM_MAX (eq. (admis), the default) or
                         HFSEM_ADM_MIN                                      */
} hfsem_hopts;

/* Admissibility of a cluster pair (tau, sigma) (Sec. 3.1, eq. (admis)):
 * MAX: max(diam tau, diam sigma) <= lambda dist(tau, sigma), as printed.
 * MIN: min(diam tau, diam sigma) <= lambda dist(tau, sigma).  The Taylor
 * expansion is always taken about the centre of the smaller cluster (Remark
 * after the Lemma), and the Lemma's bound (lambda / (2 + lambda))^R depends
 * only on that cluster's diameter over the distance, so MIN keeps the bound
 * while admitting far more blocks on geometrically graded meshes (index
 * clusters next to the refined ends are then much smaller than their
 * neighbours); on uniform meshes the two coincide. */
#define HFSEM_ADM_MAX 0
#define HFSEM_ADM_MIN 1

/* ---- right-hand sides -------------------------------------------------- */
typedef struct {
  int32_t kind;       /* HFSEM_RHS_*                                         */
  int32_t nrhs;       /* >= 1; must be equal for all instances of a call     */
  int32_t n_terms;    /* FRAC_POWERS: terms per rhs; LEGENDRE_AB: K + 1;
                         may differ between instances                    */
  const double *data; /* host.  LOAD_VECTOR: N_d x nrhs column-major (X's
                         ordering).  FRAC_POWERS: per rhs, n_terms triples
                         (coef, exponent > -1, side: 0 = (x-a), 1 = (b-x)).
                         LEGENDRE_AB: per rhs, K+1 coefficients g_k.         */
} hfsem_rhs;

typedef struct {
  int32_t iters;            /* BiCGSTAB iterations taken                    */
  int32_t status;           /* HFSEM_OK or the failure for this column      */
  double  rel_residual;     /* recursive ||r|| / ||G_lifted||               */
  double  rel_true_residual;/* ||G_lifted - A X|| / ||G_lifted|| at exit    */
} hfsem_stats;

typedef struct hfsem_system_s hfsem_system;
typedef struct hfsem_factor_s hfsem_factor;

/* Assemble n_inst >= 1 instances (Sec. 2.2): mesh geometry, the element-
 * pair moment blocks of S_l (dense path) or the block-Toeplitz symbol of
 * Sec. 4.3 (Toeplitz path), on the CUDA stream `stream` (cudaStream_t,
 * NULL = legacy default stream).  *out receives a handle owned by the
 * library.  INVALID_ARG for any parameter outside the ranges above. */
int hfsem_assemble(int32_t n_inst, const hfsem_problem *probs, void *stream,
                   hfsem_system **out);

/* N_d of instance `inst` (end of Sec. 2.2) into *nd. */
int hfsem_ndof(const hfsem_system *sys, int32_t inst, int32_t *nd);

/* y = A x for every instance (the operator of eq. (lsys), with zero boundary
 * values), x and y N_d x nrhs per instance, concatenated; 1 <= nrhs <= 64. */
int hfsem_apply(hfsem_system *sys, int32_t nrhs, const double *x, double *y);

/* The operator product of hfsem_apply for callers that cannot allocate
 * device memory while they run (the paper has no counterpart: this serves
 * applications that own every allocation themselves or call from a section
 * where cudaMalloc is not allowed).  x and y must be device pointers; no
 * cudaMalloc, cudaFree or allocating library routine is called.  Its
 * temporaries live in one file-scope device array of 32 MiB; the first
 * hfsem_assemble on a device loads that array (and the kernels this call
 * launches) there, and the device holds it until the process exits, so
 * the call itself loads and allocates nothing.  Requests needing more
 * scratch (sum of N_d, N*P, the dense column partials and the FFT buffers,
 * times nrhs) return HFSEM_ERR_INVALID_ARG, as do systems holding an
 * HFSEM_MATVEC_HMATRIX instance.  All calls share the array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it. */
int hfsem_apply_noalloc(hfsem_system *sys, int32_t nrhs, const double *x, double *y);

/* Self-check of the BF16x3 tensor-core tile that HFSEM_PREC_MIXED_TC uses (the
 * paper has no counterpart; its H-LU runs on CPU cores): one thread-block
 * cluster computes C = A B, A 128 x K and B K x N with fixed entries in
 * [-0.5, 0.5], reps times per CTA on one completion barrier, and compares
 * every entry with the product in FP64.  16 <= N <= 128 and 64 <= K <= 128,
 * both multiples of 16; 1 <= reps <= 8.  *max_rel_err receives
 * max |C - A B| / sum_k |a_mk b_kn| over the entries (the head/tail split
 * of both operands bounds it by about 2^-16 + 3K 2^-24).  HFSEM_ERR_DEVICE when a
 * product did not complete within its wait limit (about 2 ms). */
int hfsem_tc_tile_check(int32_t N, int32_t K, int32_t reps, double *max_rel_err);

/* Load vector G_i = (f, phi_i) of Sec. 2.2 for every instance, rhs[inst].
 * lifted = 1 subtracts the boundary-hat columns times (c1, c2), i.e. returns
 * the right-hand side the interior unknowns solve against. */
int hfsem_load_vector(hfsem_system *sys, const hfsem_rhs *rhs, int32_t lifted,
                      double *G);

/* Build the H-matrix approximation A~ = rho M + theta H + (1-theta) H^T of
 * Sec. 3 / eq. (approxsys) for every instance and factor it by H-LU
 * (Sec. 4.1), L_H unit lower, U_H upper, both in H-matrix format.  The
 * factor is valid for `sys` only and must be freed before it. */
int hfsem_hlu_factor(hfsem_system *sys, const hfsem_hopts *opts,
                     hfsem_factor **out);

/* Dense copy (N_d x N_d, column-major, X's ordering) of instance inst's A~
 * as built; only for factors made with build_only = 1. */
int hfsem_hmatrix_dense(const hfsem_factor *fac, int32_t inst, double *out);

/* y = (L_H U_H)^{-1} r for every instance: forward then backward
 * H-triangular substitution (Sec. 4.1).  r, y: N_d x nrhs per instance. */
int hfsem_precond_apply(hfsem_factor *fac, int32_t nrhs, const double *r,
                        double *y);

/* Direct solve of the H-matrix approximation system A~ X = G (Sec. 4.1,
 * the "H-matrix approximation system" of Sec. 5): X = (L_H U_H)^-1 G with
 * the load vector of rhs (boundary values lifted), no Krylov iteration.
 * Its accuracy is that of A~ (the Taylor rank R and Tol_HLU), which the
 * paper shows falling behind the discretisation error as N grows; solve
 * with hfsem_solve for the exact discrete solution.  X: N_d x nrhs per
 * instance (host or device). */
int hfsem_hlu_solve(hfsem_system *sys, hfsem_factor *fac, const hfsem_rhs *rhs, double *X);

/* Solve A X = G for every instance by BiCGSTAB (Sec. 4.2) right-
 * preconditioned with the H-LU factor `fac` (NULL: no preconditioner),
 * from X = 0.  rhs: n_inst entries, equal nrhs.  A column whose recursive
 * relative residual reaches tol is checked on its true relative residual
 * ||G - A X|| / ||G||: accepted when that is <= 100 tol (the recursive and
 * true residuals of the FP64 iteration may part by that much), else
 * BiCGSTAB restarts from the true residual (at most 8 times).  A restart
 * that fails to halve the true residual of the previous check shows that
 * the rounding floor of the FP64 product A X is reached; the column is then
 * accepted with that true residual (reported in stats).  A column stops as
 * NOT_CONVERGED when max_iter iterations or the restarts are spent, as
 * BREAKDOWN when rho, omega or (r^, v) vanish.  X (output only): N_d x nrhs
 * per instance, concatenated (host or device).  stats: n_inst * nrhs
 * entries (host), instance-major.  Returns the worst per-column status
 * (TIMEOUT if a preconditioner copy reached its wait limit); X holds the
 * last iterate in every case. */
int hfsem_solve(hfsem_system *sys, hfsem_factor *fac, const hfsem_rhs *rhs,
                double tol, int32_t max_iter, double *X, hfsem_stats *stats);

void hfsem_factor_free(hfsem_factor *fac);
void hfsem_system_free(hfsem_system *sys);

/* ---- serving loop (the paper has no counterpart: it solves one problem at a
 * time; this serves a stream of the Sec. 4.2 solves on one GPU) ------------
 *
 * A server runs `slots` requests at once, each on its own host worker and
 * non-blocking CUDA stream, so the work of concurrent requests overlaps on
 * the device.  A request is one problem instance with its right-hand sides:
 * it is assembled, factored (H-LU with the server's options) and solved as
 * by hfsem_assemble / hfsem_hlu_factor / hfsem_solve.  Admission: an idle
 * slot takes the oldest queued request that fits the device-memory budget
 * (resident factorisations plus the estimated needs of running requests),
 * evicting idle cached factorisations (least recently used first) when
 * that makes it fit; a request that does not fit holds back the ones
 * behind it, and one that cannot fit even on an otherwise empty budget
 * completes with HFSEM_ERR_OOM.  Reuse: after a request, its factorisation
 * stays resident (up to cache_factors idle ones); a later request with the
 * same operator (mesh, P, alpha, theta, rho, matvec: compared in full)
 * takes it instead of refactoring.  Requests with the same operator never
 * run at the same time.  Every request's result is the one hfsem_solve gives
 * for it alone: the arithmetic does not depend on what else runs. */
typedef struct hfsem_server_s hfsem_server;

typedef struct {
  int32_t     slots;          /* concurrent requests, 1..64                    */
  int64_t     budget_bytes;   /* device memory for resident factorisations and
                                 running requests; 0 = 80% of the free memory
                                 at creation                                   */
  int32_t     cache_factors;  /* idle factorisations kept resident, >= 0       */
  hfsem_hopts hopts;          /* H-LU options of every request (build_only = 0) */
  double      tol;            /* BiCGSTAB tolerance, as hfsem_solve            */
  int32_t     max_iter;
} hfsem_server_opts;

typedef struct {
  const hfsem_problem *prob;  /* one instance (h copied at submission)        */
  const hfsem_rhs     *rhs;   /* its right-hand sides (data copied)           */
  double      *X;             /* N_d x nrhs, host or device memory of the
                                 server's device; written when the request
                                 completes and must stay valid until then     */
  hfsem_stats *stats;         /* host, nrhs entries; written on completion    */
} hfsem_request;

typedef struct {
  int64_t id;                 /* as returned by hfsem_server_submit           */
  int32_t status;             /* HFSEM_* of the request                        */
  int32_t reused;             /* 1: a resident factorisation was reused        */
  double  t_submit, t_start, t_done;  /* seconds on the server's clock        */
  char    msg[128];           /* failure message ("" on success)              */
} hfsem_done;

typedef struct {
  int64_t resident_bytes, inflight_bytes, budget_bytes, peak_bytes;
  int32_t running, peak_running, cached, queued;
  int64_t builds, reuses, evictions, rejected;
} hfsem_server_counters;

/* Start a server on the current device (its workers start at once). */
int hfsem_server_create(const hfsem_server_opts *opts, hfsem_server **out);
/* Queue a request and return at once with its id; INVALID_ARG for malformed
 * sizes (problem parameters outside their ranges fail the request itself). */
int hfsem_server_submit(hfsem_server *srv, const hfsem_request *req, int64_t *id);
/* Up to max completed requests since the last poll into out[0..*n). */
int hfsem_server_poll(hfsem_server *srv, int32_t max, hfsem_done *out, int32_t *n);
/* Block until every submitted request has completed. */
int hfsem_server_drain(hfsem_server *srv);
int hfsem_server_counters_read(hfsem_server *srv, hfsem_server_counters *c);
/* Wait for the submitted requests, release everything resident, stop. */
void hfsem_server_free(hfsem_server *srv);

/* ---- kernel timing (measurement support; the paper has no counterpart) --
 * When enabled, the library brackets its main kernels with CUDA events on
 * the stream they are launched on (tags: "pairs", "symbol", "toeplitz_mv",
 * "dense_mv", "hlu_factor", "hlu_solve", "krylov_vec").  hfsem_timing_read
 * waits for the recorded events and returns, for one tag, the summed device
 * time, the number of launches and the summed algorithmic work (flops for
 * hlu_factor / hlu_solve, counted on the device from the executed shapes;
 * bytes for the operator kernels; 0 where not counted).  The tag
 * "launches" returns in *launches the number of kernels this library has
 * launched so far.  Process-wide. */
int hfsem_timing_enable(int32_t on);
int hfsem_timing_reset(void);
int hfsem_timing_read(const char *tag, double *total_ms, int64_t *launches, double *work);

/* ---- autotuner of the H-LU leaf size (Sec. 4.1 leaves the leaf size of the
 * cluster tree open; the kernels take leaves of up to 128 unknowns, 96 in
 * FP64) ------------------------------------------------------------------
 *
 * hfsem_tune groups the instances of sys into classes (factor arithmetic,
 * uniform or not, P), factors and solves 32 instances of each class (its
 * first 32, repeated when it has fewer, so that the runs launch like a large
 * batch) with every candidate leaf size (32, 48, 64, 96, 128 unknowns, capped by the
 * arithmetic), each twice (the first run builds the plans), and keeps the
 * fastest (factorisation + solve, CUDA events on sys's stream) among those
 * whose iteration count is within one of the fewest.  opts are the options
 * the factorisations will use (leaf_elems ignored, build_only must be 0); rhs
 * one per instance, all with the same nrhs; tol, max_iter as in hfsem_solve.
 * The choices enter a process-wide table that hfsem_hlu_factor consults for
 * every instance when opts->leaf_elems == 0 (instances of classes without an
 * entry keep the automatic size).  path (may be NULL): the whole table is
 * written there as text, one class per line ("fp64 kind P leaf_unknowns"),
 * which hfsem_tune_load reads back (entries merge into the table).  out (cap
 * entries, host, may be NULL when cap == 0) receives this call's choices,
 * *n_out (may be NULL) their number.  Errors of the tuning runs are
 * returned; a candidate the kernels cannot take is skipped. */
typedef struct {
  int32_t fp64;       /* 1: factored in FP64                                  */
  int32_t kind;       /* 0: uniform mesh, 1: any other                        */
  int32_t P;
  int32_t leaf_dofs;  /* chosen leaf size in unknowns                          */
  int32_t n_inst;     /* instances timed                                       */
  double  ms;         /* their factorisation + solve time at that size        */
  double  ms_default; /* the same at the automatic size                       */
} hfsem_tune_entry;

int hfsem_tune(hfsem_system *sys, const hfsem_hopts *opts, const hfsem_rhs *rhs,
               double tol, int32_t max_iter, const char *path, hfsem_tune_entry *out,
               int32_t cap, int32_t *n_out);
int hfsem_tune_load(const char *path);
/* *leaf_dofs = the table's leaf size for a class, 0 if it has none. */
int hfsem_tune_lookup(int32_t fp64, int32_t kind, int32_t P, int32_t *leaf_dofs);
int hfsem_tune_clear(void);

/* Measured ALU peak of the current device (measurement support for the
 * roofline fractions; the paper has no counterpart): independent FMA chains,
 * 8 per thread, 64 warps per SM on every SM, best of 3 timed launches.
 * kind 0: FP64, kind 1: FP32.  *tflops receives 2 x FMAs / time in TFLOP/s;
 * ms (may be NULL) the best launch time, sms (may be NULL) the SM count. */
int hfsem_alu_peak(int32_t kind, double *tflops, double *ms, int32_t *sms);

/* Static string for a status code. */
const char *hfsem_status_str(int status);

/* Message of the last call on the calling thread that failed ("" if none):
 * owned by the library, valid until that thread's next failing call. */
const char *hfsem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HFSEM_H */
