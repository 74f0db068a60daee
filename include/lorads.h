/*
 * lorads.h -- C ABI of the GB300 (sm_103a) LoRADS library.
 *
 * LoRADS solves the linear SDP of Section 1 (eq. prob:linear-SDP)
 *
 *     min <C, X>   s.t.   A(X) = b,   X PSD,     A(X)_i = <A_i, X>,  i = 1..m,
 *
 * with a Burer-Monteiro warm start (Phase I, Section 4.1) followed by the low-rank ADMM
 * splitting X = U V^T (Phase II, Algorithm 1), whose U- and V-subproblems are the linear
 * systems eq. linU / eq. linV solved by warm-started conjugate gradients (Section 4.4).
 * The output is U_hat = (U + V)/2 (Algorithm 2), X = U_hat U_hat^T, and the dual y.
 *
 * Conventions shared by every call
 *   - Symmetric matrices (C and each A_i) are passed as upper triplets (row <= col).  An
 *     off-diagonal triplet (i, j, a) stands for a at (i, j) and at (j, i), so
 *     <A, X> = sum_diag a_ii X_ii + 2 sum_{i<j} a_ij X_ij.  Duplicates add up.
 *   - Dense factors are row-major n x ld with ld >= r; the library pads r to a multiple of 4.
 *   - Indices are 0-based int32; sizes are int64.
 *   - Every call returns LORADS_OK (0) or a negative status; none aborts, throws or prints.
 *     lorads_status_string() names a status.
 *   - Host arrays passed to lorads_set_* / lorads_add_* are copied; the caller keeps them.
 *   - The library owns its device memory (one CUDA device: the current device at
 *     lorads_create).  Calls on one problem must not run concurrently from several threads.
 *   - The multiplier lambda of the augmented Lagrangian (eq. ALF) enters with a plus sign;
 *     the SDP dual returned here is y = -lambda, so that S = C - A^T(y) is PSD at an optimum.
 */
#ifndef LORADS_H
#define LORADS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
  LORADS_OK = 0,
  LORADS_ERR_ARG = -1,          /* bad argument (null pointer, index out of range, size) */
  LORADS_ERR_STATE = -2,        /* call out of order (e.g. solve before set_b)            */
  LORADS_ERR_CUDA = -3,         /* a CUDA runtime call failed                             */
  LORADS_ERR_NOMEM = -4,        /* device or host allocation failed                       */
  LORADS_ERR_MAXITER = -5,      /* iteration cap reached before the tolerance             */
  LORADS_ERR_TIMEOUT = -6,      /* time limit reached before the tolerance                */
  LORADS_ERR_NAN = -7,          /* a NaN or Inf appeared in the iterates or the input     */
  LORADS_ERR_UNSUPPORTED = -8,  /* constraint structure the device solver does not handle  */
  LORADS_ERR_DEVICE = -9,       /* a device-side wait gave up (bounded grid barrier)      */
  LORADS_ERR_TOO_LARGE = -10    /* lorads_solve_static: problem exceeds its fixed scratch */
};

/* ---------------------------------------------------------------- precision forms */
enum {
  LORADS_PREC_FP64 = 0,   /* every operator and vector in FP64                             */
  LORADS_PREC_MIXED = 1   /* CG operators (SDDMM/SpMM bulk, CG vectors) in FP32; masters   */
                          /* U, V, lambda, residual norms, CG alpha/beta, objective in FP64 */
};

/* ---------------------------------------------------------------- Phase II subproblem solvers */
enum {
  LORADS_SUB_CG = 0,          /* warm-started CG (Section 4.4)                               */
  LORADS_SUB_ROW_DIRECT = 1   /* exact row-block solve (every constraint one diagonal entry) */
};

/* ---------------------------------------------------------------- device allocator
 * Optional replacement for cudaMalloc / cudaFree, given through lorads_params (both set or
 * both NULL).  alloc returns `bytes` of device memory of the problem's device, 256-byte
 * aligned, usable by work enqueued on `stream` (the cudaStream_t of the call that
 * allocates), or NULL when it cannot (the call then returns LORADS_ERR_NOMEM).  free gets
 * back the pointer, its size and the stream it was allocated for, after every piece of
 * device work that used it has finished.  Memory that outlives a call (the problem's device
 * form and its solver state, kept for later solves and for lorads_get_solution /
 * lorads_get_state) is released through the free of the allocator that made it, at the
 * latest by lorads_destroy: the two functions and ctx must stay valid until then.  Both
 * are called from the thread that makes the library call, never concurrently for one
 * problem.  The Python binding points them at PyTorch's caching allocator. */
typedef void *(*lorads_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*lorads_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

/* ---------------------------------------------------------------- parameters
 * Defaults (lorads_default_params) follow Section 5.1 where the paper states a value and
 * the readings listed beside each field where it does not.  A negative value marked
 * "auto" is resolved at solve time from the constraint structure: when every constraint
 * is a single diagonal entry (MaxCut, Section 5.3) switch_tol = 1e-2 and h = 10,
 * otherwise switch_tol = 1e-3 and h = 1. */
typedef struct lorads_params {
  int32_t r0;              /* initial rank; 0 = ceil(log2 m)                                */
  int32_t rank_max;        /* cap for rank growth; 0 = min(floor(sqrt(2m)), n, 256)         */
  double rank_factor;      /* rank growth factor (1.5, Section 4.3)                          */
  double tol;              /* final tolerance (1e-6)                                         */
  double switch_tol;       /* Phase I -> II switch on primal infeasibility (auto)            */
  double h;                /* heuristic factor rho <- h rho at the switch (auto)             */
  double rho_max;          /* 5000 (Section 5.1)                                             */
  double rho_growth;       /* 1.2 (Section 5.1)                                              */
  int32_t rho_every;       /* 5 (Section 5.1)                                                */
  double gamma_scale;      /* gamma = gamma_scale * max_j sum_k |C_jk| (paper silent); < 0:  */
                           /*    1 when every constraint is one diagonal entry, else 2 (-1)  */
  double gamma_fixed;      /* > 0 overrides gamma                                            */
  int32_t max_admm_iter;   /* 5000 (Section 5.2)                                             */
  int32_t cg_max_iter;     /* 1000                                                           */
  double cg_rel_tol;       /* CG stops at ||R|| <= cg_rel_tol ||R_0|| ... (1e-3)             */
  double cg_abs_floor;     /* ... or ||R|| <= cg_abs_floor ||G|| (1e-13)                     */
  int32_t lbfgs_mem;       /* L-BFGS memory in Phase I (4, at most 8)                        */
  int32_t inner_max_iter;  /* L-BFGS iterations per ALM subproblem before rank growth (300)  */
  double inner_tol_factor; /* ALM subproblem stop: ||grad||/(1+||C||_F) <= min(max, f r_P)   */
  double inner_tol_max;    /*   (factor 10, max 0.1)                                         */
  int32_t max_outer;       /* ALM outer iterations (500)                                     */
  double sigma_factor;     /* ALM penalty growth when r_P fell less than 4x (2)              */
  double sigma_decrease;   /* the "4x": 0.25                                                 */
  double sigma_max;        /* cap of the ALM penalty (paper silent): 1e4, twice rho_max; an  */
                           /*    uncapped penalty overflows on constraints that converge      */
                           /*    slowly (the theta SDP)                                       */
  double new_col_std;      /* std of columns added by rank growth (1e-2)                     */
  uint64_t seed;           /* SplitMix64 seed for U_0 and rank growth                        */
  int32_t precision;       /* LORADS_PREC_FP64 or LORADS_PREC_MIXED                          */
  int32_t phase1;          /* 1: Phase I from random U_0; 0: start Phase II from lorads_set_start */
  double time_limit_s;     /* wall-clock cap of one solve on the device (60 s)               */
  int32_t threads;         /* CTA size of the solver kernels, a multiple of 32, >= 128:     */
                           /*    <= 384 for one-CTA solves and batches, <= 320 for the grid  */
                           /*    scope                                                        */
                           /*    (0 = library choice; batches autotune 128, 256, 384)         */
  int32_t grid;            /* solver CTAs (0 = library choice; 1 forces one-CTA scope)       */
  int32_t team_mult;       /* lanes per factor row = team_mult x the minimum for the rank    */
                           /* (1, 2, 4, 8; 0 = 1, or autotuned by lorads_solve_batch)         */
  int32_t kkt_dinf;        /* 1: the final test includes the dual measure                    */
                           /*    max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf) (needs      */
                           /*    lanczos_steps > 0); 0: r_P, gap and r_D only (1)             */
  int32_t lanczos_steps;   /* Lanczos steps of each lambda_min(C - A^T y) estimate, at most, */
                           /*    <= 2048; the recurrence stops earlier once the estimate moved */
                           /*    by at most 0.05 tol (1 + ||C||_inf) over its last doubling of */
                           /*    steps (checked at 128, 256, ...); 0 = no estimate (kkt_dinf   */
                           /*    must be 0) (2048)                                            */
  int32_t dinf_every;      /* after a failed dual-infeasibility test at iteration k, the next */
                           /*    waits max(dinf_every, k / 10) iterations (10)                */
  double escape_scale;     /* when a dual-infeasibility test fails less than 10% below the   */
                           /*    previous failed one, Phase II raises the rank by rank_factor */
                           /*    (up to rank_max) with the eigenvector z of lambda_min as new */
                           /*    column of U and V, scaled to escape_scale ||U_hat||_F/sqrt(r)*/
                           /*    (0.3; 0 = never)                                             */
  int32_t group;           /* CTAs per problem in lorads_solve_batch (1, 2, 4): a group     */
                           /*    shares one problem through bounded barriers; 0 = 2 when the  */
                           /*    largest problem has n >= 1024, else 1 (0)                    */
  int32_t subsolver;       /* Phase II subproblems eq. linU / linV: LORADS_SUB_CG (Section   */
                           /*    4.4) or LORADS_SUB_ROW_DIRECT, for problems whose            */
                           /*    every constraint is one diagonal entry, at most one per row  */
                           /*    (the matrix is then block diagonal, gamma I + rho a_j^2 W_j  */
                           /*    W_j^T per row, inverted by Sherman-Morrison; Section 1 admits */
                           /*    direct methods): LORADS_ERR_UNSUPPORTED otherwise (0)        */
  int32_t polish;          /* Phase III, a refinement of eq. prob:BM's stationarity (not in  */
                           /*    the paper), entered when Phase II's output passes the primal */
                           /*    test and the gap but not r_D: Newton's method on the product */
                           /*    of spheres when every row carries exactly one diagonal       */
                           /*    constraint a X_jj = b, b/a > 0 (MaxCut with n = m), else     */
                           /*    Phase I's augmented Lagrangian method continued from Phase  */
                           /*    II's output; 1 = on, 0 = Phase II alone (1)                  */
  int32_t newton_max;      /* Phase III Newton steps, at most (200)                          */
  int32_t newton_cg_max;   /* CG iterations of one Newton step, at most (1000)               */
  double *iter_log;        /* device array of iter_log_cap x 6 doubles, or NULL (no log): row */
                           /*    k of Phase II's iteration k + 1 holds (k + 1, rho, r_P of    */
                           /*    U V^T, r_P of U_hat U_hat^T, CG iterations so far, device    */
                           /*    seconds since the solve started); iterations past the cap    */
                           /*    are not logged.  Written by the device during the solve;     */
                           /*    lorads_solve_batch logs nothing.                             */
  int32_t iter_log_cap;    /* rows of iter_log (0)                                           */
  int32_t lanczos_store_mb; /* device memory (MiB) lorads_solve may add to its state to keep  */
                           /*    the Lanczos vectors of a dual test, (lanczos_steps + 1) x n */
                           /*    x 32 bytes (at most 2049 x n x 32): when they fit, the      */
                           /*    escape's eigenvector is summed from them instead of from a */
                           /*    second pass of the recurrence (same vector up to rounding */
                           /*    order); 0 = always the second pass; batches and           */
                           /*    lorads_solve_static always take the second pass (2048)    */
  int64_t barrier_polls;   /* polls a grid-wide (or CTA-group) barrier makes before it gives */
                           /*    up; the solve then ends with LORADS_ERR_DEVICE and the CUDA  */
                           /*    context stays usable (0 = 50,000,000, a few seconds)          */
  lorads_alloc_fn dev_alloc; /* device allocator (NULL with dev_free: cudaMalloc / cudaFree) */
  lorads_free_fn dev_free;
  void *alloc_ctx;         /* passed to dev_alloc and dev_free                               */
} lorads_params;

/* ---------------------------------------------------------------- result */
typedef struct lorads_result {
  int32_t status;          /* LORADS_OK when the final test passed                           */
  int32_t rank;            /* final r                                                        */
  double objective;        /* <C, U_hat U_hat^T>                                             */
  double dual_objective;   /* b^T y                                                          */
  double r_P;              /* ||A(U_hat U_hat^T) - b||_2 / (1 + ||b||_inf)   (Section 5.2)   */
  double r_P_split;        /* ||A(U V^T) - b||_2 / (1 + ||b||_inf)                           */
  double r_stop;           /* gamma ||V^{k+1} - V^k||_F / (1 + ||V^k||_F)  (eq. stop)        */
  double r_D;              /* ||(C - A^T y) U_hat||_F / (1 + ||C||_F)  (eq. def:eKKT)        */
  double gap;              /* (<C,X> - b^T y) / (1 + |<C,X>| + |b^T y|)  (Appendix B)        */
  double rho;              /* final rho                                                      */
  double gamma;            /* gamma used in Phase II                                         */
  double sigma;            /* final Phase I penalty                                          */
  int32_t admm_iters;      /* Phase II iterations                                            */
  int32_t cg_iters;        /* CG iterations summed over all subproblems (0 with             */
                           /*    LORADS_SUB_ROW_DIRECT)                                       */
  int32_t hessian_applies; /* Hessian-vector products (CG iterations + warm-start residuals; */
                           /*    with LORADS_SUB_ROW_DIRECT the passes that form R_0 and solve) */
  int32_t alm_outer;       /* Phase I outer iterations                                       */
  int32_t lbfgs_iters;     /* Phase I L-BFGS iterations                                      */
  int32_t rank_growths;    /* rank increases (Phase I and Phase II)                          */
  double time_phase1_s;    /* device time of Phase I                                         */
  double time_phase2_s;    /* device time of Phase II (and the output step without Phase III) */
  double p_infeas;         /* ||A(X) - b||_2 / (1 + ||b||_1)                    (Appendix B)  */
  double d_infeas;         /* max(0, -lambda_min) / (1 + ||vec(C)||_1)          (Appendix B)  */
  double lambda_min;       /* Lanczos estimate of lambda_min(C - A^T y) (NaN: not computed)  */
  double dual_psd;         /* max(0, -lambda_min) / (1 + ||C||_inf): the final test's dual   */
                           /*    measure (||C||_inf = max_j sum_k |C_jk|; it does not grow    */
                           /*    with n the way ||vec(C)||_1 does)                            */
  double time_phase3_s;    /* device time of Phase III and the output step (0: no Phase III) */
  int32_t polished;        /* Phase III: 0 none, 1 Newton on the product of spheres, 2 the   */
                           /*    augmented Lagrangian method of Phase I continued            */
  int32_t newton_steps;    /* Phase III Newton steps                                         */
  int32_t newton_cg_iters; /* Phase III CG iterations, summed over the Newton steps          */
  int32_t refine_outer;    /* Phase III augmented-Lagrangian outer iterations                */
  int32_t refine_lbfgs_iters; /* Phase III L-BFGS iterations                                 */
  int32_t lanczos_steps;   /* Lanczos steps of the dual tests (both passes), over the solve  */
  double time_lanczos_s;   /* device time of those Lanczos runs (part of the phase times)    */
} lorads_result;

typedef struct lorads_problem lorads_problem;

/* ---------------------------------------------------------------- problem set-up */

/* New problem with n (matrix order) and m (constraints) on the current CUDA device.
 * *out receives an opaque handle owned by the library (release with lorads_destroy). */
int lorads_create(int64_t n, int64_t m, lorads_problem **out);

/* The objective C (Section 1): nnz upper triplets.  Replaces any earlier C. */
int lorads_set_C(lorads_problem *p, int64_t nnz, const int32_t *row, const int32_t *col,
                 const double *val);

/* Adds sparse terms to constraints: for t < nnz, A_{con[t]} gets val[t] at (row[t], col[t])
 * (and its mirror).  Sparse form of the A_i of eq. prob:linear-SDP.  A constraint may carry
 * any number of entries (one for MaxCut and matrix completion, n for tr X = 1); repeated
 * (row, col) pairs of a constraint, in either order, are summed.  At the first solve a
 * constraint with no non-zero entry gives LORADS_ERR_ARG. */
int lorads_add_A_sparse(lorads_problem *p, int64_t nnz, const int32_t *con, const int32_t *row,
                        const int32_t *col, const double *val);

/* Adds a rank-one term A_con += scale * a a^T with a given by nnz (idx, a) pairs (the
 * sensor-localisation constraints of Section 2.3); repeated indices are summed.  Assembly
 * expands the term into its nnz (nnz + 1) / 2 symmetric entries (scale a_k a_l at (k, l)),
 * so it suits short vectors; above 2^29 entries in all the solve returns
 * LORADS_ERR_UNSUPPORTED. */
int lorads_add_A_rank1(lorads_problem *p, int32_t con, int64_t nnz, const int32_t *idx,
                       const double *a, double scale);

/* The right-hand side b (length m). */
int lorads_set_b(lorads_problem *p, const double *b);

/* Defaults described at lorads_params. */
void lorads_default_params(lorads_params *prm);

/* Phase II start for prm->phase1 == 0 (e.g. a learned warm start): U0 is n x r row-major
 * (U = V = U0), lambda0 of length m (NULL = 0), rho0 the initial penalty (<= 0: 100).
 * Replaces a start given by lorads_set_state. */
int lorads_set_start(lorads_problem *p, int32_t r, const double *U0, const double *lambda0,
                     double rho0);

/* ---------------------------------------------------------------- solve */

/* Algorithm 2 on the device.  stream is a cudaStream_t (NULL = the legacy default stream);
 * the call returns when the solve has finished.  res may be NULL.  The return value is
 * the solve status (also res->status).  The solve ends (LORADS_OK) when the output
 * X = U_hat U_hat^T, y = -lambda passes the final test: the paper's termination
 * r_P = ||A(X) - b||_2 / (1 + ||b||_inf) <= tol (Section 5.2), the Appendix B gap |gap| <= tol,
 * the stationarity r_D = ||(C - A^T y) U_hat||_F / (1 + ||C||_F) <= tol (eq. def:eKKT), and,
 * with kkt_dinf, the dual measure max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf) <= tol
 * (lambda_min by Lanczos, tested at most once per max(dinf_every, k/10) iterations after a
 * test that did not end the solve).  With polish = 1 the first Phase II output that passes
 * r_P and the gap is handed to Phase III, which ends the solve when r_P, r_D and the dual
 * measure pass.  Otherwise the solve ends with LORADS_ERR_MAXITER after max_admm_iter Phase II
 * iterations, newton_max Newton steps or max_outer augmented-Lagrangian iterations.
 * The solve's state (factors, CG vectors, L-BFGS history, reduction scratch and, when they fit
 * lanczos_store_mb, the Lanczos blocks of the dual tests) is one device allocation from the
 * params' allocator, kept with the problem and reused by its next solve when large enough;
 * LORADS_ERR_NOMEM when it cannot be had. */
int lorads_solve(lorads_problem *p, const lorads_params *prm, void *stream, lorads_result *res);

/* Solves count independent problems (same device) in one persistent launch: one CTA (or a
 * group of prm->group CTAs, a cooperative launch) per problem, taking problems from a
 * device-side queue, largest problems first, so uneven sizes balance across the SMs.  The device work (queue reset and the persistent kernel) is
 * captured as a CUDA graph on a private stream and the graph is launched on `stream`.
 * prm applies to every problem ("auto" fields resolved per
 * problem).  When prm->threads or prm->team_mult is 0 the library autotunes them first: it
 * times every (CTA size in {128, 256, 384}) x (lanes-per-row multiplier in {1, 2, 4}) on a
 * sample of up to 24 problems (Phase II capped at 200 iterations) and keeps the fastest;
 * the choice is returned in *tuned_threads / *tuned_team_mult (either may be NULL).  res
 * (may be NULL) receives count reports; each problem's solution is then available through
 * lorads_get_solution.  Returns LORADS_OK when the batch ran (per-problem statuses are in
 * res), or the first set-up error. */
int lorads_solve_batch(lorads_problem *const *ps, int32_t count, const lorads_params *prm,
                       void *stream, lorads_result *res, int32_t *tuned_threads,
                       int32_t *tuned_team_mult);

/* The last solve's factors and dual into caller host buffers: U, V, U_hat as n x r
 * row-major (r = result rank; any pointer may be NULL), y of length m. */
int lorads_get_solution(const lorads_problem *p, double *U, double *V, double *U_hat,
                        double *y, int32_t *r);

/* ---------------------------------------------------------------- checkpoint / resume
 * A Phase II iterate of Algorithm 1 -- (U^k, V^k, lambda^k) with the penalty rho for the
 * next iteration, the rank and the counters -- is the whole state the iteration carries from
 * one step to the next (the CG solves start from W and need no history; the Phase I -> II
 * switch of Algorithm 2 is the same kind of hand-over, with V = U).  A solve stopped by
 * max_admm_iter or time_limit_s can therefore be continued later, in this process or
 * another, by lorads_get_state after it and lorads_set_state + lorads_solve (phase1 = 0)
 * before the continuation.  The continuation keeps the iteration counter k (so the rho
 * schedule of Section 5.1, the max_admm_iter cap and the final-test schedule go on where
 * they stopped), the split penalty gamma of the checkpoint, and it reports totals (ADMM, CG,
 * Hessian, Phase I counters) including the checkpointed part.  The resumed solve recomputes
 * the row-local CG's incrementally kept products -(C W) and, in the MIXED form, re-rounds the
 * FP32 shadows of U and V from the FP64 masters; the uninterrupted solve does the same every
 * 32 iterations, so from a checkpoint with k a multiple of 32 (same launch geometry) the
 * continuation repeats the uninterrupted solve bit for bit, and from other k it agrees up
 * to rounding.  time_limit_s counts per call. */
typedef struct lorads_state {
  int64_t n, m;            /* order and constraint count of the problem it belongs to         */
  int32_t phase;           /* 2: a Phase II iterate (the only kind lorads_set_state takes)    */
  int32_t rank;            /* r: columns of U and V                                          */
  int32_t admm_iters;      /* k: Phase II iterations done                                    */
  int32_t next_dual_test;  /* first k at which the dual-infeasibility test may run again     */
  int32_t cg_iters;        /* counters of the solve so far (lorads_result meanings)          */
  int32_t hessian_applies;
  int32_t alm_outer;
  int32_t lbfgs_iters;
  int32_t rank_growths;
  int32_t reserved;        /* 0                                                              */
  double rho;              /* penalty of iteration k + 1                                     */
  double gamma;            /* split penalty of eq. linU / eq. linV                           */
  double sigma;            /* final Phase I penalty (reported only)                          */
  double prev_d_infeas;    /* dual infeasibility of the latest failed final test since the  */
                           /*    last rank growth (NaN: none), for the growth rule            */
} lorads_state;

/* The state after the last solve of p (lorads_solve, lorads_solve_batch) into *st and the
 * host buffers U, V (n x st->rank row-major) and lambda (length m, the multiplier of eq. ALF,
 * lambda = -y); each buffer may be NULL (call once with NULL buffers to learn the rank).
 * LORADS_ERR_STATE when there is no solve, or it ended in Phase I or with a NaN or device
 * status. */
int lorads_get_state(const lorads_problem *p, lorads_state *st, double *U, double *V,
                     double *lambda);

/* Makes *st with U, V (n x st->rank row-major) and lambda (length m; NULL = 0) the start of
 * the next solve with prm->phase1 == 0 (replacing lorads_set_start's).  Host data are
 * copied.  LORADS_ERR_ARG when st->n / st->m differ from p's, st->phase != 2, the rank is
 * outside [1, min(n, 256)], rho or gamma is not positive, the counters are negative, U or V
 * is NULL or a value is not finite. */
int lorads_set_state(lorads_problem *p, const lorads_state *st, const double *U,
                     const double *V, const double *lambda);

/* Allocation-free solve.  The paper has no counterpart: this is a deployment variant of
 * lorads_solve for callers that must not allocate device memory while they solve -- code
 * that runs between the set-up and the end of a latency-critical loop, processes that
 * share a GPU under a fixed memory budget, or hosts whose allocator must not be entered
 * from the solving thread.  Such a caller builds the problem once (lorads_create, the
 * set calls, and one lorads_solve or lorads_op_* call, which assemble the device form and
 * do allocate); afterwards this call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.
 *
 * The solver's working memory (factors, CG vectors, L-BFGS history, reduction scratch) is a
 * file-scope device array of LORADS_STATIC_SCRATCH_BYTES (32 MiB) that every GPU which loads
 * the library holds until the process exits.  Problems whose working set does not fit are
 * rejected with LORADS_ERR_TOO_LARGE (roughly n * 4 ceil(r_max/4) <= 150,000 for the default
 * L-BFGS memory, r_max the rank cap).  The problem must already be assembled, else
 * LORADS_ERR_STATE.
 *
 * Outputs go to caller DEVICE buffers: U_hat as n x ldu row-major doubles (ldu >= the final
 * rank, which is at most the rank cap; columns beyond the final rank are left unchanged),
 * y (length m, y = -lambda); either may be NULL.  res (host) receives the report.  The
 * problem's own solution from its last lorads_solve (what lorads_get_solution and
 * lorads_get_state return) is left as it was.
 *
 * The call that assembles the problem also prepares this one: with the problem's device
 * current it loads the library's device code (CUDA loads modules lazily by default, and
 * loading a module allocates device memory, this array included) and looks up the array's
 * device address with cudaGetSymbolAddress.  The solve launches with the geometry
 * lorads_solve picks for the same parameters (grid, threads, team_mult), so the two give
 * the same iterates (an escape's eigenvector comes from the second Lanczos pass here and,
 * within lanczos_store_mb, from the kept blocks there: the same products added in the same
 * order).  Every call shares the one array and leaves the last call's contents in it; the
 * call clears what must start at zero.  Calls that overlap on the GPU (several streams or
 * host threads at once) race on the array: serialize them.  The call blocks until the solve
 * has finished on stream and reads its report back, so it cannot be captured into a CUDA
 * graph. */
#define LORADS_STATIC_SCRATCH_BYTES (32ull << 20)
int lorads_solve_static(lorads_problem *p, const lorads_params *prm, void *stream,
                        double *U_hat, int64_t ldu, double *y, lorads_result *res);

/* Releases the problem and its device memory.  NULL is ignored. */
void lorads_destroy(lorads_problem *p);

const char *lorads_status_string(int code);

/* sizeof(lorads_params), sizeof(lorads_result) and sizeof(lorads_state) as compiled into
 * the library, so that a binding can check its mirror of the structs.  Any pointer may be
 * NULL. */
void lorads_struct_sizes(int64_t *params_bytes, int64_t *result_bytes, int64_t *state_bytes);

/* ---------------------------------------------------------------- learned warm start
 * A 3-layer message-passing network over the cost graph proposes the Phase II start
 * (U_0, y_0) in place of Phase I (the paper's Phase I is the Burer-Monteiro method,
 * Section 4.1; better warm starts are its stated future work, Section 6).  Use:
 * lorads_gnn_forward(..., U0, y0), then lorads_set_start(p, r, U0, lambda0 = -y0, rho0) and
 * lorads_solve with phase1 = 0.  Weights are BF16 on the tensor cores (FP32 accumulation,
 * FP32 master copy for Adam).  Widths: hidden 64, layers 3, r at most 16.
 *   graph    edges (ei, ej) with weights w (for MaxCut the off-diagonal entries of C)
 *   features 8 SplitMix64 normals of feature_seed, 1, log(1+deg), d/10, sum w / d
 *            (d = 1 + sum |w|), zero padding to 64
 *   layer    H = relu([H, A_hat H] Theta + b), A_hat_ij = w_ij / sqrt(d_i d_j)
 *   heads    U_0 = rows of H Theta_u (first r columns) normalised to unit length,
 *            y_0 = H theta_y + b_y
 *   loss     mean over edges (U_i.U_j - Xs_e)^2 + 0.1 mean over nodes (y_i - ys_i)^2
 * Parameter vector (FP32, lorads_gnn_param_count() entries): for l = 0..2 Theta_l
 * (128 x 64 row-major, input feature major) then b_l (64); Theta_u (64 x 16 row-major);
 * theta_y (64); b_y (1). */
typedef struct lorads_gnn lorads_gnn;

int lorads_gnn_param_count(void);

/* New network on the current device; weights ~ N(0, 1/fan_in) from the SplitMix64 seed. */
int lorads_gnn_create(uint64_t seed, lorads_gnn **out);

/* Copies the FP32 parameters to / from a host vector of lorads_gnn_param_count() floats;
 * set also resets the Adam moments. */
int lorads_gnn_get_params(const lorads_gnn *g, float *params);
int lorads_gnn_set_params(lorads_gnn *g, const float *params);

/* Loads a graph (nedges undirected edges i != j, host arrays copied) and its features. */
int lorads_gnn_load_graph(lorads_gnn *g, int64_t n, int64_t nedges, const int32_t *ei,
                          const int32_t *ej, const double *w, uint64_t feature_seed);

/* Forward pass; U0 (n x r row-major) and y0 (n) into host buffers (either may be NULL). */
int lorads_gnn_forward(lorads_gnn *g, int32_t r, double *U0, double *y0, void *stream);

/* One training step on the loaded graph with targets Xs (per edge, U_hat_i.U_hat_j of a
 * solved instance) and ys (per node, the solved dual): forward, backward, and an Adam step
 * with learning rate lr (lr = 0: gradients only).  *loss receives the loss before the step;
 * grads (may be NULL) the FP32 gradient vector. */
int lorads_gnn_train_step(lorads_gnn *g, int32_t r, const double *Xs, const double *ys,
                          double lr, double *loss, float *grads, void *stream);

void lorads_gnn_destroy(lorads_gnn *g);

/* ---------------------------------------------------------------- operators
 * The linear maps of the method on caller-owned DEVICE arrays (row-major n x ld, ld a
 * multiple of 4, ld >= r), enqueued on stream; they return after enqueueing.  prec selects
 * the element type of U, V, P, out: FP64 (double) or MIXED (float); vectors indexed by
 * constraint are double.  They exist for testing and benchmarking the kernels the solver
 * is built from. */

/* q_i = <A_i, U V^T>, i = 1..m (the sampled dense-dense product, Algorithm 1 dual step). */
int lorads_op_sddmm(lorads_problem *p, int32_t prec, int32_t r, int32_t ld, const void *U,
                    const void *V, double *q, void *stream);

/* out = (A^T(w) - C) V + gamma V (the right-hand side of eq. linU with w = rho b - lambda). */
int lorads_op_spmm(lorads_problem *p, int32_t prec, int32_t r, int32_t ld, const double *w,
                   double gamma, const void *V, void *out, void *stream);

/* out = rho A^T(A(P V^T)) V + gamma P (the matrix of eq. linU applied to P, never formed).
 * With multi-entry constraints A(P V^T) goes through m values of scratch owned by the
 * problem: calls on one problem must not overlap on the device. */
int lorads_op_hessian(lorads_problem *p, int32_t prec, int32_t r, int32_t ld, double rho,
                      double gamma, const void *V, const void *P, void *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LORADS_H */
