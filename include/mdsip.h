/*
 * mdsip -- mixed dense-sparse interior-point Newton step on one GB300 GPU.
 *
 * C ABI.  Plain pointers and sizes only.  Every call returns an mdsip_status
 * (no exceptions cross the ABI); the text of the last error of a context is
 * available from mdsip_ctx_last_error().  One context per host thread.
 *
 * Problem class (Section 2, Eqs. (obj)-(bounds)): variables x = [x_s; x_d]
 * (n = n_s + n_d), equalities g(x) = g_E (m_E), inequalities h^l <= h(x) <= h^u
 * (m_I), bounds x^l <= x <= x^u; infinite bounds are +-HUGE_VAL.  Every h_i
 * has at least one finite bound.  Assumptions A1/A2 of Section 2: no cross
 * Hessian between x_d and x_s, and the x_s Hessian block is diagonal.
 *
 * Memory: arguments tagged `mem` are host pointers when mem == MDSIP_MEM_HOST
 * and device pointers (on the context's device) when mem == MDSIP_MEM_DEVICE.
 * Pointers passed in are borrowed for the duration of the call only; the
 * library copies what it keeps.  All device work is ordered on the context's
 * stream.
 */
#ifndef MDSIP_H
#define MDSIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MDSIP_OK = 0,
    MDSIP_ERR_INVALID_ARG = 1,      /* bad size, null pointer, unknown option      */
    MDSIP_ERR_CUDA = 2,             /* a CUDA runtime call failed                  */
    MDSIP_ERR_OOM = 3,              /* device allocation failed                    */
    MDSIP_ERR_CALLBACK = 4,         /* a user callback returned nonzero            */
    MDSIP_ERR_NONFINITE = 5,        /* NaN/Inf in a model value or residual        */
    MDSIP_ERR_INERTIA = 6,          /* inertia correction exceeded dw_max (Sec 2.1)*/
    MDSIP_RESTORATION_NEEDED = 7,   /* line search reached alpha_min               */
    MDSIP_MAX_ITER = 8,             /* iteration limit reached                     */
    MDSIP_TIMEOUT = 9,              /* host wall-clock limit reached               */
    MDSIP_ERR_PRECONDITION = 10,    /* path P2 forced but its precondition fails   */
    MDSIP_ERR_DEVICE = 11           /* a device-side bounded wait expired          */
} mdsip_status;

enum { MDSIP_MEM_HOST = 0, MDSIP_MEM_DEVICE = 1 };

/* Linear-algebra path of the Newton step (option "path"):
 *   P1: dense compressed matrix of Eq. (compressed), size n_d + m;
 *   P2: two-stage elimination to size n_d + m_I (requires J_sh = 0 and rows of
 *       J_sg with disjoint column supports, so that J_sg Q_s^-1 J_sg^T is diagonal);
 *   AUTO: P2 when applicable, else P1. */
enum { MDSIP_PATH_AUTO = 0, MDSIP_PATH_P1 = 1, MDSIP_PATH_P2 = 2 };

/* Arithmetic of the condensation product (option "precision"): FP64 on the
 * DFMA pipe, or tensor cores (tcgen05) with TF32 / BF16 operands and FP32
 * accumulation, the Newton direction then refined in FP64 on the unreduced
 * system. */
enum { MDSIP_PREC_FP64 = 0, MDSIP_PREC_TF32 = 1, MDSIP_PREC_BF16 = 2 };

typedef struct mdsip_ctx mdsip_ctx;
typedef struct mdsip_problem mdsip_problem;

/* Optional device-allocation hooks (nullable).  alloc returns a device pointer
 * or NULL (reported as MDSIP_ERR_OOM); free releases it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} mdsip_alloc_hooks;

/* Create a context on `device` ordering its work on `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  `hooks` may be NULL (cudaMalloc/cudaFree). */
mdsip_status mdsip_ctx_create(int device, void *stream, const mdsip_alloc_hooks *hooks,
                              mdsip_ctx **out);
void mdsip_ctx_destroy(mdsip_ctx *ctx);
const char *mdsip_ctx_last_error(const mdsip_ctx *ctx);
const char *mdsip_status_str(mdsip_status s);

/* ------------------------------------------------------------------------- */
/* Problem: the MDS model family of the benchmark (Section 2 problem class).  */
/*                                                                            */
/*   f(x)  = 1/2 x_d^T Q x_d + sum_i 1/4 x_s,i^4 + c^T x                      */
/*   g(x)  = J_sg x_s + A x_d                (equalities g(x) = g_E)          */
/*   h_j(x)= sum_{k : h_set[k] == j} x_d,k^2 + (J_sh x_s)_j  (h^l <= h <= h^u)  */
/*                                                                            */
/* A = J_{x_d} g is dense (m_E x n_d, row-major, Section 3.2.3 container      */
/* blocks (3,1)/(3,2)); J_sg is given as COO triplets (Section 3.2.3: triplet  */
/* storage), converted once to CSR/CSC on the device; so is J_sh, the        */
/* inequalities' constant sparse block (nnz_Jsh = 0 in the benchmark family; */
/* with J_sh != 0 the two-stage path P2 does not apply and AUTO takes P1).    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n_d, n_s, m_E, m_I;
    int64_t nnz_Jsg;
    const double *Q;          /* n_d * n_d, row-major, symmetric                 */
    const double *c;          /* n_s + n_d                                       */
    const double *A;          /* m_E * n_d, row-major                            */
    const double *gE;         /* m_E                                             */
    const int32_t *Jsg_rows;  /* nnz_Jsg, in [0, m_E)                            */
    const int32_t *Jsg_cols;  /* nnz_Jsg, in [0, n_s)                            */
    const double *Jsg_vals;   /* nnz_Jsg                                         */
    const int32_t *h_set;     /* n_d: inequality index of x_d,k or -1            */
    const double *hl, *hu;    /* m_I                                             */
    const double *xl, *xu;    /* n_s + n_d                                       */
    const double *x0;         /* n_s + n_d starting point (nullable: zeros)      */
    int64_t nnz_Jsh;          /* entries of J_sh (0: J_sh = 0)                   */
    const int32_t *Jsh_rows;  /* nnz_Jsh, in [0, m_I)                            */
    const int32_t *Jsh_cols;  /* nnz_Jsh, in [0, n_s)                            */
    const double *Jsh_vals;   /* nnz_Jsh (duplicates summed)                     */
} mdsip_synth_data;

/* Copy the data to the device and build the sparse indices.  `mem` tags all
 * pointers of `data`.  Errors: INVALID_ARG (sizes, indices out of range,
 * inconsistent bounds), OOM, CUDA. */
mdsip_status mdsip_problem_create_synthetic(mdsip_ctx *ctx, const mdsip_synth_data *data, int mem,
                                            mdsip_problem **out);
/* ------------------------------------------------------------------------- */
/* Problem given by callbacks (Section 2 problem statement; Section 3.3:     */
/* dense blocks are passed as double* with a leading dimension).             */
/*                                                                           */
/* Every pointer a callback receives is a device pointer on the context's    */
/* device; `stream` is the context's stream and all the callback's device    */
/* work must be ordered on it.  A callback returns 0 on success; any other   */
/* value stops the call in progress with MDSIP_ERR_CALLBACK.  Variables are  */
/* x = [x_s (n_s); x_d (n_d)].  Requirements: J_sh = 0 (inequalities depend  */
/* on x_d only), the x_s Hessian block is diagonal (A2), no cross Hessian   */
/* (A1).                                                                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    /* f(x) into f[0] */
    int (*eval_f)(void *user, void *stream, const double *x, double *f);
    /* grad f(x) into grad[0..n) */
    int (*eval_grad_f)(void *user, void *stream, const double *x, double *grad);
    /* g(x) into g[0..m_E) and h(x) into h[0..m_I) (values, not residuals) */
    int (*eval_cons)(void *user, void *stream, const double *x, double *g, double *h);
    /* Jacobian blocks at x: Jsg_vals[e] = d g_row(e) / d x_s,col(e) in the order of the
     * triplets given at creation; A[i * lda + k] = d g_i / d x_d,k; Jdh[j * ldh + k] = d h_j / d x_d,k */
    int (*eval_jac)(void *user, void *stream, const double *x, double *Jsg_vals, double *A, int64_t lda,
                    double *Jdh, int64_t ldh);
    /* Hessian of f + y_g^T g + y_h^T h: Hss[i] = diagonal of the x_s block,
     * Hdd[p * ldd + q] = dense x_d block */
    int (*eval_hess)(void *user, void *stream, const double *x, const double *yg, const double *yh,
                     double *Hss, double *Hdd, int64_t ldd);
} mdsip_callbacks;

typedef struct {
    int64_t n_d, n_s, m_E, m_I;
    int64_t nnz_Jsg;
} mdsip_dims;

/* Create a problem evaluated by `cb` (copied; `user` is passed back
 * unchanged).  Jsg_rows/Jsg_cols (nnz_Jsg, `mem`-tagged) give the sparsity of
 * J_sg; the values come from eval_jac.  Bounds must be set with
 * mdsip_set_bounds before solving.  Errors: INVALID_ARG, OOM, CUDA. */
mdsip_status mdsip_problem_create(mdsip_ctx *ctx, const mdsip_dims *dims, const int32_t *Jsg_rows,
                                  const int32_t *Jsg_cols, const mdsip_callbacks *cb, void *user,
                                  int mem, mdsip_problem **out);

/* Bounds and right-hand sides of any problem (all `mem`-tagged; +-HUGE_VAL =
 * none): xl, xu (n), hl, hu (m_I), g_E (m_E), x0 (n, nullable = zeros).
 * Required once for a callback problem; on a synthetic problem it replaces
 * the values given at creation (a member of a parametric family). */
mdsip_status mdsip_set_bounds(mdsip_problem *p, const double *xl, const double *xu, const double *hl,
                              const double *hu, const double *gE, const double *x0, int mem);

void mdsip_problem_destroy(mdsip_problem *p);

/* Options (Section 2.1 method constants; names as in the oracle):
 *   int:    max_iter, path, max_ls, refine_max, precision (MDSIP_PREC_*),
 *           graphs (1, default: from its second use for a given order, the
 *           factorization phase -- scale of S, LDL^T, solve tiles -- runs as
 *           one captured CUDA graph; 0: separate launches),
 *           autotune (1, default: the blocked LDL^T's panel width and, for
 *           products below 4e10 multiply-adds, the FP64 product's tile edge
 *           are chosen by timing the candidates at first use per device and
 *           shape; 0: the analytic choices),
 *           ldlt_spec (1, default: the mixed-precision factorization's
 *           panels first try the verified no-interchange path described at
 *           mdsip_ldlt_factor_ex, and from order 2048 on the persistent
 *           no-interchange kernel runs first in either precision; 2: that
 *           kernel at every order; 0: every panel pivots),
 *           direction_check (0, default; 1: every step of a mixed-precision
 *           solve also computes the FP64 direction from the same iterate and
 *           shifts and logs the relative gap as dir_err_fp64 -- an extra FP64
 *           product and factorization per step, counted in the statistics;
 *           the solve itself takes the mixed-precision direction as before)
 *   double: tol, mu0, kappa_eps, kappa_mu, theta_mu, tau_min, s_max, kappa_1,
 *           kappa_2, kappa_sigma, gamma_theta, gamma_phi, delta, s_theta, s_phi,
 *           eta_phi, gamma_alpha, dw0, dw_min, dw_max, kw_minus, kw_plus,
 *           kw_plus_bar, dc_bar, kappa_c, zero_tol, time_limit_s, refine_tol,
 *           refine_fallback_tol
 *   string: path ("auto" | "p1" | "p2"), precision ("fp64" | "tf32" | "bf16"),
 *           graphs / autotune / ldlt_spec as "yes" | "no", ldlt_spec also
 *           "persistent" (2) -- the same settings as the int options of
 *           those names, by word.
 * Unknown names or values: INVALID_ARG (the option keeps its value). */
mdsip_status mdsip_set_option_int(mdsip_problem *p, const char *name, int64_t value);
mdsip_status mdsip_set_option_double(mdsip_problem *p, const char *name, double value);
mdsip_status mdsip_set_option_str(mdsip_problem *p, const char *name, const char *value);

/* Packed primal-dual layout used by set_start / get_iterate / debug_direction:
 *   [x (n) | d (m_I) | y_g (m_E) | y_h (m_I) | z_l (n) | z_u (n) | v_l (m_I) | v_u (m_I)]
 * Multipliers of infinite bounds are 0. */
int64_t mdsip_packed_size(const mdsip_problem *p);

/* Warm start: use `packed` as the starting primal-dual point and mu0 (<= 0:
 * the option mu0).  The point must be strictly inside the finite bounds.
 * packed == NULL clears the warm start (next solve starts from x0). */
mdsip_status mdsip_set_start(mdsip_problem *p, const double *packed, double mu0, int mem);

/* Run the filter line-search interior-point method (Section 2.1) to E_0 <= tol.
 * Returns the final status (OK, MAX_ITER, INERTIA, RESTORATION_NEEDED,
 * NONFINITE, TIMEOUT, or an error). */
mdsip_status mdsip_solve(mdsip_problem *p);

mdsip_status mdsip_get_iterate(mdsip_problem *p, double *packed, int mem);

/* ---- Learned warm start (not part of the paper's method) -----------------
 * A network maps the parameters of a parametric family to a predicted
 * packed primal-dual point followed by log mu0 (packed_size + 1 values); the
 * plain method started from it decides whether the result is accepted (E_0 <= tol).
 *
 * mdsip_warmstart_target: after a solve of p, write the training target for
 * that instance: the final packed iterate, then log of the barrier parameter
 * of the first logged iteration whose E_0 <= e0_level (the final one if none
 * is).  out: packed_size + 1 doubles, `mem`-tagged.  INVALID_ARG if p has not
 * been solved.
 *
 * mdsip_set_start_predicted: warm start from a prediction (packed_size + 1
 * floats, `mem`-tagged): mu0 = exp(log mu0) kept inside [tol / 10, option
 * mu0]; x and d pushed inside their bounds by the Section 3.6 rule of W&B
 * with kappa_1 = kappa_2 = push (0 < push < 0.5); each finite-bound
 * multiplier at least mu0 / its slack; multipliers of infinite bounds 0; y as
 * predicted.  Bounds must be set.  mdsip_set_start(p, NULL, ..) clears it. */
mdsip_status mdsip_warmstart_target(mdsip_problem *p, double e0_level, double *out, int mem);
mdsip_status mdsip_set_start_predicted(mdsip_problem *p, const float *pred, double push, int mem);

/* Solve `count` independent problems concurrently (the "many instances"
 * setting of Section 1.1: one IPM solve per contingency scenario).  Problems
 * whose contexts share a CUDA stream run one after another on it; problems on
 * different streams run concurrently, one host worker thread per stream, at
 * most `max_concurrent` at a time (<= 0: no limit).  statuses[i] receives
 * problem i's mdsip_solve status.  Returns OK when every problem was attempted
 * (check the statuses), or INVALID_ARG. */
mdsip_status mdsip_batch_solve(mdsip_problem *const *problems, int32_t count, int32_t max_concurrent,
                               int32_t *statuses);

typedef struct {
    int32_t status;
    int32_t iters;
    int32_t path;              /* MDSIP_PATH_P1 or MDSIP_PATH_P2 as used           */
    int32_t n_factorizations;  /* LDL^T factorizations (incl. inertia retries)     */
    int64_t n_ls_trials;
    double f, E0, inf_pr, inf_du, mu;
    double t_total_ms;
    double t_condense_ms, t_factor_ms, t_solve_ms, t_ls_ms;  /* CUDA-event phase times */
    double t_syrk_ms, t_ldlt_ms;  /* CUDA-event time of the condensation-product and the
                                     LDL^T kernels alone (stream of the launches)        */
    int32_t n_syrk, n_ldlt;       /* launches of those kernels                          */
    int64_t n_refine;             /* iterative-refinement sweeps over the solve         */
    int32_t n_fp64_fallback;      /* steps re-factored in FP64 after refinement stalled */
    int32_t precision;            /* MDSIP_PREC_* of the condensation product           */
    double t_refine_ms;           /* CUDA-event time of the direction solves incl. refinement */
} mdsip_stats;
mdsip_status mdsip_get_stats(mdsip_problem *p, mdsip_stats *out);

#define MDSIP_MAX_IC 16
typedef struct {
    int32_t iter;
    int32_t n_ic;                       /* inertia-correction attempts this step */
    int32_t n_ls;                       /* rejected trial steps                  */
    int32_t ftype;                      /* accepted as f-type (Armijo) step      */
    double mu, f, theta, E0, inf_pr, inf_du;
    double alpha, alpha_max, alpha_z, gphi;
    double ic_dw[MDSIP_MAX_IC], ic_dc[MDSIP_MAX_IC];
    int32_t ic_inertia[MDSIP_MAX_IC][3]; /* (pos, neg, zero) of the 4x4 matrix    */
    int32_t n_refine;                   /* refinement sweeps of this step         */
    int32_t fp64_fallback;              /* 1 if the step was re-factored in FP64  */
    double refine_res;                  /* final ||b - K u||inf / (||b|| + ||K u||) */
    int32_t factor_inertia[3];          /* (pos, neg, zero) of the factor the direction
                                           was solved with: after an FP64 re-factorization
                                           that factor's, which must equal the target; when
                                           it did not, Algorithm IC was rerun on FP64 factors
                                           and its attempts follow in ic_*                  */
    int32_t pad_;
    double dir_err_fp64;                /* with the option direction_check on a
                                           mixed-precision solve: ||D - D_64||_2 / ||D_64||_2
                                           between the step's direction D and the FP64
                                           direction D_64 from the same iterate and shifts
                                           (FP64 product and factorization); -1 otherwise */
} mdsip_iter_rec;
/* Copy up to `cap` per-iteration records; *n receives the number available. */
mdsip_status mdsip_get_log(mdsip_problem *p, mdsip_iter_rec *buf, int32_t cap, int32_t *n);

/* Parity hook: one Newton direction at a given packed iterate with fixed
 * shifts (no inertia correction).  dir_out receives the packed direction
 * (same layout as the iterate); inertia_out the (pos, neg, zero) inertia of
 * the 4x4 matrix of Eq. (linsys4x4) obtained by Haynsworth additivity
 * (Section 2.3).  `refine` > 0 adds up to that many iterative-refinement
 * sweeps on the unreduced operator. */
mdsip_status mdsip_debug_direction(mdsip_problem *p, const double *packed, double mu, double dw,
                                   double dc, int32_t refine, double *dir_out,
                                   int32_t inertia_out[3], int mem);

/* Number of CUDA kernels this library has launched in the process so far. */
int64_t mdsip_launch_count(void);

/* Measurement aid (the paper has no counterpart): the FP64 fused multiply-add
 * rate that bounds the FP64 condensation product and factorization.  Launches
 * `blocks` x 256 threads on the context's stream; every thread performs
 * iters x 8 independent FP64 FMAs (2 flop each) and writes one double to
 * sink (device, blocks x 256 doubles, owned by the caller).  Returns once the
 * launch is enqueued; time it with events on the context's stream.
 * blocks <= 0, iters <= 0 or sink == NULL: INVALID_ARG. */
mdsip_status mdsip_probe_fp64_fma(mdsip_ctx *ctx, int32_t blocks, int64_t iters, double *sink);

/* ------------------------------------------------------------------------- */
/* Kernel-level entry points (device pointers, context stream).              */
/* ------------------------------------------------------------------------- */

/* Condensation product of the two-stage elimination (Section 2.2 K3-type
 * update, M := M + A D B^T with A = B):
 *   C[p][q] = beta * C[p][q] + sum_i A[i][p] * A[i][q] / w[i]   for p >= q,
 * A: m x n row-major with leading dimension lda (lda >= n, lda % 2 == 0),
 * w: m (nonzero), C: n x n column-major, leading dimension ldc; only the lower
 * triangle (p >= q) is written.  beta is 0 or 1.  FP64 throughout. */
mdsip_status mdsip_syrk_scaled(mdsip_ctx *ctx, int64_t m, int64_t n, const double *A, int64_t lda,
                               const double *w, double beta, double *C, int64_t ldc);

/* The same product on the tensor cores: precision MDSIP_PREC_TF32 or
 * MDSIP_PREC_BF16 operands A[i][p] * w_i^-1/2 (rounded to that type), FP32
 * accumulation over K ranges, the ranges' partial sums added in FP32 and
 * their total added to C in FP64.  Arguments as above
 * (w > 0 required).  Relative error per entry of order the operand type's
 * unit roundoff times sum_i |A[i][p] A[i][q]| / w_i. */
mdsip_status mdsip_syrk_scaled_tc(mdsip_ctx *ctx, int64_t m, int64_t n, const double *A, int64_t lda,
                                  const double *w, double beta, double *C, int64_t ldc,
                                  int precision);

/* The two products with the dense Jacobian block that the FP64 residual of
 * Eq. (linsys4x4) needs (the A u_d and A^T u_g terms), from one pass over A in
 * double-float arithmetic (the form the refined mixed-precision path uses):
 *   Ax[i] = sum_p A[i][p] x[p]  (i < m),   ATv[p] = sum_i A[i][p] v[i]  (p < n).
 * A: m x n row-major, leading dimension lda (lda >= n, lda % 4 == 0, 16-byte
 * aligned); x: n, v: m; Ax: m, ATv: n; all device pointers owned by the
 * caller.  A is split once into A_hi = fl32(A), A_lo = fl32(A - A_hi) (library
 * scratch); every product is formed exactly on the FP32 pipes and the sums
 * are folded into FP64 every 16 terms.  Worst case, each result is within
 * 2^-36 sum_p |A[i][p] x[p]| (resp. sum_i |A[i][p] v[i]|) of the exact value
 * for n, m <= 2^20 (split and cross terms 7 2^-48, FP32 carries of a 16-term
 * block and of the block reduction about 1100 2^-48, FP64 folds n/16 2^-53,
 * each times that sum); typical errors are those of an FP64 product.
 * Returns after the results are written (synchronises the context's stream).
 * Errors: INVALID_ARG (sizes, alignment, null pointers), OOM. */
mdsip_status mdsip_gemv_pair_df(mdsip_ctx *ctx, int64_t m, int64_t n, const double *A, int64_t lda,
                                const double *x, const double *v, double *Ax, double *ATv);

/* The same pass with the first half of the refinement's next approximate
 * solve folded in (the FP32 A^T product of the two-stage elimination of
 * Section 2.3, whose input needs the whole row sum of A x).  Besides Ax and
 * ATv as in mdsip_gemv_pair_df it writes
 *   ATw[p] = sum_i A_hi[i][p] w[i],   A_hi = fl32(A),   w[i] = fl32(d[i] fl32(winv[i])),
 * d[i] the difference cpre[i] - Ax[i] formed in double-float from cpre split
 * into FP32 halves and the pass's own row sum, rounded to FP32
 * (|d[i] - (cpre[i] - Ax[i])| <= 2^-23 |cpre[i] - Ax[i]| + 2^-46 |cpre[i]|);
 * FP32 products and FP32 sums over blocks of at most ceil(m / number of SMs)
 * consecutive rows, the block sums added in FP64.  cpre, winv: m; ATw: n; device pointers owned by the caller;
 * 1 <= n <= 2048 (one slice of the pass holds a row).  Returns after the
 * results are written.  Errors: as mdsip_gemv_pair_df, and INVALID_ARG for
 * n outside 1 .. 2048 or a null operand. */
mdsip_status mdsip_gemv_pair_df_next(mdsip_ctx *ctx, int64_t m, int64_t n, const double *A, int64_t lda,
                                     const double *x, const double *v, const double *cpre,
                                     const double *winv, double *Ax, double *ATv, double *ATw);

/* Bunch-Kaufman LDL^T (Section 2.3) of the symmetric N x N matrix whose lower
 * triangle is in S (column-major, leading dimension ld).  S is overwritten
 * (used as work space).  Outputs (device):
 *   L:     N x N column-major unit lower triangular (leading dimension N)
 *   Dd:    N   diagonal of D;  Doff: N   Doff[k] = D[k+1][k] for 2x2 blocks, else 0
 *   perm:  N   P S P^T = L D L^T with (P v)[i] = v[perm[i]]
 *   kind:  N   1 = 1x1 pivot, 2 = first column of a 2x2 pivot, 0 = second column
 *   inertia: 3 (pos, neg, zero); a 1x1 pivot |d| <= zero_tol * max|S| counts zero.
 * Errors: INVALID_ARG, OOM, DEVICE (a bounded device wait expired). */
mdsip_status mdsip_ldlt_factor(mdsip_ctx *ctx, int64_t N, double *S, int64_t ld, double zero_tol,
                               double *L, double *Dd, double *Doff, int32_t *perm, int32_t *kind,
                               int32_t *inertia);

/* mdsip_ldlt_factor with options.  flags: 0, or MDSIP_LDLT_FP32_UPDATES
 * (the mixed-precision factorization of the refined path: the panels'
 * column updates and the trailing updates take FP32 products subtracted from
 * the FP64 matrix; pivot tests, D and the inertia stay FP64; the result is an
 * approximate factor meant for iterative refinement, and the unblocked kernel
 * used where thread-block clusters are unavailable ignores the flag), to
 * which MDSIP_LDLT_NO_SPECULATION may be added.  Without it, each panel of
 * the FP32-update factorization is first factored without interchanges and
 * kept only if the Bunch-Kaufman rule (Section 2.3), evaluated on the
 * computed columns, would have chosen a 1x1 pivot without interchange for
 * every column of the panel (and no pivot is below zero_tol times the
 * largest |S_ij|); otherwise the pivoting panel factors it from the
 * unchanged matrix.  The flag makes every panel take the pivoting kernel.
 * From order 2048 on (and wherever the pivoting panel does not fit shared
 * memory, N above about 16 000), and at any order with MDSIP_LDLT_PERSISTENT,
 * the no-interchange panels of either precision run in one persistent
 * cooperative kernel that stops at the first panel the rule would not keep;
 * the pivoting panels take over from there (beyond the pivoting panel's
 * limit such a panel is an INVALID_ARG error).  With FP32 updates that
 * kernel works on an FP32 copy of S (the FP32 updates are written back into
 * S before a hand-over; large trailing matrices are updated on the tensor
 * cores with a three-product TF32 split, about FP32 accuracy).  The call then
 * reads a status word back, so it synchronises the context's stream. */
#define MDSIP_LDLT_FP32_UPDATES 1
#define MDSIP_LDLT_NO_SPECULATION 2
#define MDSIP_LDLT_PERSISTENT 4
mdsip_status mdsip_ldlt_factor_ex(mdsip_ctx *ctx, int64_t N, double *S, int64_t ld, double zero_tol,
                                  int32_t flags, double *L, double *Dd, double *Doff, int32_t *perm,
                                  int32_t *kind, int32_t *inertia);

/* Panel counts of the last mdsip_ldlt_factor / mdsip_ldlt_factor_ex call on
 * ctx (host array of 2): out2[0] = panels kept by the verified
 * no-interchange path, out2[1] = panels it handed to the pivoting kernel.
 * Both are 0 when that path did not run (FP64 updates, MDSIP_LDLT_NO_SPECULATION,
 * or the unblocked kernel). */
mdsip_status mdsip_ldlt_panel_counts(mdsip_ctx *ctx, int32_t *out2);

/* Allocation-free variant of mdsip_ldlt_factor (same arguments, same
 * results).  The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc -- a host whose device memory belongs in full to
 * another allocator (a framework's caching allocator, the pre-sized arena of
 * a real-time controller), or a loop that must not pay the implicit device
 * synchronisation that allocating and freeing can cause.  Its scratch is a
 * fixed device array of the library (8 MiB plus 16 KiB, held by every GPU that
 * loads the library until the process exits), so:
 *   - N is limited to 1024 (larger N: MDSIP_ERR_INVALID_ARG);
 *   - it allocates no device memory (no cudaMalloc/cudaFree, no allocating
 *     library routine);
 *   - the first call on a device looks up the array's device address
 *     (set-up, once per device); make that first call before any stream
 *     capture.  The address is kept for the life of the process: after a
 *     cudaDeviceReset of that device do not call this entry point again;
 *   - every call shares the array: calls that overlap on the GPU (on two
 *     streams, or from two host threads) race and must not be issued.
 * The call returns after the factorization has finished (it reads a device
 * status word). */
mdsip_status mdsip_ldlt_factor_noalloc(mdsip_ctx *ctx, int64_t N, double *S, int64_t ld,
                                       double zero_tol, double *L, double *Dd, double *Doff,
                                       int32_t *perm, int32_t *kind, int32_t *inertia);

/* Solve (P^T L D L^T P) x = b in place for `nrhs` right-hand sides stored
 * column-major in B (leading dimension ldb), with the factors above. */
mdsip_status mdsip_ldlt_solve(mdsip_ctx *ctx, int64_t N, const double *L, const double *Dd,
                              const double *Doff, const int32_t *perm, int64_t nrhs, double *B,
                              int64_t ldb);

/* ---- Warm-start network ----------------------------------------------------
 * Two ReLU hidden layers of width n_hidden:
 *   h1 = relu(W1 xn + b1), h2 = relu(W2 h1 + b2), yn = W3 h2 + b3,
 * xn = (x - in_mean) / in_std per input, y = yn * out_std + out_mean per
 * output.  Training minimises L = sum (yn - (y* - out_mean) / out_std)^2 / (B
 * n_out) over a batch of B rows with Adam (bias-corrected; defaults beta1 0.9,
 * beta2 0.999, eps 1e-8).  Every contraction runs in BF16 on the tensor cores
 * with FP32 accumulation; parameters, gradients and moments are FP32.  BF16
 * rounding (to nearest even) is applied to xn, W1, W2, W3, h1, h2, dL/dyn and
 * the hidden-layer gradients dL/dz2, dL/dz1; bias gradients are sums of the
 * rounded values.
 *
 * Parameter vector (FP32): W1 (n_hidden x n_in, row-major) | b1 | W2 (n_hidden
 * x n_hidden) | b2 | W3 (n_out x n_hidden) | b3, each block starting at the
 * offset mdsip_mlp_param_offsets returns (multiples of 4 floats; gaps are
 * ignored).  New networks have zero parameters, zero means and unit standard
 * deviations.
 *
 * X (inputs) and Y (targets) are DEVICE pointers to FP64 row-major matrices
 * with row strides ldx >= n_in and ldy >= n_out; idx (device int32, nullable
 * = rows 0..batch-1) selects the batch rows.  Errors: INVALID_ARG, OOM, CUDA,
 * DEVICE (a tensor-core pipeline wait expired). */
typedef struct mdsip_mlp mdsip_mlp;

/* The contraction every layer uses: C[m][n] = sum_k A[m][k] B[n][k] with A
 * (M x K) and B (N x K) BF16 row-major (raw 16-bit patterns; rows 16-byte
 * aligned: lda, ldb multiples of 8), FP32 accumulation on the tensor cores,
 * C FP32 row-major (ldc >= N).  Device pointers. */
mdsip_status mdsip_gemm_bf16(mdsip_ctx *ctx, int64_t M, int64_t N, int64_t K, const uint16_t *A, int64_t lda,
                             const uint16_t *B, int64_t ldb, float *C, int64_t ldc);

mdsip_status mdsip_mlp_create(mdsip_ctx *ctx, int64_t n_in, int64_t n_hidden, int64_t n_out, mdsip_mlp **out);
void mdsip_mlp_destroy(mdsip_mlp *m);
int64_t mdsip_mlp_num_params(const mdsip_mlp *m);
mdsip_status mdsip_mlp_param_offsets(const mdsip_mlp *m, int64_t offsets[6]);
/* Set (`mem`-tagged, num_params floats) or read the parameters; setting them
 * resets the Adam moments and step count. */
mdsip_status mdsip_mlp_set_params(mdsip_mlp *m, const float *params, int mem);
mdsip_status mdsip_mlp_get_params(mdsip_mlp *m, float *params, int mem);
mdsip_status mdsip_mlp_set_adam(mdsip_mlp *m, double beta1, double beta2, double eps);
/* Standardisation (`mem`-tagged floats; a NULL argument leaves that vector
 * unchanged; standard deviations must be positive). */
mdsip_status mdsip_mlp_set_scaling(mdsip_mlp *m, const float *in_mean, const float *in_std, const float *out_mean,
                                   const float *out_std, int mem);
mdsip_status mdsip_mlp_get_scaling(mdsip_mlp *m, float *in_mean, float *in_std, float *out_mean, float *out_std,
                                   int mem);
/* Column means and standard deviations of `count` rows of X and Y (FP64
 * sums; a standard deviation below 1e-6 max(1, |mean|) is raised to it). */
mdsip_status mdsip_mlp_fit_scaling(mdsip_mlp *m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                                   int64_t count);
/* Prediction y for `batch` rows of X into Y (device FP32, row stride ldy). */
mdsip_status mdsip_mlp_forward(mdsip_mlp *m, const double *X, int64_t ldx, int64_t batch, float *Y, int64_t ldy);
/* Loss (host, nullable) and gradient dL/dparams (device, num_params floats,
 * nullable) of one batch, without updating the parameters. */
mdsip_status mdsip_mlp_gradient(mdsip_mlp *m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                                const int32_t *idx, int64_t batch, float *grad, double *loss);
/* One Adam step with learning rate lr on one batch.  loss (host, nullable)
 * receives the batch loss before the step; NULL avoids a synchronisation. */
mdsip_status mdsip_mlp_train_step(mdsip_mlp *m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                                  const int32_t *idx, int64_t batch, double lr, double *loss);

#ifdef __cplusplus
}
#endif
#endif /* MDSIP_H */
