/*
 * cggm.h — C ABI of the GB300 solver for l1-regularised conditional Gaussian graphical
 * models by alternating Newton coordinate descent (McCarter & Kim, "Large-Scale
 * Optimization Algorithms for Sparse Conditional Gaussian Graphical Models", AISTATS 2016).
 *
 * The problem (Eq. 1):
 *     min_{Lambda > 0, Theta}  -log|Lambda| + tr(S_yy Lambda + 2 S_xy^T Theta
 *                               + Lambda^-1 Theta^T S_xx Theta)
 *                               + lam_L ||Lambda||_1 + lam_T ||Theta||_1
 * with S_xx = X^T X / n, S_xy = X^T Y / n, S_yy = Y^T Y / n (Section 2.1); Lambda is q x q
 * (the output network), Theta is p x q (inputs to outputs).
 *
 * Conventions for every entry point below:
 *  - Matrices are dense and row-major.  X is n x p (one sample per row), Y is n x q,
 *    Lambda is q x q, Theta is p x q.
 *  - A data pointer may be host or device memory; the library tells them apart with
 *    cudaPointerGetAttributes.  Host inputs are copied to the device inside the call;
 *    host outputs are copied back before the call returns.  The caller owns every
 *    buffer it passes and the library never frees or retains them.
 *  - Every call runs on the context's device and stream and returns only after its
 *    results are complete (host-visible for host outputs, stream-ordered and synchronised
 *    for device outputs).
 *  - The return code is the only error channel; no call aborts the process.  On error
 *    the outputs are unspecified and the context stays usable.
 *  - A context is not thread-safe: one call at a time per context.
 */
#ifndef CGGM_H
#define CGGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CGGM_OK = 0,
    CGGM_EINVAL = -1,      /* bad shape, negative lambda, tol <= 0, null pointer        */
    CGGM_ENOTPD = -2,      /* Lambda (warm start or argument) is not positive definite  */
    CGGM_ENOMEM = -3,      /* device allocation failed                                  */
    CGGM_EMAXITER = -4,    /* max_iter reached before the stopping rule held            */
    CGGM_ELINESEARCH = -5, /* Armijo found no step within ls_max_trials                 */
    CGGM_ECUDA = -6,       /* a CUDA runtime call failed                                */
    CGGM_ETIMEDOUT = -7,   /* a device-side wait gave up (grid barrier deadline)        */
    CGGM_ENONFINITE = -8,  /* NaN or Inf in the inputs or in a computed quantity        */
    CGGM_ECANCELLED = -9   /* the request was cancelled                                 */
} cggm_status;

typedef enum {
    CGGM_FP64 = 0,  /* every kernel in double precision                                */
    CGGM_MIXED = 1  /* contractions and sweep state in single precision (tensor cores   */
                    /* for the products from X); Cholesky, log det, objective, Sigma    */
                    /* and Psi diagonals and coordinate coefficients in double          */
} cggm_precision;

/* Element types of X and Y (row-major n x p, n x q).  CGGM_BF16: bfloat16 values, used as
 * they are.  CGGM_I8_GENO (X only): int8 values, typically genotype counts {0, 1, 2}; the
 * library standardises every column with its mean and population standard deviation over
 * the n rows, (x - mean) / sd in double, so that diag(S_xx) = 1 (a constant column becomes
 * zero, and its Theta row stays zero).  The paper does not fix the storage; its genomic
 * inputs are genotype counts (Section 5.2). */
typedef enum { CGGM_F32 = 0, CGGM_F64 = 1, CGGM_BF16 = 2, CGGM_I8_GENO = 3 } cggm_dtype;

/* opts.sweep_batch value that lets the batch-size tuner choose (see cggm_tuned_batch). */
#define CGGM_SWEEP_BATCH_AUTO (-1)

typedef struct {
    double tol;          /* stopping ratio of Section 5.1: stop when
                            ||grad^S f||_1 < tol (||Lambda||_1 + ||Theta||_1); 0.01      */
    int max_iter;        /* Newton iterations (Algorithm 1 outer loop); 1000              */
    int precision;       /* cggm_precision; CGGM_MIXED                                    */
    double ls_sigma;     /* Armijo sufficient-decrease constant; 1e-3                     */
    double ls_beta;      /* Armijo step shrink factor; 0.5                                */
    int ls_max_trials;   /* Armijo trials before CGGM_ELINESEARCH; 50                     */
    int penalize_diag;   /* include diag(Lambda) in ||Lambda||_1; 1                       */
    int sweep_batch;     /* coordinates per blocked Gauss-Seidel batch: 32, 64, 128, or
                            256 and 512 in the mixed path; 0 = default (128 FP64, 256);
                            CGGM_SWEEP_BATCH_AUTO = chosen by the tuner (cggm_tuned_batch) */
    double target_f;     /* also stop once f <= target_f (time-to-gap runs); -inf = off  */
    int verbose;         /* per-iteration line on stderr                                  */
    int64_t sxx_rows;    /* rows of S_xx = X^T X / n held at once by the Theta pass, formed
                            from X chunk by chunk; 0 = as many as fit in 256 MiB (all p
                            rows, formed once per solve, when they fit)                    */
} cggm_opts;

typedef struct {
    int iterations;         /* Newton iterations run                                     */
    int converged;          /* stopping rule (or target_f) satisfied                     */
    double f;               /* objective (Eq. 1) at the returned point, double precision */
    double subgrad;         /* ||grad^S f||_1 at the returned point                      */
    double l1norm;          /* ||Lambda||_1 + ||Theta||_1 at the returned point          */
    int64_t m_lambda;       /* last active-set sizes                                     */
    int64_t m_theta;
    int ls_trials;          /* Armijo trials summed over iterations                      */
    double seconds;         /* device time of the solve (CUDA events)                    */
    double sec_products;    /* R, P, Psi, gradients                                      */
    double sec_factor;      /* Sigma from the accepted step's factor, and W for the Theta */
                            /* pass (the Armijo trials' factorisations: sec_linesearch)   */
    double sec_active;      /* subgradient, active sets                                  */
    double sec_sweep_lambda;  /* the Lambda pass                                         */
    double sec_linesearch;    /* Armijo: trial factorisations and objectives             */
    double sec_sweep_theta;   /* the Theta pass                                          */
    int64_t launches;       /* CUDA kernels this library launched during the call        */
    int64_t coords_lambda;  /* coordinate steps taken by all Lambda passes of the call   */
    int64_t coords_theta;   /* coordinate steps taken by all Theta passes of the call    */
} cggm_info;

typedef struct cggm_ctx cggm_ctx;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream` (a
 * cudaStream_t, or NULL for a stream owned by the context).  Allocates nothing large
 * until the first call that needs workspace.  Returns CGGM_EINVAL for a bad device. */
cggm_status cggm_create(cggm_ctx **ctx, int device, void *cuda_stream);

/* Release the context and all device workspace it owns.  NULL is ignored. */
void cggm_destroy(cggm_ctx *ctx);

/* Fill `opts` with the defaults listed beside each field. */
void cggm_opts_default(cggm_opts *opts);

/* Short English name of a status code (static storage). */
const char *cggm_status_string(int status);

/* A sparse matrix as a coordinate list: entry e is (row[e], col[e], val[e]), 0 <= e < nnz.
 * The paper keeps Lambda and Theta in sparse form (Section 5); Lambda, being symmetric, is
 * exchanged as its upper triangle (row <= col), Theta in full. */
typedef struct {
    int64_t nnz;
    int32_t *row;
    int32_t *col;
    double *val;
} cggm_coo;

/*
 * Solve Eq. 1 by alternating Newton coordinate descent (Algorithm 1): Theta <- 0,
 * Lambda <- I (or the warm start); each iteration computes Sigma = Lambda^-1 by Cholesky,
 * Psi, the gradients (Eq. 3), the stopping ratio and the active sets (Section 2.2), one
 * coordinate-descent pass for the Newton direction of Lambda (Section 3.1, Eq. 7), an
 * Armijo step on Lambda, and one coordinate-descent pass on Theta (Section 3.2, Eq. 8).
 *
 * X: n x p, dtype xdtype; Y: n x q, dtype ydtype (host or device).  lam_L, lam_T >= 0.
 * tol > 0 overrides opts->tol.  info may be NULL.  opts may be NULL (defaults).
 * Parameters are exchanged sparse:
 *  - warm_Lambda: the upper triangle (row <= col) of a symmetric positive definite q x q
 *    start, warm_Theta: the entries of a p x q start; either may be NULL (then I and 0).
 *    Their arrays may be host or device memory and stay the caller's; repeated entries
 *    add up.  An index outside the matrix (or row > col for Lambda) gives CGGM_EINVAL, a
 *    non-finite value CGGM_ENONFINITE, a warm Lambda that is not positive definite
 *    CGGM_ENOTPD.
 *  - Lambda_out (upper triangle) and Theta_out receive the nonzero entries of the solution
 *    in row-major order, exact zeros dropped, in arrays the library allocates in host
 *    memory; release them with cggm_free_coo.  Either may be NULL.  On an error return
 *    they are left empty (nnz 0, NULL arrays).
 * Returns CGGM_OK when the stopping rule held, CGGM_EMAXITER when max_iter ran out (the
 * outputs then hold the last iterate), or an error.
 */
cggm_status cggm_solve(cggm_ctx *ctx, const void *X, int xdtype, const void *Y, int ydtype,
                       int64_t n, int64_t p, int64_t q, double lam_L, double lam_T,
                       double tol, const cggm_coo *warm_Lambda, const cggm_coo *warm_Theta,
                       const cggm_opts *opts, cggm_coo *Lambda_out, cggm_coo *Theta_out,
                       cggm_info *info);

/* Release the arrays of a coordinate list returned by cggm_solve and empty it.  NULL, and
 * an already empty list, are ignored. */
void cggm_free_coo(cggm_coo *coo);

/*
 * cggm_solve with dense parameters, for callers that keep Lambda and Theta as dense
 * matrices (for instance in device memory between calls, as the regularisation-path
 * server does).  warm_Lambda (q x q, symmetric positive definite) and warm_Theta (p x q)
 * are double, host or device, and may be NULL (then I and 0).  Lambda_out (q x q) and
 * Theta_out (p x q) receive the solution in double, host or device.  Everything else as
 * for cggm_solve.
 */
cggm_status cggm_solve_dense(cggm_ctx *ctx, const void *X, int xdtype, const void *Y,
                             int ydtype, int64_t n, int64_t p, int64_t q, double lam_L,
                             double lam_T, double tol, const double *warm_Lambda,
                             const double *warm_Theta, const cggm_opts *opts,
                             double *Lambda_out, double *Theta_out, cggm_info *info);

/*
 * Prediction with a fitted model (Section 2.1): given x, y is Gaussian with mean
 * -Lambda^-1 Theta^T x, so the rows of X (n x p, dtype xdtype, host or device; genotype
 * counts are standardised as in cggm_solve) predict Yhat = X B with the regression
 * coefficients B = -Theta Sigma, Sigma = Lambda^-1.  Lambda (upper triangle) and Theta are
 * coordinate lists as cggm_solve returns them (host or device arrays).
 *   Yhat_out: n x q row-major double, B_out: p x q row-major double (host or device); either
 *   may be NULL, not both.  Double precision throughout (Cholesky of Lambda, Sigma, the
 *   product over Theta's nonzeros).
 * Errors: CGGM_EINVAL (sizes, a NULL pointer, an index outside its matrix or below the
 * diagonal of Lambda), CGGM_ENONFINITE (a non-finite value), CGGM_ENOTPD (Lambda not
 * positive definite).
 */
cggm_status cggm_predict(cggm_ctx *ctx, const void *X, int xdtype, int64_t n, int64_t p,
                         int64_t q, const cggm_coo *Lambda, const cggm_coo *Theta,
                         double *Yhat_out, double *B_out);

/*
 * f(Lambda, Theta) of Eq. 1 in double precision on the device.  Lambda must be positive
 * definite (CGGM_ENOTPD otherwise).  penalize_diag as in cggm_opts.
 */
cggm_status cggm_objective(cggm_ctx *ctx, const void *X, int xdtype, const void *Y,
                           int ydtype, int64_t n, int64_t p, int64_t q,
                           const double *Lambda, const double *Theta, double lam_L,
                           double lam_T, int penalize_diag, double *f_out);

/*
 * Gradients of the smooth part (Eq. 3) in double precision:
 *     G_Lambda = S_yy - Sigma - Psi (q x q),  G_Theta = 2 S_xy + 2 S_xx Theta Sigma (p x q),
 * computed from X as (2/n) X^T (Y + X Theta Sigma), so S_xx is never formed.
 */
cggm_status cggm_grad(cggm_ctx *ctx, const void *X, int xdtype, const void *Y, int ydtype,
                      int64_t n, int64_t p, int64_t q, const double *Lambda,
                      const double *Theta, double *G_Lambda, double *G_Theta);

/*
 * Step-level entry points: one kernel of the Newton iteration each, on caller data, so
 * that every step can be checked on its own.  All matrices double, host or device.
 */

/* Cholesky Lambda = L L^T (lower L, row-major q x q, upper part of L_out set to 0),
 * log|Lambda| = 2 sum log L_ii, and Sigma = Lambda^-1 (Section 2.3's Cholesky
 * initialisation of Sigma), all in double (`precision` is ignored).  Lambda is read, the
 * outputs written, in host or device memory owned by the caller; L_out, logdet_out and
 * Sigma_out may each be NULL.  Errors: CGGM_EINVAL for q <= 0 or a null Lambda;
 * CGGM_ENOTPD if Lambda is not positive definite (a pivot <= 0 or not finite). */
cggm_status cggm_cholesky(cggm_ctx *ctx, int64_t q, const double *Lambda, double *L_out,
                          double *logdet_out, double *Sigma_out, int precision);

/* One coordinate-descent pass for the Newton direction of Lambda (Section 3.1, Eq. 7;
 * coordinate step of Appendix A.1 with the curvature of the exact quadratic model).
 * Sigma, Psi, Syy, Lambda: q x q row-major double.  (ai[k], aj[k]), ai <= aj, k < m, are
 * the active coordinates in visiting order.  D_out (q x q) receives the symmetric
 * direction.  precision: CGGM_FP64 (caches in double, batches of 128) or CGGM_MIXED
 * (caches in float, batches of 256).  All buffers host or device, owned by the caller.
 * Errors: CGGM_EINVAL for q <= 0, m < 0, a null pointer, another precision, or an index
 * pair outside 0 <= ai <= aj < q (checked on the host before any kernel runs);
 * CGGM_ETIMEDOUT if a device wait of the pass gave up; CGGM_ENONFINITE for a NaN or Inf
 * met in a step. */
cggm_status cggm_lambda_sweep(cggm_ctx *ctx, int64_t q, const double *Sigma,
                              const double *Psi, const double *Syy, const double *Lambda,
                              int64_t m, const int32_t *ai, const int32_t *aj, double lam_L,
                              int penalize_diag, int precision, double *D_out);

/* One coordinate-descent pass on Theta with Lambda fixed (Section 3.2, Eq. 8; Appendix
 * A.1 coordinate step with curvature 2 Sigma_jj (S_xx)_ii).  X is n x p (double), S_xy
 * p x q, Sigma q x q, all row-major; (ti[k], tj[k]), k < m, the active coordinates in
 * visiting order, any order (a list in ascending rows, as the active sets are, runs
 * fastest).  Theta (p x q) is read from Theta_in and the result written to
 * Theta_out (may alias).  precision as for cggm_lambda_sweep.  All buffers host or
 * device, owned by the caller.  Errors: CGGM_EINVAL for sizes <= 0, m < 0, a null
 * pointer, another precision, or an index outside 0 <= ti < p, 0 <= tj < q (checked on
 * the host before any kernel runs); CGGM_ETIMEDOUT and CGGM_ENONFINITE as for
 * cggm_lambda_sweep. */
cggm_status cggm_theta_sweep(cggm_ctx *ctx, int64_t n, int64_t p, int64_t q,
                             const double *X, const double *Sxy, const double *Sigma,
                             const double *Theta_in, int64_t m, const int32_t *ti,
                             const int32_t *tj, double lam_T, int precision,
                             double *Theta_out);

/* Active sets of Section 2.2 from gradients and parameters: Lambda entries (i <= j) with
 * |G_Lambda| > lam_L or Lambda != 0, Theta entries with |G_Theta| > lam_T or Theta != 0,
 * both in row-major order (with penalize_diag = 0 every diagonal entry is active).
 * G_Lambda, Lambda: q x q; G_Theta, Theta: p x q; row-major double, host or device.  The
 * caller's index buffers must hold q(q+1)/2 (li, lj) and p q (ti, tj) entries; the counts
 * are returned in *m_lambda and *m_theta.  Errors: CGGM_EINVAL for sizes <= 0 or a null
 * pointer. */
cggm_status cggm_active_sets(cggm_ctx *ctx, int64_t p, int64_t q, const double *G_Lambda,
                             const double *G_Theta, const double *Lambda,
                             const double *Theta, double lam_L, double lam_T,
                             int penalize_diag, int32_t *li, int32_t *lj, int64_t *m_lambda,
                             int32_t *ti, int32_t *tj, int64_t *m_theta);

/*
 * Regularisation-path server (not in the paper: a serving layer over Algorithm 1).
 * Requests arrive at any time through cggm_server_submit; each carries X (n x p), Y (n x q)
 * in host or device memory (kept alive by the caller until the request is done) and a grid
 * of lambda values solved in order with lam_Lambda = lam_Theta = lambdas[k], every solve
 * warm-started from the previous one with Lambda and Theta kept in device memory.  A request
 * is admitted when one of `slots` worker contexts is free and its device footprint
 * (cggm_footprint) fits the budget (the oldest request that fits goes first; a request larger
 * than the whole budget runs alone).  Admitted requests run concurrently, each on its own
 * stream, so their kernels overlap on the GPU; the results of a request do not depend on the
 * others (every kernel reduces in a fixed order).  Times are seconds on the server's clock
 * (steady clock from cggm_server_create).
 */
typedef struct cggm_server cggm_server;

typedef struct {
    const void *X;        /* n x p, row-major, host or device                            */
    int xdtype;           /* cggm_dtype                                                  */
    const void *Y;        /* n x q                                                       */
    int ydtype;
    int64_t n, p, q;
    int n_lambda;         /* points of the path (> 0)                                    */
    const double *lambdas;/* host, n_lambda values >= 0, copied at submission           */
    double tol;           /* stopping ratio of Section 5.1 for every point               */
    int max_iter;         /* per point; <= 0: default                                    */
    int precision;        /* cggm_precision                                              */
    double *Lambda_out;   /* host or device, n_lambda x q x q, or NULL                   */
    double *Theta_out;    /* host or device, n_lambda x p x q, or NULL                   */
} cggm_request;

typedef struct {
    int done;             /* 1 once the request has finished (or was cancelled)          */
    int status;           /* CGGM_OK, or the first error of the path                     */
    double arrival_s;     /* submission time                                             */
    double start_s;       /* admission time                                              */
    double finish_s;      /* completion time                                             */
    int iterations;       /* Newton iterations summed over the path                      */
    double f_last;        /* objective at the last point                                 */
    int64_t footprint;    /* device bytes accounted to the request                       */
} cggm_result;

/* Start `slots` worker threads on `device`; hbm_budget_bytes <= 0 means 80 % of the free
 * device memory at creation. */
cggm_status cggm_server_create(cggm_server **srv, int device, int slots, int64_t hbm_budget_bytes);
/* Queue a request; *id identifies it for cggm_server_poll. */
cggm_status cggm_server_submit(cggm_server *srv, const cggm_request *req, uint64_t *id);
/* Copy the request's state into *out; with wait != 0 block until it is done. */
cggm_status cggm_server_poll(cggm_server *srv, uint64_t id, int wait, cggm_result *out);
/* Cancel requests not yet admitted, wait for the running ones, release everything. */
void cggm_server_destroy(cggm_server *srv);
/* The coordinate passes of the requests that run at once share cooperative launches: a pass
 * that becomes ready waits briefly (until every running request has one ready, or 200 us)
 * for the passes of other requests, and up to eight passes of one precision and batch size
 * then run in one launch, each on its own group of SMs (the result of a pass does not depend
 * on how many SMs it gets).  Counts since creation: launches, passes launched, and launches
 * that held more than one pass; each pointer may be NULL.  Not in the paper (a serving layer). */
cggm_status cggm_server_stats(cggm_server *srv, int64_t *pass_launches, int64_t *passes,
                              int64_t *shared_launches);
/* Device bytes a request of this size is accounted for (workspace of cggm_solve plus the
 * request's own device copies); -1 for invalid sizes. */
int64_t cggm_footprint(int64_t n, int64_t p, int64_t q, int precision);

/* The batch size (the tile shape of the coordinate-pass kernels) that the tuner chose for a
 * size class: precision (cggm_precision), q and the Lambda active-set size m, each rounded up
 * to a power of two.  A solve with opts.sweep_batch = CGGM_SWEEP_BATCH_AUTO times the Lambda
 * pass at every candidate batch size in its first Newton iteration of a class it has not
 * seen, keeps the fastest for the process (shared by all contexts and threads), and uses it
 * for both passes.  Returns the chosen size, 0 if the class has not been tuned yet, -1 for
 * bad arguments.  The paper has no counterpart (its passes visit one coordinate at a time). */
int cggm_tuned_batch(int64_t q, int64_t m, int precision);

/* The tuner's table (the batch size chosen per size class) saved to and loaded from a text
 * file, so that a deployment tunes a size class once and later processes start with the
 * choice instead of timing their first iteration again.  The choices belong to the GPU
 * model they were timed on.  Format: '#' comment lines, then "precision log2_q log2_m
 * batch" per class (log2 rounded up, as cggm_tuned_batch rounds).  Host code.
 *   cggm_tuner_save writes every class tuned so far; cggm_tuner_load merges a file's
 *   classes into the table (replacing a class already present).  count_out (optional):
 *   classes written or read.
 * Errors: CGGM_EINVAL for a null path, a file that cannot be opened or written, or (load)
 * a malformed line, an unknown precision or a batch size the precision does not allow;
 * a load that fails merges nothing.  The paper has no counterpart. */
cggm_status cggm_tuner_save(const char *path, int64_t *count_out);
cggm_status cggm_tuner_load(const char *path, int64_t *count_out);

/* Dense contraction on the tensor cores, the form every product from X takes in the mixed
 * path (R = X Theta, P = R Sigma, Psi = P^T P / n, X^T (Y + P); Section 2.3 lists them):
 *     C = alpha A B^T + beta C,
 * A M x K, B N x K, C M x N, row-major float in device memory; lda, ldb, ldc in elements,
 * lda and ldb multiples of 4 with 16-byte aligned bases (CGGM_EINVAL otherwise).
 * mode 0: one TF32 product (10-bit mantissa operands, FP32 accumulation); mode 1: three
 * TF32 products on a high/low split of both operands (close to FP32 accuracy). */
cggm_status cggm_contract(cggm_ctx *ctx, int64_t M, int64_t N, int64_t K, float alpha,
                          const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
                          float *C, int64_t ldc, int mode);

/* Sparse symmetric positive definite solve by conjugate gradient.  Section 4 (the block
 * regime of Algorithm 2) never forms Sigma = Lambda^-1 whole: it computes blocks of its
 * columns by conjugate gradient on the sparse Lambda, and P = R Sigma through
 * Lambda P^T = R^T.  This entry point solves Lambda X = B for k right-hand sides at once.
 *   Lambda: q x q in CSR (row_ptr[q + 1] int64, col[nnz] int32, val[nnz] double; host or
 *           device), symmetric positive definite, both triangles stored.
 *   B:      q x k row-major double (host or device), or NULL for the identity columns
 *           c0 .. c0 + k - 1 (then X = Sigma[:, c0 : c0 + k]; 0 <= c0, c0 + k <= q).
 *   X:      q x k row-major double output (host or device).
 * Jacobi-preconditioned CG in double, all k columns advancing together; stops when every
 * column's residual norm is <= tol times its right-hand side's norm (tol > 0), or after
 * max_iter iterations (CGGM_EMAXITER; X holds the last iterate).  iters_out, resid_out
 * (optional): iterations run and the largest residual ratio at exit.  Errors: CGGM_EINVAL
 * (shapes, tol, a malformed CSR: row pointers not non-decreasing from 0 to nnz or a column
 * outside [0, q)), CGGM_ENOTPD (a non-positive diagonal or curvature), CGGM_ENOMEM. */
cggm_status cggm_spd_solve(cggm_ctx *ctx, int64_t q, const int64_t *row_ptr, const int32_t *col,
                           const double *val, int64_t k, const double *B, int64_t c0, double tol,
                           int max_iter, double *X, int *iters_out, double *resid_out);

/* A block of columns C = c0 .. c0 + k - 1 of the Lambda gradient (Eq. 3),
 * G_Lambda[:, C] = S_yy[:, C] - Sigma[:, C] - Psi[:, C], without forming Sigma or Psi whole:
 * the block regime of Section 4 visits Lambda column block by column block, and the
 * block's active set (Section 2.2) is the threshold of this gradient.  Sigma[:, C] and
 * P^T = Sigma R^T (R = X Theta) come from conjugate-gradient solves on the sparse Lambda
 * (as cggm_spd_solve, tolerance tol, at most max_iter iterations each), Psi[:, C] = P^T P_C / n
 * and S_yy[:, C] = Y^T Y_C / n from products over the n samples.
 *   X, Y: as for cggm_solve.  Lambda: q x q CSR as for cggm_spd_solve.  Theta: p x q
 *   row-major double (host or device).  G_out: q x k row-major double (host or device).
 *   iters_out (optional): the larger iteration count of the two solves.
 * Errors: as cggm_spd_solve (CGGM_EMAXITER if a solve did not reach tol), and CGGM_EINVAL
 * for c0 + k > q. */
cggm_status cggm_grad_lambda_block(cggm_ctx *ctx, const void *X, int xdtype, const void *Y,
                                   int ydtype, int64_t n, int64_t p, int64_t q,
                                   const int64_t *row_ptr, const int32_t *col, const double *val,
                                   const double *Theta, int64_t c0, int64_t k, double tol,
                                   int max_iter, double *G_out, int *iters_out);

/* Column partition for the block coordinate descent of Algorithm 2 (Section 4): the q
 * columns are cut into blocks of at most max_block columns, and the cut is chosen by graph
 * clustering (Section 4.1 for Lambda, where an active coordinate between two blocks costs
 * a cache miss; the paper uses METIS).  The graph has q vertices and the m edges
 * (ei[t], ej[t]) of weight w[t] (w = NULL: weight 1); self loops are ignored and repeated
 * edges add their weights.  For Lambda, pass the active coordinates as the edges.
 *   block_out: q int32 (caller-owned, host), the block of every column, ids 0..k-1 with
 *   no empty block, numbered by the lowest column they hold.  nblocks_out (optional): k.
 *   cut_out (optional): total weight of the edges between blocks.
 * The method, a host heuristic with no GPU use: three candidates, of which the one of
 * lowest cut is returned - components in Cuthill-McKee order cut into the fewest pieces,
 * and a multilevel scheme (heavy-edge matching, pieces grown around strongly connected
 * columns on the coarsest graph, refined level by level) with two growing rules - each
 * with pieces joined along their heaviest links, packed first-fit decreasing, and
 * refined by moves and exchanges of boundary columns that lower the cut.  Deterministic.
 * A q = 20000 graph with 40000 edges takes a fraction of a second.
 * Errors: CGGM_EINVAL for q < 0, m < 0, max_block < 1, an index outside [0, q), a
 * negative or non-finite weight, or a null pointer that the sizes need. */
cggm_status cggm_partition_columns(int64_t q, int64_t m, const int32_t *ei, const int32_t *ej,
                                   const double *w, int64_t max_block, int32_t *block_out,
                                   int64_t *nblocks_out, double *cut_out);

/* Column partition for the blocked Theta pass of Algorithm 2 (Section 4.2): a block
 * (i, C_r) with active entries costs one row (S_xx)_i, so the partition should keep the
 * active columns of each row together.  The graph joins columns j and k when a row holds
 * active entries (i, j) and (i, k); a row with d active columns adds weight 1/(d - 1) to
 * each of its pairs when d <= 16, and joins them as a path (ascending columns, weight 1)
 * when d is larger.  That graph is cut as by cggm_partition_columns.
 *   ti, tj: the m active coordinates (0 <= ti < p, 0 <= tj < q; any order; repeats
 *   allowed).  block_out, nblocks_out: as for cggm_partition_columns.
 *   row_blocks_out (optional): the cost Section 4.2 minimises, the number of pairs
 *   (row i, block r) that hold an active entry.
 * Errors: CGGM_EINVAL for negative sizes, max_block < 1, an index out of range, or a null
 * pointer that the sizes need. */
cggm_status cggm_partition_theta_columns(int64_t p, int64_t q, int64_t m, const int32_t *ti,
                                         const int32_t *tj, int64_t max_block,
                                         int32_t *block_out, int64_t *nblocks_out,
                                         int64_t *row_blocks_out);

/* Number of blocks of Algorithm 2 for a memory budget, by Section 4's rule: the smallest k
 * such that the columns a block holds fit in budget_bytes, values of bytes_per_value bytes.
 *   kind 0 (Lambda, Section 4.1): a block holds 2q/k columns of Sigma and 2q/k of Psi, so
 *   k is the least with 4 q ceil(q/k) bytes_per_value <= budget_bytes.
 *   kind 1 (Theta, Section 4.2): q/k columns of Sigma, q ceil(q/k) bytes_per_value.
 *   *k_out: the number of blocks; *max_block_out: ceil(q / k), the cap to give
 *   cggm_partition_columns (blocks of equal size up to one fit the budget).  Host code.
 * Errors: CGGM_EINVAL for another kind, a size below 1 or a null pointer; CGGM_ENOMEM when
 * the budget does not hold a single block column. */
cggm_status cggm_block_count(int kind, int64_t q, int64_t bytes_per_value, int64_t budget_bytes,
                             int64_t *k_out, int64_t *max_block_out);

/* Visiting order of the blocked coordinate passes of Algorithm 2 for a column partition
 * (one block id per column, ids 0..k-1, none empty), and the cache counts of Section 4.
 *   kind 0 (Lambda): (ci[t], cj[t]) with 0 <= ci <= cj < q; a coordinate belongs to the
 *   block pair (z, r), z <= r, of its indices' blocks, a being the index in block z; the
 *   pass runs by z, then r, then a, then b.  It forms Sigma (and Psi) columns for every
 *   block once and again for block r at each off-diagonal pair holding a coordinate:
 *   *columns_out = q + the sizes of those blocks, *misses_out = the number of such pairs.
 *   kind 1 (Theta): (ci[t], cj[t]) = (i, j) with i >= 0, 0 <= j < q; the pass runs by the
 *   block of j, then i, then j; *columns_out = q (Sigma once), *misses_out = the number of
 *   non-empty (i, block) pairs, each one row of S_xx formed.
 *   order_out (m, caller-owned host): positions into the input list in visiting order.
 *   columns_out, misses_out: optional.  Host code, no GPU use.
 * Errors: CGGM_EINVAL for another kind, negative sizes, a null pointer the sizes need, a
 * block id outside [0, q) or an empty block, or an index out of range. */
cggm_status cggm_block_order(int kind, int64_t q, int64_t m, const int32_t *ci,
                             const int32_t *cj, const int32_t *block, int32_t *order_out,
                             int64_t *columns_out, int64_t *misses_out);

/* Pivot orders for cggm_chol_symbolic. */
typedef enum {
    CGGM_ORDER_NATURAL = 0, /* columns as numbered                                        */
    CGGM_ORDER_RCM = 1,     /* reverse Cuthill-McKee: small profile on chain-like patterns */
    CGGM_ORDER_GIVEN = 2,   /* the caller's permutation perm_in                            */
    CGGM_ORDER_MINDEG = 3,  /* minimum degree: little fill on chains with few extra links; */
                            /* none on a forest                                            */
    CGGM_ORDER_AMD = 4      /* minimum degree with approximate degrees on the quotient    */
                            /* graph: about the same fill at a fraction of the cost       */
} cggm_ordering;

/* Symbolic analysis of the sparse Cholesky factor of a q x q symmetric pattern: the block
 * regime of Algorithm 2 keeps Lambda sparse, and its line search needs log det of
 * Lambda + alpha D (Section 4) from a sparse factor, whose structure depends only on the
 * pattern and the pivot order.  Host code, no GPU use.
 *   row_ptr (q + 1), col: the pattern in CSR, either triangle or both (the union with its
 *   transpose is used; the diagonal is always taken as present; repeats allowed).
 *   ordering: a cggm_ordering; perm_in (q, used with CGGM_ORDER_GIVEN): perm_in[k] is
 *   the original column of pivot k.
 *   perm_out (q): the pivot order used, as perm_in.  parent_out (q): the elimination tree
 *   of the permuted pattern, parent of pivot k (-1 for a root; parent > k).
 *   colcount_out (q): entries of column k of L, the diagonal included.
 *   nnz_L_out (optional): their sum.  All caller-owned host memory.
 * The tree comes from path compression over the ancestors found so far and the counts
 * from row subtrees (every entry of L is counted once), so the cost is O(nnz(L)) after
 * the order; the minimum-degree order works on the explicit elimination graph, with its
 * cost growing with the fill: a chain of 20000 columns with 2000 extra links takes 0.15 s,
 * of 50000 with 5000 links 2.6 s, of 100000 with 10000 links 18 s; a random network of
 * degree 4 over 20000 columns 6.4 s.  The approximate-degree order (CGGM_ORDER_AMD) takes
 * well under a second on each of these and a few seconds for 200000 columns.
 * Errors: CGGM_EINVAL for q < 0, a null pointer that q needs, a malformed CSR (row_ptr[0]
 * != 0, decreasing, or a column outside [0, q)), another ordering, or a perm_in that is
 * not a permutation of 0..q-1. */
cggm_status cggm_chol_symbolic(int64_t q, const int64_t *row_ptr, const int32_t *col,
                               int ordering, const int32_t *perm_in, int32_t *perm_out,
                               int32_t *parent_out, int64_t *colcount_out,
                               int64_t *nnz_L_out);

/* Row structure of the supernodes (cggm_chol_supernodes) of the sparse Cholesky factor
 * analysed by cggm_chol_symbolic: for supernode s, the sorted rows (pivot numbering) of its
 * dense block of L, its own columns first.  A numeric factorisation allocates and
 * addresses L from it.  Host code, no GPU use.
 *   row_ptr, col: the pattern as given to cggm_chol_symbolic; perm, parent, colcount: its
 *   outputs; nsuper, super_start: cggm_chol_supernodes' outputs.
 *   rows_ptr_out (nsuper + 1): offsets, rows_ptr_out[s + 1] - rows_ptr_out[s] =
 *   colcount[super_start[s]]; rows_out (rows_ptr_out[nsuper] entries, or NULL to get the
 *   offsets only).  Caller-owned host memory.
 * Errors: CGGM_EINVAL for sizes out of range, a null pointer the sizes need, a malformed
 * CSR, perm not a permutation, a supernode list not increasing from 0 to q, or inputs not
 * from one analysis (a structure whose size disagrees with the column counts). */
cggm_status cggm_chol_structure(int64_t q, const int64_t *row_ptr, const int32_t *col,
                                const int32_t *perm, const int32_t *parent,
                                const int64_t *colcount, int64_t nsuper,
                                const int64_t *super_start, int64_t *rows_ptr_out,
                                int32_t *rows_out);

/* Symmetric permutation of a q x q CSR matrix, B = P A P^T with B[k][l] = A[perm[k]][perm[l]]
 * (perm[k] = the original index of new index k): with the order of a column partition's
 * blocks it makes every block a contiguous range of columns, the layout the blocked passes
 * of Algorithm 2 and a sparse factorisation work on.  Host code, no GPU use.
 *   row_ptr (q + 1), col, val (nnz = row_ptr[q]; val and out_val may be NULL for a pattern
 *   only): the input; out_row_ptr (q + 1), out_col, out_val (nnz): caller-owned host
 *   output, columns ascending within each row (entries repeated in the input stay
 *   repeated, in their input order).
 * Errors: CGGM_EINVAL for q < 0, a null pointer the sizes need, a malformed CSR, or a
 * perm that is not a permutation of 0..q-1. */
cggm_status cggm_permute_csr(int64_t q, const int64_t *row_ptr, const int32_t *col,
                             const double *val, const int32_t *perm, int64_t *out_row_ptr,
                             int32_t *out_col, double *out_val);

/* Fundamental supernodes of the factor analysed by cggm_chol_symbolic: maximal runs of
 * consecutive pivots whose columns share one row pattern below the run (a dense block of
 * L), the unit of work of a supernodal numeric factorisation.  Pivot k + 1 continues the
 * run of pivot k when k is its only child in the elimination tree and column k holds
 * exactly one entry more than column k + 1 (then column k below its diagonal is column
 * k + 1's pattern).
 *   parent, colcount (q): as returned by cggm_chol_symbolic.
 *   start_out (q + 1 entries, caller-owned host memory): start_out[s] is the first pivot of
 *   supernode s, s < *nsuper_out, and start_out[*nsuper_out] = q.
 * Errors: CGGM_EINVAL for q < 0, a null pointer, a parent outside (k, q) or -1, or a
 * count outside [1, q - k]. */
cggm_status cggm_chol_supernodes(int64_t q, const int32_t *parent, const int64_t *colcount,
                                 int64_t *start_out, int64_t *nsuper_out);

/* Numeric sparse Cholesky factorisation in double precision on the GPU.  Section 4 keeps
 * Lambda sparse in the block regime of Algorithm 2, and the Armijo rule of Algorithm 1
 * needs log det(Lambda + alpha D) and the positive definiteness that a Cholesky factor
 * certifies (Section 2.3 takes both from the factor); columns of Sigma = Lambda^-1 follow
 * from two triangular solves with it.  With the pivot order P (perm[k] = the original
 * index of pivot k), P A P^T = L L^T, L lower triangular with a positive diagonal (so L is
 * unique).  L is stored by supernodes (cggm_chol_supernodes): supernode s owns pivots
 * super_start[s] .. super_start[s+1]-1 (nc of them) and its rows rows[rows_ptr[s] ..
 * rows_ptr[s+1]) (nr of them, its own pivots first, ascending), and keeps the dense nr x nc
 * block L[rows, own pivots] row-major at blocks[block_ptr[s] ..]; the strict upper triangle
 * of its top nc x nc square is zero.
 *
 * cggm_spchol_create: symbolic analysis (host: cggm_chol_symbolic, cggm_chol_supernodes,
 *   cggm_chol_structure) of a q x q symmetric pattern and the device structures of the
 *   numeric work, on the context's device.
 *   row_ptr (q + 1), col: the matrix in CSR (host memory), both triangles or the lower one:
 *   the values used are those of entries with col <= row (the lower triangle with the
 *   diagonal); entries above the diagonal only add to the pattern.  ordering, perm_in: as
 *   for cggm_chol_symbolic.  *out: the plan, released by cggm_spchol_destroy, which must be
 *   called before the context is destroyed; one thread at a time per plan, and it shares
 *   the context's stream.
 *   Errors: CGGM_EINVAL (q < 1, a null pointer, a malformed CSR, a bad ordering or perm_in),
 *   CGGM_ENOMEM (device memory, or one supernode's block beyond 2^31 entries).
 * cggm_spchol_factor: factor the matrix with values val (row_ptr[q] doubles in the CSR
 *   order given to cggm_spchol_create, host or device memory; repeated entries add up).
 *   logdet_out (optional): log det A = 2 sum_k log L_kk.  Errors: CGGM_ENOTPD (a pivot not
 *   positive: A is not positive definite), CGGM_ENONFINITE (a value not finite),
 *   CGGM_ETIMEDOUT (a device-side wait gave up), CGGM_EINVAL.
 * cggm_spchol_solve: X = A^-1 B with the last successful factorisation.  B: q x k row-major
 *   double (host or device), or NULL for the identity columns c0 .. c0 + k - 1 (then X =
 *   Sigma[:, c0 : c0 + k]); X: q x k row-major double (host or device).  CGGM_EINVAL for
 *   k < 1, columns outside [0, q) or no factorisation yet.
 * cggm_spchol_export: the structure and the factor (host memory, each output optional):
 *   nsuper, nblock (entries of blocks), nnz_L (entries of L); perm (q), super_start,
 *   rows_ptr and block_ptr (nsuper + 1 each), rows (rows_ptr[nsuper]), blocks (nblock;
 *   CGGM_EINVAL before a successful factorisation).
 * cggm_spchol_destroy: releases the plan (NULL is allowed). */
typedef struct cggm_spchol cggm_spchol;
cggm_status cggm_spchol_create(cggm_ctx *ctx, int64_t q, const int64_t *row_ptr,
                               const int32_t *col, int ordering, const int32_t *perm_in,
                               cggm_spchol **out);
cggm_status cggm_spchol_factor(cggm_spchol *f, const double *val, double *logdet_out);
cggm_status cggm_spchol_solve(cggm_spchol *f, int64_t k, const double *B, int64_t c0,
                              double *X);
cggm_status cggm_spchol_export(cggm_spchol *f, int64_t *nsuper_out, int64_t *nblock_out,
                               int64_t *nnz_L_out, int32_t *perm_out,
                               int64_t *super_start_out, int64_t *rows_ptr_out,
                               int32_t *rows_out, int64_t *block_ptr_out, double *blocks_out);
cggm_status cggm_spchol_destroy(cggm_spchol *f);

/*
 * No-allocation variant of cggm_lambda_sweep (the paper has no counterpart: this is an
 * interface for embedding).  Some callers cannot call cudaMalloc: code that runs under
 * an allocator that owns all device memory (a framework's caching allocator or a fixed
 * memory pool sized up front), and latency-critical loops where the implicit device
 * synchronisation of cudaMalloc/cudaFree is not acceptable.  This entry point computes
 * the same Lambda direction as cggm_lambda_sweep (double precision) but allocates
 * nothing: its working memory is one device array inside the library, of
 * CGGM_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library holds until
 * the process exits.
 *
 *  - q <= CGGM_NOALLOC_MAX_Q and 0 <= m <= q (q + 1) / 2; larger sizes return
 *    CGGM_EINVAL without touching the GPU.
 *  - Every pointer must be device memory of the current device (CGGM_EINVAL otherwise):
 *    Sigma, Psi, Syy, Lambda (q x q double), ai, aj (m int32, ai <= aj, visiting order),
 *    D_out (q x q double, overwritten).  The index pairs are checked on the device before
 *    the pass reads them: a pair outside 0 <= ai <= aj < q returns CGGM_EINVAL (D_out is
 *    then zero).  The call runs on cuda_stream (a cudaStream_t; NULL = the legacy default
 *    stream) and returns after the pass has finished and D_out is written (also for
 *    m = 0, where D_out is set to zero).
 *  - The first call on a device looks up the device address of the array (once per
 *    device, with that device current); make that first call before any stream capture.
 *    The address is kept for the life of the process: do not use this entry point on a
 *    device after cudaDeviceReset has been called on it.
 *  - All calls share the one array and it keeps the last call's contents (the call
 *    clears what must start at zero).  Calls that overlap on the GPU - from two host
 *    threads or on two streams - race on it; serialise them.
 */
#define CGGM_NOALLOC_MAX_Q 256
#define CGGM_NOALLOC_SCRATCH_BYTES (3u << 20)
cggm_status cggm_lambda_sweep_noalloc(int64_t q, const double *Sigma, const double *Psi,
                                      const double *Syy, const double *Lambda, int64_t m,
                                      const int32_t *ai, const int32_t *aj, double lam_L,
                                      int penalize_diag, double *D_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CGGM_H */
