/*
 * oem.h -- C ABI of the GB300 (sm_103a) OEM penalized least-squares library.
 *
 * The library computes the data-parallel hot path of the orthogonalizing EM
 * (OEM) method for penalized linear regression on tall data (Huling & Qian,
 * "Fast penalized regression and cross validation for tall data with the oem
 * package", arXiv 1801.09661):
 *   - the sufficient statistics X^T X, X^T y, y^T y in one pass over X, split
 *     into per-fold partial sums for cross validation (Section 3);
 *   - the OEM constant d >= lambda_1(X^T X / n) (Section 2.1, by Lanczos);
 *   - warm-started OEM paths beta <- threshold(X^T y/n + d beta - (X^T X/n) beta)
 *     for the lasso, elastic net, MCP, SCAD and group lasso (Section 2.2);
 *   - K-fold cross validation from the fold statistics (Sections 3, 5.5).
 *
 * Conventions (all entry points):
 *   - Array arguments are DEVICE pointers owned by the caller, unless a
 *     parameter says "host". The library never frees caller memory.
 *   - Exception, X in host memory: oem_gram, oem_fold_grams, oem_fit and
 *     oem_cv also accept X (and then y, fold, on either side) in host memory,
 *     pinned or pageable (the paper's out-of-memory big.oem, Section 5.7, done
 *     as a stream): row blocks of about 256 MB are copied into two device
 *     staging buffers on a copy stream while the previous block's Gram pass
 *     runs, and the blocks' fold sums are added up; pinned memory overlaps
 *     the copies with the passes. The work is ordered after `stream`'s
 *     earlier work and before its later work; the call returns without
 *     waiting for the device, so the host buffers must stay valid until
 *     `stream` has reached that point. With X in device memory, y and fold
 *     must be in device memory too (OEM_EINVAL otherwise). oem_fit_logistic
 *     takes device memory only.
 *   - CUDA graphs: oem_gram, oem_fold_grams, oem_spectral_d, oem_fit_path,
 *     oem_fit and oem_cv (X in device memory) may be captured into a graph
 *     once the same call has run outside the capture on the same context:
 *     that call sizes the context's workspace, which cannot grow inside a
 *     capture (OEM_EINVAL), and fixes the autotuned layout (the autotuner
 *     does not run inside a capture). Host data a call uploads (penalty and
 *     task tables, user lambdas, d) travel inside the captured launches, so
 *     the graph replays the call on whatever the device buffers hold.
 *     oem_fit_logistic (a host loop over outer steps) and the server are not
 *     capturable.
 *   - Matrices are row-major (C order). X is n x p with leading dimension
 *     ldx >= p (elements); ldx * sizeof(element) must be a multiple of 16 and
 *     X, y must be 16-byte aligned, else OEM_EINVAL.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = the
 *     legacy default stream) and the call returns without waiting, except
 *     where a parameter is a host output. Argument errors are returned before
 *     anything is launched. Conditions found on the device (non-finite input,
 *     a bounded device wait that expired) are recorded in the context and
 *     returned by oem_sync().
 *   - Workspace comes from a per-context arena that never exceeds the byte
 *     budget given to oem_create (OEM_EBUDGET otherwise). A context is used by
 *     one host thread and one stream at a time.
 *   - Objective (reading of the paper's scaling, Section 2.1 and the oem.xtx
 *     example of Section 5.6): minimise (1/2n)||y - X beta||^2 + P_lambda(beta),
 *     i.e. beta^T G beta / 2 - c^T beta + P_lambda(beta) with G = X^T X / n,
 *     c = X^T y / n.
 */
#ifndef OEM_GB300_H
#define OEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oem_ctx oem_ctx;

/* Status codes. Negative = error, 0 = ok, positive = warning. */
enum {
  OEM_OK = 0,
  OEM_WARN_NOTCONV = 1,   /* some (lambda, penalty) hit max_iter */
  OEM_EINVAL = -1,        /* bad argument (size, pointer, alignment, option) */
  OEM_ENOMEM = -2,        /* device allocation failed */
  OEM_EBUDGET = -3,       /* workspace would exceed the context's byte budget */
  OEM_ECUDA = -4,         /* a CUDA runtime call failed */
  OEM_ENONFINITE = -5,    /* NaN/Inf in X or y */
  OEM_ETIMEOUT = -6,      /* a bounded device wait expired; results invalid */
  OEM_EUNSUPPORTED = -7   /* valid request this build does not serve */
};

/* Element type of X (and y). y is float64 when X is float64, else float32. */
enum { OEM_F64 = 0, OEM_F32 = 1, OEM_BF16 = 2 };

/* How the Gram pass forms products and sums (Section 3, O(np^2) step):
 *   FP64       : float64 products and sums on CUDA cores (X float64 or float32).
 *   FP32       : float32 products, float32 sums over short row blocks, float64
 *                across blocks, on CUDA cores (the plain form).
 *   TF32       : tcgen05 tensor cores, kind::tf32 (X float32), float32
 *                accumulation in tensor memory, compensated across blocks.
 *   BF16       : tcgen05 kind::f16 with bfloat16 operands (X bfloat16: exact
 *                products; the float32 y is carried exactly as three bfloat16
 *                columns hi + mid + lo).
 *   SPLIT_BF16 : tcgen05 kind::f16, X float32 split as hi + lo bfloat16
 *                (X float32). The TMA-fed path (the default whenever the
 *                packed copy fits the budget) forms hi*hi + hi*lo + lo*hi,
 *                plus lo*lo on the diagonal 128 x 128 tiles (where lo_i^2
 *                would otherwise bias G_ii); the converting kernel (small
 *                budgets and oem_gram_noalloc) forms all four products on
 *                every tile. Both hold the same error bound.
 *   AUTO       : SPLIT_BF16 for float32, BF16 for bfloat16, FP64 for float64. */
enum {
  OEM_GRAM_FP64 = 0,
  OEM_GRAM_FP32 = 1,
  OEM_GRAM_TF32 = 2,
  OEM_GRAM_BF16 = 3,
  OEM_GRAM_SPLIT_BF16 = 4,
  OEM_GRAM_AUTO = 5
};

/* Penalties of Table 1 (Section 2.2 updates). */
enum {
  OEM_LASSO = 0, OEM_ENET = 1, OEM_MCP = 2, OEM_SCAD = 3, OEM_GROUP_LASSO = 4,
  OEM_GROUP_MCP = 5,            /* Eq. gmcp: M(||u_g||, c_k lambda, gamma, d) u_g / ||u_g|| */
  OEM_GROUP_SCAD = 6,           /* Eq. gscad: C(||u_g||, c_k lambda, gamma, d) u_g / ||u_g|| */
  OEM_SPARSE_GROUP_LASSO = 7    /* Eq. sglasso: v = S(u, w lambda tau, d), then
                                   beta_g = v_g (1 - c_k lambda (1 - tau) / (d ||v_g||))_+ */
};

/* Precision of the OEM iteration: float32 mat-vec with a compensated
 * (float32 hi + lo) running u, or float64 throughout. */
enum { OEM_ITER_F32 = 0, OEM_ITER_F64 = 1 };

typedef struct oem_penalty {
  int32_t kind;          /* OEM_LASSO .. OEM_SPARSE_GROUP_LASSO */
  double alpha;          /* elastic net mixing alpha in [0,1] (Eq. net); for the
                            sparse group lasso its tau in [0,1] (Table 1) */
  double gamma;          /* MCP and group MCP gamma > 1 (Eqs. mcp, gmcp), SCAD
                            and group SCAD gamma > 2 (Eqs. scad, gscad) */
  const double* w;       /* host, p variable weights w_j >= 0, or NULL (all 1);
                            lasso, elastic net, MCP, SCAD, sparse group lasso */
  const int32_t* group;  /* host, p group ids in [0, ngroups), group penalties
                            only; each group's variables must be contiguous */
  const double* cg;      /* host, ngroups group weights c_k >= 0, or NULL (sqrt|g_k|) */
  int32_t ngroups;
} oem_penalty;

typedef struct oem_options {
  int32_t nlambda;          /* lambdas per path (default 100) */
  double lambda_min_ratio;  /* smallest / largest lambda (default 1e-3) */
  const double* lambdas;    /* host, npen x nlambda user grid, or NULL (computed) */
  double tol;               /* stop when max|dbeta| <= tol*max(1,max|beta|) (1e-7) */
  int64_t max_iter;         /* iteration cap per lambda (default 10000) */
  int32_t lanczos_steps;    /* Lanczos steps for d (default 64) */
  int32_t gram_mode;        /* OEM_GRAM_* (default OEM_GRAM_AUTO) */
  int32_t iter_precision;   /* OEM_ITER_F32 (default) or OEM_ITER_F64 */
  int32_t cluster_ctas;     /* CTAs cooperating on one Gram in the iteration
                               (0 = chosen by the library; 1,2,4,8,16: one
                               thread-block cluster exchanging through
                               distributed shared memory; 17..4096: a group of
                               that many CTAs of a cooperative launch, at most
                               one per SM, exchanging through L2) */
  int32_t instances_per_task; /* penalties of one Gram iterated together by
                               one cluster (0 = chosen by the library; else
                               1,2,4,8); results do not depend on it */
  int32_t autotune;         /* 1 (default): when cluster_ctas and
                               instances_per_task are both 0, the first call
                               for a new (p, Grams, penalties, precision)
                               shape times the candidate layouts for a few
                               iterations on its own inputs (synchronising the
                               stream once) and the context keeps the fastest;
                               skipped while the stream is being captured.
                               0: the library's fixed rule */
  int32_t intercept;        /* oem_fit / oem_cv: 1 = fit an unpenalised
                               intercept by centring X and y by their means
                               over the rows of each fit; default 0 */
  int32_t standardize;      /* oem_fit / oem_cv: 1 = divide column j by its
                               standard deviation sd_j (population, of the
                               centred column with an intercept, else the
                               root second moment) before fitting; penalties
                               apply to the standardized coefficients, results
                               are reported on the original scale; a column
                               with zero variance (or below 1e-14 of its
                               second moment) gets a zero coefficient.
                               Section 2.1 assumes standardized columns; the
                               API follows glmnet's (Section 5). Default 0 */
} oem_options;

/* Fill *opt with the defaults listed above. */
void oem_options_default(oem_options* opt);

/* Create a context on CUDA device `device` whose workspace arena may grow to
 * mem_budget_bytes (0 = 8 GiB). Returns OEM_OK and sets *ctx, or an error. */
int oem_create(oem_ctx** ctx, int device, size_t mem_budget_bytes);

/* Free the context and its workspace (synchronises the device first). */
int oem_destroy(oem_ctx* ctx);

/* Text of the last error recorded in ctx (static storage inside ctx). */
const char* oem_last_error(const oem_ctx* ctx);

/* Wait for all work enqueued on `stream`, then return (and clear) the worst
 * device-side status recorded since the last oem_sync: OEM_OK,
 * OEM_WARN_NOTCONV, OEM_ENONFINITE or OEM_ETIMEOUT. */
int oem_sync(oem_ctx* ctx, void* stream);

/* Number of kernels this context has launched so far (for accounting). */
int64_t oem_kernel_launches(const oem_ctx* ctx);

/* OEM iterations of the last oem_fit_path / oem_fit / oem_cv call on ctx
 * (Section 2.1 Step 2: one iteration = one update u, beta of one instance).
 * Waits for `stream`, then reads that call's per-lambda iteration counts:
 * *iterations = their sum over every instance (penalty, and fold Gram for
 * oem_cv) and lambda; *loop_trips = the largest sum of one instance, i.e.
 * the loop trips of the persistent launch that runs all instances side by
 * side. Valid until the next call on ctx (the counts live in its
 * workspace). Returns OEM_OK, OEM_EINVAL (no fit yet) or OEM_ECUDA. */
int oem_iter_stats(oem_ctx* ctx, void* stream, int64_t* iterations, int64_t* loop_trips);

/* Per-kernel device timing. While enabled, every launch of this context is
 * bracketed by CUDA events on its stream; oem_profile_get() waits for the
 * pending events and returns the accumulated device milliseconds and launch
 * count of one kernel class (0 <= kernel < OEM_PROF_NKERNELS, names from
 * oem_profile_name). Enabling (again) clears the totals. OEM_PROF_GRAM_TC
 * ("gram_tc_pass") covers the tensor-core Gram pass: the packing pass and
 * the TMA-fed kernel, or the converting kernel. */
enum {
  OEM_PROF_FOLD_SORT = 0, OEM_PROF_CHUNKS = 1, OEM_PROF_GRAM_SIMT = 2, OEM_PROF_GRAM_TC = 3,
  OEM_PROF_GRAM_REDUCE = 4, OEM_PROF_ASSEMBLE = 5, OEM_PROF_LANCZOS = 6, OEM_PROF_LAMBDA = 7,
  OEM_PROF_ITER = 8, OEM_PROF_CV = 9, OEM_PROF_COPY = 10, OEM_PROF_LOGIT = 11, OEM_PROF_NKERNELS = 12
};
int oem_profile_enable(oem_ctx* ctx, int enable);
int oem_profile_get(oem_ctx* ctx, int kernel, double* ms, int64_t* launches);
const char* oem_profile_name(int kernel);

/* Full-data sufficient statistics (Section 3: X^T X and X^T y).
 * X: n x p (ldx), element type xtype; y: n (float64 if xtype == OEM_F64, else
 * float32). Outputs RAW sums (not divided by n), float64, device:
 * G: p x p row-major, full symmetric; c: p; yty: 1. mode: OEM_GRAM_*.
 * n >= 1, p >= 1. */
int oem_gram(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p,
             int64_t ldx, const void* y, int32_t mode,
             double* G, double* c, double* yty, void* stream);

/* oem_gram without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when
 * they call -- code running under a framework that owns the whole device
 * memory pool, loops that must not allocate once they have started, or a
 * caller with no oem_ctx at all (this call needs none). It computes what
 * oem_gram computes (same arguments and outputs, same kernels; the caller
 * still passes X, y and the outputs G, c, yty) with all working memory in one
 * 48 MiB array that the library declares in device memory at file scope;
 * every GPU that loads the library holds that array until the process exits.
 * Limits: p <= 1024 (OEM_EBUDGET beyond it, or when the rows need more tile
 * partials than the array holds); n <= 2^31 - 1.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Every call shares the one array and leaves its contents behind: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must
 * not be issued. X, y, G, c and yty must be device memory (or managed memory) of the
 * current device: host memory, pinned or not, and memory of another device
 * give OEM_EINVAL (this entry point has no streamed host path). A bounded
 * device wait of the Gram pass that expires (about 2 s: a device that stopped
 * making progress) leaves NaN in every element of G, c and yty, since no
 * status word is read back. Non-finite values in X or y are not reported
 * (they show up in G, c, yty). Returns OEM_OK, OEM_EINVAL, OEM_EBUDGET or
 * OEM_ECUDA; work is enqueued on `stream` and the call does not wait. */
int oem_gram_noalloc(const void* X, int32_t xtype, int64_t n, int64_t p, int64_t ldx,
                     const void* y, int32_t mode, double* G, double* c, double* yty,
                     void* stream);

/* Per-fold raw sums in one pass (Section 3: X_k^T X_k, X_k^T y_k for every k).
 * fold: n uint8 labels in [0, K). Outputs: Gk K x p x p, ck K x p, ytyk K,
 * nk K (int64) -- all device. A fold with no rows gets zeros. 1 <= K <= 64. */
int oem_fold_grams(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p,
                   int64_t ldx, const void* y, const uint8_t* fold, int32_t K,
                   int32_t mode, double* Gk, double* ck, double* ytyk, int64_t* nk,
                   void* stream);

/* d_b >= lambda_1(G_b) for b < batch (Section 2.1, computed by Lanczos).
 * G_b = G + b*strideG, p x p float64 symmetric with leading dimension ldg.
 * steps: Lanczos steps (<= 0: 64; capped at p). d: batch float64, device.
 * d_b = theta + r, theta the largest Ritz value and r its residual norm;
 * an all-zero G_b gives d_b = 1. */
int oem_spectral_d(oem_ctx* ctx, const double* G, int64_t p, int64_t ldg,
                   int32_t batch, int64_t strideG, int32_t steps, double* d,
                   void* stream);

/* Warm-started OEM paths from SCALED statistics (Section 5.6, oem.xtx):
 * G = X^T X / n (p x p float64, device), c = X^T y / n (p float64, device).
 * d > 0: use it; d <= 0: computed by Lanczos (opt->lanczos_steps).
 * pens, npen (1..8), opt: host. Outputs (device): beta npen x nlambda x p
 * float64; lambdas_out npen x nlambda float64; iters npen x nlambda int32;
 * converged npen x nlambda uint8. Lambda grid per penalty (when
 * opt->lambdas is NULL): lambda_max (the smallest lambda with beta = 0)
 * down to lambda_min_ratio * lambda_max, log-spaced. */
int oem_fit_path(oem_ctx* ctx, const double* G, const double* c, int64_t p, double d,
                 const oem_penalty* pens, int32_t npen, const oem_options* opt,
                 double* beta, double* lambdas_out, int32_t* iters,
                 uint8_t* converged, void* stream);

/* oem(): Gram pass over X (opt->gram_mode), d, lambda grid and paths, in one
 * call (Section 5.1-5.2: several penalties from one Gram). Outputs as for
 * oem_fit_path, plus d_out (1 float64, device, may be NULL; d of the
 * standardized problem when opt->standardize) and beta0 (npen x nlambda
 * float64, device, may be NULL: the intercepts, 0 without opt->intercept).
 * With opt->intercept or opt->standardize the Gram pass also forms the column
 * sums (a column of ones appended to [X | y], on X and y shifted by the
 * column means of a sample of rows so that centring loses no precision), and
 * the paths run on the centred / scaled statistics: beta is then on the
 * original scale and beta0 = mean(y) - mean(X) beta. A bfloat16 Gram request
 * with an intercept runs in split mode (the shifted X is not bfloat16). */
int oem_fit(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p,
            int64_t ldx, const void* y, const oem_penalty* pens, int32_t npen,
            const oem_options* opt, double* beta, double* lambdas_out,
            int32_t* iters, uint8_t* converged, double* d_out, double* beta0, void* stream);

/* xval.oem(): K-fold cross validation by per-fold statistics (Section 3).
 * One pass forms every fold's sums; leave-fold-out statistics by
 * subtraction; d per Gram; the full-data lambda grid per penalty; paths for
 * the full data and each of the K leave-fold-out fits (all in one batched
 * launch); held-out MSE_k(lambda) = ||y_k - X_k beta_{-k}(lambda)||^2 / n_k.
 * Outputs (device): beta_full npen x nlambda x p float64 (full-data paths);
 * lambdas_out npen x nlambda; cvm, cvsd npen x nlambda (mean over folds and
 * sample sd / sqrt(K)); idx_min, idx_1se npen int32 (lambda.min: argmin cvm,
 * ties to the larger lambda; lambda.1se: largest lambda with
 * cvm <= cvm_min + cvsd_min); best_penalty 1 int32 (lowest cvm at its
 * lambda.min). 2 <= K <= 64; every fold must have >= 1 row (OEM_EINVAL after
 * the fold count pass otherwise, reported by oem_sync). With opt->intercept
 * / opt->standardize every fit (full data and each leave-fold-out set)
 * centres and scales by its own rows' statistics, the held-out error is that
 * of beta_0 + x^T beta, and beta0_full (npen x nlambda float64, device, may
 * be NULL) receives the full-data intercepts. */
int oem_cv(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p,
           int64_t ldx, const void* y, const uint8_t* fold, int32_t K,
           const oem_penalty* pens, int32_t npen, const oem_options* opt,
           double* beta_full, double* lambdas_out, double* cvm, double* cvsd,
           int32_t* idx_min, int32_t* idx_1se, int32_t* best_penalty, double* beta0_full,
           void* stream);

/* Penalised logistic regression (Section 4): minimise
 *   -(1/n) sum_i { y_i eta_i - log(1 + exp(eta_i)) } + P_lambda(beta),
 *   eta_i = x_i^T beta (+ beta_0 with opt->intercept, unpenalised),
 * by the proximal Newton algorithm with the Hessian weights replaced by their
 * upper bound 1/4: G = Z^T Z / (4n) (Z = [X | 1] with an intercept) comes
 * from one Gram pass and stays fixed; each outer step makes one pass over X
 * for the score g = Z^T (y - mu) / n of every penalty's current beta and
 * solves the surrogate 1/2 b^T G b - (G beta + g)^T b + P_lambda(b) by OEM
 * iterations warm-started at beta (d >= lambda_1(G) by Lanczos). The outer
 * loop stops by the inner stopping rule applied to successive outer iterates
 * (at most 100 steps per lambda). lambda_max and the first warm start are
 * the null model's (beta = 0, beta_0 = logit(mean y)).
 * X n x p (float32, bfloat16 or float64; p <= 1023), y n values in {0, 1}
 * (float32; float64 for float64 X). pens: lasso, elastic net, MCP, SCAD
 * (npen 1..8). opt->standardize is not supported (OEM_EUNSUPPORTED).
 * Outputs (device): beta npen x nlambda x p; beta0 npen x nlambda (may be
 * NULL; 0 without an intercept); lambdas_out npen x nlambda; iters npen x
 * nlambda (inner OEM iterations summed over the outer steps); converged
 * npen x nlambda (the outer loop met its stopping rule); d_out (may be NULL).
 * The host waits for the stream once per outer step. */
int oem_fit_logistic(oem_ctx* ctx, const void* X, int32_t xtype, int64_t n, int64_t p,
                     int64_t ldx, const void* y, const oem_penalty* pens, int32_t npen,
                     const oem_options* opt, double* beta, double* beta0, double* lambdas_out,
                     int32_t* iters, uint8_t* converged, double* d_out, void* stream);

/* ------------------------------------------------------------------------
 * Serving: a request loop that admits fit and cross-validation jobs of mixed
 * n and p as they arrive, under a device-memory budget, and runs them with
 * continuous batching (the paper's OEM path per job, Sections 2-3; the
 * request loop itself has no counterpart in the paper).
 *
 * OEM_SERVE_BATCHED: each admitted job's Gram pass (split-bfloat16 tensor
 * cores), d and lambda grid run on the job's own stream, overlapping
 * whatever else is on the GPU; the job's Grams, d and path state stay
 * resident; the OEM iterations of every job whose Grams are ready run
 * together in rounds of one cluster launch (a bounded number of iterations
 * per round, state saved between rounds), so jobs join and leave the batch
 * as they become ready and finish.
 * OEM_SERVE_PLAIN: jobs one at a time in arrival order, float32 CUDA-core
 * Gram, and one kernel launch plus a host convergence check per OEM
 * iteration (the plain per-job GPU form, for comparison; lasso, elastic net,
 * MCP and SCAD only).
 * A job is DONE when its results are in host memory. Results of a job do not
 * depend on the other jobs in the batch.
 * ---------------------------------------------------------------------- */
typedef struct oem_server oem_server;

enum { OEM_SERVE_BATCHED = 0, OEM_SERVE_PLAIN = 1 };
enum { OEM_JOB_QUEUED = 0, OEM_JOB_PREP = 1, OEM_JOB_ITER = 2, OEM_JOB_FINISH = 3,
       OEM_JOB_DONE = 4, OEM_JOB_FAILED = 5 };

/* One request: a fit (K = 0) or a K-fold cross validation (2 <= K <= 64) of
 * one penalty. X (n x p, ldx), y and fold are DEVICE pointers that must stay
 * valid and unchanged until the job is DONE. gram_mode as in oem_options
 * (ignored by the plain form, which uses OEM_GRAM_FP32). */
typedef struct oem_job {
  const void* X;
  int32_t xtype;
  int64_t n, p, ldx;
  const void* y;
  const uint8_t* fold;
  int32_t K;
  oem_penalty pen;
  int32_t nlambda;
  double lambda_min_ratio;
  double tol;
  int64_t max_iter;
  int32_t gram_mode;
} oem_job;

/* Start a server on `device` with a device-memory budget for job data
 * (0 = 8 GiB), a form (OEM_SERVE_*) and the OEM iterations per batched
 * round (<= 0: 2000). A worker thread runs the loop until oem_server_destroy. */
int oem_server_create(oem_server** srv, int device, size_t mem_budget_bytes, int32_t form,
                      int64_t iters_per_round);

/* Queue a job; returns at once with its id. OEM_EINVAL for a bad job,
 * OEM_EBUDGET for a job that can never fit in the budget. */
int oem_server_submit(oem_server* srv, const oem_job* job, int64_t* id);

/* State (OEM_JOB_*) of a job and, once DONE, its latency from submission to
 * results in host memory, in milliseconds (may be NULL). */
int oem_server_poll(oem_server* srv, int64_t id, int32_t* state, double* latency_ms);

/* Results of a DONE job, copied to HOST arrays (each may be NULL): beta
 * nlambda x p (full-data path), lambdas nlambda; for CV jobs cvm and cvsd
 * (nlambda) and idx_min, idx_1se; iters = OEM iterations over all of the
 * job's paths. OEM_EINVAL if the job is not DONE. */
int oem_server_result(oem_server* srv, int64_t id, double* beta, double* lambdas, double* cvm,
                      double* cvsd, int32_t* idx_min, int32_t* idx_1se, int64_t* iters);

/* Server counters: jobs done, paths done (a CV job counts K+1 paths), kernel
 * launches, batched rounds, peak device bytes in use. */
int oem_server_stats(oem_server* srv, int64_t* jobs_done, int64_t* paths_done, int64_t* launches,
                     int64_t* rounds, int64_t* peak_bytes);

/* Finish every queued and running job, stop the worker and free the server. */
int oem_server_destroy(oem_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* OEM_GB300_H */
