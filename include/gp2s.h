/*
 * gp2s.h -- C ABI of the GB300 (sm_103a) engine for the exact sparse-kernel Gaussian-process
 * log marginal likelihood of gp2Scale (Noack, Risser, Luo, Tekriwal, Pandolfi; arXiv 2512.06143).
 *
 * The problem (Sec. 3, Background): data X (n points in R^d) and observations y; a compactly
 * supported non-stationary kernel
 *     k(xi, xj) = phi(|xi - xj| / r) * ( sum_l b_l(xi) b_l(xj) + w0 )            (Sec. 4.1, 4.3)
 * with the Wendland taper phi (Eq. 3; "C2" reading by default), bump functions
 *     b_l(x) = a_l exp(beta (1 - 1/(1 - |x - c_l|^2 / rho_l^2)))   inside |x - c_l| < rho_l (Eq. 7)
 * and noise V = sigma2 I.  A = K + sigma2 I is sparse because phi vanishes for |xi - xj| >= r.
 * The engine evaluates
 *     LML = -1/2 y^T A^{-1} y - 1/2 log|A| - n/2 log(2 pi)                          (Sec. 3)
 * and its gradient with respect to theta = [centers (L x d), radii (L), amps (L), r, sigma2].
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA tensors).  Pointers whose
 *     name says "host" are host memory.  X and y may be either: the engine asks the CUDA driver
 *     which one it got and stages host buffers through its own device workspace.
 *   - X is n x d, row-major, FP64.  y is n, FP64.  Hyperparameter arrays are host FP64.
 *   - All device work is issued on the context's stream.  A call returns when its host-visible
 *     outputs are written (it synchronises that stream once at the end, plus at most one small
 *     device->host read per Krylov convergence check).
 *   - Errors are returned as gp2s_status; gp2s_last_error() gives a one-line message.  Nothing
 *     aborts, prints or traps; a CUDA error reported by the runtime is returned as GP2S_ECUDA.
 *   - The context owns every intermediate (sorted points, cell table, CSR, Krylov vectors); it
 *     keeps them until the next gp2s_assemble / gp2s_lml* call or gp2s_destroy.
 *   - One context per host thread; calls on one context must not overlap.
 */
#ifndef GP2S_H
#define GP2S_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GP2S_OK = 0,
    GP2S_EINVAL = 1,      /* invalid argument (sizes, d, r <= 0, sigma2 < 0, NaN, null pointer) */
    GP2S_ENOMEM = 2,      /* device allocation failed (or exceeded GP2S_MEM_LIMIT bytes) */
    GP2S_ECUDA = 3,       /* a CUDA runtime call failed */
    GP2S_ENOCONV = 4,     /* a Krylov solve hit max_iter before its tolerance */
    GP2S_EBREAKDOWN = 5,  /* CG breakdown: p^T A p <= 0 or NaN while the column's residual is still
                             above the rounding level of its precision (a column whose residual has
                             reached it just stops: its Krylov space is exhausted) */
    GP2S_ETIMEOUT = 6,    /* reserved: a bounded device-side wait gave up */
    GP2S_EOVERFLOW = 7,   /* nnz would exceed 2^31 - 1 (int32 column / row-pointer limit) */
    GP2S_ENOTPD = 8,      /* A not positive definite (zero diagonal, Cholesky pivot <= 0) */
    GP2S_ENOTREADY = 9    /* the call needs an earlier gp2s_assemble / gp2s_solve on this context */
} gp2s_status;

typedef enum {
    GP2S_WENDLAND_C2 = 0,        /* (1-t)^4 (4t+1) for d <= 3, (1-t)^5 (5t+1) for d = 4 */
    GP2S_WENDLAND_C6_PAPER = 1   /* Eq. 3: (1-t)^8 (32t^3 + 25t^2 + 8t + 1), d <= 3 */
} gp2s_wendland;

typedef enum {
    GP2S_PREC_FP64 = 0,   /* FP64 values, FP64 SpMV/CG (the plain FP64 GPU form) */
    GP2S_PREC_MIXED = 1   /* FP32 values + int32 indices for assembly/SpMM/CG; FP64 dots, FP64
                             residual refinement, FP64 tridiagonal eigensolve and reductions */
} gp2s_precision;

typedef enum {
    GP2S_SOLVER_CG = 0,
    GP2S_SOLVER_MINRES = 1
} gp2s_solver;

typedef enum {
    GP2S_LOGDET_AUTO = 0,   /* EXACT when n <= n_exact, else SLQ */
    GP2S_LOGDET_EXACT = 1,  /* dense FP64 Cholesky of A: log|A| = 2 sum log L_ii */
    GP2S_LOGDET_SLQ = 2     /* stochastic Lanczos quadrature on D^{-1/2} A D^{-1/2} */
} gp2s_logdet_method;

/* Kernel families.
 *   GP2S_KERNEL_PRODUCT (Sec. 4.1 / 4.3): k = phi(|xi - xj| / r) (sum_l b_l(xi) b_l(xj) + w0), the
 *     bumps b_l of Eq. 7; support |xi - xj| < r.
 *   GP2S_KERNEL_WENDCONV (Eq. 6, Sec. 4.2): the non-stationary Wendland kernel by convolution,
 *       k = s(xi) s(xj) |S_i|^(1/4) |S_j|^(1/4) / |(S_i + S_j)/2|^(1/2) phi(sqrt(Q) / r),
 *       Q = (xi - xj)^T ((S_i + S_j)/2)^{-1} (xi - xj),  support Q < r^2,
 *     with the paper's parametric fields read as S(x) = diag(lambda_k(x)),
 *       lambda_k(x) = ell_k^2 + sum_l G_lk psi_l(x),   s(x) = w0 + sum_l amps_l psi_l(x),
 *       psi_l(x) = (1 - |x - c_l|^2 / rho_l^2)^3 inside the bump l (centers c, radii rho), else 0.
 *     Its hyperparameter vector is [centers (L x d), radii (L), amps (L), G (L x d), ell (d), w0,
 *     r, sigma2]; beta is unused.
 *   GP2S_KERNEL_FARFIELD (Sec. 4.5, small core length scales): the bumps' far-field term tied to
 *     a globally supported core, active only inside the bumps,
 *       k = w0 phi(|xi - xj| / r) + kappa(|xi - xj|) sum_l b_l(xi) b_l(xj),
 *       kappa(rho) = exp(-rho^2 / (2 lc^2)),  lc = ell[0],
 *     stored where |xi - xj| < r or where both points lie strictly inside one bump (L <= 31).
 *     Its hyperparameter vector is [centers (L x d), radii (L), amps (L), lc, w0, r, sigma2].
 *     gp2s_posterior does not take this family. */
typedef enum {
    GP2S_KERNEL_PRODUCT = 0,
    GP2S_KERNEL_WENDCONV = 1,
    GP2S_KERNEL_FARFIELD = 2
} gp2s_kernel_family;

/* Kernel hyperparameters (Eq. 3, Eq. 6, Eq. 7, Sec. 4.3) and noise (Sec. 3).  Host memory. */
typedef struct {
    int32_t d;               /* input dimension, 1..4 */
    int32_t L;               /* number of bumps, 0..32 */
    int32_t kind;            /* gp2s_wendland */
    int32_t reserved;
    double r;                /* Wendland support radius r0 > 0 */
    double sigma2;           /* noise variance >= 0 */
    double beta;             /* bump shape parameter (not differentiated) */
    double w0;               /* constant added to the bump sum (not differentiated) */
    const double *centers;   /* host, L x d row-major */
    const double *radii;     /* host, L */
    const double *amps;      /* host, L */
    int32_t family;          /* gp2s_kernel_family: PRODUCT (0), WENDCONV (1) or FARFIELD (2) */
    int32_t reserved2;
    const double *ell;       /* WENDCONV: host, d base length-scale factors (> 0); FARFIELD: ell[0] = lc */
    const double *G;         /* WENDCONV: host, L x d weights (>= 0) of the length-scale field */
} gp2s_hyper;

/* Options.  gp2s_opts_default() fills the defaults listed here. */
typedef struct {
    int32_t precision;       /* gp2s_precision, default MIXED */
    int32_t logdet;          /* gp2s_logdet_method, default AUTO */
    int32_t n_exact;         /* AUTO threshold for the dense path, default 20000 */
    int32_t probes;          /* Rademacher probes m for SLQ / Hutchinson: 0, 16, 32, 48, 64, 96 or 128;
                                default 64 */
    int32_t lanczos_steps;   /* SLQ steps k per probe, default 100 */
    int32_t max_iter;        /* iteration cap per CG solve, default 20000 */
    double tol_inner;        /* relative residual at which an FP32 y solve without reliable updates
                                stops before an FP64 refinement step (the MIXED y column with the
                                block-Jacobi preconditioner and at least 2^18 rows instead replaces
                                its recursive residual by the true FP64 residual at every gain of
                                a factor 33 and stops at tol_refine), default 1e-6 */
    double tol_refine;       /* target |y - A a| / |y| of the y solve (FP64 residual), default 1e-8 */
    double tol_probe;        /* relative residual of the probe solves used by the gradient, default 1e-5 */
    uint64_t seed;           /* probe seed, default 0 */
    int32_t precond;         /* 1 = Jacobi scaling Ah = D^{-1/2} A D^{-1/2} (0 is read as 1);
                                2 = block-Jacobi on Morton-consecutive blocks of bj_block rows of
                                Ah on top of it (MIXED precision; FP64 precision runs 1).
                                Default 2. */
    int32_t exact_support;   /* 1 = skip the FP32 guard-band pre-test (every candidate pair is
                                decided by the FP64 test); default 0 */
    int32_t max_outer;       /* refinement steps (restarted FP64-residual solves) cap, default 8 */
    int32_t profile;         /* 1 = time every SpMM launch with CUDA events (gp2s_lml_info.ms_spmm); default 0 */
    int32_t bj_block;        /* rows per block-Jacobi block (precond = 2): 64, 128, or 0 =
                                automatic (128 when A has at least 64 stored entries per row and
                                at least 768 rows per SM, else 64); default 0 */
    int32_t pattern_cache;   /* 0 = reuse the last assembly's pattern when X (fingerprint), n, d,
                                r, exact_support and precision are unchanged: only the bump
                                tables and values are recomputed; 1 = always rebuild; default 0 */
    int32_t solver;          /* solver of the y column: GP2S_SOLVER_CG (default; multi-RHS with the
                                probes, FP32 in MIXED precision with FP64 reliable updates and
                                refinement) or
                                GP2S_SOLVER_MINRES (App. B.6's solver: FP64 MINRES on
                                D^{-1/2} A D^{-1/2}, restarted on the FP64 residual until
                                tol_refine); the probe columns always run CG */
    int32_t reserved;
} gp2s_opts;

typedef struct {
    int64_t n, nnz;
    int64_t candidates;      /* candidate pairs tested (3^d stencil) */
    int64_t band_pairs;      /* pairs the FP32 guard band sent to the FP64 test */
    int64_t ncells;          /* occupied cells */
    int32_t nnz_row_min, nnz_row_max;
    double guard_delta;      /* relative guard band used by the FP32 pre-test */
    double cell_h;           /* cell edge */
    float ms_geometry, ms_count, ms_fill, ms_values64;
    int32_t pattern_reused;  /* 1 when the pattern of the previous assembly was reused */
    int32_t reserved;
} gp2s_assemble_info;

typedef struct {
    int32_t iters;           /* FP32 (or FP64) CG iterations of the y column, all refinement steps */
    int32_t outer;           /* refinement steps (0 when the reliable updates met tol_refine) */
    double relres;           /* final |y - A a| / |y|, FP64 residual */
    float ms;
} gp2s_solve_info;

typedef struct {
    int32_t method;          /* GP2S_LOGDET_EXACT or GP2S_LOGDET_SLQ */
    int32_t probes, steps;
    int32_t reserved;
    double logdet_diag;      /* sum log D_ii (SLQ) */
    double logdet_hat;       /* SLQ estimate of log|D^{-1/2} A D^{-1/2}| */
    double stderr_hat;       /* standard error of logdet_hat from the probe spread */
    float ms;
} gp2s_logdet_info;

typedef struct {
    double lml, quad, logdet, logdet_stderr, relres;
    int64_t n, nnz;
    int32_t iters_y, iters_probes, outer, logdet_method;
    float ms_assemble, ms_solve, ms_logdet, ms_grad, ms_total;
    int64_t launches;        /* kernels this call launched */
    int64_t spmm_launches;   /* multi-RHS SpMM launches of the Krylov solves (y plus probe
                                columns; the y-only SpMV launches are not counted) */
    double spmm_bytes;       /* algorithmic bytes of those launches: CSR values + indices + row
                                pointers + each input and output vector element once */
    float ms_spmm;           /* summed CUDA-event time of those launches (opts.profile = 1) */
    float reserved_f;
    int32_t bj_block;        /* rows per block-Jacobi block of the probe columns (0: no block-Jacobi) */
    int32_t spmm_seg_tiles;  /* largest number of row-block tiles per reduction segment in the
                                multi-RHS SpMM launches (1: every tile is its own segment) */
    int32_t pattern_reused;  /* 1 when the assembly reused the previous pattern */
    int32_t batch_config;    /* gp2s_lml_batched: the autotuner's launch configuration for this
                                problem (0: 64-row blocks, 1: 128-row blocks, 2 and 3: the same with
                                CUDA-graph replay), -1 when not tuned */
} gp2s_lml_info;

typedef struct gp2s_ctx gp2s_ctx;

/* Fill *opts with the defaults above. */
void gp2s_opts_default(gp2s_opts *opts);

/* Number of hyperparameters of gp2s_lml_grad: L (d + 2) + 2 (product kernel). */
int32_t gp2s_num_params(int32_t d, int32_t L);
/* The same for a given family: L (d + 2) + 2 (PRODUCT), L (2 d + 2) + d + 3 (WENDCONV) or
 * L (d + 2) + 4 (FARFIELD). */
int32_t gp2s_num_params_family(int32_t d, int32_t L, int32_t family);

/* Create a context on CUDA device `device` that issues all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the handle. */
gp2s_status gp2s_create(gp2s_ctx **ctx, int device, void *cuda_stream);

/* Release every device and host buffer of the context. */
void gp2s_destroy(gp2s_ctx *ctx);

/* One-line description of the last failure on this context ("" if none).  Owned by ctx. */
const char *gp2s_last_error(const gp2s_ctx *ctx);

/*
 * Sec. 4.6 (covariance computation) re-designed: assemble A = K + sigma2 I as CSR.
 * Points are sorted along a Morton curve of a uniform cell grid with edge h >= r; a pair (i, j)
 * is stored iff i == j or d2(i, j) < r*r with d2 = ((D0*D0 + D1*D1) + D2*D2) + ... in FP64
 * (round to nearest, no fused multiply-add).  Rows and columns use the sorted numbering;
 * columns ascend within a row.  In MIXED precision the stored FP32 values are those of the
 * Jacobi-scaled matrix Ah = D^{-1/2} A D^{-1/2} (D = diag A); FP64 values of Ah are stored too.
 *   n: number of points (>= 1).  X: n x d FP64, host or device.
 *   info: optional (NULL allowed).
 */
gp2s_status gp2s_assemble(gp2s_ctx *ctx, int64_t n, const double *X, const gp2s_hyper *hyper,
                          const gp2s_opts *opts, gp2s_assemble_info *info);

/*
 * Read-only view of the assembled matrix, borrowed from the context (valid until the next
 * assemble / lml call or destroy).  All pointers are device pointers, sorted numbering:
 *   rowptr (n + 1, int32), col (nnz, int32), val32 (nnz, FP32 values of Ah, NULL in FP64 mode),
 *   val64 (nnz, FP64 values of Ah), dscale (n, FP64, D^{-1/2}), perm (n, int32: sorted index ->
 *   original index).  A_ij = Ah_ij / (dscale_i dscale_j) in FP64.
 */
typedef struct {
    int64_t n, nnz;
    const int32_t *rowptr, *col, *perm;
    const float *val32;
    const double *val64, *dscale;
} gp2s_csr_view;
gp2s_status gp2s_csr(gp2s_ctx *ctx, gp2s_csr_view *view);

/*
 * Sec. 3 / App. B.7 "K^{-1} y": solve A a = y on the last assembled matrix by Jacobi-scaled
 * conjugate gradients; MIXED precision runs FP32 inner CG and FP64 residual refinement until
 * |y - A a| / |y| <= opts->tol_refine (FP64 values).  y, a: n FP64 in ORIGINAL point order,
 * host or device.  The solution is also kept in the context (App. B.7 keeps K^{-1} y).
 */
gp2s_status gp2s_solve(gp2s_ctx *ctx, const double *y, double *a, gp2s_solve_info *info);

/*
 * log|A| of the last assembled matrix (Sec. 3; the method is left open in Sec. 4.6 / App. B.7):
 * EXACT = dense FP64 Cholesky; SLQ = stochastic Lanczos quadrature with opts->probes Rademacher
 * probes (SplitMix64, seed) and opts->lanczos_steps steps on Ah, plus sum log D_ii.
 *   logdet: host.  stderr_hat: host, optional (0 for EXACT).
 */
gp2s_status gp2s_logdet(gp2s_ctx *ctx, double *logdet, double *stderr_hat, gp2s_logdet_info *info);

/*
 * The LML of Sec. 3: assemble + solve + log-determinant + reduction, in one call.
 *   lml: host.  info: optional.
 */
gp2s_status gp2s_lml(gp2s_ctx *ctx, int64_t n, const double *X, const double *y,
                     const gp2s_hyper *hyper, const gp2s_opts *opts, double *lml,
                     gp2s_lml_info *info);

/*
 * LML and its gradient d LML / d theta = 1/2 a^T (dA/dtheta) a - 1/2 tr(A^{-1} dA/dtheta),
 * theta = [centers (L x d), radii (L), amps (L), r, sigma2].  The trace uses Hutchinson's
 * estimator with opts->probes Rademacher probes in both log-determinant modes (u_s = A^{-1} z_s
 * are the probe columns of the shared multi-RHS CG; in SLQ mode they are the SLQ probes, solved
 * to opts->tol_probe); the quadratic term a^T dA a is exact.  dA/dtheta is formed pair by pair
 * on A's pattern and contracted on the fly; it is never stored.
 *   grad_host: host, gp2s_num_params(d, L) doubles.
 */
gp2s_status gp2s_lml_grad(gp2s_ctx *ctx, int64_t n, const double *X, const double *y,
                          const gp2s_hyper *hyper, const gp2s_opts *opts, double *lml,
                          double *grad_host, gp2s_lml_info *info);

/*
 * Many independent problems in one call (the batched form): problem b has n[b] points of
 * dimension hyper[b].d, X[b] (n[b] x d) and y[b] (n[b]), host or device.  Each problem runs the
 * gp2s_lml path (assembly, multi-RHS CG over y plus opts->probes probe columns, FP64 refinement,
 * SLQ; EXACT only when opts->logdet == EXACT, AUTO is read as SLQ).  The problems are spread over
 * a pool of worker contexts owned by ctx, each with its own CUDA stream and workspace (at most 16,
 * or GP2S_BATCH_WORKERS), largest problems first; the call first synchronises ctx's stream so
 * that device inputs produced there are complete.  In MIXED precision with precond = 2 and
 * bj_block = 0 an autotuner picks, per shape class (family, d, floor(log2 n)), the block-Jacobi
 * block size and CUDA-graph replay from timings of the class's first problems: each of the four
 * configurations runs one problem, and once all four have been timed the fastest (mean time per
 * point) is fixed for the class, in this call and later ones on ctx (GP2S_BATCH_TUNE=0 turns the
 * autotuner off).  Each problem's result equals that of a single
 * gp2s_lml call with the same options and opts.bj_block = info.bj_block, bit for bit.
 * lml_host: B doubles (NaN for a failed problem).
 * info_host: optional, B entries.  On failure the status and message are those of the first
 * failing problem ("problem b: ...").
 */
gp2s_status gp2s_lml_batched(gp2s_ctx *ctx, int32_t B, const int64_t *n, const double *const *X,
                             const double *const *y, const gp2s_hyper *hyper,
                             const gp2s_opts *opts, double *lml_host, gp2s_lml_info *info_host);

/*
 * Posterior of Eq. 2 (Sec. 3) at n_test new points, on the last solved problem (after gp2s_lml,
 * gp2s_lml_grad or gp2s_solve on this context; the solution a = A^{-1} y is kept, as App. B.7
 * keeps K^{-1} y).  With zero prior mean and A = K + sigma2 I in place of the paper's K:
 *     mean_i = k(X, x*_i)^T a
 *     var_i  = k(x*_i, x*_i) - k(X, x*_i)^T A^{-1} k(X, x*_i)       (latent f*, add sigma2 for y*)
 * k(X, x*) holds the training points with d2 < r*r (the training matrix's FP64 support test and
 * kernel value, no noise term), found through the training cell grid.  The mean is one FP64 pass.
 * The variance solves A v = k(X, x*) for batches of up to 64 test points as the columns of one
 * multi-RHS CG in the problem's precision (block-Jacobi PCG in MIXED) to opts.tol_probe of the
 * last assembly, and evaluates k^T A^{-1} k in its second-order (energy) form
 * 2 k^T v - v^T A v in FP64; it overwrites the probe solutions of the last gp2s_lml_grad (the
 * gradient was already returned).
 *   Xtest: n_test x d FP64, host or device.  mean: n_test FP64, host or device.  var: n_test FP64,
 *   host or device, or NULL to skip the variance solves.  info: optional.
 * Returns GP2S_ENOTREADY without a solved problem, GP2S_ENOCONV if a variance solve hits max_iter.
 */
typedef struct {
    int64_t n_test;
    int64_t cross_entries;   /* nonzero k(x*_i, x_j) found */
    int32_t batches;         /* variance solves */
    int32_t iters_max;       /* largest CG iteration count of those solves */
    float ms_mean, ms_var;
} gp2s_posterior_info;
gp2s_status gp2s_posterior(gp2s_ctx *ctx, int64_t n_test, const double *Xtest, double *mean, double *var,
                           gp2s_posterior_info *info);

/*
 * Block Metropolis-Hastings training of theta (Sec. 4.6, App. D).  Each iteration sweeps the
 * parameter blocks in order; block b proposes theta' = theta + step * z on its components
 * (z standard normal), rejects theta' outside [lower, upper] (a flat prior), and otherwise
 * evaluates LML(theta') with gp2s_lml (opts, with pattern reuse forced on: blocks that leave r
 * alone recompute only the values) and accepts when log u < LML(theta') - LML(theta).
 * A proposal the engine refuses (GP2S_EINVAL, GP2S_ENOTPD) is a rejection.
 *   block: P = gp2s_num_params_family(d, L, family) ints, the block of each theta component (in
 *          the order gp2s_lml_grad returns them; -1 = held fixed); a block
 *          without members is skipped.
 *   step:  P proposal standard deviations.  lower / upper: P bounds each, or NULL (unbounded).
 *   normals (iters x P) / uniforms (iters x nblocks): the random numbers, or NULL to let the
 *          driver draw them (SplitMix64 counter stream keyed by seed; Box-Muller normals).
 *   checkpoint: file written every checkpoint_every iterations (and after the last), or NULL.
 *   resume = 1: continue from that file (its iteration count, theta and LML); rows before the
 *          resumed iteration are not written.
 *   chain: host, iters x (P + 1): theta after each iteration's sweep, then its LML.
 *   accept: host, iters x nblocks acceptance flags, or NULL.
 */
typedef struct {
    int32_t iters;
    int32_t nblocks;                 /* 1..64 */
    const int32_t *block;
    const double *step;
    const double *lower, *upper;
    const double *normals, *uniforms;
    uint64_t seed;
    const char *checkpoint;
    int32_t checkpoint_every;
    int32_t resume;
} gp2s_mcmc_opts;
typedef struct {
    int32_t start, done;             /* first iteration run by this call, iterations completed */
    int32_t evals;                   /* LML evaluations */
    int32_t pattern_reused;          /* of which reused the previous pattern */
    int32_t accepted;                /* accepted proposals over the whole chain */
    int32_t reserved;
    double lml;                      /* LML of the final state */
    float ms;
    float reserved_f;
} gp2s_mcmc_info;
gp2s_status gp2s_mcmc(gp2s_ctx *ctx, int64_t n, const double *X, const double *y, const gp2s_hyper *hyper0,
                      const gp2s_opts *opts, const gp2s_mcmc_opts *mcmc, double *chain, int32_t *accept,
                      gp2s_mcmc_info *info);

/*
 * Allocation-free exact LML for small problems.  The paper has no counterpart: this is a service
 * entry point for callers that cannot allocate device memory, e.g. code that issues work while a
 * CUDA stream is being captured into a graph (cudaMalloc is not allowed there), or a process whose
 * device memory is entirely reserved by another allocator (a framework's caching pool, a serving
 * runtime with a fixed budget) so that the library must not create allocations of its own.
 *
 * It computes what gp2s_lml computes with GP2S_PREC_FP64 and GP2S_LOGDET_EXACT, for n <=
 * GP2S_NOALLOC_MAX_N points: the dense FP64 matrix A = K + sigma2 I (same exact support test and
 * kernel as the CSR path), its Cholesky factor, log|A|, a = A^{-1} y, and the LML.  All scratch
 * lives in one fixed-size array compiled into the library (about 2.1 MB of every GPU that loads the
 * library, held until the process exits); the call makes no cudaMalloc / cudaFree and calls no
 * allocating library routine.
 *   n: 1..GP2S_NOALLOC_MAX_N; larger n returns GP2S_EINVAL and does nothing.
 *   X_dev (n x d FP64), y_dev (n FP64): DEVICE pointers, original point order.
 *   hyper: host, as for gp2s_lml; the product kernel family only (WENDCONV returns GP2S_EINVAL).
 *   out_dev: DEVICE pointer to 3 doubles receiving {LML, y^T A^{-1} y, log|A|}; NaN if a Cholesky
 *   pivot is not positive.
 *   cuda_stream: the stream all work is issued on (NULL = legacy default stream).  It must belong
 *   to the calling thread's current device: a stream of another device returns GP2S_EINVAL when
 *   it is not being captured.  While it is being captured this is not checked (the runtime does
 *   not permit asking a capturing stream for its device), so the caller answers for it.
 * The call is asynchronous: it returns after queueing the work on cuda_stream.  The first call on
 * each device looks up the scratch array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture begins.  Every call on a device shares
 * the one scratch array and leaves its contents behind: calls whose work overlaps on the GPU (two
 * streams, or two host threads) race and give wrong results, so serialise them.
 */
#define GP2S_NOALLOC_MAX_N 512
gp2s_status gp2s_lml_exact_noalloc(int64_t n, const double *X_dev, const double *y_dev,
                                   const gp2s_hyper *hyper, double *out_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GP2S_H */
