// gp2s_internal.cuh -- shared declarations of the GB300 engine (device helpers, context, launchers).
// Internal to the library; the public ABI is include/gp2s.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gp2s.h"

namespace gp2s {

constexpr int kMaxDim = 4;
constexpr int kMaxBumps = 32;
constexpr int kWarp = 32;

// The CG scalar block: kScal doubles per column c (y = 0, probes 1..m) at sc + c kScal:
// [rho, alpha, beta, b2, pq, rr, steps, tol2b2, rho of the previous step, why an active column
// stopped (1: in the beta kernel, its direction update still pending; 2: in the alpha kernel)]
constexpr int kScal = 10;
enum { S_RHO = 0, S_ALPHA, S_BETA, S_B2, S_PQ, S_RR, S_STEPS, S_TOL, S_RHO_PREV, S_STOP };

// ------------------------------------------------------------------------------------------
// Kernel hyperparameters passed by value to kernels (Eq. 3, Eq. 7, Sec. 4.3).
// ------------------------------------------------------------------------------------------
struct KernelParams {
    int d, L, kind, family;
    double r, inv_r, sigma2, beta, w0;
    double centers[kMaxBumps * kMaxDim];
    double radii[kMaxBumps];
    double amps[kMaxBumps];
    double ell[kMaxDim];              // Wendland convolution (family 1): base length-scale factors
    double G[kMaxBumps * kMaxDim];    // family 1: weights of the length-scale field
};

// Geometry of the cell grid: cell edge h >= r, FP64 origin, F fine bits per dimension below the
// cell level, B bits per dimension in total (d * B <= 64).
struct GridParams {
    int d, fine_bits, bits, pad;
    double origin[kMaxDim];
    double inv_h;             // 1 / h
    double h;
    int64_t dims[kMaxDim];    // cells per dimension
};

// FP32 guard band of the support pre-test: accept if d2_f32 < thr_lo, reject if d2_f32 > thr_hi,
// otherwise decide with the exact FP64 test.
struct SupportParams {
    float thr_lo, thr_hi;
    double r2;                // r * r in FP64 (the exact test's threshold)
};

// ------------------------------------------------------------------------------------------
// Device buffers (grow-only).
// ------------------------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

struct HostPinned {
    void *p = nullptr;
    size_t bytes = 0;
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// The assembled single problem.
struct Assembled {
    bool valid = false;
    int64_t n = 0, nnz = 0, ncells = 0, nitems = 0;
    int d = 0, L = 0, precision = GP2S_PREC_MIXED;
    KernelParams kp{};
    GridParams gp{};
    SupportParams sp{};
    gp2s_opts opts{};
    gp2s_assemble_info info{};
    double wc_lmax = 0.0;     // Wendland convolution: largest lambda_k over the points (cell edge r sqrt)
};

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
};

}  // namespace gp2s

struct gp2s_ctx {
    int device = 0;
    int num_sms = 152;
    cudaStream_t stream = nullptr;
    std::string err;
    size_t mem_limit = 0;     // GP2S_MEM_LIMIT (0 = none)
    size_t mem_in_use = 0;
    // geometry / sort
    gp2s::DevBuf Xin, yin, keys, keys2, idx, idx2, perm, iperm;
    gp2s::DevBuf Xs64, Xhi, Xlo, ys64;
    gp2s::DevBuf bbox_part, bbox;
    gp2s::DevBuf hist, scan_tmp, scan_tmp2;
    gp2s::DevBuf cell_start, cell_flag, items, item_cnt;
    // bumps / diagonal
    gp2s::DevBuf B64, B32, D64, s64, s32;
    // Wendland convolution: length-scale field (double4 per point) and signal field
    gp2s::DevBuf wc_lam, wc_sig;
    // far-field kernel: bump membership masks, member lists and the union pattern's buffers
    gp2s::DevBuf ff_mask, ff_flag, ff_mptr, ff_mcol, ff_ucnt, ff_uptr, ff_ucol;
    // CSR
    gp2s::DevBuf rowcnt, rowptr, col, val32, val64, counters;
    // Krylov
    gp2s::DevBuf vec, vec64, partials, scal, Z, Zf, rec, rsplit;   // Zf: probe signs as FP32 +-1 (gradient)
    // row-block (8 rows) copy of the FP32 matrix for the multi-RHS SpMM
    gp2s::DevBuf rb_cnt, rb_ptr, rb_col, rb_val, rb_tpart, rb_seg;
    bool rb_valid = false;
    int64_t rb_entries = 0;
    // block-Jacobi preconditioner: FP32 M^{-1} per 64-row block and the block log-determinants
    gp2s::DevBuf bj_Minv, bj_ld, bj_Minv_y;
    bool bj_valid = false;
    int bj_size = 64;               // rows per block-Jacobi block of the probe columns
    int bj_size_y = 64;             // rows per block of the y column (64 or 128)
    double bj_logdet = 0.0;
    bool probes_for_grad = false;   // the probe solves feed the Hutchinson gradient
    bool use_graphs = true;         // replay runs of CG iterations as CUDA graphs (GP2S_GRAPHS=0: off)
    bool pc_async = true;           // probe-group PCG step on the bulk-copy pipelined kernel
    bool pc_async64 = true;         // ... also with 64-row block-Jacobi blocks (two per stage)
    bool spmm_half = false;         // 16 and 32 columns on half-warp entry groups (KH = 1, 2)
    int spmm_tma = 0;               // 16, 32, 64 columns: rows per 32 gathered by tensor copies (0: none)
    bool pc_fuse_y = true;          // the y column's PCG update inside the probe kernel
    bool reliable_y = true;         // reliable updates of the y column instead of restarted refinement
    double reliable_delta = 0.03;   // residual replacement at every gain of this factor
    int64_t reliable_min_rows = int64_t(1) << 18;   // reliable updates of the y column from here
                                    // (GP2S_PC_ASYNC=0: the staged kernel)
    cudaStream_t capture_stream = nullptr;   // private stream the graphs are captured on
    // SLQ's tridiagonal quadratures run on a side stream once the probes' k steps are recorded,
    // beside the rest of the probe solves (slq_start_async); slq_logdet waits for them
    cudaStream_t side_stream = nullptr;
    cudaEvent_t slq_ev_rec = nullptr, slq_ev_done = nullptr;
    bool slq_pending = false;
    bool slq_async = true;
    int slq_m = 0, slq_k = 0;
    gp2s::DevBuf slq_work;
    // batched form: worker contexts (own stream and workspace each), created on first use
    std::vector<gp2s_ctx *> workers;
    std::vector<cudaStream_t> worker_streams;
    int batch_workers_max = 16;
    // batched autotuner: per shape class, the summed score (seconds per point) and the number of
    // problems each launch configuration ran, and which configurations were handed out
    struct TuneState {
        std::vector<double> score;
        std::vector<int> count, issued;
        int chosen = -1;   // fixed once every configuration has a measurement
    };
    std::map<int, TuneState> tune;
    std::mutex tune_mu;
    // dense
    gp2s::DevBuf dense;
    // adjoint
    gp2s::DevBuf H, gpart;
    // posterior (test points, their bump values / prior variances / outputs, counters, partials)
    gp2s::DevBuf post_X, post_B, post_cnt, post_part;
    // MINRES vectors and scalars
    gp2s::DevBuf mr_vec;
    // MCMC driver: the chain's inputs staged once
    gp2s::DevBuf mc_X, mc_y;
    // host staging
    gp2s::HostPinned hbuf;
    gp2s::Assembled A;
    // pattern cache: the last assembly's points (fingerprint), size and support radius; a later
    // assembly with the same ones reuses the pattern and recomputes only the values
    bool pat_valid = false;
    int64_t pat_n = 0;
    int pat_d = 0, pat_exact = 0, pat_precision = 0;
    double pat_r = 0.0;
    uint64_t pat_hash = 0;
    bool rb_pattern_valid = false;   // the RB8 union structure matches the current pattern
    // last solve
    bool have_solution = false;
    bool have_probes = false;
    int32_t solve_iters = 0, solve_outer = 0;
    double solve_relres = 0.0;
    int32_t probe_iters = 0;
    bool have_exact = false;   // dense factor of the current matrix is in `dense`
    double exact_lhat = 0.0;   // its 2 sum log L_ii
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // launch accounting and optional SpMM timing
    int64_t launches = 0;
    int64_t spmm_launches = 0;
    double spmm_bytes = 0.0;
    int spmm_seg_tiles = 0;   // largest tiles-per-segment of this call's multi-RHS SpMM launches
    bool profile = false;
    std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop) per profiled SpMM launch
    size_t prof_used = 0;
    double prof_ms = 0.0;
};

namespace gp2s {

// Status helpers ---------------------------------------------------------------------------
gp2s_status set_err(gp2s_ctx *c, gp2s_status st, const std::string &msg);
gp2s_status cuda_err(gp2s_ctx *c, cudaError_t e, const char *where);
gp2s_status ensure(gp2s_ctx *c, DevBuf &b, size_t bytes);
gp2s_status ensure_host(gp2s_ctx *c, HostPinned &b, size_t bytes);
// Raise a kernel's dynamic shared-memory limit to at least smem bytes (thread-safe, grow-only).
gp2s_status smem_attr(gp2s_ctx *c, const void *func, size_t smem);

#define GP2S_CUDA(ctx, expr)                                     \
    do {                                                         \
        cudaError_t e__ = (expr);                                \
        if (e__ != cudaSuccess) return gp2s::cuda_err((ctx), e__, #expr); \
    } while (0)
#define GP2S_TRY(expr)                                           \
    do {                                                         \
        gp2s_status s__ = (expr);                                \
        if (s__ != GP2S_OK) return s__;                          \
    } while (0)
#define GP2S_LAUNCH(ctx)                                         \
    do {                                                         \
        ++(ctx)->launches;                                       \
        cudaError_t e__ = cudaGetLastError();                    \
        if (e__ != cudaSuccess) return gp2s::cuda_err((ctx), e__, "kernel launch"); \
    } while (0)

// Primitives (prim.cu) -----------------------------------------------------------------------
// Exclusive scan of n int32 counts into out (n + 1 entries, out[n] = total), int64 accumulation.
// *total_host receives the total (the call synchronises the stream to read it).
gp2s_status scan_counts_i32(gp2s_ctx *c, const int32_t *in, int32_t *out, int64_t n, int64_t *total_host);
gp2s_status scan_counts_i64(gp2s_ctx *c, const int32_t *in, int64_t *out, int64_t n, int64_t *total_host);
// Stable LSD radix sort of (64-bit key, 32-bit value) pairs on the low `bits` key bits.
// Results end in keys/vals (the alternate buffers are scratch of the same size).
gp2s_status radix_sort_pairs(gp2s_ctx *c, uint64_t *keys, uint64_t *keys_alt, int32_t *vals,
                             int32_t *vals_alt, int64_t n, int bits);

// Geometry + assembly (geometry.cu, assemble.cu) ---------------------------------------------
gp2s_status assemble_problem(gp2s_ctx *c, int64_t n, const double *X_dev, const gp2s_hyper *h,
                             const gp2s_opts *o);

// Krylov (krylov.cu) ---------------------------------------------------------------------------
// Multi-RHS CG on the assembled Ah for the y column (scaled rhs s * y) and m probe columns.
struct CGResult {
    int iters_y = 0, iters_probes = 0, outer = 0;
    double relres = 0.0;
    gp2s_status status = GP2S_OK;
};
gp2s_status krylov_solve(gp2s_ctx *c, const double *y_sorted_dev, bool with_probes, int m,
                         int ksteps, CGResult *res);
gp2s_status slq_logdet(gp2s_ctx *c, int m, int ksteps, double *logdet_hat, double *stderr_hat);
// Start SLQ's quadratures on the side stream from the coefficients recorded so far (every probe
// column has its k steps or has stopped); the stream order of c->stream is the dependency.
gp2s_status slq_start_async(gp2s_ctx *c, int m, int ksteps);
// c->stream waits for a pending SLQ launch (before its inputs are overwritten).
gp2s_status slq_fence(gp2s_ctx *c);
// FP64 MINRES on Ah (minres.cu): b (device, sorted order) -> x, until |b - Ah x| <= tol |b|.
gp2s_status minres_solve(gp2s_ctx *c, const double *b, double *x, double tol, int maxit, int *steps);
// Multi-RHS (P)CG on caller-supplied columns (no y column, no SLQ records): krylov_columns_buffers
// gives the probe group's right-hand-side block rz (n x m, row-major, vector precision of the
// assembled problem) to fill, and its solution block xz; krylov_columns_solve then runs the
// columns to relative residual tol (xz: solutions, rz: final recursively updated residuals).
gp2s_status krylov_columns_buffers(gp2s_ctx *c, int m, void **rz, void **xz);
gp2s_status krylov_columns_solve(gp2s_ctx *c, int m, double tol, int *iters);
gp2s_status exact_logdet_solve(gp2s_ctx *c, const double *y_sorted_dev, double *logdet_hat,
                               bool want_inverse);
// Reductions used by several stages
gp2s_status sum_log_diag(gp2s_ctx *c, double *out_host);
gp2s_status dot_f64(gp2s_ctx *c, const double *a, const double *b, int64_t n, double *out_host);

// Adjoint (adjoint.cu) ---------------------------------------------------------------------------
gp2s_status adjoint_gradient(gp2s_ctx *c, int m, double *grad_host);

// Posterior (posterior.cu) -------------------------------------------------------------------
gp2s_status posterior(gp2s_ctx *c, int64_t ns, const double *Xs, double *mean, double *var,
                      gp2s_posterior_info *info);

// Block Metropolis-Hastings driver (mcmc.cu) ----------------------------------------------------
gp2s_status mcmc_run(gp2s_ctx *c, int64_t n, const double *X, const double *y, const gp2s_hyper *h0,
                     const gp2s_opts *o, const gp2s_mcmc_opts *mo, double *chain, int32_t *accept,
                     gp2s_mcmc_info *info);

// Batched engine (batched.cu) ----------------------------------------------------------------
gp2s_status batched_lml(gp2s_ctx *c, int32_t B, const int64_t *n, const double *const *X,
                        const double *const *y, const gp2s_hyper *hyper, const gp2s_opts *opts,
                        double *lml_host, gp2s_lml_info *info_host);

// Device helpers -------------------------------------------------------------------------------
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace gp2s
