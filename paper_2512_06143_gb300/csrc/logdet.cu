// logdet.cu -- log|A| (Sec. 3; the method is left open in Sec. 4.6 / App. B.7):
//   * SLQ: stochastic Lanczos quadrature (Ubaru, Chen & Saad 2017) on Ah = D^{-1/2} A D^{-1/2}.
//     For every probe z_s the tridiagonal T_s comes from the recorded CG coefficients (CG-Lanczos
//     relation); its eigenvalues theta_j and eigenvector first components tau_j come from an
//     implicit-shift symmetric tridiagonal QR iteration with Wilkinson shifts (Golub & Van Loan,
//     Sec. 8.3), one thread per probe in FP64, and log|Ah| ~= (n/m) sum_s sum_j tau_sj^2 log theta_sj.
//   * EXACT: dense FP64 Cholesky of Ah (right-looking, 32-wide panels: diagonal-block factor,
//     panel triangular solve, symmetric rank-32 update of the trailing lower triangle), then
//     log|Ah| = 2 sum log L_ii and the y solve by forward/backward substitution.
//   log|A| = sum log D_ii + log|Ah| in both cases.
#include <cmath>
#include <cstring>
#include <mutex>

#include "gp2s_internal.cuh"
#include "gp2s_kernel_math.cuh"

namespace gp2s {

namespace {

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------------------------
// Symmetric tridiagonal eigenvalues + first eigenvector components, implicit QR with Wilkinson
// shift and bulge chasing, deflating negligible off-diagonals.  a: diagonal (k), b: off-diagonal
// (k - 1), q: first row of the accumulated rotations (k).  Returns false if it fails to converge.
// ---------------------------------------------------------------------------------------------
__host__ __device__ bool tridiag_eig(double *a, double *b, double *q, int k)
{
    const double eps = 2.220446049250313e-16;
    for (int i = 0; i < k; ++i) q[i] = i == 0 ? 1.0 : 0.0;
    int hi = k - 1;
    int guard = 0;
    while (hi > 0) {
        // deflate from the bottom
        if (fabs(b[hi - 1]) <= eps * (fabs(a[hi - 1]) + fabs(a[hi]))) {
            b[hi - 1] = 0.0;
            --hi;
            continue;
        }
        // start of the unreduced block ending at hi
        int lo = hi - 1;
        while (lo > 0 && fabs(b[lo - 1]) > eps * (fabs(a[lo - 1]) + fabs(a[lo]))) --lo;
        if (lo > 0) b[lo - 1] = 0.0;
        if (++guard > 60 * k) return false;
        // Wilkinson shift from the trailing 2x2 block
        const double bb = b[hi - 1];
        const double dd = 0.5 * (a[hi - 1] - a[hi]);
        const double rr = hypot(dd, bb);
        const double mu = a[hi] - bb * bb / (dd + (dd >= 0.0 ? rr : -rr));
        // bulge chase over [lo, hi]
        double x = a[lo] - mu, z = b[lo];
        for (int j = lo; j < hi; ++j) {
            double r = hypot(x, z);
            double c = r > 0.0 ? x / r : 1.0;
            double s = r > 0.0 ? -z / r : 0.0;
            if (j > lo) b[j - 1] = r;   // the rotation folds the bulge into b[j-1]
            // 2x2 similarity on rows/cols j, j+1 with P = [[c, s], [-s, c]]
            const double aj = a[j], aj1 = a[j + 1], bj = b[j];
            const double cc = c * c, ss = s * s, cs = c * s;
            a[j] = aj * cc - 2.0 * bj * cs + aj1 * ss;
            a[j + 1] = aj * ss + 2.0 * bj * cs + aj1 * cc;
            b[j] = (aj - aj1) * cs + bj * (cc - ss);
            if (j + 1 < hi) {
                // the next off-diagonal b[j+1] is rotated into the new bulge at (j + 2, j)
                x = b[j];
                z = -s * b[j + 1];
                b[j + 1] = c * b[j + 1];
            }
            // accumulate the first row of Q <- Q P
            const double qj = q[j], qj1 = q[j + 1];
            q[j] = qj * c - qj1 * s;
            q[j + 1] = qj * s + qj1 * c;
        }
    }
    return true;
}

// One CTA per probe (its first thread runs the sequential QR iteration on arrays in shared
// memory): T from CG coefficients, eigen-decomposition, Gauss quadrature of log.
__global__ void k_slq(const double *__restrict__ rec, const double *__restrict__ sc, int m, int ksteps,
                      double *__restrict__ work, double *__restrict__ out, int *__restrict__ bad)
{
    extern __shared__ double slq_sh[];
    const int s = blockIdx.x;
    if (s >= m || threadIdx.x != 0) return;
    (void)work;
    double *a = slq_sh;
    double *b = a + ksteps;
    double *q = b + ksteps;
    // number of recorded steps for this probe column (column s + 1 of the CG scalar block)
    int steps = (int)sc[(s + 1) * kScal + S_STEPS];
    int k = steps < ksteps ? steps : ksteps;
    if (k <= 0) { out[s] = 0.0; atomicOr(bad, 1); return; }
    const double *al = rec + (int64_t)s * ksteps * 2;
    // CG-Lanczos relation: T_00 = 1/alpha_0; T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1};
    // T_{j,j+1} = sqrt(beta_j)/alpha_j
    for (int j = 0; j < k; ++j) {
        double aj = al[2 * j];
        a[j] = 1.0 / aj + (j > 0 ? al[2 * (j - 1) + 1] / al[2 * (j - 1)] : 0.0);
        if (j + 1 < k) b[j] = sqrt(al[2 * j + 1]) / aj;
    }
    if (!tridiag_eig(a, b, q, k)) { out[s] = nan(""); atomicOr(bad, 2); return; }
    double g = 0.0;
    for (int j = 0; j < k; ++j) {
        if (!(a[j] > 0.0)) { atomicOr(bad, 4); out[s] = nan(""); return; }
        g += q[j] * q[j] * log(a[j]);
    }
    out[s] = g;
}

__global__ void k_sum_log(const double *__restrict__ D, int64_t n, double *__restrict__ part)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += log(D[i]);
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_dot64(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                        double *__restrict__ part)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------------------------
// Dense FP64 Cholesky (lower, column-major-free: row-major n x n, only the lower triangle used)
// ---------------------------------------------------------------------------------------------
constexpr int NB = 32;

__global__ void k_densify(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                          const double *__restrict__ val, int64_t n, double *__restrict__ Ad)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw)
        for (int p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) Ad[i * n + col[p]] = val[p];
}

// Factor the NB x NB diagonal block at (kb, kb) in shared memory.
__global__ void k_potrf_diag(double *__restrict__ Ad, int64_t n, int kb, int *__restrict__ bad)
{
    __shared__ double S[NB][NB + 1];
    const int nbk = (int)(n - kb < NB ? n - kb : NB);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int i = t / NB, j = t % NB;
        S[i][j] = (i < nbk && j < nbk) ? Ad[(int64_t)(kb + i) * n + kb + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < nbk; ++j) {
        if (threadIdx.x == 0) {
            double d = S[j][j];
            if (!(d > 0.0)) { atomicOr(bad, 1); d = 1.0; }
            S[j][j] = sqrt(d);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < nbk; i += blockDim.x) S[i][j] /= S[j][j];
        __syncthreads();
        for (int t = threadIdx.x; t < nbk * nbk; t += blockDim.x) {
            int i = t / nbk, l = t % nbk;
            if (i > j && l > j && l <= i) S[i][l] -= S[i][j] * S[l][j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nbk * nbk; t += blockDim.x) {
        int i = t / nbk, j = t % nbk;
        if (j <= i) Ad[(int64_t)(kb + i) * n + kb + j] = S[i][j];
    }
}

// Panel: rows r >= kb + NB, columns kb..kb+NB: L21 = A21 L11^{-T}.  One thread per row.
__global__ void k_trsm_panel(double *__restrict__ Ad, int64_t n, int kb)
{
    __shared__ double Lk[NB][NB + 1];
    const int nbk = (int)(n - kb < NB ? n - kb : NB);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int i = t / NB, j = t % NB;
        Lk[i][j] = (i < nbk && j <= i) ? Ad[(int64_t)(kb + i) * n + kb + j] : 0.0;
    }
    __syncthreads();
    int64_t r = kb + nbk + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double x[NB];
    double *row = Ad + r * n + kb;
    for (int j = 0; j < nbk; ++j) {
        double v = row[j];
        for (int l = 0; l < j; ++l) v -= x[l] * Lk[j][l];
        x[j] = v / Lk[j][j];
    }
    for (int j = 0; j < nbk; ++j) row[j] = x[j];
}

// Trailing update of the lower triangle: A[i][j] -= sum_l L[i][kb+l] L[j][kb+l] for
// i >= j >= kb + NB.  64 x 64 output tiles, 256 threads, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) k_syrk(double *__restrict__ Ad, int64_t n, int kb)
{
    const int64_t t0 = kb + NB;
    const int64_t ti = t0 + (int64_t)blockIdx.y * 64, tj = t0 + (int64_t)blockIdx.x * 64;
    if (tj > ti + 63) return;   // strictly upper tile
    __shared__ double Li[64][NB + 1], Lj[64][NB + 1];
    const int nbk = (int)(n - kb < NB ? n - kb : NB);
    for (int t = threadIdx.x; t < 64 * NB; t += blockDim.x) {
        int r = t / NB, l = t % NB;
        Li[r][l] = (ti + r < n && l < nbk) ? Ad[(ti + r) * n + kb + l] : 0.0;
        Lj[r][l] = (tj + r < n && l < nbk) ? Ad[(tj + r) * n + kb + l] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int l = 0; l < nbk; ++l) {
        double vi[4], vj[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) { vi[a] = Li[ty + 16 * a][l]; vj[a] = Lj[tx + 16 * a][l]; }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(vi[a], vj[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int64_t i = ti + ty + 16 * a, j = tj + tx + 16 * b;
            if (i < n && j <= i) Ad[i * n + j] -= acc[a][b];
        }
}

__global__ void k_logdiag(const double *__restrict__ Ad, int64_t n, double *__restrict__ part)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += log(Ad[i * n + i]);
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// Forward substitution L z = b, block kb: solve the NB x NB diagonal block (one CTA).
__global__ void k_trsv_diag(const double *__restrict__ Ad, int64_t n, int kb, double *__restrict__ x, int trans)
{
    __shared__ double xs[NB];
    const int nbk = (int)(n - kb < NB ? n - kb : NB);
    if (threadIdx.x == 0) {
        if (!trans) {
            for (int j = 0; j < nbk; ++j) {
                double v = x[kb + j];
                for (int l = 0; l < j; ++l) v -= Ad[(int64_t)(kb + j) * n + kb + l] * xs[l];
                xs[j] = v / Ad[(int64_t)(kb + j) * n + kb + j];
            }
        } else {
            for (int j = nbk - 1; j >= 0; --j) {
                double v = x[kb + j];
                for (int l = j + 1; l < nbk; ++l) v -= Ad[(int64_t)(kb + l) * n + kb + j] * xs[l];
                xs[j] = v / Ad[(int64_t)(kb + j) * n + kb + j];
            }
        }
        for (int j = 0; j < nbk; ++j) x[kb + j] = xs[j];
    }
}

// Forward: x[i] -= sum_l L[i][kb+l] x[kb+l] for i >= kb + NB (one warp per row).
// Backward (trans): x[j] -= sum_l L[kb+l][j] x[kb+l] for j < kb (one thread per column j).
__global__ void k_trsv_update(const double *__restrict__ Ad, int64_t n, int kb, double *__restrict__ x, int trans)
{
    const int nbk = (int)(n - kb < NB ? n - kb : NB);
    if (!trans) {
        const int lane = threadIdx.x & 31;
        const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t i = kb + nbk + w0; i < n; i += nw) {
            double v = lane < nbk ? Ad[i * n + kb + lane] * x[kb + lane] : 0.0;
            v = warp_sum_d(v);
            if (lane == 0) x[i] -= v;
        }
    } else {
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < kb; j += (int64_t)gridDim.x * blockDim.x) {
            double v = 0.0;
            for (int l = 0; l < nbk; ++l) v = fma(Ad[(int64_t)(kb + l) * n + j], x[kb + l], v);
            x[j] -= v;
        }
    }
}

__global__ void k_gp2s_mul(int64_t n, const double *a, const double *b, double *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

gp2s_status reduce_parts(gp2s_ctx *c, const double *part, int cnt, double *out_host)
{
    std::vector<double> h(cnt);
    GP2S_CUDA(c, cudaMemcpyAsync(h.data(), part, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    double s = 0.0;
    for (int k = 0; k < cnt; ++k) s += h[k];
    *out_host = s;
    return GP2S_OK;
}

}  // namespace

gp2s_status sum_log_diag(gp2s_ctx *c, double *out_host)
{
    const int nb = 152 * 2;
    GP2S_TRY(ensure(c, c->gpart, sizeof(double) * (2 * nb + 8)));
    k_sum_log<<<nb, 256, 0, c->stream>>>(c->D64.as<double>(), c->A.n, c->gpart.as<double>());
    GP2S_LAUNCH(c);
    return reduce_parts(c, c->gpart.as<double>(), nb, out_host);
}

gp2s_status dot_f64(gp2s_ctx *c, const double *a, const double *b, int64_t n, double *out_host)
{
    const int nb = 152 * 2;
    GP2S_TRY(ensure(c, c->gpart, sizeof(double) * (2 * nb + 8)));
    k_dot64<<<nb, 256, 0, c->stream>>>(a, b, n, c->gpart.as<double>());
    GP2S_LAUNCH(c);
    return reduce_parts(c, c->gpart.as<double>(), nb, out_host);
}

// SLQ scratch: per probe 3 k doubles of work, the m quadratures, the failure flag, and a snapshot
// of the CG scalar block (the step counts k_slq reads) taken when the launch is queued.
static double *slq_layout(gp2s_ctx *c, int m, int ksteps, double **out, int **bad, double **snap)
{
    double *work = c->slq_work.as<double>();
    *out = work + (size_t)m * 3 * ksteps;
    *bad = reinterpret_cast<int *>(*out + m);
    *snap = *out + m + 8;
    return work;
}

static gp2s_status slq_launch(gp2s_ctx *c, cudaStream_t wait_on, cudaStream_t run_on, int m, int ksteps)
{
    GP2S_TRY(ensure(c, c->slq_work, sizeof(double) * ((size_t)m * 3 * ksteps + m + 8 + (size_t)kScal * (m + 1)) + 64));
    double *out, *snap;
    int *bad;
    double *work = slq_layout(c, m, ksteps, &out, &bad, &snap);
    GP2S_CUDA(c, cudaMemcpyAsync(snap, c->scal.as<double>(), sizeof(double) * kScal * (m + 1), cudaMemcpyDeviceToDevice,
                                 wait_on));
    GP2S_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), wait_on));
    if (run_on != wait_on) {
        GP2S_CUDA(c, cudaEventRecord(c->slq_ev_rec, wait_on));
        GP2S_CUDA(c, cudaStreamWaitEvent(run_on, c->slq_ev_rec, 0));
    }
    const size_t smem = sizeof(double) * 3 * (size_t)ksteps;
    GP2S_TRY(smem_attr(c, (const void *)k_slq, smem));
    k_slq<<<m, 32, smem, run_on>>>(c->rec.as<double>(), snap, m, ksteps, work, out, bad);
    GP2S_LAUNCH(c);
    return GP2S_OK;
}

gp2s_status slq_start_async(gp2s_ctx *c, int m, int ksteps)
{
    if (!c->side_stream) {
        GP2S_CUDA(c, cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
        GP2S_CUDA(c, cudaEventCreateWithFlags(&c->slq_ev_rec, cudaEventDisableTiming));
        GP2S_CUDA(c, cudaEventCreateWithFlags(&c->slq_ev_done, cudaEventDisableTiming));
    }
    GP2S_TRY(slq_fence(c));
    GP2S_TRY(slq_launch(c, c->stream, c->side_stream, m, ksteps));
    GP2S_CUDA(c, cudaEventRecord(c->slq_ev_done, c->side_stream));
    c->slq_pending = true;
    c->slq_m = m;
    c->slq_k = ksteps;
    return GP2S_OK;
}

gp2s_status slq_fence(gp2s_ctx *c)
{
    if (c->slq_pending) GP2S_CUDA(c, cudaStreamWaitEvent(c->stream, c->slq_ev_done, 0));
    return GP2S_OK;
}

gp2s_status slq_logdet(gp2s_ctx *c, int m, int ksteps, double *logdet_hat, double *stderr_hat)
{
    if (m <= 0 || !c->have_probes) return set_err(c, GP2S_ENOTREADY, "SLQ needs the probe CG run");
    if (c->slq_pending && c->slq_m == m && c->slq_k == ksteps) {
        GP2S_TRY(slq_fence(c));   // queued beside the probe solves, from the same recorded steps
    } else {
        GP2S_TRY(slq_fence(c));
        GP2S_TRY(slq_launch(c, c->stream, c->stream, m, ksteps));
    }
    c->slq_pending = false;
    double *out, *snap;
    int *bad;
    slq_layout(c, m, ksteps, &out, &bad, &snap);
    std::vector<double> g(m);
    int hbad = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(g.data(), out, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hbad) return set_err(c, GP2S_EBREAKDOWN, "SLQ: tridiagonal eigensolve failed or non-positive Ritz value");
    const double n = (double)c->A.n;
    double mean = 0.0;
    for (int s = 0; s < m; ++s) mean += n * g[s];
    mean /= m;
    double var = 0.0;
    for (int s = 0; s < m; ++s) var += (n * g[s] - mean) * (n * g[s] - mean);
    var = m > 1 ? var / (m - 1) : 0.0;
    *logdet_hat = mean;
    if (stderr_hat) *stderr_hat = std::sqrt(var / m);
    return GP2S_OK;
}

gp2s_status exact_logdet_solve(gp2s_ctx *c, const double *y_sorted_dev, double *logdet_hat, bool want_inverse)
{
    (void)want_inverse;
    const Assembled &A = c->A;
    const int64_t n = A.n;
    const size_t bytes = sizeof(double) * (size_t)n * (size_t)n;
    GP2S_TRY(ensure(c, c->dense, bytes + 64));
    double *Ad = c->dense.as<double>();
    GP2S_CUDA(c, cudaMemsetAsync(Ad, 0, bytes, c->stream));
    {
        unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n * 32, 256), 152 * 16);
        k_densify<<<gb, 256, 0, c->stream>>>(c->rowptr.as<int32_t>(), c->col.as<int32_t>(), c->val64.as<double>(), n, Ad);
        GP2S_LAUNCH(c);
    }
    GP2S_TRY(ensure(c, c->counters, 256));
    int *bad = reinterpret_cast<int *>(c->counters.as<char>() + 192);
    GP2S_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    for (int64_t kb = 0; kb < n; kb += NB) {
        k_potrf_diag<<<1, 256, 0, c->stream>>>(Ad, n, (int)kb, bad);
        GP2S_LAUNCH(c);
        int64_t rest = n - kb - NB;
        if (rest > 0) {
            k_trsm_panel<<<(unsigned)ceil_div(rest, 64), 64, 0, c->stream>>>(Ad, n, (int)kb);
            GP2S_LAUNCH(c);
            unsigned tiles = (unsigned)ceil_div(rest, 64);
            k_syrk<<<dim3(tiles, tiles), 256, 0, c->stream>>>(Ad, n, (int)kb);
            GP2S_LAUNCH(c);
        }
    }
    int hbad = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hbad) return set_err(c, GP2S_ENOTPD, "dense Cholesky: non-positive pivot");
    const int nb = 152 * 2;
    GP2S_TRY(ensure(c, c->gpart, sizeof(double) * (2 * nb + 8)));
    k_logdiag<<<nb, 256, 0, c->stream>>>(Ad, n, c->gpart.as<double>());
    GP2S_LAUNCH(c);
    double half = 0.0;
    GP2S_TRY(reduce_parts(c, c->gpart.as<double>(), nb, &half));
    *logdet_hat = 2.0 * half;
    c->have_exact = true;
    c->exact_lhat = *logdet_hat;

    if (y_sorted_dev) {
        // a = s * (Ah^{-1} (s * y)) by forward / backward substitution in vec64 slot 3
        GP2S_TRY(ensure(c, c->vec64, sizeof(double) * (size_t)n * 4 + 256));
        double *b64 = c->vec64.as<double>();
        double *xh = b64 + n, *a64 = b64 + 3 * n;
        GP2S_TRY(ensure(c, c->gpart, sizeof(double) * (2 * nb + 8)));
        const unsigned gbn = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
        // b64 = s * y ; xh = b64
        k_gp2s_mul<<<gbn, 256, 0, c->stream>>>(n, c->s64.as<double>(), y_sorted_dev, b64);
        GP2S_LAUNCH(c);
        GP2S_CUDA(c, cudaMemcpyAsync(xh, b64, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        const unsigned gbu = (unsigned)std::min<int64_t>(ceil_div(n * 32, 256), 152 * 8);
        for (int64_t kb = 0; kb < n; kb += NB) {
            k_trsv_diag<<<1, 32, 0, c->stream>>>(Ad, n, (int)kb, xh, 0);
            GP2S_LAUNCH(c);
            if (kb + NB < n) {
                k_trsv_update<<<gbu, 256, 0, c->stream>>>(Ad, n, (int)kb, xh, 0);
                GP2S_LAUNCH(c);
            }
        }
        for (int64_t kb = ((n - 1) / NB) * NB; kb >= 0; kb -= NB) {
            k_trsv_diag<<<1, 32, 0, c->stream>>>(Ad, n, (int)kb, xh, 1);
            GP2S_LAUNCH(c);
            if (kb > 0) {
                k_trsv_update<<<gbn, 256, 0, c->stream>>>(Ad, n, (int)kb, xh, 1);
                GP2S_LAUNCH(c);
            }
        }
        k_gp2s_mul<<<gbn, 256, 0, c->stream>>>(n, c->s64.as<double>(), xh, a64);
        GP2S_LAUNCH(c);
        c->have_solution = true;
    }
    return GP2S_OK;
}

}  // namespace gp2s

// =============================================================================================
// Allocation-free exact LML for small problems (gp2s_lml_exact_noalloc).
//
// For callers that may not allocate device memory (work issued during CUDA stream capture, or a
// device whose memory is owned by another allocator), every intermediate of this path lives in one
// fixed array compiled into the library.  The dense matrix is built pair by pair with the same
// exact FP64 support test and FP64 kernel value as the CSR path, then factored by the same blocked
// Cholesky kernels as the EXACT log-determinant above.
// =============================================================================================
namespace gp2s {

namespace {

constexpr int kNoAllocMaxN = GP2S_NOALLOC_MAX_N;
constexpr size_t kNoAllocA = (size_t)kNoAllocMaxN * kNoAllocMaxN;              // dense A / its factor
constexpr size_t kNoAllocX = kNoAllocA;                                          // y, then a = A^{-1} y
constexpr size_t kNoAllocB = kNoAllocX + kNoAllocMaxN;                           // bump table n x L
constexpr size_t kNoAllocFlag = kNoAllocB + (size_t)kNoAllocMaxN * kMaxBumps;    // pivot flag (int)
constexpr size_t kNoAllocDoubles = kNoAllocFlag + 32;

// The scratch array: every call on a device shares it (about 2.1 MB per device).
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {};   // device address of g_noalloc_scratch per device ordinal

template <int D>
__global__ void k_noalloc_bumps(const double *__restrict__ X, int n, KernelParams kp, double *__restrict__ B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int l = 0; l < kp.L; ++l) {
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double dk = X[(int64_t)i * D + k] - kp.centers[l * D + k];
            q = q + dk * dk;
        }
        double rho = kp.radii[l];
        double s = q / (rho * rho);
        double e = s < 1.0 ? exp(kp.beta * (1.0 - 1.0 / (1.0 - s))) : 0.0;
        B[(int64_t)i * kp.L + l] = kp.amps[l] * e;
    }
}

// Lower triangle of the dense A = K + sigma2 I (every entry written, so no clearing is needed).
template <int D>
__global__ void k_noalloc_dense(const double *__restrict__ X, int n, KernelParams kp, const double *__restrict__ B,
                                double *__restrict__ A)
{
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
        if (j > i) continue;
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double dk = __dsub_rn(X[(int64_t)i * D + k], X[(int64_t)j * D + k]);
            q = __dadd_rn(q, __dmul_rn(dk, dk));
        }
        double v = 0.0;
        if (i == j || q < kp.r * kp.r) {
            double S = 0.0;
            for (int l = 0; l < kp.L; ++l) S = fma(B[(int64_t)i * kp.L + l], B[(int64_t)j * kp.L + l], S);
            v = wendland<double>(kp.kind, D, sqrt(q) * kp.inv_r) * (S + kp.w0);
            if (i == j) v += kp.sigma2;
        }
        A[e] = v;
    }
}

// {LML, y^T a, log|A|} from the factor's diagonal and the solution; NaN when a pivot failed.
__global__ void k_noalloc_finish(const double *__restrict__ A, int n, const double *__restrict__ y,
                                 const double *__restrict__ a, const int *__restrict__ bad, double *__restrict__ out)
{
    __shared__ double sh[2][32];
    double ld = 0.0, qd = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        ld += log(A[(int64_t)i * n + i]);
        qd = fma(y[i], a[i], qd);
    }
    ld = warp_sum_d(ld);
    qd = warp_sum_d(qd);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = ld;
        sh[1][threadIdx.x >> 5] = qd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L2 = 0.0, Q = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { L2 += sh[0][w]; Q += sh[1][w]; }
        double logdet = 2.0 * L2;
        double lml = -0.5 * Q - 0.5 * logdet - 0.5 * (double)n * log(2.0 * 3.141592653589793);
        if (*bad) { lml = nan(""); Q = nan(""); logdet = nan(""); }
        out[0] = lml;
        out[1] = Q;
        out[2] = logdet;
    }
}

// Device address of the scratch array on the current device, looked up once per device.
gp2s_status noalloc_scratch(double **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return GP2S_ECUDA; }
    if (dev < 0 || dev >= 64) return GP2S_ECUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { cudaGetLastError(); return GP2S_ECUDA; }
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *ptr = g_noalloc_ptr[dev];
    return GP2S_OK;
}

template <int D>
void launch_noalloc_build(const double *X, int n, const KernelParams &kp, double *B, double *A, cudaStream_t s)
{
    k_noalloc_bumps<D><<<(n + 127) / 128, 128, 0, s>>>(X, n, kp, B);
    const int64_t tot = (int64_t)n * n;
    unsigned gb = (unsigned)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096);
    k_noalloc_dense<D><<<gb, 256, 0, s>>>(X, n, kp, B, A);
}

}  // namespace

gp2s_status validate_hyper(gp2s_ctx *c, const gp2s_hyper *h);   // assemble.cu
KernelParams make_kernel_params(const gp2s_hyper *h);             // assemble.cu

}  // namespace gp2s

extern "C" gp2s_status gp2s_lml_exact_noalloc(int64_t n, const double *X_dev, const double *y_dev,
                                              const gp2s_hyper *hyper, double *out_dev, void *cuda_stream)
{
    using namespace gp2s;
    if (n < 1 || n > kNoAllocMaxN) return GP2S_EINVAL;
    if (!X_dev || !y_dev || !out_dev) return GP2S_EINVAL;
    if (validate_hyper(nullptr, hyper) != GP2S_OK) return GP2S_EINVAL;
    if (hyper->family != GP2S_KERNEL_PRODUCT) return GP2S_EINVAL;   // the product kernel only
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    // the scratch address is per device: a stream of another device would get this device's
    // address, so such a stream is refused (the legacy and per-thread default streams follow the
    // current device).  The stream's device is not asked for while the stream is being captured,
    // where that query invalidates the capture: a capture records on the stream's own device, and
    // the caller answers for the device being current.
    if (s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
            cudaGetLastError();
            return GP2S_ECUDA;
        }
        if (cs == cudaStreamCaptureStatusNone) {
            int cur = 0, sdev = 0;
            if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
                cudaGetLastError();
                return GP2S_ECUDA;
            }
            if (sdev != cur) return GP2S_EINVAL;
        }
    }
    double *base = nullptr;
    gp2s_status st = noalloc_scratch(&base);
    if (st != GP2S_OK) return st;
    const int nn = (int)n;
    const KernelParams kp = make_kernel_params(hyper);
    double *A = base;                          // nn x nn, leading dimension nn
    double *x = base + kNoAllocX;
    double *B = base + kNoAllocB;
    int *bad = reinterpret_cast<int *>(base + kNoAllocFlag);
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) { cudaGetLastError(); return GP2S_ECUDA; }
    if (cudaMemcpyAsync(x, y_dev, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return GP2S_ECUDA;
    }
    switch (hyper->d) {
    case 1: launch_noalloc_build<1>(X_dev, nn, kp, B, A, s); break;
    case 2: launch_noalloc_build<2>(X_dev, nn, kp, B, A, s); break;
    case 3: launch_noalloc_build<3>(X_dev, nn, kp, B, A, s); break;
    default: launch_noalloc_build<4>(X_dev, nn, kp, B, A, s); break;
    }
    // blocked Cholesky A = L L^T (lower triangle, in place)
    for (int kb = 0; kb < nn; kb += NB) {
        k_potrf_diag<<<1, 256, 0, s>>>(A, nn, kb, bad);
        int rest = nn - kb - NB;
        if (rest > 0) {
            k_trsm_panel<<<(rest + 63) / 64, 64, 0, s>>>(A, nn, kb);
            unsigned tiles = (unsigned)((rest + 63) / 64);
            k_syrk<<<dim3(tiles, tiles), 256, 0, s>>>(A, nn, kb);
        }
    }
    // a = L^{-T} L^{-1} y, in place in x
    for (int kb = 0; kb < nn; kb += NB) {
        k_trsv_diag<<<1, 32, 0, s>>>(A, nn, kb, x, 0);
        if (kb + NB < nn) k_trsv_update<<<(unsigned)((nn * 32 + 255) / 256), 256, 0, s>>>(A, nn, kb, x, 0);
    }
    for (int kb = ((nn - 1) / NB) * NB; kb >= 0; kb -= NB) {
        k_trsv_diag<<<1, 32, 0, s>>>(A, nn, kb, x, 1);
        if (kb > 0) k_trsv_update<<<(unsigned)((kb + 255) / 256), 256, 0, s>>>(A, nn, kb, x, 1);
    }
    k_noalloc_finish<<<1, 256, 0, s>>>(A, nn, y_dev, x, bad, out_dev);
    if (cudaGetLastError() != cudaSuccess) return GP2S_ECUDA;
    return GP2S_OK;
}
