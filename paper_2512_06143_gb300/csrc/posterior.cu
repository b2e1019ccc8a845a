// posterior.cu -- the GP posterior at test points (Eq. 2, Sec. 3) on the assembled training
// problem, with zero prior mean and A = K + sigma^2 I in place of the paper's K:
//     mean(x*) = k(X, x*)^T a,                      a = A^{-1} y (kept from the last solve),
//     var(x*)  = k(x*, x*) - k(X, x*)^T A^{-1} k(X, x*)   (latent f*, without the noise term).
// The cross-covariance k(X, x*) has the training points within r of x* as its only nonzeros; they
// lie in the 3^d cells around x*'s cell of the training grid, found by binary search in the sorted
// cell-key table the assembly left behind.  Every (x*, x_j) pair there takes the same FP64 support
// test and kernel value as the training matrix (no noise term: x* is a new location).
//
// The variance needs one solve per test point: batches of up to 64 test points become the columns
// of one multi-RHS (P)CG on the Jacobi-scaled matrix, Ah v = s k(X, x*) with s = D^{-1/2}.  From
// the approximate solution v (taken as exact input to FP64 arithmetic),
//     k^T A^{-1} k  ~=  2 (s k)^T v - v^T Ah v        (Ah with its FP64 values),
// the Galerkin (energy) form: its error is -e^T Ah e for the solution error e, second order in the
// solve's accuracy whatever the precision the solve ran in.
#include <cmath>
#include <cstring>
#include <vector>

#include "gp2s_geometry.cuh"
#include "gp2s_kernel_math.cuh"
#include "gp2s_internal.cuh"

namespace gp2s {

namespace {

constexpr int kPostThreads = 256;
constexpr int kPostBatch = 64;   // test points per variance solve (the probe group's width)

struct PostArgs {
    const double *Xs;             // ns x d, caller order
    const double *Bs;             // ns x L bump values of the test points (FP64); Wendland convolution:
                                  // ns x 5, [s, lambda_1..4]
    int64_t ns;
    const double4_16a *X64;       // training points, sorted order
    const double *B64;            // n x L
    const double *s64;            // n, D^{-1/2}
    const int32_t *cell_start;    // ncells + 1
    const uint64_t *cell_key;     // ncells
    int64_t ncells;
    const double4_16a *Lam;       // Wendland convolution: training lambda (sorted order)
    const double *Sig;            // Wendland convolution: training s
    int sw;                       // stencil half-width in cells (1; more when a test point's length
                                  // scale exceeds every training point's)
};

// The Wendland convolution kernel's fields at a point (the assembly's arithmetic, Eq. 6 reading):
// psi_l = (1 - |x - c_l|^2 / rho_l^2)^3, s = w0 + sum a_l psi_l, lambda_k = ell_k^2 + sum G_lk psi_l.
template <int D>
__device__ __forceinline__ void post_wc_fields(const double *x, const KernelParams &kp, double &sig, double *lam)
{
    double sg = 0.0, acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.0;
    for (int l = 0; l < kp.L; ++l) {
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double dk = __dsub_rn(x[k], kp.centers[l * D + k]);
            q = __dadd_rn(q, __dmul_rn(dk, dk));
        }
        const double rho = kp.radii[l];
        const double s = __ddiv_rn(q, __dmul_rn(rho, rho));
        double ps = 0.0;
        if (s < 1.0) {
            const double u = __dsub_rn(1.0, s);
            ps = __dmul_rn(__dmul_rn(u, u), u);
        }
        sg = __dadd_rn(sg, __dmul_rn(kp.amps[l], ps));
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = __dadd_rn(acc[k], __dmul_rn(kp.G[l * D + k], ps));
    }
    sig = __dadd_rn(kp.w0, sg);
#pragma unroll
    for (int k = 0; k < D; ++k) lam[k] = __dadd_rn(__dmul_rn(kp.ell[k], kp.ell[k]), acc[k]);
}

__device__ __forceinline__ int64_t lower_bound_key(const uint64_t *__restrict__ keys, int64_t n, uint64_t k)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Calls fn(j, k(x*, x_j)) for every training point j (sorted index) with d2(x*, x_j) < r^2; the
// lanes of the calling warp split each cell's points.
template <int D, class Fn>
__device__ __forceinline__ void for_each_neighbour(const PostArgs &a, const GridParams &g, const KernelParams &kp,
                                                   int64_t t, Fn &&fn)
{
    const int lane = threadIdx.x & 31;
    double x[D];
    int64_t cc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        x[k] = a.Xs[t * D + k];
        double y = __dmul_rn(__dsub_rn(x[k], g.origin[k]), g.inv_h);   // cell units, as the training keys
        // far outside the grid no cell is adjacent: clamp before the integer conversion
        y = fmin(fmax(y, -4.0 - a.sw), (double)g.dims[k] + 4.0 + a.sw);
        cc[k] = (int64_t)floor(y);
    }
    const double r2 = kp.r * kp.r;
    const int L = kp.L;
    const int span = 2 * a.sw + 1;
    int ncomb = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) ncomb *= span;
    for (int o = 0; o < ncomb; ++o) {
        int64_t nc[D];
        bool inside = true;
        int rest = o;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            nc[k] = cc[k] + (rest % span) - a.sw;
            rest /= span;
            inside = inside && nc[k] >= 0 && nc[k] < g.dims[k];
        }
        if (!inside) continue;
        const uint64_t key = coarse_key<D>(nc, g);
        const int64_t f = lower_bound_key(a.cell_key, a.ncells, key);
        if (f >= a.ncells || a.cell_key[f] != key) continue;
        const int p1 = a.cell_start[f + 1];
        for (int p = a.cell_start[f] + lane; p < p1; p += kWarp) {
            const double4_16a xv = a.X64[p];
            const double xj[4] = {xv.x, xv.y, xv.z, xv.w};
            double q = 0.0;
            if (kp.family == 1) {
                // Q = sum_k D_k D_k / ((lambda*_k + lambda_jk) * 0.5), support Q < r^2 (Eq. 6)
                const double4_16a lv = a.Lam[p];
                const double lj[4] = {lv.x, lv.y, lv.z, lv.w};
                const double *ls = a.Bs + t * 5 + 1;
                double pref = 1.0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const double dk = __dsub_rn(x[k], xj[k]);
                    const double m = __dmul_rn(__dadd_rn(ls[k], lj[k]), 0.5);
                    q = __dadd_rn(q, __ddiv_rn(__dmul_rn(dk, dk), m));
                    pref = pref * (sqrt(sqrt(ls[k] * lj[k])) / sqrt(m));
                }
                if (!(q < r2)) continue;
                fn(p, a.Bs[t * 5] * a.Sig[p] * pref * wendland<double>(kp.kind, D, sqrt(q) * kp.inv_r));
                continue;
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double dk = __dsub_rn(x[k], xj[k]);
                q = __dadd_rn(q, __dmul_rn(dk, dk));
            }
            if (!(q < r2)) continue;
            const double phi = wendland<double>(kp.kind, D, sqrt(q) * kp.inv_r);
            double S = 0.0;
            for (int l = 0; l < L; ++l) S = fma(a.Bs[t * L + l], a.B64[(int64_t)p * L + l], S);
            fn(p, phi * (S + kp.w0));
        }
    }
}

__device__ __forceinline__ double warp_sum_post(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// b_l(x*) of Eq. 7 for every test point (FP64) and the prior variance k(x*, x*) = phi(0)
// (sum_l b_l(x*)^2 + w0) = sum_l b_l(x*)^2 + w0.
template <int D>
__global__ void k_post_bumps(const double *__restrict__ Xs, int64_t ns, KernelParams kp, double *__restrict__ Bs,
                             double *__restrict__ kss)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += (int64_t)gridDim.x * blockDim.x) {
        if (kp.family == 1) {
            double x[D], sig, lam[D];
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = Xs[t * D + k];
            post_wc_fields<D>(x, kp, sig, lam);
            Bs[t * 5] = sig;
            for (int k = 0; k < 4; ++k) Bs[t * 5 + 1 + k] = k < D ? lam[k < D ? k : 0] : 1.0;
            kss[t] = sig * sig;   // Q = 0 and the prefactor is 1 at zero distance
            continue;
        }
        double S = 0.0;
        for (int l = 0; l < kp.L; ++l) {
            double q = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double dk = Xs[t * D + k] - kp.centers[l * D + k];
                q = q + dk * dk;
            }
            const double rho = kp.radii[l];
            const double s = q / (rho * rho);
            const double b = s < 1.0 ? kp.amps[l] * exp(kp.beta * (1.0 - 1.0 / (1.0 - s))) : 0.0;
            Bs[t * kp.L + l] = b;
            S = S + b * b;
        }
        kss[t] = S + kp.w0;
    }
}

// mean(x*_t) = sum_j k(x*_t, x_j) a_j, one warp per test point (FP64); counts the nonzeros.
template <int D>
__global__ void __launch_bounds__(kPostThreads)
k_post_mean(PostArgs a, GridParams g, KernelParams kp, const double *__restrict__ asol, double *__restrict__ mean,
            unsigned long long *__restrict__ nnz)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cnt = 0;
    for (int64_t t = w0; t < a.ns; t += nw) {
        double acc = 0.0;
        for_each_neighbour<D>(a, g, kp, t, [&](int p, double v) {
            acc = fma(v, asol[p], acc);
            ++cnt;
        });
        acc = warp_sum_post(acc);
        if (lane == 0) mean[t] = acc;
    }
    atomicAdd(nnz, cnt);
}

// Right-hand sides of one variance batch: column c (test point t0 + c) gets s_j k(x_j, x*) in row j
// (the block was zeroed; each (j, c) is written once).
template <int D, class T>
__global__ void __launch_bounds__(kPostThreads)
k_post_rhs(PostArgs a, GridParams g, KernelParams kp, int64_t t0, int nb, int m, T *__restrict__ rz)
{
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = w0; c < nb; c += nw)
        for_each_neighbour<D>(a, g, kp, t0 + c, [&](int p, double v) { rz[(int64_t)p * m + c] = (T)(a.s64[p] * v); });
}

// Column quadratic forms x_c^T Ah x_c of the n x m solution block in FP64 (FP64 values, the
// stored x taken as exact): one warp per row, lane l owns columns l, l + 32 (m <= 64); per-CTA
// partials in part[c * gridDim.x + block].
template <class T>
__global__ void __launch_bounds__(kPostThreads)
k_post_xax(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const double *__restrict__ val,
           int64_t n, int m, const T *__restrict__ x, double *__restrict__ part)
{
    __shared__ double sh[kPostThreads / 32][kPostBatch];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc0 = 0.0, acc1 = 0.0;
    const bool c1 = lane + 32 < m;
    for (int64_t i = w0; i < n; i += nw) {
        double s0 = 0.0, s1 = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const int j = col[p];
            const double v = val[p];
            s0 = fma(v, (double)x[(int64_t)j * m + lane], s0);
            if (c1) s1 = fma(v, (double)x[(int64_t)j * m + lane + 32], s1);
        }
        acc0 = fma((double)x[i * m + lane], s0, acc0);
        if (c1) acc1 = fma((double)x[i * m + lane + 32], s1, acc1);
    }
    sh[wid][lane] = acc0;
    if (m > 32) sh[wid][lane + 32] = acc1;
    __syncthreads();
    if ((int)threadIdx.x < m) {
        double t = 0.0;
        for (int w = 0; w < kPostThreads / 32; ++w) t += sh[w][threadIdx.x];
        part[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// var(x*_t) = k(x*, x*) - (2 (s k)^T x - x^T Ah x) for the batch's test points, one warp each.
template <int D, class T>
__global__ void __launch_bounds__(kPostThreads)
k_post_var(PostArgs a, GridParams g, KernelParams kp, int64_t t0, int nb, int m, const T *__restrict__ xz,
           const double *__restrict__ part, int nblk, const double *__restrict__ kss, double *__restrict__ var)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = w0; c < nb; c += nw) {
        double acc = 0.0;
        for_each_neighbour<D>(a, g, kp, t0 + c, [&](int p, double v) {
            acc = fma(a.s64[p] * v, (double)xz[(int64_t)p * m + c], acc);
        });
        acc = warp_sum_post(acc);
        if (lane == 0) {
            double xax = 0.0;
            for (int b = 0; b < nblk; ++b) xax += part[(int64_t)c * nblk + b];
            var[t0 + c] = kss[t0 + c] - (2.0 * acc - xax);
        }
    }
}

template <int D>
gp2s_status posterior_d(gp2s_ctx *c, const PostArgs &pa, double *mean_dev, double *var_dev, double *kss,
                        gp2s_posterior_info *info)
{
    const Assembled &A = c->A;
    const int64_t n = A.n, ns = pa.ns;
    const bool mixed = A.precision == GP2S_PREC_MIXED;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c->post_cnt.p);
    GP2S_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), c->stream));
    const unsigned gw = (unsigned)std::min<int64_t>(ceil_div(ns * kWarp, kPostThreads), (int64_t)c->num_sms * 16);
    cudaEvent_t e0, e1, e2;
    GP2S_CUDA(c, cudaEventCreate(&e0));
    GP2S_CUDA(c, cudaEventCreate(&e1));
    GP2S_CUDA(c, cudaEventCreate(&e2));
    struct G { cudaEvent_t a, b, d; ~G() { cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(d); } } guard{e0, e1, e2};
    GP2S_CUDA(c, cudaEventRecord(e0, c->stream));
    k_post_mean<D><<<gw, kPostThreads, 0, c->stream>>>(pa, A.gp, A.kp, c->vec64.as<double>() + 3 * n, mean_dev, cnt);
    GP2S_LAUNCH(c);
    GP2S_CUDA(c, cudaEventRecord(e1, c->stream));
    int batches = 0, iters_max = 0;
    if (var_dev) {
        const int nblk = (int)std::min<int64_t>(ceil_div(n, kPostThreads / kPostBatch), (int64_t)c->num_sms * 4);
        GP2S_TRY(ensure(c, c->post_part, sizeof(double) * (size_t)kPostBatch * nblk));
        const size_t es = mixed ? sizeof(float) : sizeof(double);
        for (int64_t t0 = 0; t0 < ns; t0 += kPostBatch) {
            const int nb = (int)std::min<int64_t>(kPostBatch, ns - t0);
            const int m = nb <= 32 ? 32 : 64;   // the probe group's width: zero columns stay idle
            void *rz = nullptr, *xz = nullptr;
            GP2S_TRY(krylov_columns_buffers(c, m, &rz, &xz));
            GP2S_CUDA(c, cudaMemsetAsync(rz, 0, es * (size_t)n * m, c->stream));
            const unsigned gb = (unsigned)std::max<int64_t>(1, ceil_div((int64_t)nb * kWarp, kPostThreads));
            if (mixed) k_post_rhs<D, float><<<gb, kPostThreads, 0, c->stream>>>(pa, A.gp, A.kp, t0, nb, m, (float *)rz);
            else k_post_rhs<D, double><<<gb, kPostThreads, 0, c->stream>>>(pa, A.gp, A.kp, t0, nb, m, (double *)rz);
            GP2S_LAUNCH(c);
            int it = 0;
            GP2S_TRY(krylov_columns_solve(c, m, A.opts.tol_probe, &it));
            iters_max = std::max(iters_max, it);
            ++batches;
            const int nbk = (int)std::min<int64_t>(ceil_div(n, kPostThreads / 32), nblk);
            const int32_t *rp = c->rowptr.as<int32_t>(), *cl = c->col.as<int32_t>();
            if (mixed)
                k_post_xax<float><<<nbk, kPostThreads, 0, c->stream>>>(rp, cl, c->val64.as<double>(), n, m,
                                                                       (const float *)xz, c->post_part.as<double>());
            else
                k_post_xax<double><<<nbk, kPostThreads, 0, c->stream>>>(rp, cl, c->val64.as<double>(), n, m,
                                                                        (const double *)xz, c->post_part.as<double>());
            GP2S_LAUNCH(c);
            if (mixed)
                k_post_var<D, float><<<gb, kPostThreads, 0, c->stream>>>(pa, A.gp, A.kp, t0, nb, m, (const float *)xz,
                                                                         c->post_part.as<double>(), nbk, kss, var_dev);
            else
                k_post_var<D, double><<<gb, kPostThreads, 0, c->stream>>>(pa, A.gp, A.kp, t0, nb, m, (const double *)xz,
                                                                          c->post_part.as<double>(), nbk, kss, var_dev);
            GP2S_LAUNCH(c);
        }
    }
    GP2S_CUDA(c, cudaEventRecord(e2, c->stream));
    unsigned long long hcnt = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&hcnt, cnt, sizeof(hcnt), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (info) {
        info->n_test = ns;
        info->cross_entries = (int64_t)hcnt;
        info->batches = batches;
        info->iters_max = iters_max;
        cudaEventElapsedTime(&info->ms_mean, e0, e1);
        cudaEventElapsedTime(&info->ms_var, e1, e2);
    }
    return GP2S_OK;
}

bool is_device_ptr_post(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

gp2s_status posterior(gp2s_ctx *c, int64_t ns, const double *Xs, double *mean, double *var,
                      gp2s_posterior_info *info)
{
    const Assembled &A = c->A;
    if (!A.valid || !c->have_solution)
        return set_err(c, GP2S_ENOTREADY, "gp2s_posterior needs a solved problem (gp2s_lml, gp2s_lml_grad or gp2s_solve)");
    if (ns < 0) return set_err(c, GP2S_EINVAL, "n_test must be >= 0");
    if (A.kp.family == 2) return set_err(c, GP2S_EINVAL, "gp2s_posterior takes the product and convolution kernels");
    if (ns == 0) {
        if (info) std::memset(info, 0, sizeof(*info));
        return GP2S_OK;
    }
    if (!Xs || !mean) return set_err(c, GP2S_EINVAL, "Xtest / mean is NULL");
    const int d = A.d, L = A.L;
    // inputs: test points on the device; outputs: device buffers, copied out when the caller's are host
    const double *xs_dev = Xs;
    if (!is_device_ptr_post(Xs)) {
        GP2S_TRY(ensure(c, c->post_X, sizeof(double) * (size_t)ns * d));
        GP2S_CUDA(c, cudaMemcpyAsync(c->post_X.p, Xs, sizeof(double) * (size_t)ns * d, cudaMemcpyHostToDevice, c->stream));
        xs_dev = c->post_X.as<double>();
    }
    const int bw = A.kp.family == 1 ? 5 : (L > 0 ? L : 1);   // per-test-point values
    GP2S_TRY(ensure(c, c->post_B, sizeof(double) * (size_t)ns * bw + sizeof(double) * (size_t)ns * 3));
    double *Bs = c->post_B.as<double>();
    double *kss = Bs + (size_t)ns * bw;
    double *mean_buf = kss + ns, *var_buf = mean_buf + ns;
    const bool mean_dev = is_device_ptr_post(mean);
    const bool var_dev = var && is_device_ptr_post(var);
    double *mean_out = mean_dev ? mean : mean_buf;
    double *var_out = var ? (var_dev ? var : var_buf) : nullptr;
    GP2S_TRY(ensure(c, c->post_cnt, 64));
    {
        const unsigned gb = (unsigned)std::min<int64_t>(ceil_div(ns, 256), (int64_t)c->num_sms * 8);
        switch (d) {
        case 1: k_post_bumps<1><<<gb, 256, 0, c->stream>>>(xs_dev, ns, A.kp, Bs, kss); break;
        case 2: k_post_bumps<2><<<gb, 256, 0, c->stream>>>(xs_dev, ns, A.kp, Bs, kss); break;
        case 3: k_post_bumps<3><<<gb, 256, 0, c->stream>>>(xs_dev, ns, A.kp, Bs, kss); break;
        default: k_post_bumps<4><<<gb, 256, 0, c->stream>>>(xs_dev, ns, A.kp, Bs, kss); break;
        }
        GP2S_LAUNCH(c);
    }
    PostArgs pa;
    pa.Xs = xs_dev;
    pa.Bs = Bs;
    pa.ns = ns;
    pa.X64 = c->Xs64.as<double4_16a>();
    pa.B64 = c->B64.as<double>();
    pa.s64 = c->s64.as<double>();
    pa.cell_start = c->cell_start.as<int32_t>();
    pa.cell_key = cell_keys_ptr(c, A.ncells);
    pa.ncells = A.ncells;
    pa.Lam = c->wc_lam.as<double4_16a>();
    pa.Sig = c->wc_sig.as<double>();
    pa.sw = 1;
    if (A.kp.family == 1) {
        // a test point reaches |D_k| < r sqrt((lambda*_k + lambda_jk) / 2); cells have edge
        // >= r sqrt(max training lambda): widen the stencil if a test point's field is larger
        std::vector<double> hb((size_t)ns * 5);
        GP2S_CUDA(c, cudaMemcpyAsync(hb.data(), Bs, sizeof(double) * (size_t)ns * 5, cudaMemcpyDeviceToHost, c->stream));
        GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
        double lmax = 0.0;
        for (int64_t t = 0; t < ns; ++t)
            for (int k = 0; k < d; ++k) lmax = std::fmax(lmax, hb[(size_t)t * 5 + 1 + k]);
        const double reach = std::sqrt(0.5 * (lmax + A.wc_lmax)) * A.kp.r;
        pa.sw = std::max(1, (int)std::ceil(reach / A.gp.h * (1.0 + 1e-12)));
        if (pa.sw > 4) return set_err(c, GP2S_EINVAL, "test points' length scales exceed the training grid's reach by more than 4 cells");
    }
    switch (d) {
    case 1: GP2S_TRY(posterior_d<1>(c, pa, mean_out, var_out, kss, info)); break;
    case 2: GP2S_TRY(posterior_d<2>(c, pa, mean_out, var_out, kss, info)); break;
    case 3: GP2S_TRY(posterior_d<3>(c, pa, mean_out, var_out, kss, info)); break;
    default: GP2S_TRY(posterior_d<4>(c, pa, mean_out, var_out, kss, info)); break;
    }
    if (!mean_dev) GP2S_CUDA(c, cudaMemcpyAsync(mean, mean_out, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->stream));
    if (var && !var_dev) GP2S_CUDA(c, cudaMemcpyAsync(var, var_out, sizeof(double) * ns, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    return GP2S_OK;
}

}  // namespace gp2s
