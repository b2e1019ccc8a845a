// minres.cu -- MINRES (Paige & Saunders 1975), the solver the paper uses for K^{-1} y (App. B.6),
// in FP64 on the Jacobi-scaled matrix Ah = D^{-1/2} A D^{-1/2}: the Lanczos process on the
// right-hand side with the tridiagonal's QR factorisation by Givens rotations, which minimises
// |b - Ah x| over the Krylov space at every step.  With beta_1 v_1 = b and G_k = [[c_k, s_k],
// [-s_k, c_k]]:
//     u = Ah v_k - beta_k v_{k-1},  alpha_k = v_k^T u,  u -= alpha_k v_k,  beta_{k+1} = |u|,
//     eps_k = s_{k-2} beta_k,  dbar_k = c_{k-2} beta_k,
//     delta_k = c_{k-1} dbar_k + s_{k-1} alpha_k,  gbar_k = -s_{k-1} dbar_k + c_{k-1} alpha_k,
//     gamma_k = |(gbar_k, beta_{k+1})|,  c_k = gbar_k / gamma_k,  s_k = beta_{k+1} / gamma_k,
//     tau_k = c_k phibar_{k-1},  phibar_k = -s_k phibar_{k-1},
//     w_k = (v_k - delta_k w_{k-1} - eps_k w_{k-2}) / gamma_k,  x += tau_k w_k,
// and |b - Ah x_k| = |phibar_k|.  Each step is five kernels (SpMV + alpha partials, alpha, the
// orthogonalisation + |u|^2 partials, the rotations, the vector updates); the scalars live in
// device memory, so the host only reads the stop flag every few steps.
#include <cmath>

#include "gp2s_internal.cuh"

namespace gp2s {

namespace {

constexpr int kMrThreads = 256;
constexpr int kMrParts = 152 * 4;

struct MrScal {
    double beta, beta1, phibar, c1, s1, c2, s2;   // beta_k, |b|, phibar, rotations k-1 and k-2
    double alpha, eps, delta, gamma, tau, beta_next, tol;
    int active;   // still iterating
    int upd;      // this step updates x and the directions
    int steps;
    int pad;
};

__device__ __forceinline__ double mr_warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of one double per thread into part[blockIdx.x] (fixed order).
__device__ __forceinline__ void mr_block_part(double v, double *__restrict__ part)
{
    __shared__ double sh[kMrThreads / 32];
    v = mr_warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kMrThreads / 32; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__device__ __forceinline__ double mr_sum_parts(const double *__restrict__ part, int cnt)
{
    double s = 0.0;
    for (int b = 0; b < cnt; ++b) s += part[b];
    return s;
}

// |b|^2 partials, then the start: v = b / beta_1, v_prev = w_{k-1} = w_{k-2} = x = 0.
__global__ void __launch_bounds__(kMrThreads) k_mr_norm(const double *__restrict__ b, int64_t n, double *__restrict__ part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(b[i], b[i], acc);
    mr_block_part(acc, part);
}

__global__ void k_mr_init_scal(const double *__restrict__ part, int nparts, double tol, MrScal *__restrict__ sc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double b1 = sqrt(mr_sum_parts(part, nparts));
    sc->beta = b1;
    sc->beta1 = b1;
    sc->phibar = b1;
    sc->c1 = sc->c2 = 1.0;
    sc->s1 = sc->s2 = 0.0;
    sc->tol = tol;
    sc->active = b1 > 0.0 ? 1 : 0;
    sc->upd = 0;
    sc->steps = 0;
}

__global__ void __launch_bounds__(kMrThreads)
k_mr_init_vec(const double *__restrict__ b, int64_t n, const MrScal *__restrict__ sc, double *__restrict__ v,
              double *__restrict__ vprev, double *__restrict__ w1, double *__restrict__ w2, double *__restrict__ x)
{
    const double inv = sc->beta1 > 0.0 ? 1.0 / sc->beta1 : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        v[i] = b[i] * inv;
        vprev[i] = 0.0;
        w1[i] = 0.0;
        w2[i] = 0.0;
        x[i] = 0.0;
    }
}

// u = Ah v - beta_k v_prev (warp per row, FP64 values), partials of v^T u.
__global__ void __launch_bounds__(kMrThreads)
k_mr_spmv(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const double *__restrict__ val,
          int64_t n, const double *__restrict__ v, const double *__restrict__ vprev, const MrScal *__restrict__ sc,
          double *__restrict__ u, double *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double beta = sc->beta;
    double acc = 0.0;
    for (int64_t i = w0; i < n; i += nw) {
        double s = 0.0;
        for (int p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) s = fma(val[p], v[col[p]], s);
        s = mr_warp_sum(s);
        if (lane == 0) {
            const double ui = s - beta * vprev[i];
            u[i] = ui;
            acc = fma(v[i], ui, acc);
        }
    }
    mr_block_part(acc, part);
}

__global__ void k_mr_alpha(const double *__restrict__ part, int nparts, MrScal *__restrict__ sc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) sc->alpha = mr_sum_parts(part, nparts);
}

// u -= alpha v, partials of |u|^2.
__global__ void __launch_bounds__(kMrThreads)
k_mr_orth(int64_t n, const double *__restrict__ v, const MrScal *__restrict__ sc, double *__restrict__ u,
          double *__restrict__ part)
{
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ui = u[i] - alpha * v[i];
        u[i] = ui;
        acc = fma(ui, ui, acc);
    }
    mr_block_part(acc, part);
}

// The rotations of step k and the stop test (|phibar_k| <= tol beta_1, or an exhausted Krylov space).
__global__ void k_mr_givens(const double *__restrict__ part, int nparts, MrScal *__restrict__ sc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!sc->active) {
        sc->upd = 0;
        return;
    }
    const double bn = sqrt(mr_sum_parts(part, nparts));
    const double beta = sc->beta, alpha = sc->alpha;
    const double eps = sc->s2 * beta;
    const double dbar = sc->c2 * beta;
    const double delta = sc->c1 * dbar + sc->s1 * alpha;
    const double gbar = -sc->s1 * dbar + sc->c1 * alpha;
    const double gamma = hypot(gbar, bn);
    if (!(gamma > 0.0)) {   // singular tridiagonal: no further progress is possible
        sc->upd = 0;
        sc->active = 0;
        return;
    }
    const double ck = gbar / gamma, sk = bn / gamma;
    sc->eps = eps;
    sc->delta = delta;
    sc->gamma = gamma;
    sc->tau = ck * sc->phibar;
    sc->phibar = -sk * sc->phibar;
    sc->beta_next = bn;
    sc->c2 = sc->c1;
    sc->s2 = sc->s1;
    sc->c1 = ck;
    sc->s1 = sk;
    sc->upd = 1;
    sc->steps += 1;
    if (fabs(sc->phibar) <= sc->tol * sc->beta1 || !(bn > 0.0)) sc->active = 0;
}

// w_k = (v_k - delta w_{k-1} - eps w_{k-2}) / gamma (written over w_{k-2}), x += tau w_k,
// v_{k+1} = u / beta_{k+1} (written over u); beta_k <- beta_{k+1}.
__global__ void __launch_bounds__(kMrThreads)
k_mr_update(int64_t n, const double *__restrict__ v, double *__restrict__ u, const double *__restrict__ wkm1,
            double *__restrict__ wkm2, double *__restrict__ x, MrScal *__restrict__ sc)
{
    if (!sc->upd) return;
    const double delta = sc->delta, eps = sc->eps, ig = 1.0 / sc->gamma, tau = sc->tau;
    const double bn = sc->beta_next;
    const double ib = bn > 0.0 ? 1.0 / bn : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double w = (v[i] - delta * wkm1[i] - eps * wkm2[i]) * ig;
        wkm2[i] = w;
        x[i] = fma(tau, w, x[i]);
        u[i] = u[i] * ib;
    }
}

__global__ void k_mr_shift_beta(MrScal *__restrict__ sc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && sc->upd) sc->beta = sc->beta_next;
}

}  // namespace

// MINRES on Ah for the right-hand side b (n FP64, device, sorted order) into x; stops when
// |b - Ah x| <= tol |b| (the recurrence's residual norm) or after maxit steps.
gp2s_status minres_solve(gp2s_ctx *c, const double *b, double *x, double tol, int maxit, int *steps)
{
    const Assembled &A = c->A;
    const int64_t n = A.n;
    GP2S_TRY(ensure(c, c->mr_vec, sizeof(double) * (size_t)n * 5 + sizeof(MrScal) + sizeof(double) * 2 * kMrParts + 512));
    double *base = c->mr_vec.as<double>();
    double *vb[5] = {base, base + n, base + 2 * n, base + 3 * n, base + 4 * n};
    MrScal *sc = reinterpret_cast<MrScal *>(base + 5 * n);
    double *part = reinterpret_cast<double *>(sc + 1);
    double *part2 = part + kMrParts;
    const unsigned gv = (unsigned)std::min<int64_t>(ceil_div(n, kMrThreads), kMrParts);
    const unsigned gs = (unsigned)std::min<int64_t>(ceil_div(n * 32, kMrThreads), kMrParts);
    // roles: v_prev, v, u (next v), w_{k-1}, w_{k-2} (next w)
    int vp = 0, vc = 1, vu = 2, w1 = 3, w2 = 4;
    k_mr_norm<<<gv, kMrThreads, 0, c->stream>>>(b, n, part);
    GP2S_LAUNCH(c);
    k_mr_init_scal<<<1, 32, 0, c->stream>>>(part, (int)gv, tol, sc);
    GP2S_LAUNCH(c);
    k_mr_init_vec<<<gv, kMrThreads, 0, c->stream>>>(b, n, sc, vb[vc], vb[vp], vb[w1], vb[w2], x);
    GP2S_LAUNCH(c);
    GP2S_TRY(ensure_host(c, c->hbuf, 4096));
    int *hflag = reinterpret_cast<int *>(c->hbuf.p);
    const int check_every = 8;
    int it = 0;
    while (it < maxit) {
        const int len = std::min(check_every, maxit - it);
        for (int r = 0; r < len; ++r, ++it) {
            k_mr_spmv<<<gs, kMrThreads, 0, c->stream>>>(c->rowptr.as<int32_t>(), c->col.as<int32_t>(),
                                                         c->val64.as<double>(), n, vb[vc], vb[vp], sc, vb[vu], part);
            GP2S_LAUNCH(c);
            k_mr_alpha<<<1, 32, 0, c->stream>>>(part, (int)gs, sc);
            GP2S_LAUNCH(c);
            k_mr_orth<<<gv, kMrThreads, 0, c->stream>>>(n, vb[vc], sc, vb[vu], part2);
            GP2S_LAUNCH(c);
            k_mr_givens<<<1, 32, 0, c->stream>>>(part2, (int)gv, sc);
            GP2S_LAUNCH(c);
            k_mr_update<<<gv, kMrThreads, 0, c->stream>>>(n, vb[vc], vb[vu], vb[w1], vb[w2], x, sc);
            GP2S_LAUNCH(c);
            k_mr_shift_beta<<<1, 32, 0, c->stream>>>(sc);
            GP2S_LAUNCH(c);
            // rotate the roles: the new v is u, the new w_{k-1} was written over w_{k-2}
            const int t = vp;
            vp = vc;
            vc = vu;
            vu = t;
            std::swap(w1, w2);
        }
        GP2S_CUDA(c, cudaMemcpyAsync(hflag, &sc->active, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
        GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
        if (!hflag[0]) break;
    }
    GP2S_CUDA(c, cudaMemcpyAsync(hflag, &sc->active, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    *steps = hflag[2];
    return GP2S_OK;
}

}  // namespace gp2s
