// adjoint.cu -- gradient of the LML (Sec. 3) with respect to theta = [bump centers (L x d), bump
// radii (L), bump amplitudes (L), Wendland radius r, noise sigma^2]:
//     d LML / d theta_p = 1/2 a^T (dA/dtheta_p) a - 1/2 tr(A^{-1} dA/dtheta_p),   a = A^{-1} y.
// The trace uses Hutchinson's estimator with the SLQ probes: with s = D^{-1/2}, u_s = s * Ah^{-1} z_s
// (the probe columns of the multi-RHS CG) and v_s = s * z_s,
//     tr(A^{-1} dA) ~= (1/m) sum_s u_s^T dA v_s.
// Both terms are contracted with dA on A's own pattern in one pass over the CSR, never storing dA:
//     W_ij = a_i a_j - (1/m) sum_s (u_is v_js + u_js v_is) / 2
//     H_il = sum_j phi_ij W_ij b_l(x_j)                        (bump parameters, per row)
//     g_r  = 1/2 sum_ij (sum_l b_l(x_i) b_l(x_j) + w0) dphi_ij/dr W_ij
//     g_s2 = 1/2 sum_i W_ii
// and a per-point pass finishes g_{l,p} = sum_i (d b_l(x_i) / d theta_{l,p}) H_il with the bump
// derivatives of Eq. 7.
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "gp2s_kernel_math.cuh"

#include "gp2s_internal.cuh"

namespace gp2s {

namespace {

__device__ __forceinline__ uint64_t sm64_first(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Probe sign bits: bit s-1 of word (s-1)/32 of row i is 1 when z_s(i) = -1.
__global__ void k_probe_bits(const int32_t *__restrict__ perm, int64_t n, int m, uint64_t seed,
                             uint32_t *__restrict__ bits)
{
    const int W = (m + 31) / 32;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * W; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / W;
        int w = (int)(e - i * W);
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            int s = w * 32 + b + 1;
            if (s > m) break;
            uint64_t key = seed ^ (((uint64_t)s << 32) + (uint64_t)(uint32_t)perm[i]);
            word |= (uint32_t)(sm64_first(key) >> 63) << b;
        }
        bits[e] = word;
    }
}

// The same signs as FP32 +-1, row-major n x m (for the FP32 gradient's vectorised probe sums).
__global__ void k_probe_signs(const uint32_t *__restrict__ bits, int64_t n, int m, float *__restrict__ zf)
{
    const int W = (m + 31) / 32;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m;
        const int s = (int)(e - i * m);
        zf[e] = (bits[i * W + s / 32] >> (s % 32)) & 1u ? -1.0f : 1.0f;
    }
}

__device__ __forceinline__ double warp_sum_adj(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

// sum_s (xa_s z_b,s + xb_s z_a,s) over the m probes (z as sign bits), accumulated in the vectors'
// precision (FP32 in MIXED, FP64 in the FP64 form).
template <class T>
__device__ __forceinline__ T flip_t(T x, uint32_t bit) { return bit ? -x : x; }

template <class T, int M>
__device__ __forceinline__ T probe_cross(const T *__restrict__ xa, const uint32_t *__restrict__ za,
                                         const T *__restrict__ xb, const uint32_t *__restrict__ zb)
{
    T acc = T(0);
#pragma unroll
    for (int w = 0; w < (M + 31) / 32; ++w) {
        const uint32_t ba = za[w], bb = zb[w];
        constexpr int NB = M < 32 ? M : 32;
#pragma unroll 8
        for (int b = 0; b < NB; ++b) {
            const int s = w * 32 + b;
            if (s >= M) break;
            acc += flip_t<T>(xa[s], (bb >> b) & 1u) + flip_t<T>(xb[s], (ba >> b) & 1u);
        }
    }
    return acc;
}

// The same sum in FP32 with four probes per step: row i's solutions and signs staged in shared
// memory (ui, zi), row j's read as float4 from U and the +-1 signs zf, two packed FP32x2
// accumulators (multiplying by +-1 is exact, so only the order of the additions differs).
template <int M>
__device__ __forceinline__ float probe_cross4(const float4 *__restrict__ ui, const float4 *__restrict__ zi,
                                              const float *__restrict__ uj, const float *__restrict__ zj)
{
    float2 s0 = make_float2(0.0f, 0.0f), s1 = s0;
    const float4 *uj4 = reinterpret_cast<const float4 *>(uj);
    const float4 *zj4 = reinterpret_cast<const float4 *>(zj);
#pragma unroll 4
    for (int k = 0; k < M / 4; ++k) {
        const float4 a = ui[k], za = zi[k], b = __ldg(uj4 + k), zb = __ldg(zj4 + k);
        s0 = __ffma2_rn(make_float2(a.x, a.y), make_float2(zb.x, zb.y), s0);
        s1 = __ffma2_rn(make_float2(a.z, a.w), make_float2(zb.z, zb.w), s1);
        s0 = __ffma2_rn(make_float2(b.x, b.y), make_float2(za.x, za.y), s0);
        s1 = __ffma2_rn(make_float2(b.z, b.w), make_float2(za.z, za.w), s1);
    }
    return (s0.x + s0.y) + (s1.x + s1.y);
}

struct AdjArgs {
    const int32_t *rowptr, *col;
    const float4 *Xhi, *Xlo;
    const float *B32;          // n x L
    const double *a;           // n (sorted order)
    const double *s64;         // n
    const void *U;             // n x m probe solutions of Ah (FP32 or FP64)
    const uint32_t *zbits;     // n x (m/32)
    const float *zf;           // n x m signs as +-1 (FP32 form, m a multiple of 4)
    int64_t n;
    int m;
    float *H;                  // n x L
    double *part;              // per block: [g_r, g_s2]
};

template <int D, class T, int M>
__global__ void __launch_bounds__(256) k_adjoint(AdjArgs g, KernelParams kp)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int L = kp.L;
    const T *U = reinterpret_cast<const T *>(g.U);
    constexpr int WZ = M > 0 ? (M + 31) / 32 : 1;
    const float inv_r = (float)kp.inv_r;
    const float inv2m = M > 0 ? 0.5f / (float)M : 0.0f;
    // far-field kernel (family 2): kappa = exp(-q / (2 lc^2)) weights the bump term, w0 the taper
    const bool ff = kp.family == 2;
    const float lc = ff ? (float)kp.ell[0] : 1.0f;
    const float inv2lc2 = 0.5f / (lc * lc);
    // FP32 form: row i's probe solutions and signs in shared memory for the vectorised sums
    constexpr bool V4 = std::is_same<T, float>::value && M > 0 && M % 4 == 0 && M <= 128;
    __shared__ float4 s_uz[V4 ? 8 : 1][2][V4 ? M / 4 : 1];
    const int wl = (int)(threadIdx.x >> 5);
    double gr = 0.0, gs = 0.0, glc = 0.0, gw0 = 0.0;
    for (int64_t i = w0; i < g.n; i += nw) {
        const float4 hi_i = g.Xhi[i], lo_i = g.Xlo[i];
        const float ai = (float)g.a[i];
        const float si = (float)g.s64[i];
        const T *Ui = U + i * M;
        if constexpr (V4) {
            __syncwarp();
            for (int k = lane; k < M / 4; k += 32) {
                s_uz[wl][0][k] = reinterpret_cast<const float4 *>(Ui)[k];
                s_uz[wl][1][k] = reinterpret_cast<const float4 *>(g.zf + i * M)[k];
            }
            __syncwarp();
        }
        uint32_t zi[WZ];
#pragma unroll
        for (int w = 0; w < WZ; ++w) zi[w] = M > 0 && !V4 ? g.zbits[i * WZ + w] : 0u;
        float Hacc[kMaxBumps];
        for (int l = 0; l < L; ++l) Hacc[l] = 0.0f;
        float grr = 0.0f, gss = 0.0f, glcr = 0.0f, gw0r = 0.0f;
        const int p1 = g.rowptr[i + 1];
        for (int p = g.rowptr[i] + lane; p < p1; p += 32) {
            const int j = g.col[p];
            const float aj = (float)g.a[j];
            const float sj = (float)g.s64[j];
            float tr = 0.0f;
            if constexpr (V4) {
                tr = probe_cross4<M>(s_uz[wl][0], s_uz[wl][1], reinterpret_cast<const float *>(U) + (int64_t)j * M,
                                     g.zf + (int64_t)j * M);
            } else if (M > 0) {
                uint32_t zj[WZ];
#pragma unroll
                for (int w = 0; w < WZ; ++w) zj[w] = g.zbits[(int64_t)j * WZ + w];
                tr = (float)probe_cross<T, M>(Ui, zi, U + (int64_t)j * M, zj);
            }
            const float W = ai * aj - si * sj * tr * inv2m;
            if (j == i) {
                gss += W;
            }
            // distance (hi/lo split), Wendland value and d/dr
            const float4 hi_j = g.Xhi[j], lo_j = g.Xlo[j];
            const float hi[4] = {hi_i.x, hi_i.y, hi_i.z, hi_i.w}, lo[4] = {lo_i.x, lo_i.y, lo_i.z, lo_i.w};
            const float hj[4] = {hi_j.x, hi_j.y, hi_j.z, hi_j.w}, lj[4] = {lo_j.x, lo_j.y, lo_j.z, lo_j.w};
            float q = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                float dk = (hi[k] - hj[k]) + (lo[k] - lj[k]);
                q = fmaf(dk, dk, q);
            }
            const float t = sqrtf(q) * inv_r;
            const float phi = wendland<float>(kp.kind, D, t);
            const float dphi_dr = -wendland_dt<float>(kp.kind, D, t) * t * inv_r;
            float S = 0.0f;
            const float kap = ff ? expf(-q * inv2lc2) : 1.0f;
            const float pw = (ff ? kap : phi) * W;
            for (int l = 0; l < L; ++l) {
                const float bj = g.B32[(int64_t)j * L + l];
                S = fmaf(g.B32[i * L + l], bj, S);
                Hacc[l] = fmaf(pw, bj, Hacc[l]);
            }
            if (ff) {
                grr += (float)kp.w0 * dphi_dr * W;
                glcr += S * kap * q / (lc * lc * lc) * W;
                gw0r += phi * W;
            } else {
                grr += (S + (float)kp.w0) * dphi_dr * W;
            }
        }
        // reduce the row's H over the warp
        for (int l = 0; l < L; ++l) {
            float v = Hacc[l];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) g.H[i * L + l] = v;
        }
        gr += (double)grr;
        gs += (double)gss;
        glc += (double)glcr;
        gw0 += (double)gw0r;
    }
    // block reduction of the g_r, g_s2 (and far-field g_lc, g_w0) partial sums
    __shared__ double sh[4][8];
    double v4[4] = {gr, gs, glc, gw0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v4[k] = warp_sum_adj(v4[k]);
        if (lane == 0) sh[k][threadIdx.x >> 5] = v4[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[threadIdx.x][w];
        g.part[blockIdx.x * 4 + threadIdx.x] = a;
    }
}

// (The far-field kernel (family 2) takes the same pass with kappa in place of phi in H and the
// extra sums g_lc = 1/2 sum W_ij S_ij dkappa/dlc and g_w0 = 1/2 sum W_ij phi_ij.)
// g_{l,p} = sum_i d b_l(x_i) / d theta_{l,p} * H_il (FP64), per-block partials of the
// L (d + 2) bump parameters: [centers (L x d), radii (L), amps (L)].
// Thread t of a block handles bump l = t % L for points i = t / L, t / L + R, ... (R = threads / L
// points per block step); blockDim.x is a multiple of L.
template <int D>
__global__ void __launch_bounds__(256)
k_bump_grad(const double4_16a *__restrict__ X64, const float *__restrict__ H, int64_t n, KernelParams kp,
            double *__restrict__ part)
{
    const int L = kp.L;
    const int P = L * (D + 2);
    extern __shared__ double acc_sh[];   // blockDim.x x (D + 2)
    const int l = threadIdx.x % L;
    const int R = blockDim.x / L;
    double acc[D + 2];
#pragma unroll
    for (int p = 0; p < D + 2; ++p) acc[p] = 0.0;
    const double rho = kp.radii[l];
    for (int64_t i = (int64_t)blockIdx.x * R + threadIdx.x / L; i < n; i += (int64_t)gridDim.x * R) {
        const double h = (double)H[i * L + l];
        if (h == 0.0) continue;
        const double4_16a xv = X64[i];
        const double x[4] = {xv.x, xv.y, xv.z, xv.w};
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double dk = x[k] - kp.centers[l * D + k];
            q = q + dk * dk;
        }
        const double s = q / (rho * rho);
        if (!(s < 1.0)) continue;
        const double om = 1.0 - s;
        const double e = exp(kp.beta * (1.0 - 1.0 / om));
        if (!(e > 0.0)) continue;
        const double b = kp.amps[l] * e;
        const double dbds = -kp.beta * b / (om * om);            // d b / d s
#pragma unroll
        for (int k = 0; k < D; ++k)                               // d s / d c_k = -2 (x_k - c_k) / rho^2
            acc[k] += h * dbds * (-2.0 * (x[k] - kp.centers[l * D + k]) / (rho * rho));
        acc[D] += h * dbds * (-2.0 * s / rho);                    // d s / d rho = -2 s / rho
        acc[D + 1] += h * e;                                      // d b / d a
    }
#pragma unroll
    for (int p = 0; p < D + 2; ++p) acc_sh[threadIdx.x * (D + 2) + p] = acc[p];
    __syncthreads();
    // threads 0..L-1 sum their bump's rows of the block (fixed order)
    if ((int)threadIdx.x < L) {
        double v[D + 2];
#pragma unroll
        for (int p = 0; p < D + 2; ++p) v[p] = 0.0;
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int p = 0; p < D + 2; ++p) v[p] += acc_sh[(r * L + threadIdx.x) * (D + 2) + p];
        double *out = part + (int64_t)blockIdx.x * P;
#pragma unroll
        for (int k = 0; k < D; ++k) out[threadIdx.x * D + k] = v[k];
        out[L * D + threadIdx.x] = v[D];
        out[L * D + L + threadIdx.x] = v[D + 1];
    }
}

// ---------------------------------------------------------------------------------------------
// Wendland convolution kernel (Eq. 6): with W_ij as above and, for a stored pair i != j,
//     dk/ds_i      = s_j P phi,
//     dk/dlambda_ik = s_i s_j P [phi (1/(4 lambda_ik) - 1/(4 m_k)) - (phi'(t)/t) / (2 r^2) D_k^2 / (2 m_k^2)],
//     dk/dr        = s_i s_j P phi'(t) (-t / r),
// (P the determinant prefactor, m_k = (lambda_ik + lambda_jk)/2, t = sqrt(Q)/r; on the diagonal
// k_ii = s_i^2 and only dk/ds_i = s_i remains), the row sums Hs_i = sum_j W_ij dk/ds_i and
// Hl_ik = sum_j W_ij dk/dlambda_ik carry every field parameter (the sum over ordered pairs counts
// each point once as the first argument: g = sum_i ds_i/dtheta Hs_i + dlambda_ik/dtheta Hl_ik),
// and g_r = 1/2 sum_ij W_ij dk/dr, g_sigma2 = 1/2 sum_i W_ii.  FP64 per pair.
// ---------------------------------------------------------------------------------------------
struct AdjWcArgs {
    const int32_t *rowptr, *col;
    const double4_16a *X64, *Lam;
    const double *Sig;
    const double *a, *s64;
    const void *U;
    const uint32_t *zbits;
    int64_t n;
    int m;
    double *Hs;               // n
    double *Hl;               // n x 4
    double *part;             // per block: [g_r, g_s2]
};

template <int D, class T, int M>
__global__ void __launch_bounds__(256) k_adjoint_wc(AdjWcArgs g, KernelParams kp)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const T *U = reinterpret_cast<const T *>(g.U);
    constexpr int WZ = M > 0 ? (M + 31) / 32 : 1;
    const double inv2m = M > 0 ? 0.5 / (double)M : 0.0;
    const double r = kp.r;
    double gr = 0.0, gs = 0.0;
    for (int64_t i = w0; i < g.n; i += nw) {
        const double4_16a xiv = g.X64[i], liv = g.Lam[i];
        const double xi[4] = {xiv.x, xiv.y, xiv.z, xiv.w}, li[4] = {liv.x, liv.y, liv.z, liv.w};
        const double ai = g.a[i], si = g.s64[i], sgi = g.Sig[i];
        const T *Ui = U + i * M;
        uint32_t zi[WZ];
#pragma unroll
        for (int w = 0; w < WZ; ++w) zi[w] = M > 0 ? g.zbits[i * WZ + w] : 0u;
        double hs = 0.0, hl[D];
#pragma unroll
        for (int k = 0; k < D; ++k) hl[k] = 0.0;
        const int p1 = g.rowptr[i + 1];
        for (int p = g.rowptr[i] + lane; p < p1; p += 32) {
            const int j = g.col[p];
            double tr = 0.0;
            if (M > 0) {
                uint32_t zj[WZ];
#pragma unroll
                for (int w = 0; w < WZ; ++w) zj[w] = g.zbits[(int64_t)j * WZ + w];
                tr = (double)probe_cross<T, M>(Ui, zi, U + (int64_t)j * M, zj);
            }
            const double W = ai * g.a[j] - si * g.s64[j] * tr * inv2m;
            const double sgj = g.Sig[j];
            if (j == i) {
                gs += W;
                hs += W * sgi;
                continue;
            }
            const double4_16a xjv = g.X64[j], ljv = g.Lam[j];
            const double xj[4] = {xjv.x, xjv.y, xjv.z, xjv.w}, lj[4] = {ljv.x, ljv.y, ljv.z, ljv.w};
            double q = 0.0, pref = 1.0, dd[D], mm[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double dk = xi[k] - xj[k];
                mm[k] = (li[k] + lj[k]) * 0.5;
                dd[k] = dk * dk;
                q += dd[k] / mm[k];
                pref *= sqrt(sqrt(li[k] * lj[k])) / sqrt(mm[k]);
            }
            const double t = sqrt(q) / r;
            const double phi = wendland<double>(kp.kind, D, t);
            const double dphit = wendland_dt_over_t<double>(kp.kind, D, t);
            const double ss = sgi * sgj;
            hs += W * sgj * pref * phi;
#pragma unroll
            for (int k = 0; k < D; ++k)
                hl[k] += W * ss * pref * (phi * (0.25 / li[k] - 0.25 / mm[k]) - dphit / (2.0 * r * r) * dd[k] / (2.0 * mm[k] * mm[k]));
            gr += W * ss * pref * (dphit * t) * (-t / r);
        }
        // the row's sums over the warp
        hs = warp_sum_adj(hs);
#pragma unroll
        for (int k = 0; k < D; ++k) hl[k] = warp_sum_adj(hl[k]);
        if (lane == 0) {
            g.Hs[i] = hs;
#pragma unroll
            for (int k = 0; k < D; ++k) g.Hl[i * 4 + k] = hl[k];
        }
    }
    __shared__ double sh[2][8];
    gr = warp_sum_adj(gr);
    gs = warp_sum_adj(gs);
    if (lane == 0) {
        sh[0][threadIdx.x >> 5] = gr;
        sh[1][threadIdx.x >> 5] = gs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh[0][w]; b += sh[1][w]; }
        g.part[blockIdx.x * 2 + 0] = a;
        g.part[blockIdx.x * 2 + 1] = b;
    }
}

// Field parameters of the convolution kernel from the row sums: thread t of a block handles bump
// l = t % L for points i = t / L, t / L + R, ... (R = threads / L); for psi_l at x_i,
//     w = Hs_i a_l + sum_k Hl_ik G_lk   ->   centers: w dpsi/dc,  radii: w dpsi/drho,
//     amps: Hs_i psi,  G_lk: Hl_ik psi;
// threads of bump 0 also sum ell_k: 2 ell_k Hl_ik and w0: Hs_i.  Per-block partials of the
// parameters [centers, radii, amps, G, ell, w0] in that order.
template <int D>
__global__ void __launch_bounds__(256)
k_wc_field_grad(const double4_16a *__restrict__ X64, const double *__restrict__ Hs, const double *__restrict__ Hl,
                int64_t n, KernelParams kp, double *__restrict__ part)
{
    const int L = kp.L;
    constexpr int NA = 3 * D + 3;                 // per thread: 2 D + 2 bump terms, D + 1 shared terms
    const int Pf = L * (2 * D + 2) + D + 1;
    extern __shared__ double wacc_sh[];           // blockDim.x x NA
    const int l = L > 0 ? (int)threadIdx.x % L : 0;
    const int R = L > 0 ? (int)blockDim.x / L : (int)blockDim.x;
    double acc[NA];
#pragma unroll
    for (int p = 0; p < NA; ++p) acc[p] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * R + threadIdx.x / (L > 0 ? L : 1); i < n && (int)threadIdx.x < R * (L > 0 ? L : 1);
         i += (int64_t)gridDim.x * R) {
        const double hs = Hs[i];
        double hl[D];
#pragma unroll
        for (int k = 0; k < D; ++k) hl[k] = Hl[i * 4 + k];
        if (l == 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) acc[2 * D + 2 + k] += 2.0 * kp.ell[k] * hl[k];
            acc[3 * D + 2] += hs;
        }
        if (L == 0) continue;
        const double4_16a xv = X64[i];
        const double x[4] = {xv.x, xv.y, xv.z, xv.w};
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double dk = x[k] - kp.centers[l * D + k];
            q += dk * dk;
        }
        const double rho = kp.radii[l];
        const double s = q / (rho * rho);
        if (!(s < 1.0)) continue;
        const double u = 1.0 - s;
        const double psi = u * u * u;
        const double dpds = -3.0 * u * u;
        double w = hs * kp.amps[l];
#pragma unroll
        for (int k = 0; k < D; ++k) w += hl[k] * kp.G[l * D + k];
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] += w * dpds * (-2.0 * (x[k] - kp.centers[l * D + k]) / (rho * rho));
        acc[D] += w * dpds * (-2.0 * s / rho);
        acc[D + 1] += hs * psi;
#pragma unroll
        for (int k = 0; k < D; ++k) acc[D + 2 + k] += hl[k] * psi;
    }
#pragma unroll
    for (int p = 0; p < NA; ++p) wacc_sh[threadIdx.x * NA + p] = acc[p];
    __syncthreads();
    double *out = part + (int64_t)blockIdx.x * Pf;
    if ((int)threadIdx.x < L) {
        double v[2 * D + 2];
#pragma unroll
        for (int p = 0; p < 2 * D + 2; ++p) v[p] = 0.0;
        for (int rr = 0; rr < R; ++rr)
#pragma unroll
            for (int p = 0; p < 2 * D + 2; ++p) v[p] += wacc_sh[(rr * L + threadIdx.x) * NA + p];
        const int t = threadIdx.x;
#pragma unroll
        for (int k = 0; k < D; ++k) out[t * D + k] = v[k];
        out[L * D + t] = v[D];
        out[L * D + L + t] = v[D + 1];
#pragma unroll
        for (int k = 0; k < D; ++k) out[L * D + 2 * L + t * D + k] = v[D + 2 + k];
    }
    if (threadIdx.x == 0) {
        double v[D + 1];
#pragma unroll
        for (int p = 0; p <= D; ++p) v[p] = 0.0;
        const int stride = L > 0 ? L : 1;
        for (int rr = 0; rr < R; ++rr)
#pragma unroll
            for (int p = 0; p <= D; ++p) v[p] += wacc_sh[(rr * stride) * NA + 2 * D + 2 + p];
#pragma unroll
        for (int p = 0; p <= D; ++p) out[L * (2 * D + 2) + p] = v[p];
    }
}

template <int D, class T>
gp2s_status launch_adjoint_wc(gp2s_ctx *c, const AdjWcArgs &g, const KernelParams &kp, unsigned gb)
{
    switch (g.m) {
    case 0: k_adjoint_wc<D, T, 0><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 16: k_adjoint_wc<D, T, 16><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 32: k_adjoint_wc<D, T, 32><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 48: k_adjoint_wc<D, T, 48><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 64: k_adjoint_wc<D, T, 64><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 96: k_adjoint_wc<D, T, 96><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 128: k_adjoint_wc<D, T, 128><<<gb, 256, 0, c->stream>>>(g, kp); break;
    default: return set_err(c, GP2S_EINVAL, "probes must be 0, 16, 32, 48, 64, 96 or 128");
    }
    GP2S_LAUNCH(c);
    return GP2S_OK;
}

template <int D, class T>
gp2s_status launch_adjoint(gp2s_ctx *c, const AdjArgs &g, const KernelParams &kp, unsigned gb)
{
    switch (g.m) {
    case 0: k_adjoint<D, T, 0><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 16: k_adjoint<D, T, 16><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 32: k_adjoint<D, T, 32><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 48: k_adjoint<D, T, 48><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 64: k_adjoint<D, T, 64><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 96: k_adjoint<D, T, 96><<<gb, 256, 0, c->stream>>>(g, kp); break;
    case 128: k_adjoint<D, T, 128><<<gb, 256, 0, c->stream>>>(g, kp); break;
    default: return set_err(c, GP2S_EINVAL, "probes must be 0, 16, 32, 48, 64, 96 or 128");
    }
    GP2S_LAUNCH(c);
    return GP2S_OK;
}

template <class T>
gp2s_status dispatch_adjoint(gp2s_ctx *c, int d, const AdjArgs &g, const KernelParams &kp, unsigned gb)
{
    switch (d) {
    case 1: return launch_adjoint<1, T>(c, g, kp, gb);
    case 2: return launch_adjoint<2, T>(c, g, kp, gb);
    case 3: return launch_adjoint<3, T>(c, g, kp, gb);
    default: return launch_adjoint<4, T>(c, g, kp, gb);
    }
}

}  // namespace

static gp2s_status adjoint_gradient_wc(gp2s_ctx *c, int m, double *grad_host);

gp2s_status adjoint_gradient(gp2s_ctx *c, int m, double *grad_host)
{
    if (c->A.kp.family == 1) return adjoint_gradient_wc(c, m, grad_host);
    const Assembled &A = c->A;
    const int64_t n = A.n;
    const int d = A.d, L = A.L;
    const bool ff = A.kp.family == 2;
    const int P = ff ? L * (d + 2) + 4 : L * (d + 2) + 2;
    if (!c->have_solution) return set_err(c, GP2S_ENOTREADY, "gradient needs the solve");
    if (m > 0 && !c->have_probes) return set_err(c, GP2S_ENOTREADY, "gradient needs the probe solves");
    const bool mixed = A.precision == GP2S_PREC_MIXED;
    const int W = m > 0 ? (m + 31) / 32 : 0;
    GP2S_TRY(ensure(c, c->Z, sizeof(uint32_t) * (size_t)n * (W > 0 ? W : 1) + 64));
    GP2S_TRY(ensure(c, c->H, sizeof(float) * (size_t)n * (L > 0 ? L : 1) + 64));
    const int nb = 152 * 8;
    const int nbf = 152 * 2;
    GP2S_TRY(ensure(c, c->gpart, sizeof(double) * ((size_t)nb * 4 + (size_t)nbf * P + 64)));
    double *part = c->gpart.as<double>();
    double *bpart = part + (size_t)nb * 4;
    if (m > 0) {
        unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n * W, 256), 152 * 8);
        k_probe_bits<<<gb, 256, 0, c->stream>>>(c->perm.as<int32_t>(), n, m, A.opts.seed, c->Z.as<uint32_t>());
        GP2S_LAUNCH(c);
        if (mixed && m % 4 == 0) {
            GP2S_TRY(ensure(c, c->Zf, sizeof(float) * (size_t)n * m + 64));
            const unsigned gs = (unsigned)std::min<int64_t>(ceil_div(n * m, 256), 152 * 16);
            k_probe_signs<<<gs, 256, 0, c->stream>>>(c->Z.as<uint32_t>(), n, m, c->Zf.as<float>());
            GP2S_LAUNCH(c);
        }
    }
    AdjArgs g;
    std::memset(&g, 0, sizeof(g));
    g.rowptr = c->rowptr.as<int32_t>();
    g.col = c->col.as<int32_t>();
    g.Xhi = c->Xhi.as<float4>();
    g.Xlo = c->Xlo.as<float4>();
    g.B32 = c->B32.as<float>();
    g.a = c->vec64.as<double>() + 3 * n;
    g.s64 = c->s64.as<double>();
    g.U = c->vec.p;          // probe-group x (first block of the Krylov vectors)
    g.zbits = c->Z.as<uint32_t>();
    g.zf = mixed && m > 0 && m % 4 == 0 ? c->Zf.as<float>() : nullptr;
    g.n = n;
    g.m = m;
    g.H = c->H.as<float>();
    g.part = part;
    if (mixed) GP2S_TRY(dispatch_adjoint<float>(c, d, g, A.kp, nb));
    else GP2S_TRY(dispatch_adjoint<double>(c, d, g, A.kp, nb));
    // bump parameters
    const int Pb = L * (d + 2);
    if (Pb > 0) {
        const int thr = L * (256 / L);
        size_t smem = sizeof(double) * (size_t)thr * (d + 2);
        switch (d) {
        case 1: k_bump_grad<1><<<nbf, thr, smem, c->stream>>>(c->Xs64.as<double4_16a>(), c->H.as<float>(), n, A.kp, bpart); break;
        case 2: k_bump_grad<2><<<nbf, thr, smem, c->stream>>>(c->Xs64.as<double4_16a>(), c->H.as<float>(), n, A.kp, bpart); break;
        case 3: k_bump_grad<3><<<nbf, thr, smem, c->stream>>>(c->Xs64.as<double4_16a>(), c->H.as<float>(), n, A.kp, bpart); break;
        default: k_bump_grad<4><<<nbf, thr, smem, c->stream>>>(c->Xs64.as<double4_16a>(), c->H.as<float>(), n, A.kp, bpart); break;
        }
        GP2S_LAUNCH(c);
    }
    std::vector<double> hp((size_t)nb * 4), hb((size_t)nbf * (Pb > 0 ? Pb : 1));
    GP2S_CUDA(c, cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb * 4, cudaMemcpyDeviceToHost, c->stream));
    if (Pb > 0)
        GP2S_CUDA(c, cudaMemcpyAsync(hb.data(), bpart, sizeof(double) * (size_t)nbf * Pb, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    // fixed-order host sums of the (few hundred) block partials
    for (int p = 0; p < P; ++p) grad_host[p] = 0.0;
    for (int b = 0; b < nbf && Pb > 0; ++b)
        for (int p = 0; p < Pb; ++p) grad_host[p] += hb[(size_t)b * Pb + p];
    double gr = 0.0, gs = 0.0, glc = 0.0, gw0 = 0.0;
    for (int b = 0; b < nb; ++b) {
        gr += hp[4 * b];
        gs += hp[4 * b + 1];
        glc += hp[4 * b + 2];
        gw0 += hp[4 * b + 3];
    }
    if (ff) {
        grad_host[P - 4] = 0.5 * glc;
        grad_host[P - 3] = 0.5 * gw0;
    }
    grad_host[P - 2] = 0.5 * gr;
    grad_host[P - 1] = 0.5 * gs;
    return GP2S_OK;
}

// The Wendland convolution kernel's gradient: [centers, radii, amps, G, ell, w0, r, sigma2].
static gp2s_status adjoint_gradient_wc(gp2s_ctx *c, int m, double *grad_host)
{
    const Assembled &A = c->A;
    const int64_t n = A.n;
    const int d = A.d, L = A.L;
    const int P = L * (2 * d + 2) + d + 3;
    const int Pf = P - 2;
    if (!c->have_solution) return set_err(c, GP2S_ENOTREADY, "gradient needs the solve");
    if (m > 0 && !c->have_probes) return set_err(c, GP2S_ENOTREADY, "gradient needs the probe solves");
    const bool mixed = A.precision == GP2S_PREC_MIXED;
    const int W = m > 0 ? (m + 31) / 32 : 0;
    GP2S_TRY(ensure(c, c->Z, sizeof(uint32_t) * (size_t)n * (W > 0 ? W : 1) + 64));
    GP2S_TRY(ensure(c, c->H, sizeof(double) * (size_t)n * 5 + 64));
    const int nb = 152 * 8;
    const int nbf = 152 * 2;
    GP2S_TRY(ensure(c, c->gpart, sizeof(double) * ((size_t)nb * 2 + (size_t)nbf * Pf + 64)));
    double *part = c->gpart.as<double>();
    double *fpart = part + (size_t)nb * 2;
    if (m > 0) {
        unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n * W, 256), 152 * 8);
        k_probe_bits<<<gb, 256, 0, c->stream>>>(c->perm.as<int32_t>(), n, m, A.opts.seed, c->Z.as<uint32_t>());
        GP2S_LAUNCH(c);
    }
    AdjWcArgs g;
    std::memset(&g, 0, sizeof(g));
    g.rowptr = c->rowptr.as<int32_t>();
    g.col = c->col.as<int32_t>();
    g.X64 = c->Xs64.as<double4_16a>();
    g.Lam = c->wc_lam.as<double4_16a>();
    g.Sig = c->wc_sig.as<double>();
    g.a = c->vec64.as<double>() + 3 * n;
    g.s64 = c->s64.as<double>();
    g.U = c->vec.p;
    g.zbits = c->Z.as<uint32_t>();
    g.n = n;
    g.m = m;
    g.Hs = c->H.as<double>();
    g.Hl = g.Hs + n;
    g.part = part;
#define GP2S_AWC(DD)                                                                         \
    (mixed ? launch_adjoint_wc<DD, float>(c, g, A.kp, nb) : launch_adjoint_wc<DD, double>(c, g, A.kp, nb))
    switch (d) {
    case 1: GP2S_TRY(GP2S_AWC(1)); break;
    case 2: GP2S_TRY(GP2S_AWC(2)); break;
    case 3: GP2S_TRY(GP2S_AWC(3)); break;
    default: GP2S_TRY(GP2S_AWC(4)); break;
    }
#undef GP2S_AWC
    {
        const int thr = L > 0 ? L * (256 / L) : 256;
        const size_t smem = sizeof(double) * (size_t)thr * (3 * d + 3);
        const double *Hs = g.Hs, *Hl = g.Hl;
        const double4_16a *x64 = c->Xs64.as<double4_16a>();
        switch (d) {
        case 1: k_wc_field_grad<1><<<nbf, thr, smem, c->stream>>>(x64, Hs, Hl, n, A.kp, fpart); break;
        case 2: k_wc_field_grad<2><<<nbf, thr, smem, c->stream>>>(x64, Hs, Hl, n, A.kp, fpart); break;
        case 3: k_wc_field_grad<3><<<nbf, thr, smem, c->stream>>>(x64, Hs, Hl, n, A.kp, fpart); break;
        default: k_wc_field_grad<4><<<nbf, thr, smem, c->stream>>>(x64, Hs, Hl, n, A.kp, fpart); break;
        }
        GP2S_LAUNCH(c);
    }
    std::vector<double> hp((size_t)nb * 2), hb((size_t)nbf * Pf);
    GP2S_CUDA(c, cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb * 2, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaMemcpyAsync(hb.data(), fpart, sizeof(double) * (size_t)nbf * Pf, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int p = 0; p < P; ++p) grad_host[p] = 0.0;
    for (int b = 0; b < nbf; ++b)
        for (int p = 0; p < Pf; ++p) grad_host[p] += hb[(size_t)b * Pf + p];
    double gr = 0.0, gs = 0.0;
    for (int b = 0; b < nb; ++b) { gr += hp[2 * b]; gs += hp[2 * b + 1]; }
    grad_host[P - 2] = 0.5 * gr;
    grad_host[P - 1] = 0.5 * gs;
    return GP2S_OK;
}

}  // namespace gp2s
