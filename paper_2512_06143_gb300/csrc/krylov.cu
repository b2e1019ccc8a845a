// krylov.cu -- multi-RHS conjugate gradients on the Jacobi-scaled matrix Ah = D^{-1/2} A D^{-1/2},
// FP64 residual refinement of the y column, Rademacher probes and the CG coefficient records that
// stochastic Lanczos quadrature needs.
//
// The paper solves K^{-1} y by MINRES on the host (App. B.7) and leaves the log-determinant method
// open (Sec. 3.6).  A = K + sigma^2 I is symmetric positive definite, so conjugate gradients solve
// the same system; running the y column and the m probe columns together lets one pass over the CSR
// serve all of them (the SpMM), and the CG step lengths / direction coefficients of each probe column
// are its Lanczos tridiagonal (the CG-Lanczos relation), which is what SLQ needs.
//
// Column 0 is y (right-hand side s * y, s = D^{-1/2}); columns 1..m are the probes z_s.  Vectors are
// row-major: the y group is n values, the probe group n x m values.  In MIXED precision vectors are
// FP32, dot products use compensated FP32 partial sums that are combined in FP64, and the scalars
// (alpha, beta, rho) are FP64.  In FP64 precision everything is FP64.
#include <cmath>
#include <cstring>

#include "gp2s_internal.cuh"

namespace gp2s {

namespace {

constexpr int kSpmmThreads = 256;
constexpr int kSpmmWarps = kSpmmThreads / kWarp;
constexpr int kMaxPartBlocks = 152 * 8;
constexpr int kScal = 8;   // doubles per column in the scalar block
constexpr int kMaxCols = 129;   // y + up to 128 probes

// scalar block layout per column c: [rho, alpha, beta, b2, pq, rr, steps, tol2b2]
enum { S_RHO = 0, S_ALPHA, S_BETA, S_B2, S_PQ, S_RR, S_STEPS, S_TOL };

// ---------------------------------------------------------------------------------------------
// SplitMix64 Rademacher probes (same definition as the oracle's, written independently):
// z = 1 - 2 * (top bit of splitmix64(seed ^ (s << 32 | i_orig))), s = 1..m.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_first(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class T>
__global__ void k_probes(const int32_t *__restrict__ perm, int64_t n, int m, uint64_t seed, T *__restrict__ Z)
{
    int64_t tot = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / m;
        int s = (int)(e - i * m) + 1;
        uint64_t key = seed ^ (((uint64_t)s << 32) + (uint64_t)(uint32_t)perm[i]);
        Z[e] = (splitmix64_first(key) >> 63) ? T(-1) : T(1);
    }
}

// ---------------------------------------------------------------------------------------------
// Compensated accumulation for FP32 dot products (TwoProduct via FMA + TwoSum).
// ---------------------------------------------------------------------------------------------
struct Acc32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        float t = s + x;
        float z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ void fma2(float a, float b)
    {
        float p = a * b;
        float pe = __fmaf_rn(a, b, -p);
        add(p);
        c += pe;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
struct Acc64 {
    double s = 0.0;
    __device__ __forceinline__ void fma2(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <class T> struct AccOf;
template <> struct AccOf<float> { using type = Acc32; };
template <> struct AccOf<double> { using type = Acc64; };

template <class T, int K>
__device__ __forceinline__ void load_k(const T *__restrict__ p, T (&v)[K])
{
    if constexpr (sizeof(T) == 4 && K == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (sizeof(T) == 4 && K == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else if constexpr (sizeof(T) == 8 && K == 2) {
        double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else if constexpr (sizeof(T) == 8 && K == 4) {
        double2 t0 = reinterpret_cast<const double2 *>(p)[0], t1 = reinterpret_cast<const double2 *>(p)[1];
        v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = p[k];
    }
}
template <class T, int K>
__device__ __forceinline__ void store_k(T *__restrict__ p, const T (&v)[K])
{
    if constexpr (sizeof(T) == 4 && K == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (sizeof(T) == 4 && K == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else if constexpr (sizeof(T) == 8 && K == 2) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = v[k];
    }
}

// Block-reduce one double per (warp lane-set) into part[col * pstride + blockIdx.x].
// vals[k] holds this lane's contribution to column col0 + lane * K + k (probe group) or the y
// column.  Deterministic: fixed shuffle tree, fixed warp order.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------------------------
// SpMM: Q = Ah P for the y column (lanes over a row's entries) and the m probe columns (all lanes
// per entry, K = m / 32 columns per lane), plus the partial dots p_c^T q_c.
// One CTA owns a contiguous range of rows; its warps take rows round-robin.
// ---------------------------------------------------------------------------------------------
template <class T, class V, int K, bool HAS_Y>
__global__ void __launch_bounds__(kSpmmThreads)
k_spmm(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const V *__restrict__ val,
       int64_t n, int64_t rows_per_block, const T *__restrict__ py, const T *__restrict__ pz,
       T *__restrict__ qy, T *__restrict__ qz, double *__restrict__ part, int pstride,
       const int *__restrict__ active)
{
    using Acc = typename AccOf<T>::type;
    constexpr int M = 32 * K;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r_end = min(n, r_begin + rows_per_block);
    Acc dz[K > 0 ? K : 1];
    Acc dy;
    for (int64_t i = r_begin + wid; i < r_end; i += kSpmmWarps) {
        const int p0 = rowptr[i], p1 = rowptr[i + 1];
        T acc[K > 0 ? K : 1];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = T(0);
        T accy = T(0);
        for (int pb = p0; pb < p1; pb += kWarp) {
            const int p = pb + lane;
            int cj = 0;
            T cv = T(0);
            if (p < p1) {
                cj = col[p];
                cv = (T)val[p];
            }
            if (HAS_Y) accy += cv * py[cj];
            if (K > 0) {
                const int cnt = min(kWarp, p1 - pb);
                for (int t = 0; t < cnt; ++t) {
                    const int j = __shfl_sync(0xffffffffu, cj, t);
                    const T v = __shfl_sync(0xffffffffu, cv, t);
                    T pv[K > 0 ? K : 1];
                    load_k<T, (K > 0 ? K : 1)>(pz + (int64_t)j * M + lane * K, pv);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc[k] += v * pv[k];
                }
            }
        }
        if (K > 0) {
            store_k<T, (K > 0 ? K : 1)>(qz + i * M + lane * K, acc);
            T pi[K > 0 ? K : 1];
            load_k<T, (K > 0 ? K : 1)>(pz + i * M + lane * K, pi);
#pragma unroll
            for (int k = 0; k < K; ++k) dz[k].fma2(pi[k], acc[k]);
        }
        if (HAS_Y) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) accy += __shfl_xor_sync(0xffffffffu, accy, o);
            if (lane == 0) {
                qy[i] = accy;
                dy.fma2(py[i], accy);
            }
        }
    }
    // block reduction of the partial dots: y column (lane 0 of each warp) and probe columns
    __shared__ double red[kSpmmWarps][M + 1];
    if (HAS_Y) {
        double v = lane == 0 ? dy.value() : 0.0;
        if (lane == 0) red[wid][M] = v;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) red[wid][lane * K + k] = dz[k].value();
    __syncthreads();
    for (int cidx = threadIdx.x; cidx < M + 1; cidx += kSpmmThreads) {
        if (cidx == M && !HAS_Y) continue;
        double s = 0.0;
        for (int w = 0; w < kSpmmWarps; ++w) s += red[w][cidx];
        const int c = cidx == M ? 0 : cidx + 1;
        part[(int64_t)c * pstride + blockIdx.x] = s;
    }
    (void)active;
}

// CSR SpMV in FP64 (refinement residual): out = b - Ah x.
__global__ void __launch_bounds__(256)
k_residual64(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
             const double *__restrict__ val, int64_t n, const double *__restrict__ x,
             const double *__restrict__ b, double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        double s = 0.0;
        for (int p = rowptr[i] + lane; p < rowptr[i + 1]; p += kWarp) s = fma(val[p], x[col[p]], s);
        s = warp_sum(s);
        if (lane == 0) out[i] = b[i] - s;
    }
}

// ---------------------------------------------------------------------------------------------
// Scalar kernels: one CTA per column, fixed-order FP64 reduction of the per-block partials.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(const double *__restrict__ p, int cnt)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < cnt; b += blockDim.x) s += p[b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
    }
    return t;   // valid in thread 0
}

// Initial scalars: rho = b^T b (partials in part), b2 = rho, tol2 = tol^2 b2, alpha = beta = 0.
__global__ void k_scal_init(const double *__restrict__ part, int pstride, int nparts_y, int nparts_z,
                            double *__restrict__ sc, int *__restrict__ active, double tol_y, double tol_z)
{
    const int c = blockIdx.x;
    double s = block_sum(part + (int64_t)c * pstride, c == 0 ? nparts_y : nparts_z);
    if (threadIdx.x == 0) {
        double *q = sc + c * kScal;
        q[S_RHO] = s;
        q[S_B2] = s;
        double tol = c == 0 ? tol_y : tol_z;
        q[S_TOL] = tol * tol * s;
        q[S_ALPHA] = 0.0;
        q[S_BETA] = 0.0;
        q[S_STEPS] = 0.0;
        active[c] = s > 0.0 ? 1 : 0;
    }
}

// alpha_c = rho_c / (p_c^T q_c); breakdown if p^T q <= 0 or NaN.
__global__ void k_scal_alpha(const double *__restrict__ part, int pstride, int nparts, double *__restrict__ sc,
                             int *__restrict__ active, int *__restrict__ flags, double *__restrict__ rec,
                             int ksteps)
{
    const int c = blockIdx.x;
    double s = block_sum(part + (int64_t)c * pstride, nparts);
    if (threadIdx.x == 0) {
        double *q = sc + c * kScal;
        q[S_PQ] = s;
        if (!active[c]) {
            q[S_ALPHA] = 0.0;
            return;
        }
        if (!(s > 0.0)) {
            active[c] = 0;
            q[S_ALPHA] = 0.0;
            atomicOr(&flags[0], 1);   // breakdown
            return;
        }
        double a = q[S_RHO] / s;
        q[S_ALPHA] = a;
        int st = (int)q[S_STEPS];
        if (c > 0 && rec && st < ksteps) rec[((int64_t)(c - 1) * ksteps + st) * 2 + 0] = a;
    }
}

// beta_c = rr_c / rho_c, rho_c = rr_c, convergence test |r|^2 <= tol^2 |b|^2 once at least
// kmin steps are recorded (the probe columns keep iterating to give SLQ its k Lanczos steps).
__global__ void k_scal_beta(const double *__restrict__ part, int pstride, int nparts_y, int nparts_z,
                            double *__restrict__ sc, int *__restrict__ active, int *__restrict__ count,
                            double *__restrict__ rec, int ksteps, int kmin_probe)
{
    const int c = blockIdx.x;
    double s = block_sum(part + (int64_t)c * pstride, c == 0 ? nparts_y : nparts_z);
    if (threadIdx.x == 0) {
        double *q = sc + c * kScal;
        if (!active[c]) {
            q[S_BETA] = 0.0;
            return;
        }
        q[S_RR] = s;
        double b = s / q[S_RHO];
        int st = (int)q[S_STEPS];
        if (c > 0 && rec && st < ksteps) rec[((int64_t)(c - 1) * ksteps + st) * 2 + 1] = b;
        q[S_BETA] = b;
        q[S_RHO] = s;
        q[S_STEPS] = (double)(st + 1);
        bool conv = s <= q[S_TOL];
        int kmin = c == 0 ? 0 : kmin_probe;
        if ((conv && st + 1 >= kmin) || !(s == s)) {
            active[c] = 0;
            // p is not updated for inactive columns (beta unused)
        } else {
            atomicAdd(count, 1);
        }
    }
}

// x += alpha p ; r -= alpha q ; partial r^T r.  Probe group: thread t owns column t % m.
template <class T>
__global__ void k_update(int64_t n, int m, T *__restrict__ xz, T *__restrict__ rz, const T *__restrict__ pz,
                         const T *__restrict__ qz, T *__restrict__ xy, T *__restrict__ ry, const T *__restrict__ py,
                         const T *__restrict__ qy, const double *__restrict__ sc, double *__restrict__ part,
                         int pstride, int nbz)
{
    using Acc = typename AccOf<T>::type;
    __shared__ double shv[kSpmmThreads / 32 + 1][32];
    Acc acc;
    if ((int)blockIdx.x < nbz) {
        // probe group: element e = i * m + c
        const int c = threadIdx.x % m;
        const double alpha = sc[(c + 1) * kScal + S_ALPHA];
        const T a = (T)alpha;
        const int rows_per_step = blockDim.x / m;
        const int64_t r0 = threadIdx.x / m;
        for (int64_t i = (int64_t)blockIdx.x * rows_per_step + r0; i < n; i += (int64_t)nbz * rows_per_step) {
            int64_t e = i * m + c;
            T r = rz[e];
            if (alpha != 0.0) {
                xz[e] = xz[e] + a * pz[e];
                r = r - a * qz[e];
                rz[e] = r;
            }
            acc.fma2(r, r);
        }
        // reduce threads of the same column: threads c, c+m, c+2m, ... (rows_per_step of them)
        __shared__ double red[1024];
        red[threadIdx.x] = acc.value();
        __syncthreads();
        if ((int)threadIdx.x < m) {
            double s = 0.0;
            for (int k = 0; k < rows_per_step; ++k) s += red[k * m + threadIdx.x];
            part[(int64_t)(threadIdx.x + 1) * pstride + blockIdx.x] = s;
        }
    } else {
        const int b = blockIdx.x - nbz;
        const int nby = gridDim.x - nbz;
        const double alpha = sc[0 * kScal + S_ALPHA];
        const T a = (T)alpha;
        for (int64_t i = (int64_t)b * blockDim.x + threadIdx.x; i < n; i += (int64_t)nby * blockDim.x) {
            T r = ry[i];
            if (alpha != 0.0) {
                xy[i] = xy[i] + a * py[i];
                r = r - a * qy[i];
                ry[i] = r;
            }
            acc.fma2(r, r);
        }
        double v = warp_sum(acc.value());
        if ((threadIdx.x & 31) == 0) shv[threadIdx.x >> 5][0] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += shv[w][0];
            part[(int64_t)0 * pstride + b] = s;
        }
    }
}

// p = r + beta p for active columns.
template <class T>
__global__ void k_direction(int64_t n, int m, const T *__restrict__ rz, T *__restrict__ pz, const T *__restrict__ ry,
                            T *__restrict__ py, const double *__restrict__ sc, const int *__restrict__ active)
{
    const int64_t tz = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tz + n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < tz) {
            int c = (int)(e % m) + 1;
            if (active[c]) pz[e] = rz[e] + (T)sc[c * kScal + S_BETA] * pz[e];
        } else {
            int64_t i = e - tz;
            if (active[0]) py[i] = ry[i] + (T)sc[S_BETA] * py[i];
        }
    }
}

// Initial state: x = 0, r = p = rhs; partial b^T b.  rhs_y is FP64 (s * y or the refinement residual).
template <class T>
__global__ void k_cg_init(int64_t n, int m, const double *__restrict__ rhs_y, T *__restrict__ xz, T *__restrict__ rz,
                          T *__restrict__ pz, T *__restrict__ xy, T *__restrict__ ry, T *__restrict__ py,
                          double *__restrict__ part, int pstride, int nbz)
{
    using Acc = typename AccOf<T>::type;
    Acc acc;
    __shared__ double red[1024];
    __shared__ double shv[32];
    if ((int)blockIdx.x < nbz) {
        const int c = threadIdx.x % m;
        const int rows_per_step = blockDim.x / m;
        const int64_t r0 = threadIdx.x / m;
        for (int64_t i = (int64_t)blockIdx.x * rows_per_step + r0; i < n; i += (int64_t)nbz * rows_per_step) {
            int64_t e = i * m + c;
            T z = rz[e];     // probes were written into rz
            xz[e] = T(0);
            pz[e] = z;
            acc.fma2(z, z);
        }
        red[threadIdx.x] = acc.value();
        __syncthreads();
        if ((int)threadIdx.x < m) {
            double s = 0.0;
            for (int k = 0; k < rows_per_step; ++k) s += red[k * m + threadIdx.x];
            part[(int64_t)(threadIdx.x + 1) * pstride + blockIdx.x] = s;
        }
    } else {
        const int b = blockIdx.x - nbz;
        const int nby = gridDim.x - nbz;
        for (int64_t i = (int64_t)b * blockDim.x + threadIdx.x; i < n; i += (int64_t)nby * blockDim.x) {
            T v = (T)rhs_y[i];
            xy[i] = T(0);
            ry[i] = v;
            py[i] = v;
            acc.fma2(v, v);
        }
        double v = warp_sum(acc.value());
        if ((threadIdx.x & 31) == 0) shv[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += shv[w];
            part[b] = s;
        }
    }
}

__global__ void k_scale64(int64_t n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

template <class T>
__global__ void k_accum64(int64_t n, const T *__restrict__ e, double *__restrict__ x)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)e[i];
}

// Partial sums of (r_i / s_i)^2 and y_i^2 (original-space residual norm), per block.
__global__ void k_resnorm(int64_t n, const double *__restrict__ r, const double *__restrict__ s,
                          const double *__restrict__ y, double *__restrict__ part, int nb)
{
    __shared__ double sh[2][32];
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = r[i] / s[i];
        a = fma(t, t, a);
        b = fma(y[i], y[i], b);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a;
        sh[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa += sh[0][w]; sb += sh[1][w]; }
        part[blockIdx.x] = sa;
        part[nb + blockIdx.x] = sb;
    }
}

__global__ void k_sum_parts(const double *__restrict__ part, int cnt, int groups, double *__restrict__ out)
{
    for (int g = 0; g < groups; ++g) {
        double s = block_sum(part + (int64_t)g * cnt, cnt);
        if (threadIdx.x == 0) out[g] = s;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------------------------
struct CGBuffers {
    void *xz, *rz, *pz, *qz, *xy, *ry, *py, *qy;
};

template <class T, class V>
gp2s_status launch_spmm(gp2s_ctx *c, int m, bool has_y, const V *val, const CGBuffers &B, double *part,
                        int pstride, int nb, int64_t rpb, const int *active)
{
    const Assembled &A = c->A;
    const int32_t *rp = c->rowptr.as<int32_t>(), *cl = c->col.as<int32_t>();
    const T *py = (const T *)B.py, *pz = (const T *)B.pz;
    T *qy = (T *)B.qy, *qz = (T *)B.qz;
#define GP2S_SPMM_CASE(KK, HY)                                                                    \
    k_spmm<T, V, KK, HY><<<nb, kSpmmThreads, 0, c->stream>>>(rp, cl, val, A.n, rpb, py, pz, qy, qz, \
                                                             part, pstride, active)
    int K = m / 32;
    // algorithmic bytes: values + column indices + row pointers + every input and output element once
    c->spmm_bytes += (double)A.nnz * (sizeof(V) + sizeof(int32_t)) + 4.0 * (double)(A.n + 1) +
                     2.0 * (double)A.n * (double)(m + (has_y ? 1 : 0)) * sizeof(T);
    ++c->spmm_launches;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    if (c->profile) {
        if (c->prof_used + 2 > c->prof_ev.size()) {
            for (int k = 0; k < 64; ++k) {
                cudaEvent_t e;
                GP2S_CUDA(c, cudaEventCreate(&e));
                c->prof_ev.push_back(e);
            }
        }
        ev_a = c->prof_ev[c->prof_used];
        ev_b = c->prof_ev[c->prof_used + 1];
        c->prof_used += 2;
        GP2S_CUDA(c, cudaEventRecord(ev_a, c->stream));
    }
    if (has_y) {
        switch (K) {
        case 0: GP2S_SPMM_CASE(0, true); break;
        case 1: GP2S_SPMM_CASE(1, true); break;
        case 2: GP2S_SPMM_CASE(2, true); break;
        case 3: GP2S_SPMM_CASE(3, true); break;
        default: GP2S_SPMM_CASE(4, true); break;
        }
    } else {
        switch (K) {
        case 1: GP2S_SPMM_CASE(1, false); break;
        case 2: GP2S_SPMM_CASE(2, false); break;
        case 3: GP2S_SPMM_CASE(3, false); break;
        default: GP2S_SPMM_CASE(4, false); break;
        }
    }
#undef GP2S_SPMM_CASE
    GP2S_LAUNCH(c);
    if (c->profile) GP2S_CUDA(c, cudaEventRecord(ev_b, c->stream));
    return GP2S_OK;
}

// Sum the recorded SpMM event pairs into c->prof_ms (synchronises on the last event).
gp2s_status flush_profile(gp2s_ctx *c)
{
    if (!c->profile || c->prof_used == 0) return GP2S_OK;
    GP2S_CUDA(c, cudaEventSynchronize(c->prof_ev[c->prof_used - 1]));
    for (size_t k = 0; k + 1 < c->prof_used; k += 2) {
        float ms = 0.0f;
        GP2S_CUDA(c, cudaEventElapsedTime(&ms, c->prof_ev[k], c->prof_ev[k + 1]));
        c->prof_ms += ms;
    }
    c->prof_used = 0;
    return GP2S_OK;
}

// One CG run (x0 = 0) on columns [y | probes]; the probe right-hand sides must already be in rz.
template <class T, class V>
gp2s_status cg_run(gp2s_ctx *c, int m, const V *val, const CGBuffers &B, const double *rhs_y, double tol_y,
                   double tol_z, int kmin_probe, int ksteps, double *rec, int max_iter, int *iters_y,
                   int *iters_z, bool *breakdown)
{
    const Assembled &A = c->A;
    const int64_t n = A.n;
    const int k = 1 + m;
    const int nb = (int)std::min<int64_t>(kMaxPartBlocks, std::max<int64_t>(1, ceil_div(n, 64)));
    const int64_t rpb = ceil_div(n, nb);
    const int pstride = kMaxPartBlocks;
    // update-kernel geometry
    const int ut = m > 0 ? m * std::max(1, 256 / m) : 256;
    const int nbz = m > 0 ? (int)std::min<int64_t>(152 * 4, std::max<int64_t>(1, ceil_div(n, ut / m))) : 0;
    const int nby = (int)std::min<int64_t>(152 * 2, std::max<int64_t>(1, ceil_div(n, ut)));
    GP2S_TRY(ensure(c, c->partials, sizeof(double) * (size_t)pstride * k));
    // fixed layout: scalars of column c at sc[c * kScal] for up to kMaxCols columns, then the
    // active flags, then the breakdown / active-count words (a later y-only run must not touch
    // the probe columns' records)
    GP2S_TRY(ensure(c, c->scal, sizeof(double) * kScal * kMaxCols + sizeof(int) * (kMaxCols + 8)));
    double *part = c->partials.as<double>();
    double *sc = c->scal.as<double>();
    int *active = reinterpret_cast<int *>(sc + kScal * kMaxCols);
    int *flags = active + k;       // [0] breakdown, [1] active count
    GP2S_CUDA(c, cudaMemsetAsync(flags, 0, sizeof(int) * 4, c->stream));

    k_cg_init<T><<<nbz + nby, ut, 0, c->stream>>>(n, m > 0 ? m : 1, rhs_y, (T *)B.xz, (T *)B.rz, (T *)B.pz,
                                                  (T *)B.xy, (T *)B.ry, (T *)B.py, part, pstride, nbz);
    GP2S_LAUNCH(c);
    k_scal_init<<<k, 256, 0, c->stream>>>(part, pstride, nby, nbz, sc, active, tol_y, tol_z);
    GP2S_LAUNCH(c);

    const int check_every = 8;
    int it = 0;
    int *hcount = reinterpret_cast<int *>(c->hbuf.p);
    for (; it < max_iter; ++it) {
        GP2S_TRY((launch_spmm<T, V>(c, m, true, val, B, part, pstride, nb, rpb, active)));
        k_scal_alpha<<<k, 256, 0, c->stream>>>(part, pstride, nb, sc, active, flags, rec, ksteps);
        GP2S_LAUNCH(c);
        GP2S_CUDA(c, cudaMemsetAsync(flags + 1, 0, sizeof(int), c->stream));
        k_update<T><<<nbz + nby, ut, 0, c->stream>>>(n, m > 0 ? m : 1, (T *)B.xz, (T *)B.rz, (const T *)B.pz,
                                                     (const T *)B.qz, (T *)B.xy, (T *)B.ry, (const T *)B.py,
                                                     (const T *)B.qy, sc, part, pstride, nbz);
        GP2S_LAUNCH(c);
        k_scal_beta<<<k, 256, 0, c->stream>>>(part, pstride, nby, nbz, sc, active, flags + 1, rec, ksteps,
                                              kmin_probe);
        GP2S_LAUNCH(c);
        {
            int64_t tot = n * (int64_t)(m + 1);
            unsigned gb = (unsigned)std::min<int64_t>(ceil_div(tot, 256), 152 * 8);
            k_direction<T><<<gb, 256, 0, c->stream>>>(n, m > 0 ? m : 1, (const T *)B.rz, (T *)B.pz,
                                                       (const T *)B.ry, (T *)B.py, sc, active);
            GP2S_LAUNCH(c);
        }
        if ((it + 1) % check_every == 0 || it + 1 == max_iter) {
            GP2S_CUDA(c, cudaMemcpyAsync(hcount, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->stream));
            GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
            GP2S_TRY(flush_profile(c));
            if (hcount[1] == 0) { ++it; break; }
        }
    }
    // iteration counts per column group
    std::vector<double> hs((size_t)kScal * k);
    GP2S_CUDA(c, cudaMemcpyAsync(hs.data(), sc, sizeof(double) * kScal * k, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaMemcpyAsync(hcount, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    GP2S_TRY(flush_profile(c));
    *iters_y = (int)hs[S_STEPS];
    int mz = 0;
    for (int cc = 1; cc < k; ++cc) mz = std::max(mz, (int)hs[cc * kScal + S_STEPS]);
    *iters_z = mz;
    *breakdown = hcount[0] != 0;
    return GP2S_OK;
}

}  // namespace

// r64 = b64 - Ah64 xhat (vec64 slots 0, 1 -> 2) and |r64 / s| / |y| (original-space relative
// residual of the y solve, FP64).
gp2s_status y_residual(gp2s_ctx *c, const double *y_sorted_dev, double *relres)
{
    const int64_t n = c->A.n;
    double *b64 = c->vec64.as<double>();
    double *xh = b64 + n, *r64 = b64 + 2 * n;
    const unsigned gbw = (unsigned)std::min<int64_t>(ceil_div(n * 32, 256), 152 * 32);
    const int nbr = 152 * 2;
    GP2S_TRY(ensure(c, c->gpart, sizeof(double) * (2 * nbr + 8)));
    double *rp = c->gpart.as<double>();
    k_residual64<<<gbw, 256, 0, c->stream>>>(c->rowptr.as<int32_t>(), c->col.as<int32_t>(), c->val64.as<double>(),
                                             n, xh, b64, r64);
    GP2S_LAUNCH(c);
    k_resnorm<<<nbr, 256, 0, c->stream>>>(n, r64, c->s64.as<double>(), y_sorted_dev, rp, nbr);
    GP2S_LAUNCH(c);
    k_sum_parts<<<1, 256, 0, c->stream>>>(rp, nbr, 2, rp + 2 * nbr);
    GP2S_LAUNCH(c);
    double h2[2];
    GP2S_CUDA(c, cudaMemcpyAsync(h2, rp + 2 * nbr, sizeof(h2), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    *relres = h2[1] > 0 ? std::sqrt(h2[0] / h2[1]) : 0.0;
    return GP2S_OK;
}

gp2s_status krylov_solve(gp2s_ctx *c, const double *y_sorted_dev, bool with_probes, int m, int ksteps,
                         CGResult *res)
{
    Assembled &A = c->A;
    const int64_t n = A.n;
    if (!with_probes) m = 0;
    const bool mixed = A.precision == GP2S_PREC_MIXED;
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    const int mm = m > 0 ? m : 0;
    // vectors: y group 4 n, probe group 4 n m
    GP2S_TRY(ensure(c, c->vec, es * (size_t)n * (4 + 4 * (size_t)mm) + 256));
    CGBuffers B;
    char *base = c->vec.as<char>();
    size_t nz = es * (size_t)n * mm;
    B.xz = base; B.rz = base + nz; B.pz = base + 2 * nz; B.qz = base + 3 * nz;
    char *yb = base + 4 * nz;
    B.xy = yb; B.ry = yb + es * n; B.py = yb + 2 * es * n; B.qy = yb + 3 * es * n;
    // FP64 refinement vectors: b64, xhat64, res64, a64 (solution in sorted order)
    GP2S_TRY(ensure(c, c->vec64, sizeof(double) * (size_t)n * 4 + 256));
    double *b64 = c->vec64.as<double>();
    double *xh = b64 + n, *r64 = b64 + 2 * n, *a64 = b64 + 3 * n;
    GP2S_TRY(ensure_host(c, c->hbuf, 4096));
    if (mm > 0) GP2S_TRY(ensure(c, c->rec, sizeof(double) * (size_t)mm * ksteps * 2 + 64));
    double *rec = mm > 0 ? c->rec.as<double>() : nullptr;
    if (rec) GP2S_CUDA(c, cudaMemsetAsync(rec, 0, sizeof(double) * (size_t)mm * ksteps * 2, c->stream));

    const unsigned gbn = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    k_scale64<<<gbn, 256, 0, c->stream>>>(n, c->s64.as<double>(), y_sorted_dev, b64);
    GP2S_LAUNCH(c);
    if (mm > 0) {
        unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n * mm, 256), 152 * 16);
        if (mixed)
            k_probes<float><<<gb, 256, 0, c->stream>>>(c->perm.as<int32_t>(), n, mm, A.opts.seed, (float *)B.rz);
        else
            k_probes<double><<<gb, 256, 0, c->stream>>>(c->perm.as<int32_t>(), n, mm, A.opts.seed, (double *)B.rz);
        GP2S_LAUNCH(c);
    }
    const gp2s_opts &o = A.opts;
    const double tol_first = mixed ? o.tol_inner : std::min(o.tol_inner, 0.1 * o.tol_refine);
    int iy = 0, iz = 0;
    bool brk = false;
    if (mixed)
        GP2S_TRY((cg_run<float, float>(c, mm, c->val32.as<float>(), B, b64, tol_first, o.tol_probe, mm > 0 ? ksteps : 0,
                                       ksteps, rec, o.max_iter, &iy, &iz, &brk)));
    else
        GP2S_TRY((cg_run<double, double>(c, mm, c->val64.as<double>(), B, b64, tol_first, o.tol_probe,
                                         mm > 0 ? ksteps : 0, ksteps, rec, o.max_iter, &iy, &iz, &brk)));
    res->iters_probes = iz;
    int total_y = iy;
    if (brk) {
        res->status = GP2S_EBREAKDOWN;
        return set_err(c, GP2S_EBREAKDOWN, "CG breakdown (p^T A p <= 0 or NaN)");
    }
    // xhat = x_y (FP64 accumulate)
    GP2S_CUDA(c, cudaMemsetAsync(xh, 0, sizeof(double) * n, c->stream));
    if (mixed) k_accum64<float><<<gbn, 256, 0, c->stream>>>(n, (const float *)B.xy, xh);
    else k_accum64<double><<<gbn, 256, 0, c->stream>>>(n, (const double *)B.xy, xh);
    GP2S_LAUNCH(c);

    // refinement: r = b - Ah xhat in FP64; original-space residual |r / s| / |y|
    double relres = 0.0;
    int outer = 0;
    for (;;) {
        GP2S_TRY(y_residual(c, y_sorted_dev, &relres));
        if (!(relres > o.tol_refine) || outer >= o.max_outer) break;
        ++outer;
        int iy2 = 0, iz2 = 0;
        if (mixed)
            GP2S_TRY((cg_run<float, float>(c, 0, c->val32.as<float>(), B, r64, o.tol_inner, o.tol_probe, 0, 0, nullptr,
                                           o.max_iter, &iy2, &iz2, &brk)));
        else
            GP2S_TRY((cg_run<double, double>(c, 0, c->val64.as<double>(), B, r64, std::min(o.tol_inner, 0.1 * o.tol_refine),
                                             o.tol_probe, 0, 0, nullptr, o.max_iter, &iy2, &iz2, &brk)));
        total_y += iy2;
        if (brk) return set_err(c, GP2S_EBREAKDOWN, "CG breakdown in refinement");
        if (mixed) k_accum64<float><<<gbn, 256, 0, c->stream>>>(n, (const float *)B.xy, xh);
        else k_accum64<double><<<gbn, 256, 0, c->stream>>>(n, (const double *)B.xy, xh);
        GP2S_LAUNCH(c);
    }
    // a = s * xhat (sorted order)
    k_scale64<<<gbn, 256, 0, c->stream>>>(n, c->s64.as<double>(), xh, a64);
    GP2S_LAUNCH(c);
    res->iters_y = total_y;
    res->outer = outer;
    res->relres = relres;
    c->have_solution = true;
    c->have_probes = mm > 0;
    c->solve_iters = total_y;
    c->solve_outer = outer;
    c->solve_relres = relres;
    c->probe_iters = iz;
    if (relres > o.tol_refine) {
        res->status = GP2S_ENOCONV;
        return set_err(c, GP2S_ENOCONV, "y solve did not reach tol_refine within max_outer refinement steps");
    }
    return GP2S_OK;
}

}  // namespace gp2s
