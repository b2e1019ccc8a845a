// krylov.cu -- multi-RHS conjugate gradients on the Jacobi-scaled matrix Ah = D^{-1/2} A D^{-1/2},
// FP64 residual refinement of the y column, Rademacher probes and the CG coefficient records that
// stochastic Lanczos quadrature needs.
//
// The paper solves K^{-1} y by MINRES on the host (App. B.7) and leaves the log-determinant method
// open (Sec. 4.6).  A = K + sigma^2 I is symmetric positive definite, so conjugate gradients solve
// the same system; running the y column and the m probe columns together lets one pass over the CSR
// serve all of them (the SpMM), and the CG step lengths / direction coefficients of each probe column
// are its Lanczos tridiagonal (the CG-Lanczos relation), which is what SLQ needs.
//
// Column 0 is y (right-hand side s * y, s = D^{-1/2}); columns 1..m are the probes z_s.  Vectors are
// row-major: the y group is n values, the probe group n x m values.  In MIXED precision vectors are
// FP32, dot products use compensated FP32 partial sums that are combined in FP64, and the scalars
// (alpha, beta, rho) are FP64.  In FP64 precision everything is FP64.
#include <climits>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "gp2s_internal.cuh"

namespace gp2s {

namespace {

constexpr int kSpmmThreads = 1024;
constexpr int kSpmmWarps = kSpmmThreads / kWarp;
constexpr int kMaxPartBlocks = 152 * 8;
constexpr int kRBWorkOffset = 224;   // byte offset of the RB8 SpMM's tile counter in c->counters
constexpr int kMaxCols = 129;   // y + up to 128 probes

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
    } else if constexpr (sizeof(T) == 4 && K % 4 == 0) {
#pragma unroll
        for (int k = 0; k < K; k += 4) {
            float4 t = reinterpret_cast<const float4 *>(p)[k / 4];
            v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
        }
    } else if constexpr (sizeof(T) == 4 && K % 2 == 0) {
#pragma unroll
        for (int k = 0; k < K; k += 2) {
            float2 t = reinterpret_cast<const float2 *>(p)[k / 2];
            v[k] = t.x; v[k + 1] = t.y;
        }
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
    } else if constexpr (sizeof(T) == 8 && K == 4) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    } else if constexpr (sizeof(T) == 4 && K % 4 == 0) {
#pragma unroll
        for (int k = 0; k < K; k += 4)
            reinterpret_cast<float4 *>(p)[k / 4] = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    } else if constexpr (sizeof(T) == 4 && K % 2 == 0) {
#pragma unroll
        for (int k = 0; k < K; k += 2) reinterpret_cast<float2 *>(p)[k / 2] = make_float2(v[k], v[k + 1]);
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
// One CTA per SM owns a contiguous range of rows holding an equal share of the entries
// (row_split), so the P rows its warps gather (the Morton neighbourhood of the range) stay in that
// SM's L1; its warps take consecutive rows round-robin.  Each warp stages 32 (column, value)
// entries of its row in shared memory and broadcasts them with one shared load per entry, with
// four independent P-row loads in flight.
// ---------------------------------------------------------------------------------------------
template <class T> struct Staged;
template <> struct Staged<float> { int j; float v; };
template <> struct Staged<double> { int j; int pad; double v; };

template <class T, class V, int M, bool HAS_Y>
__global__ void __launch_bounds__(kSpmmThreads, 1)
k_spmm(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const V *__restrict__ val,
       int64_t n, const int32_t *__restrict__ row_split, const T *__restrict__ py, const T *__restrict__ pz,
       T *__restrict__ qy, T *__restrict__ qz, double *__restrict__ part, int pstride,
       const int *__restrict__ active)
{
    using Acc = typename AccOf<T>::type;
    // K columns per lane; with M < 32 (or not a multiple of 32) the last lanes hold none
    constexpr int K = (M + 31) / 32;
    const bool lon = (int)(threadIdx.x & 31) * K < M;
    __shared__ Staged<T> stage[kSpmmWarps][kWarp];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r_begin = row_split[blockIdx.x];
    const int64_t r_end = row_split[blockIdx.x + 1];
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
            int cj = (int)i;     // padding entries: a valid row with value 0
            T cv = T(0);
            if (p < p1) {
                cj = col[p];
                cv = (T)val[p];
            }
            if (HAS_Y) accy += cv * py[cj];
            if (K > 0) {
                Staged<T> e;
                e.j = cj;
                e.v = cv;
                stage[wid][lane] = e;
                __syncwarp();
                const int cnt = min(kWarp, p1 - pb);
#pragma unroll 4
                for (int t = 0; t < cnt; ++t) {
                    const Staged<T> s = stage[wid][t];
                    T pv[K > 0 ? K : 1];
                    if (lon) load_k<T, (K > 0 ? K : 1)>(pz + (int64_t)s.j * M + lane * K, pv);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc[k] += lon ? s.v * pv[k] : T(0);
                }
                __syncwarp();
            }
        }
        if (K > 0 && lon) {
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
    // block reduction of the partial dots: y column (lane 0 of each warp) and probe columns, in
    // two halves to keep the shared buffer small (fixed order: deterministic)
    constexpr int HW = kSpmmWarps / 2;
    __shared__ double red[HW][M + 1];
    if (wid >= HW) {
        if (HAS_Y && lane == 0) red[wid - HW][M] = dy.value();
        if (lon) {
#pragma unroll
            for (int k = 0; k < K; ++k) red[wid - HW][lane * K + k] = dz[k].value();
        }
    }
    __syncthreads();
    if (wid < HW) {
        if (HAS_Y && lane == 0) red[wid][M] += dy.value();
        if (lon) {
#pragma unroll
            for (int k = 0; k < K; ++k) red[wid][lane * K + k] += dz[k].value();
        }
    }
    __syncthreads();
    for (int cidx = threadIdx.x; cidx < M + 1; cidx += kSpmmThreads) {
        if (cidx == M && !HAS_Y) continue;
        double s = 0.0;
        for (int w = 0; w < HW; ++w) s += red[w][cidx];
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
        for (int p = rowptr[i] + lane; p < rowptr[i + 1]; p += kWarp) s = fma(__ldcs(val + p), x[__ldcs(col + p)], s);
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
// For a preconditioned column (pc_y for column 0, pc_z for the probe columns) part holds r^T z
// and part_rr holds r^T r; for a plain CG column part holds r^T r.
__global__ void k_scal_init(const double *__restrict__ part, const double *__restrict__ part_rr, int pstride,
                            int nparts_y, int nparts_z, double *__restrict__ sc, int *__restrict__ active,
                            double tol_y, double tol_z, int pc_y, int pc_z)
{
    const int c = blockIdx.x;
    const int np = c == 0 ? nparts_y : nparts_z;
    const bool pc = c == 0 ? pc_y : pc_z;
    double s = block_sum(part + (int64_t)c * pstride, np);
    __syncthreads();
    double s2 = pc ? block_sum(part_rr + (int64_t)c * pstride, np) : s;
    if (threadIdx.x == 0) {
        double *q = sc + c * kScal;
        q[S_RHO] = s;
        q[S_B2] = s2;
        double tol = c == 0 ? tol_y : tol_z;
        q[S_TOL] = tol * tol * s2;
        q[S_ALPHA] = 0.0;
        q[S_BETA] = 0.0;
        q[S_STEPS] = 0.0;
        q[S_RR] = s2;
        q[S_RHO_PREV] = 0.0;
        q[S_STOP] = 0.0;
        active[c] = s > 0.0 ? 1 : 0;
    }
}

// alpha_c = rho_c / (p_c^T q_c).  p^T q <= 0 (or NaN) is a breakdown, except when the column's
// residual has already fallen to the rounding level of the vector precision (|r|^2 <= lucky
// |b|^2): then the Krylov space is exhausted and the column simply stops, with the steps it has
// recorded (a small problem, or an operator with few distinct eigenvalues).
__global__ void k_scal_alpha(const double *__restrict__ part, int pstride, int nparts, double *__restrict__ sc,
                             int *__restrict__ active, int *__restrict__ flags, double *__restrict__ rec,
                             int ksteps, double lucky)
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
            q[S_STOP] = 2.0;
            if (!(q[S_RR] <= lucky * q[S_B2])) atomicOr(&flags[0], 1);   // breakdown
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
__global__ void k_scal_beta(const double *__restrict__ part, const double *__restrict__ part_rr, int pstride,
                            int nparts_y, int nparts_z, double *__restrict__ sc, int *__restrict__ active,
                            int *__restrict__ count, double *__restrict__ rec, int ksteps, int kmin_probe, int pc_y,
                            int pc_z, double lucky)
{
    const int c = blockIdx.x;
    const int np = c == 0 ? nparts_y : nparts_z;
    const bool pc = c == 0 ? pc_y : pc_z;
    double s = block_sum(part + (int64_t)c * pstride, np);
    __syncthreads();
    double s2 = pc ? block_sum(part_rr + (int64_t)c * pstride, np) : s;
    if (threadIdx.x == 0) {
        double *q = sc + c * kScal;
        if (!active[c]) {
            q[S_BETA] = 0.0;
            return;
        }
        q[S_RR] = s2;
        double b = s / q[S_RHO];
        int st = (int)q[S_STEPS];
        if (c > 0 && rec && st < ksteps) rec[((int64_t)(c - 1) * ksteps + st) * 2 + 1] = b;
        q[S_BETA] = b;
        q[S_RHO_PREV] = q[S_RHO];
        q[S_RHO] = s;
        q[S_STEPS] = (double)(st + 1);
        bool conv = s2 <= q[S_TOL];
        int kmin = c == 0 ? 0 : kmin_probe;
        // a residual at the rounding level ends the column even before kmin steps: the steps after
        // it would only record rounding noise as Lanczos coefficients
        const bool exhausted = s2 <= lucky * q[S_B2];
        if ((conv && st + 1 >= kmin) || exhausted || !(s == s)) {
            active[c] = 0;
            q[S_STOP] = 1.0;
            // p is not updated for inactive columns (beta unused)
        } else {
            atomicAdd(count, 1);
            if (c > 0) atomicAdd(count + 1, 1);
        }
    }
}

// Restart of the probe columns as PCG: rho = r^T z for the still active columns.
__global__ void k_scal_restart(const double *__restrict__ part, int pstride, int nparts, double *__restrict__ sc,
                               const int *__restrict__ active)
{
    const int c = blockIdx.x + 1;
    double s = block_sum(part + (int64_t)c * pstride, nparts);
    if (threadIdx.x == 0 && active[c]) sc[c * kScal + S_RHO] = s;
}

// Reliable update of the y column (column 0) after its residual was replaced by the true one.
// The column stopped in the beta kernel of some step j, before that step's direction update: the
// recurrence continues there with the replaced residual, rho' = r'^T z', beta = rho' / rho_j
// (p = z' + beta p follows in the direction kernel).  A column that stopped in the alpha kernel
// (p^T A p at the rounding level) restarts its direction, beta = 0.  The new |r|^2 becomes the
// reference of the rounding-level rule (b2) and the column stops again once |r| has fallen by
// the factor delta.
__global__ void k_scal_replace(const double *__restrict__ part, const double *__restrict__ part_rr, int nparts,
                               double *__restrict__ sc, int *__restrict__ active, double delta)
{
    double s = block_sum(part, nparts);
    __syncthreads();
    double s2 = block_sum(part_rr, nparts);
    if (threadIdx.x == 0) {
        const bool cont = sc[S_STOP] == 1.0 && sc[S_RHO_PREV] > 0.0;
        sc[S_BETA] = cont ? s / sc[S_RHO_PREV] : 0.0;
        sc[S_RHO_PREV] = sc[S_RHO];
        sc[S_RHO] = s;
        sc[S_RR] = s2;
        sc[S_B2] = s2;
        sc[S_TOL] = delta * delta * s2;
        sc[S_ALPHA] = 0.0;
        sc[S_STOP] = 0.0;
        active[0] = s > 0.0 ? 1 : 0;
    }
}

// Plain-CG step of the FP32 probe group, four columns per thread: r -= alpha q and the partial
// r^T r of each column (x += alpha p is left to the direction kernel, which reads p anyway).
// Thread t owns columns 4 (t % (m/4)) .. +3 and strides over rows; per column the CTA's partial
// sums the threads in thread order.
__global__ void __launch_bounds__(256)
k_update_z4(int64_t n, int m, float *__restrict__ rz, const float *__restrict__ qz, const double *__restrict__ sc,
            double *__restrict__ part, int pstride)
{
    __shared__ double red[256 * 4];
    const int cgs = m / 4;
    const int rps = blockDim.x / cgs;
    const bool on = (int)threadIdx.x < cgs * rps;
    const int cg = threadIdx.x % cgs, r0 = threadIdx.x / cgs;
    float a4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a4[q] = (float)sc[(cg * 4 + q + 1) * kScal + S_ALPHA];
    Acc32 acc[4];
    if (on) {
        for (int64_t i = (int64_t)blockIdx.x * rps + r0; i < n; i += (int64_t)gridDim.x * rps) {
            const int64_t e = i * m + cg * 4;
            float r4[4], q4[4];
            load_k<float, 4>(rz + e, r4);
            load_k<float, 4>(qz + e, q4);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (a4[q] != 0.0f) r4[q] = r4[q] - a4[q] * q4[q];
                acc[q].fma2(r4[q], r4[q]);
            }
            store_k<float, 4>(rz + e, r4);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[threadIdx.x * 4 + q] = on ? acc[q].value() : 0.0;
    __syncthreads();
    if ((int)threadIdx.x < m) {
        const int g = threadIdx.x / 4, q = threadIdx.x % 4;
        double t = 0.0;
        for (int u = g; u < cgs * rps; u += cgs) t += red[u * 4 + q];
        part[(int64_t)(threadIdx.x + 1) * pstride + blockIdx.x] = t;
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

// p = r + beta p for active columns.  CTAs [0, gz) cover the probe group: thread t owns the four
// columns 4 (t % (m/4)) .. +3 for the whole launch (beta and the active flags stay in registers)
// and strides over rows; the remaining CTAs cover the y column.  With upd_x the probe group's
// x += alpha p (alpha of this iteration, 0 for a column that was already idle) is applied first,
// from the same read of p (the asynchronous block-Jacobi step leaves x to this kernel).
template <class T>
__global__ void k_direction(int64_t n, int m, const T *__restrict__ rz, T *__restrict__ pz, const T *__restrict__ ry,
                            T *__restrict__ py, const double *__restrict__ sc, const int *__restrict__ active, int gz,
                            T *__restrict__ xz, int upd_x)
{
    if ((int)blockIdx.x < gz) {
        const int cgs = m / 4;
        const int rows_per_step = blockDim.x / cgs;
        if ((int)threadIdx.x >= cgs * rows_per_step) return;
        const int cg = threadIdx.x % cgs;
        const int c0 = cg * 4;
        T b[4], al[4];
        bool act[4], all = true;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            act[q] = active[c0 + q + 1] != 0;
            b[q] = (T)sc[(c0 + q + 1) * kScal + S_BETA];
            al[q] = (T)sc[(c0 + q + 1) * kScal + S_ALPHA];
            all = all && act[q];
        }
        for (int64_t i = (int64_t)blockIdx.x * rows_per_step + threadIdx.x / cgs; i < n;
             i += (int64_t)gz * rows_per_step) {
            const int64_t e = i * m + c0;
            T r4[4], p4[4];
            load_k<T, 4>(rz + e, r4);
            load_k<T, 4>(pz + e, p4);
            if (upd_x) {
                T x4[4];
                load_k<T, 4>(xz + e, x4);
#pragma unroll
                for (int q = 0; q < 4; ++q) x4[q] = x4[q] + al[q] * p4[q];
                store_k<T, 4>(xz + e, x4);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) p4[q] = (all || act[q]) ? r4[q] + b[q] * p4[q] : p4[q];
            store_k<T, 4>(pz + e, p4);
        }
    } else {
        if (!active[0]) return;
        const T b = (T)sc[S_BETA];
        const int gy = gridDim.x - gz;
        for (int64_t i = (int64_t)(blockIdx.x - gz) * blockDim.x + threadIdx.x; i < n; i += (int64_t)gy * blockDim.x)
            py[i] = ry[i] + b * py[i];
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
    void *zz, *zy;   // preconditioned residuals (block-Jacobi PCG)
};

template <int KH, int NG>
gp2s_status launch_rb(gp2s_ctx *c, const CGBuffers &B, double *part, int pstride, int nb, int *nparts);
template <int NG>
gp2s_status launch_rb4_et(gp2s_ctx *c, const CGBuffers &B, double *part, int pstride, int nb, int *nparts, int *err,
                          int et, bool *done);

// y-only SpMV (the y column after every probe column has stopped, and the refinement solves):
// one warp per row, lanes over the row's entries, many warps per SM to keep enough independent
// loads in flight; per-CTA partial dot p^T q.
constexpr int kSpmvThreads = 256;
constexpr int kSpmvBlocks = 152 * 8;
template <class T, class V>
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv_y(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const V *__restrict__ val, int64_t n,
         const T *__restrict__ py, T *__restrict__ qy, double *__restrict__ part)
{
    using Acc = typename AccOf<T>::type;
    __shared__ double sh[kSpmvThreads / kWarp];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Acc d;
    for (int64_t i = w0; i < n; i += nw) {
        const int p1 = rowptr[i + 1];
        T s = T(0);
        // four independent entries per lane in flight (rows of up to 128 entries in one pass)
        for (int p = rowptr[i] + lane; p < p1; p += 4 * kWarp) {
            V v[4];
            int cj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = p + u * kWarp;
                v[u] = q < p1 ? __ldcs(val + q) : V(0);
                cj[u] = q < p1 ? __ldcs(col + q) : 0;
            }
            T g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) g[u] = py[cj[u]];
#pragma unroll
            for (int u = 0; u < 4; ++u) s += (T)v[u] * g[u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            qy[i] = s;
            d.fma2(py[i], s);
        }
    }
    if (lane == 0) sh[wid] = d.value();
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kSpmvThreads / kWarp; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// The FP32 multi-RHS SpMM runs on the RB8 copy when it has been built.
template <class T>
bool rb_launch(gp2s_ctx *c, int m, bool has_y)
{
    return std::is_same<T, float>::value && c->rb_valid && m > 0 && has_y;
}

// Row ranges of the SpMM CTAs with equal shares of the entries: split[b] = first row whose entries
// start at or after b * nnz / nb.
__global__ void k_row_split(const int32_t *__restrict__ rowptr, int64_t n, int nb, int32_t *__restrict__ split)
{
    const int64_t nnz = rowptr[n];
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) {
        if (b == 0) { split[0] = 0; continue; }
        if (b == nb) { split[nb] = (int32_t)n; continue; }
        const int64_t target = nnz * b / nb;
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (rowptr[mid] < target) lo = mid + 1; else hi = mid;
        }
        split[b] = (int32_t)lo;
    }
}

template <class T, class V>
gp2s_status launch_spmm(gp2s_ctx *c, int m, bool has_y, const V *val, const CGBuffers &B, double *part,
                        int pstride, int nb, const int32_t *rsplit, const int *active, int *nparts, int *err)
{
    *nparts = nb;
    const Assembled &A = c->A;
    const int32_t *rp = c->rowptr.as<int32_t>(), *cl = c->col.as<int32_t>();
    const T *py = (const T *)B.py, *pz = (const T *)B.pz;
    T *qy = (T *)B.qy, *qz = (T *)B.qz;
#define GP2S_SPMM_CASE(MM, HY)                                                                    \
    k_spmm<T, V, MM, HY><<<nb, kSpmmThreads, 0, c->stream>>>(rp, cl, val, A.n, rsplit, py, pz, qy, qz, \
                                                             part, pstride, active)
    // multi-RHS launches: algorithmic bytes = values + column indices + row pointers + every input
    // and output element once
    const bool counted = m > 0;
    if (counted) {
        c->spmm_bytes += (double)A.nnz * (sizeof(V) + sizeof(int32_t)) + 4.0 * (double)(A.n + 1) +
                         2.0 * (double)A.n * (double)(m + (has_y ? 1 : 0)) * sizeof(T);
        ++c->spmm_launches;
    }
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    if (c->profile && counted) {
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
    if (rb_launch<T>(c, m, has_y)) {
        // 16, 32 and 64 columns can take the gather-copy form (ET copied rows per 32-entry batch)
        bool done = false;
        if (c->spmm_tma > 0 && !c->spmm_half) {
            const int et = c->spmm_tma;
            switch (m) {
            case 16: GP2S_TRY((launch_rb4_et<8>(c, B, part, pstride, nb, nparts, err, et, &done))); break;
            case 32: GP2S_TRY((launch_rb4_et<4>(c, B, part, pstride, nb, nparts, err, et, &done))); break;
            case 64: GP2S_TRY((launch_rb4_et<2>(c, B, part, pstride, nb, nparts, err, et, &done))); break;
            default: break;
            }
        }
        if (!done) switch (m) {
        // every lane covers KH = 4 columns where the column count allows (groups of 4, 8 or 16
        // lanes per entry); 48 and 96 columns take half-warps with KH = 3 and 6
        case 16:
            GP2S_TRY((c->spmm_half ? launch_rb<1, 2>(c, B, part, pstride, nb, nparts)
                                   : launch_rb<4, 8>(c, B, part, pstride, nb, nparts)));
            break;
        case 32:
            GP2S_TRY((c->spmm_half ? launch_rb<2, 2>(c, B, part, pstride, nb, nparts)
                                   : launch_rb<4, 4>(c, B, part, pstride, nb, nparts)));
            break;
        case 48: GP2S_TRY((launch_rb<3, 2>(c, B, part, pstride, nb, nparts))); break;
        case 64: GP2S_TRY((launch_rb<4, 2>(c, B, part, pstride, nb, nparts))); break;
        case 96: GP2S_TRY((launch_rb<6, 2>(c, B, part, pstride, nb, nparts))); break;
        default: GP2S_TRY((launch_rb<8, 2>(c, B, part, pstride, nb, nparts))); break;
        }
        if (ev_b) GP2S_CUDA(c, cudaEventRecord(ev_b, c->stream));
        return GP2S_OK;
    }
    if (has_y && m == 0) {
        const int nbv = (int)std::min<int64_t>(std::min(kSpmvBlocks, pstride),
                                               std::max<int64_t>(1, ceil_div(A.n * kWarp, kSpmvThreads)));
        k_spmv_y<T, V><<<nbv, kSpmvThreads, 0, c->stream>>>(rp, cl, val, A.n, py, qy, part);
        GP2S_LAUNCH(c);
        *nparts = nbv;
        if (ev_b) GP2S_CUDA(c, cudaEventRecord(ev_b, c->stream));
        return GP2S_OK;
    }
    if (has_y) {
        switch (m) {
        case 0: GP2S_SPMM_CASE(0, true); break;
        case 16: GP2S_SPMM_CASE(16, true); break;
        case 32: GP2S_SPMM_CASE(32, true); break;
        case 48: GP2S_SPMM_CASE(48, true); break;
        case 64: GP2S_SPMM_CASE(64, true); break;
        case 96: GP2S_SPMM_CASE(96, true); break;
        default: GP2S_SPMM_CASE(128, true); break;
        }
    } else {
        switch (m) {
        case 16: GP2S_SPMM_CASE(16, false); break;
        case 32: GP2S_SPMM_CASE(32, false); break;
        case 48: GP2S_SPMM_CASE(48, false); break;
        case 64: GP2S_SPMM_CASE(64, false); break;
        case 96: GP2S_SPMM_CASE(96, false); break;
        default: GP2S_SPMM_CASE(128, false); break;
        }
    }
#undef GP2S_SPMM_CASE
    GP2S_LAUNCH(c);
    if (ev_b) GP2S_CUDA(c, cudaEventRecord(ev_b, c->stream));
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

// ---------------------------------------------------------------------------------------------
// Row-block (RB8) SpMM for the FP32 multi-RHS solves.
//
// With m = 64 probe columns every stored entry of the CSR makes the warp gather a 256-byte row of
// P through L1, and the SpMM is L1-bandwidth bound.  Consecutive rows in Morton order share most
// of their columns, so the RB8 copy of Ah groups 8 consecutive rows into a block that stores the
// union of their column lists once, with the 8 values of each union column (0 for a row that does
// not hold it).  A gathered P row then feeds 8 rows from registers: the L1 traffic per stored entry
// drops about four-fold at the cost of some multiplications by zero.
// ---------------------------------------------------------------------------------------------
constexpr int kRB = 8;

// Union of the 8 sorted column lists of a row block by a warp-wide 8-way merge: lane r < 8 holds
// the head of row r; each step emits the smallest head, with the value of every row that holds it.
template <bool FILL>
__global__ void __launch_bounds__(256)
k_rb_build(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const float *__restrict__ val,
           int64_t n, int64_t nblk, int32_t *__restrict__ cnt, const int32_t *__restrict__ bptr,
           int32_t *__restrict__ ucol, float *__restrict__ uval)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = w0; b < nblk; b += nw) {
        const int64_t r = b * kRB + lane;
        int pos = 0, end = 0;
        if (lane < kRB && r < n) {
            pos = rowptr[r];
            end = rowptr[r + 1];
        }
        int head = pos < end ? col[pos] : INT_MAX;
        int64_t e = FILL ? bptr[b] : 0;
        int emitted = 0;
        for (;;) {
            int mn = head;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            if (mn == INT_MAX) break;
            const bool mine = head == mn;
            if (FILL) {
                if (lane < kRB) uval[e * kRB + lane] = mine ? val[pos] : 0.0f;
                if (lane == 0) ucol[e] = mn;
                ++e;
            }
            if (mine) {
                ++pos;
                head = pos < end ? col[pos] : INT_MAX;
            }
            ++emitted;
        }
        if (!FILL && lane == 0) cnt[b] = emitted;
    }
}

template <int K> struct RBCfg {
    static constexpr int threads = 512;   // 16 warps, ~128 registers each: deep unrolled gathers
    static constexpr int warps = threads / kWarp;
};

// Work distribution of the RB8 SpMM.  The row blocks are cut into tiles of `tile_blocks`
// consecutive blocks; warps take tiles from a global counter in increasing order (the next index
// is fetched while the current tile runs), so an SM that runs slower, or a warp that drew denser
// blocks, takes fewer tiles instead of holding the whole launch back, and the tiles in flight stay
// a narrow window of the Morton order whose gathered P rows stay in L2.  The partial dots must
// not depend on which warp ran which tile: every tile writes its own (tpart[tile][col]), and the
// warp that completes the last tile of a segment of `seg_tiles` tiles sums the segment's tiles in
// tile order into part[col * pstride + segment], which the scalar kernels sum in segment order.
// The last CTA to finish puts the tile counter back to zero for the next launch on the stream;
// each segment's reducer does the same for its segment counter.
struct RBWork {
    unsigned long long next;   // next tile index
    unsigned int done;         // CTAs finished
    unsigned int pad;
};

// ---------------------------------------------------------------------------------------------
// mbarrier and bulk-copy helpers.  Every wait is bounded: after about a second without the phase
// completing the caller sets an error flag that the host turns into GP2S_ETIMEOUT.
// ---------------------------------------------------------------------------------------------
constexpr uint32_t kPPMaxSpins = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of bar; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t spin = 0; spin < kPPMaxSpins; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if (spin > 32) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Row block bcur of the RB8 SpMM is complete: a butterfly over the warp's NG entry groups (lane
// masks 16, 8, 4) leaves each group the full sums of 8 / NG rows, which it stores and folds into the
// tile's dots; the row accumulators go back to zero.
template <int KH, int NG, bool HAS_Y>
__device__ __forceinline__ void rb_block_end(float2 (&acc)[kRB / 2][KH], float (&ay)[kRB], Acc32 (&dz)[KH], Acc32 &dy,
                                             int64_t bcur, int64_t n, const float *__restrict__ py,
                                             const float *__restrict__ pz, float *__restrict__ qy,
                                             float *__restrict__ qz, int lane)
{
    constexpr int LG = kWarp / NG;
    constexpr int M = LG * KH;
    const int gl = lane % LG;
    const int64_t r0 = bcur * kRB;
    const int nrows = (int)(n - r0 < kRB ? n - r0 : kRB);
    const int b16 = (lane >> 4) & 1, b8 = (lane >> 3) & 1, b4 = (lane >> 2) & 1;
    float2 h2[2][KH];   // rows 4 b16 + 2q, 4 b16 + 2q + 1
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < KH; ++k) {
            const float2 keep = b16 ? acc[2 + q][k] : acc[q][k];
            const float2 send = b16 ? acc[q][k] : acc[2 + q][k];
            float2 got;
            got.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
            got.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
            h2[q][k] = make_float2(keep.x + got.x, keep.y + got.y);
        }
    if constexpr (NG == 2) {
#pragma unroll
        for (int rr = 0; rr < kRB / 2; ++rr) {
            const int r = 4 * b16 + rr;
            if (r < nrows) {
                const int64_t i = r0 + r;
                float qr[KH];
#pragma unroll
                for (int k = 0; k < KH; ++k) qr[k] = (rr & 1) ? h2[rr / 2][k].y : h2[rr / 2][k].x;
                store_k<float, KH>(qz + i * M + gl * KH, qr);
                float pi[KH];
                load_k<float, KH>(pz + i * M + gl * KH, pi);
#pragma unroll
                for (int k = 0; k < KH; ++k) dz[k].fma2(pi[k], qr[k]);
            }
        }
    } else {
        float2 h1[KH];   // rows 4 b16 + 2 b8, + 1
#pragma unroll
        for (int k = 0; k < KH; ++k) {
            const float2 keep = b8 ? h2[1][k] : h2[0][k];
            const float2 send = b8 ? h2[0][k] : h2[1][k];
            float2 got;
            got.x = __shfl_xor_sync(0xffffffffu, send.x, 8);
            got.y = __shfl_xor_sync(0xffffffffu, send.y, 8);
            h1[k] = make_float2(keep.x + got.x, keep.y + got.y);
        }
        if constexpr (NG == 4) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int r = 4 * b16 + 2 * b8 + rr;
                if (r < nrows) {
                    const int64_t i = r0 + r;
                    float qr[KH];
#pragma unroll
                    for (int k = 0; k < KH; ++k) qr[k] = rr ? h1[k].y : h1[k].x;
                    store_k<float, KH>(qz + i * M + gl * KH, qr);
                    float pi[KH];
                    load_k<float, KH>(pz + i * M + gl * KH, pi);
#pragma unroll
                    for (int k = 0; k < KH; ++k) dz[k].fma2(pi[k], qr[k]);
                }
            }
        } else {
            float qr[KH];   // row 4 b16 + 2 b8 + b4
#pragma unroll
            for (int k = 0; k < KH; ++k) {
                const float keep = b4 ? h1[k].y : h1[k].x;
                const float send = b4 ? h1[k].x : h1[k].y;
                qr[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            const int r = 4 * b16 + 2 * b8 + b4;
            if (r < nrows) {
                const int64_t i = r0 + r;
                store_k<float, KH>(qz + i * M + gl * KH, qr);
                float pi[KH];
                load_k<float, KH>(pz + i * M + gl * KH, pi);
#pragma unroll
                for (int k = 0; k < KH; ++k) dz[k].fma2(pi[k], qr[k]);
            }
        }
    }
#pragma unroll
    for (int rp = 0; rp < kRB / 2; ++rp)
#pragma unroll
        for (int k = 0; k < KH; ++k) acc[rp][k] = make_float2(0.0f, 0.0f);
    if (HAS_Y) {
#pragma unroll
        for (int r = 0; r < kRB; ++r) {
            float v = ay[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && r < nrows) {
                qy[r0 + r] = v;
                dy.fma2(py[r0 + r], v);
            }
            ay[r] = 0.0f;
        }
    }
}

// The tile's dot of each probe column (the groups' rows combined in a fixed order: lane masks 16,
// then 8, then 4, the lower group first) goes to part directly when every tile is a segment of its
// own, else to tpart[t], and the segment's last tile sums its tiles in tile order into part.
template <int KH, int NG, bool HAS_Y>
__device__ __forceinline__ void rb_tile_end(Acc32 (&dz)[KH], Acc32 &dy, unsigned long long t,
                                            double *__restrict__ part, int pstride, double *__restrict__ tpart,
                                            int *__restrict__ seg_cnt, int seg_tiles, int ntiles, int lane)
{
    constexpr int LG = kWarp / NG;
    constexpr int M = LG * KH;
    const int grp = lane / LG, gl = lane % LG;
    double dzt[KH];
#pragma unroll
    for (int k = 0; k < KH; ++k) {
        double v = dz[k].value();
#pragma unroll
        for (int o = 16; o >= LG; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = (lane & o) ? w + v : v + w;
        }
        dzt[k] = v;
    }
    if (seg_tiles == 1) {
        // every tile is a segment of its own: its partial dots go straight to part
        if (grp == 0) {
#pragma unroll
            for (int k = 0; k < KH; ++k) part[(int64_t)(1 + gl * KH + k) * pstride + (int64_t)t] = dzt[k];
        }
        if (lane == 0) part[(int64_t)t] = HAS_Y ? dy.value() : 0.0;
        return;
    }
    // the tile's partial dots, then the segment count; the segment's last tile reduces it
    double *tp = tpart + (int64_t)t * (M + 1);
    if (grp == 0) {
#pragma unroll
        for (int k = 0; k < KH; ++k) tp[1 + gl * KH + k] = dzt[k];
    }
    if (lane == 0) tp[0] = HAS_Y ? dy.value() : 0.0;
    __threadfence();
    __syncwarp();
    const int sg = (int)(t / (unsigned long long)seg_tiles);
    const int nseg = (ntiles + seg_tiles - 1) / seg_tiles;
    const int need = sg == nseg - 1 ? ntiles - sg * seg_tiles : seg_tiles;
    int last = 0;
    if (lane == 0) last = atomicAdd(&seg_cnt[sg], 1) == need - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
        __threadfence();
        const double *q = tpart + (int64_t)sg * seg_tiles * (M + 1);
        // column cc = lane, lane + 32, ...: the segment's tiles in tile order
        for (int cc = lane; cc < M; cc += kWarp) {
            double sz = 0.0;
#pragma unroll 4
            for (int i = 0; i < need; ++i) sz += __ldcg(q + (int64_t)i * (M + 1) + 1 + cc);
            part[(int64_t)(1 + cc) * pstride + sg] = sz;
        }
        if (lane == 0) {
            double sy = 0.0;
            for (int i = 0; i < need; ++i) sy += __ldcg(q + (int64_t)i * (M + 1));
            part[sg] = sy;
            seg_cnt[sg] = 0;
        }
    }
}

template <int KH, int NG, bool HAS_Y>
__global__ void __launch_bounds__(RBCfg<KH>::threads, 1)
k_spmm_rb(const int32_t *__restrict__ bptr, const int32_t *__restrict__ ucol, const float *__restrict__ uval,
          int64_t n, const float *__restrict__ py, const float *__restrict__ pz, float *__restrict__ qy,
          float *__restrict__ qz, double *__restrict__ part, int pstride, RBWork *__restrict__ work,
          int tile_blocks, int ntiles, double *__restrict__ tpart, int *__restrict__ seg_cnt, int seg_tiles)
{
    // The warp splits into NG groups of LG = 32 / NG lanes.  Each group covers all M = LG KH probe
    // columns (KH per lane) and the groups take interleaved union entries of the same row block:
    // one shared-memory broadcast of an entry's column and 8 values feeds 8 x KH products per
    // lane, and every lane keeps PD independent 4 KH-byte gathers in flight.  NG = 2 (half-warps)
    // for M >= 48; M = 32 and M = 16 take NG = 4 and 8 with KH = 4, so that every lane does the
    // same 16 packed FMAs per gathered entry whatever the column count.
    // (A double-buffered form with 4 + 4 gathers spilled registers at KH = 4 and measured slower:
    // 1.03 against 0.90 ms per launch at N = 1M.)
    constexpr int LG = kWarp / NG;
    constexpr int M = LG * KH;
    // runs of PD entries per group, at most the 32 / NG entries of a staged batch
    constexpr int PD = (KH >= 6 ? 4 : 8) < kWarp / NG ? (KH >= 6 ? 4 : 8) : kWarp / NG;
    constexpr int W = RBCfg<KH>::warps;
    static_assert(NG == 2 || NG == 4 || NG == 8, "entry groups of 16, 8 or 4 lanes");
    static_assert((kWarp / NG) % PD == 0, "runs tile the staged batch");
    extern __shared__ __align__(16) unsigned char rb_sh[];
    int *s_col = reinterpret_cast<int *>(rb_sh);                                    // W x 32
    float4 *s_val = reinterpret_cast<float4 *>(rb_sh + sizeof(int) * W * kWarp);  // W x 32 x 2
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int grp = lane / LG, gl = lane % LG;
    const int64_t nblk = (n + kRB - 1) / kRB;
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(&work->next, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    while (t < (unsigned long long)ntiles) {
        unsigned long long tn = 0;
        if (lane == 0) tn = atomicAdd(&work->next, 1ull);
        const int64_t bb = (int64_t)t * tile_blocks;
        const int64_t be = bb + tile_blocks < nblk ? bb + tile_blocks : nblk;
        Acc32 dz[KH];
        Acc32 dy;
        // the tile's entries are contiguous: stream them in 32-entry batches that never straddle
        // a block, the next batch's column and values loaded while the current one is consumed
        // (evict-first: the matrix is read once per launch, the gathered P rows are what L2
        // should keep; 4.67 -> 4.37 ms per launch at N = 10M); lanes past the block's last entry
        // stage a zero entry on the block's first row
        int64_t b = bb;
        int e1 = bptr[b + 1];
        int eb = bptr[b];
        int cj_n = (int)(b * kRB);
        float4 v0_n = make_float4(0.f, 0.f, 0.f, 0.f), v1_n = v0_n;
        if (eb + lane < e1) {
            cj_n = __ldcs(ucol + eb + lane);
            v0_n = __ldcs(reinterpret_cast<const float4 *>(uval) + (int64_t)(eb + lane) * 2);
            v1_n = __ldcs(reinterpret_cast<const float4 *>(uval) + (int64_t)(eb + lane) * 2 + 1);
        }
        // accumulators of row pairs (2p, 2p + 1) for each of the lane's columns: one packed FP32x2
        // FMA per pair (each half rounds exactly like a scalar fmaf)
        float2 acc[kRB / 2][KH];
        float ay[kRB];
#pragma unroll
        for (int r = 0; r < kRB; ++r) ay[r] = 0.0f;
#pragma unroll
        for (int rp = 0; rp < kRB / 2; ++rp)
#pragma unroll
            for (int k = 0; k < KH; ++k) acc[rp][k] = make_float2(0.0f, 0.0f);
        while (b < be) {
            const int cj = cj_n;
            const float4 v0 = v0_n, v1 = v1_n;
            const int cnt = min(kWarp, e1 - eb);
            const int64_t bcur = b;
            // advance to the next batch and issue its loads
            eb += kWarp;
            const bool block_end = eb >= e1;
            if (block_end) {
                ++b;
                if (b < be) {
                    eb = e1;
                    e1 = bptr[b + 1];
                }
            }
            cj_n = (int)(b * kRB);
            v0_n = make_float4(0.f, 0.f, 0.f, 0.f);
            v1_n = v0_n;
            if (b < be && eb + lane < e1) {
                cj_n = __ldcs(ucol + eb + lane);
                v0_n = __ldcs(reinterpret_cast<const float4 *>(uval) + (int64_t)(eb + lane) * 2);
                v1_n = __ldcs(reinterpret_cast<const float4 *>(uval) + (int64_t)(eb + lane) * 2 + 1);
            }
            if (HAS_Y) {
                const float yj = py[cj];
                ay[0] = fmaf(v0.x, yj, ay[0]); ay[1] = fmaf(v0.y, yj, ay[1]);
                ay[2] = fmaf(v0.z, yj, ay[2]); ay[3] = fmaf(v0.w, yj, ay[3]);
                ay[4] = fmaf(v1.x, yj, ay[4]); ay[5] = fmaf(v1.y, yj, ay[5]);
                ay[6] = fmaf(v1.z, yj, ay[6]); ay[7] = fmaf(v1.w, yj, ay[7]);
            }
            s_col[wid * kWarp + lane] = cj;
            s_val[(wid * kWarp + lane) * 2] = v0;
            s_val[(wid * kWarp + lane) * 2 + 1] = v1;
            __syncwarp();
            // group g takes entries NG u + g, u < ceil(cnt / NG), in runs of PD (the staged entries
            // past cnt are zeros, so a run may pass cnt)
            const int nrun = (cnt + NG - 1) / NG;
            const int *scol = s_col + wid * kWarp + grp;
            const float4 *sval = s_val + (wid * kWarp + grp) * 2;
#pragma unroll 1
            for (int u0 = 0; u0 < nrun; u0 += PD) {
                int jj[PD];
#pragma unroll
                for (int d = 0; d < PD; ++d) jj[d] = scol[NG * (u0 + d)];
                float pv[PD][KH];
#pragma unroll
                for (int d = 0; d < PD; ++d) load_k<float, KH>(pz + (int64_t)jj[d] * M + gl * KH, pv[d]);
#pragma unroll
                for (int d = 0; d < PD; ++d) {
                    const float4 a0 = sval[2 * NG * (u0 + d)], a1 = sval[2 * NG * (u0 + d) + 1];
                    const float2 vp[kRB / 2] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w),
                                                make_float2(a1.x, a1.y), make_float2(a1.z, a1.w)};
#pragma unroll
                    for (int k = 0; k < KH; ++k) {
                        const float2 pk = make_float2(pv[d][k], pv[d][k]);
#pragma unroll
                        for (int rp = 0; rp < kRB / 2; ++rp) acc[rp][k] = __ffma2_rn(vp[rp], pk, acc[rp][k]);
                    }
                }
            }
            __syncwarp();
            if (block_end) rb_block_end<KH, NG, HAS_Y>(acc, ay, dz, dy, bcur, n, py, pz, qy, qz, lane);
        }
        rb_tile_end<KH, NG, HAS_Y>(dz, dy, t, part, pstride, tpart, seg_cnt, seg_tiles, ntiles, lane);
        t = __shfl_sync(0xffffffffu, tn, 0);
    }
    // every warp of this CTA has made its last (failed) grab: count the CTA out, and let the last
    // one reset the counter for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(&work->done, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&work->next, 0ull);
            atomicExch(&work->done, 0u);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// RB8 SpMM with part of the gathered probe rows brought in by the tensor-memory accelerator.  Row
// blocks, tiles, entry groups, the order of every FMA and the reductions are those of k_spmm_rb,
// so the results are the same; what changes is where a gathered row comes from.  Of a warp's
// 32-entry batch, the first ET rows are fetched by tile::gather4 tensor copies (four rows each,
// issued by lanes 0, 4, ..., ET - 4) into one of the warp's two shared-memory slots during the
// previous batch; the other rows are gathered into registers at the start of the batch and are
// in flight while the copied rows are multiplied.  The two paths to memory work side by side: the
// copy engine's cost per row bounds the copies (all 32 rows by copies measured slower than the
// register gathers alone), the registers bound the loads in flight.  The matrix stream's columns
// run two batches ahead (a batch's copies are issued an iteration before it), its values one.
// Every wait on a slot's mbarrier is bounded: a warp whose copies do not land sets err, waits
// (bounded) for its copies in flight and stops.
// ---------------------------------------------------------------------------------------------
template <int NG, int ET> struct RB4Cfg {
    static constexpr int KH = 4;
    static constexpr int M = kWarp / NG * KH;                      // 64, 32 or 16 probe columns
    static constexpr int RG = (kWarp - ET) / NG;                   // register-gathered entries per group
    static constexpr uint32_t slot = ET * M * sizeof(float);      // the copied rows of one batch
    static constexpr int warps = 12;                               // up to 168 registers a thread
    static constexpr int threads = warps * kWarp;
    static constexpr size_t per_warp =
        2 * slot + 2 * kWarp * sizeof(float4) + kWarp * sizeof(int) + 2 * sizeof(uint64_t);
    static constexpr size_t smem = 128 + (size_t)warps * per_warp;
    static_assert(ET > 0 && ET <= kWarp && ET % 4 == 0 && ET % NG == 0,
                  "copied entries: whole gather4 copies and whole runs of every group");
};

// Four rows r0..r3, columns x .. x + box - 1 of the tensor map's 2-D tensor, to dst (four boxes
// back to back); completion is counted in bytes on bar.
__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *tm, int x, int r0, int r1, int r2, int r3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}

// One 32-entry batch of a row block: the lane's entry's column and where the batch sits.
struct RB4Batch {
    int cj;                    // column (past the batch's entries: the block's first row)
    int eb;                    // the batch's first entry
    int b, t;                  // row block, tile
    int cnt;                   // entries of the batch; 0: no batch
    bool bend, tend;           // the block's / the tile's last batch
};

template <int NG, int ET, bool HAS_Y>
__global__ void __launch_bounds__(RB4Cfg<NG, ET>::threads, 1)
k_spmm_rb4(const __grid_constant__ CUtensorMap tmz, const int32_t *__restrict__ bptr,
           const int32_t *__restrict__ ucol, const float *__restrict__ uval, int64_t n, const float *__restrict__ py,
           const float *__restrict__ pz, float *__restrict__ qy, float *__restrict__ qz, double *__restrict__ part,
           int pstride, RBWork *__restrict__ work, int tile_blocks, int ntiles, double *__restrict__ tpart,
           int *__restrict__ seg_cnt, int seg_tiles, int *__restrict__ err)
{
    using C = RB4Cfg<NG, ET>;
    constexpr int KH = C::KH, M = C::M, W = C::warps, LG = kWarp / NG, RG = C::RG, EC = ET / NG;
    extern __shared__ __align__(16) unsigned char rb4_sh[];
    unsigned char *base = rb4_sh + ((128u - (smem_addr(rb4_sh) & 127u)) & 127u);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int grp = lane / LG, gl = lane % LG;
    float *ring = reinterpret_cast<float *>(base + (size_t)wid * 2 * C::slot);   // this warp's two slots
    unsigned char *tail = base + (size_t)W * 2 * C::slot;
    float4 *s_val = reinterpret_cast<float4 *>(tail) + wid * 2 * kWarp;
    tail += (size_t)W * 2 * kWarp * sizeof(float4);
    int *s_col = reinterpret_cast<int *>(tail) + wid * kWarp;
    tail += (size_t)W * kWarp * sizeof(int);
    uint64_t *bar = reinterpret_cast<uint64_t *>(tail) + wid * 2;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t nblk = (n + kRB - 1) / kRB;
    const float4 *uval4 = reinterpret_cast<const float4 *>(uval);

    // The cursor (warp-uniform): the next batch to read from the matrix stream.  The tile after the
    // cursor's is taken from the counter on entering a tile, and the end of the block after the
    // cursor's is read on entering a block, so that neither load is waited for at once.
    unsigned long long ct, ctn = 0;
    int64_t cb = 0, cbe = 0;
    int ceb = 0, ce1 = 0, ce2 = 0;
    bool cval;
    auto grab = [&]() {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(&work->next, 1ull);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    auto enter = [&]() {
        ctn = grab();
        cb = (int64_t)ct * tile_blocks;
        cbe = cb + tile_blocks < nblk ? cb + tile_blocks : nblk;
        ceb = bptr[cb];
        ce1 = bptr[cb + 1];
        ce2 = cb + 1 < cbe ? bptr[cb + 2] : 0;
    };
    auto advance = [&]() {
        ceb += kWarp;
        if (ceb >= ce1) {
            ++cb;
            if (cb < cbe) {
                ceb = ce1;
                ce1 = ce2;
                ce2 = cb + 1 < cbe ? bptr[cb + 2] : 0;
            } else {
                ct = ctn;
                cval = ct < (unsigned long long)ntiles;
                if (cval) enter();
            }
        }
    };
    // the batch at the cursor (its columns: evict-first loads, the matrix is read once per
    // launch), then the cursor moves on
    auto take = [&]() {
        RB4Batch q;
        q.cj = 0;
        q.eb = 0;
        q.b = 0;
        q.t = 0;
        q.cnt = 0;
        q.bend = q.tend = false;
        if (!cval) return q;
        q.cj = (int)(cb * kRB);
        if (ceb + lane < ce1) q.cj = __ldcs(ucol + ceb + lane);
        q.eb = ceb;
        q.cnt = min(kWarp, ce1 - ceb);
        q.b = (int)cb;
        q.t = (int)ct;
        q.bend = ceb + kWarp >= ce1;
        q.tend = q.bend && cb + 1 >= cbe;
        advance();
        return q;
    };
    // the values of the lane's entry of a batch (zeros past its entries)
    auto values = [&](const RB4Batch &q, float4 &v0, float4 &v1) {
        v0 = make_float4(0.f, 0.f, 0.f, 0.f);
        v1 = v0;
        if (lane < q.cnt) {
            v0 = __ldcs(uval4 + (int64_t)(q.eb + lane) * 2);
            v1 = __ldcs(uval4 + (int64_t)(q.eb + lane) * 2 + 1);
        }
    };
    // the copies of a batch's first ET rows into slot s
    auto issue = [&](const RB4Batch &q, int s) {
        const int r1 = __shfl_down_sync(0xffffffffu, q.cj, 1);
        const int r2 = __shfl_down_sync(0xffffffffu, q.cj, 2);
        const int r3 = __shfl_down_sync(0xffffffffu, q.cj, 3);
        if (lane == 0) mbar_expect_tx(&bar[s], C::slot);
        __syncwarp();
        if ((lane & 3) == 0 && lane < ET)
            tma_gather4(ring + (size_t)s * ET * M + lane * M, &tmz, 0, q.cj, r1, r2, r3, &bar[s]);
    };

    ct = grab();
    cval = ct < (unsigned long long)ntiles;
    if (cval) enter();
    RB4Batch cur = take();
    RB4Batch nxt = take();
    float4 v0, v1;
    values(cur, v0, v1);
    float yj = 0.0f;
    if (cur.cnt) {
        issue(cur, 0);
        if (HAS_Y) yj = py[cur.cj];
    }
    Acc32 dz[KH];
    Acc32 dy;
    float2 acc[kRB / 2][KH];
    float ay[kRB];
#pragma unroll
    for (int r = 0; r < kRB; ++r) ay[r] = 0.0f;
#pragma unroll
    for (int rp = 0; rp < kRB / 2; ++rp)
#pragma unroll
        for (int k = 0; k < KH; ++k) acc[rp][k] = make_float2(0.0f, 0.0f);
    // acc[rp][.] += (values of rows 2 rp, 2 rp + 1 of staged entry e) x (the lane's KH columns of its row)
    auto fma_entry = [&](int e, const float (&pv)[KH]) {
        const float4 a0 = s_val[2 * e], a1 = s_val[2 * e + 1];
        const float2 vp[kRB / 2] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                                    make_float2(a1.z, a1.w)};
#pragma unroll
        for (int kk = 0; kk < KH; ++kk) {
            const float2 pk = make_float2(pv[kk], pv[kk]);
#pragma unroll
            for (int rp = 0; rp < kRB / 2; ++rp) acc[rp][kk] = __ffma2_rn(vp[rp], pk, acc[rp][kk]);
        }
    };
    uint32_t k = 0;
    bool failed = false;
    while (cur.cnt) {
        // batch k + 1's copies go out (its columns were read an iteration ago)
        if (nxt.cnt) issue(nxt, (k + 1) & 1);
        // stage batch k's columns and values
        s_col[lane] = cur.cj;
        s_val[lane * 2] = v0;
        s_val[lane * 2 + 1] = v1;
        if (HAS_Y) {
            ay[0] = fmaf(v0.x, yj, ay[0]); ay[1] = fmaf(v0.y, yj, ay[1]);
            ay[2] = fmaf(v0.z, yj, ay[2]); ay[3] = fmaf(v0.w, yj, ay[3]);
            ay[4] = fmaf(v1.x, yj, ay[4]); ay[5] = fmaf(v1.y, yj, ay[5]);
            ay[6] = fmaf(v1.z, yj, ay[6]); ay[7] = fmaf(v1.w, yj, ay[7]);
        }
        __syncwarp();
        // group g's entries NG u + g: u < EC from the copies, the RG after them gathered into
        // registers now; entries past cnt are skipped (zero values)
        const int nrun = (cur.cnt + NG - 1) / NG;
        float pv[RG > 0 ? RG : 1][KH];
#pragma unroll
        for (int d = 0; d < RG; ++d) {
            const int e = ET + NG * d + grp;
            if (e < cur.cnt) {
                load_k<float, KH>(pz + (int64_t)s_col[e] * M + gl * KH, pv[d]);
            } else {
#pragma unroll
                for (int kk = 0; kk < KH; ++kk) pv[d][kk] = 0.0f;
            }
        }
        // batch k + 1's values and y values, batch k + 2's columns
        float4 v0n, v1n;
        values(nxt, v0n, v1n);
        const float yj_n = HAS_Y && nxt.cnt ? py[nxt.cj] : 0.0f;
        const RB4Batch nn = take();
        const int s = (int)(k & 1);
        if (!mbar_wait_bounded(&bar[s], (k >> 1) & 1)) {
            failed = true;
            break;
        }
        const float *rs = ring + (size_t)s * ET * M + gl * KH;
#pragma unroll 4
        for (int u = 0; u < EC; ++u) {
            if (u < nrun) {
                const float4 p4 = *reinterpret_cast<const float4 *>(rs + (NG * u + grp) * M);
                const float pc[KH] = {p4.x, p4.y, p4.z, p4.w};
                fma_entry(NG * u + grp, pc);
            }
        }
#pragma unroll
        for (int d = 0; d < RG; ++d)
            if (EC + d < nrun) fma_entry(ET + NG * d + grp, pv[d]);
        // the slot's reads are ordered before the copies that will refill it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (cur.bend) rb_block_end<KH, NG, HAS_Y>(acc, ay, dz, dy, (int64_t)cur.b, n, py, pz, qy, qz, lane);
        if (cur.tend) {
            rb_tile_end<KH, NG, HAS_Y>(dz, dy, (unsigned long long)cur.t, part, pstride, tpart, seg_cnt, seg_tiles,
                                       ntiles, lane);
#pragma unroll
            for (int kk = 0; kk < KH; ++kk) dz[kk] = Acc32();
            dy = Acc32();
        }
        cur = nxt;
        nxt = nn;
        v0 = v0n;
        v1 = v1n;
        yj = yj_n;
        ++k;
    }
    if (failed) {
        if (lane == 0) atomicExch(err, 1);
        // the copies this warp still has in flight must land before the CTA's shared memory goes
        mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1);
        if (nxt.cnt) mbar_wait_bounded(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1);
    }
    // every warp of this CTA has made its last grab: count the CTA out, and let the last one reset
    // the counter for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(&work->done, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&work->next, 0ull);
            atomicExch(&work->done, 0u);
        }
    }
}

template <int KH>
size_t rb_smem()
{
    constexpr int W = RBCfg<KH>::warps;
    return sizeof(int) * W * kWarp + sizeof(float4) * W * kWarp * 2;
}

// Tiles of the RB8 SpMM: about 32 per warp of the grid (a warp's last tile is a small share of
// its work, so the SMs finish together), and segments of seg_tiles tiles, at most kMaxPartBlocks
// of them (the partial-dot stride).
// A small matrix takes fewer CTAs (about eight row blocks per warp): the SMs it leaves free run
// the other problems' kernels when many problems share the GPU on separate streams.
struct RBTiles {
    int ctas, tile_blocks, ntiles, seg_tiles, nseg;
};
inline RBTiles rb_tiles(int64_t nblk, int nb)
{
    RBTiles t;
    t.ctas = (int)std::max<int64_t>(1, std::min<int64_t>(nb, ceil_div(nblk, (int64_t)RBCfg<1>::warps * 8)));
    const int64_t want = (int64_t)t.ctas * RBCfg<1>::warps * 32;
    int64_t tb = std::max<int64_t>(1, ceil_div(nblk, want));
    // a small matrix takes tiles large enough that every tile is its own segment (no segment
    // counters, fences or second reduction pass), as long as every warp still gets a tile
    const int64_t tb_one = ceil_div(nblk, kMaxPartBlocks);
    if (ceil_div(nblk, tb_one) >= (int64_t)t.ctas * RBCfg<1>::warps) tb = std::max<int64_t>(tb, tb_one);
    t.tile_blocks = (int)tb;
    t.ntiles = (int)ceil_div(nblk, tb);
    t.seg_tiles = (int)ceil_div(t.ntiles, kMaxPartBlocks);
    t.nseg = (int)ceil_div(t.ntiles, t.seg_tiles);
    return t;
}

template <int KH, int NG>
gp2s_status launch_rb(gp2s_ctx *c, const CGBuffers &B, double *part, int pstride, int nb, int *nparts)
{
    constexpr int M = kWarp / NG * KH;
    const size_t smem = rb_smem<KH>();
    auto kern = k_spmm_rb<KH, NG, true>;
    GP2S_TRY(smem_attr(c, (const void *)kern, smem));
    const RBTiles tl = rb_tiles(ceil_div(c->A.n, kRB), nb);
    GP2S_TRY(ensure(c, c->rb_tpart, sizeof(double) * (size_t)tl.ntiles * (M + 1)));
    RBWork *work = reinterpret_cast<RBWork *>(c->counters.as<char>() + kRBWorkOffset);
    kern<<<tl.ctas, RBCfg<KH>::threads, smem, c->stream>>>(c->rb_ptr.as<int32_t>(), c->rb_col.as<int32_t>(),
                                                     c->rb_val.as<float>(), c->A.n, (const float *)B.py,
                                                     (const float *)B.pz, (float *)B.qy, (float *)B.qz, part,
                                                     pstride, work, tl.tile_blocks, tl.ntiles,
                                                     c->rb_tpart.as<double>(), c->rb_seg.as<int>(), tl.seg_tiles);
    GP2S_LAUNCH(c);
    *nparts = tl.nseg;
    c->spmm_seg_tiles = std::max(c->spmm_seg_tiles, tl.seg_tiles);
    return GP2S_OK;
}

// The tensor map of the row-major n x M FP32 probe block for the gather copies (one box = one row);
// false when the driver has no encoder or the block does not fit the map's limits.
static bool rb4_map(CUtensorMap *tm, const float *p, int64_t n, int M)
{
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    if (!encode || n <= 0 || n > INT_MAX || (reinterpret_cast<uintptr_t>(p) & 15u) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)M * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)M, 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(p), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The gather-copy form of the RB8 SpMM (M = 16, 32, 64; ET of every 32 gathered rows by copies);
// *done = false when it cannot run here (no tensor-map encoder, or an ET without a kernel), and
// the register-gather form takes the launch.
template <int NG, int ET>
gp2s_status launch_rb4(gp2s_ctx *c, const CGBuffers &B, double *part, int pstride, int nb, int *nparts, int *err,
                       bool *done)
{
    using C = RB4Cfg<NG, ET>;
    *done = false;
    CUtensorMap tm;
    if (!err || !rb4_map(&tm, (const float *)B.pz, c->A.n, C::M)) return GP2S_OK;
    auto kern = k_spmm_rb4<NG, ET, true>;
    GP2S_TRY(smem_attr(c, (const void *)kern, C::smem));
    const RBTiles tl = rb_tiles(ceil_div(c->A.n, kRB), nb);
    GP2S_TRY(ensure(c, c->rb_tpart, sizeof(double) * (size_t)tl.ntiles * (C::M + 1)));
    RBWork *work = reinterpret_cast<RBWork *>(c->counters.as<char>() + kRBWorkOffset);
    kern<<<tl.ctas, C::threads, C::smem, c->stream>>>(tm, c->rb_ptr.as<int32_t>(), c->rb_col.as<int32_t>(),
                                                     c->rb_val.as<float>(), c->A.n, (const float *)B.py,
                                                     (const float *)B.pz, (float *)B.qy, (float *)B.qz, part,
                                                     pstride, work, tl.tile_blocks, tl.ntiles,
                                                     c->rb_tpart.as<double>(), c->rb_seg.as<int>(), tl.seg_tiles, err);
    GP2S_LAUNCH(c);
    *nparts = tl.nseg;
    c->spmm_seg_tiles = std::max(c->spmm_seg_tiles, tl.seg_tiles);
    *done = true;
    return GP2S_OK;
}

template <int NG>
gp2s_status launch_rb4_et(gp2s_ctx *c, const CGBuffers &B, double *part, int pstride, int nb, int *nparts, int *err,
                          int et, bool *done)
{
    *done = false;
    // half or all of every batch's rows by copies (8 and 24 measured no faster than 16)
    switch (et) {
    case 16: return launch_rb4<NG, 16>(c, B, part, pstride, nb, nparts, err, done);
    case 32: return launch_rb4<NG, 32>(c, B, part, pstride, nb, nparts, err, done);
    default: return GP2S_OK;
    }
}

// ---------------------------------------------------------------------------------------------
// Block-Jacobi preconditioner on Morton-consecutive blocks of BJ = 64 or 128 rows.
//
// The paper leaves the solver's preconditioning open.  M = blockdiag(Ah_bb) = L L^T over blocks
// of BJ consecutive rows of the Morton order: spatially close points whose mutual covariances are
// the largest entries of their rows, so these small dense blocks cut the iteration count
// several-fold against plain Jacobi scaling.  The probe columns run their first k steps as plain
// CG on Ah (those coefficients are Ah's Lanczos tridiagonal for SLQ; SLQ on the preconditioned
// operator L^{-1} Ah L^{-T} would have a far larger probe variance) and are then restarted as PCG
// with M to finish the solves the gradient needs; the y column runs PCG throughout.
// ---------------------------------------------------------------------------------------------
constexpr int kPCThreads = 256;

// One CTA per block of BJ rows (BJ = 64 or 128): the dense block of Ah (FP32 values) from the
// CSR, Cholesky L L^T, L^{-1} in place, then M^{-1} = L^{-T} L^{-1} (symmetric bit for bit: both
// triangles come from the same products in the same order) and the block's log|M_b|.  FP32 is
// enough for a preconditioner (a block's condition number is bounded by about 1 / sigma^2 of the
// Jacobi-scaled matrix) and runs on the full-rate FP32 pipes; rows beyond n (last block) are
// padded with the identity.
template <int BJ>
__global__ void __launch_bounds__(kPCThreads)
k_bj_build(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const float *__restrict__ val32,
           int64_t n, float *__restrict__ Minv32, double *__restrict__ logdet_blk,
           int *__restrict__ bad)
{
    extern __shared__ float bjf_sh[];
    float (*S)[BJ + 1] = reinterpret_cast<float (*)[BJ + 1]>(bjf_sh);   // L, then L^{-1} (lower)
    float *tmp = bjf_sh + BJ * (BJ + 1);                                // one column of L
    const int64_t b = blockIdx.x;
    const int64_t i0 = b * BJ;
    const int nb = (int)(n - i0 < BJ ? n - i0 : BJ);
    for (int t = threadIdx.x; t < BJ * BJ; t += blockDim.x) {
        int i = t / BJ, j = t % BJ;
        S[i][j] = (i == j && i >= nb) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = wid; i < nb; i += kPCThreads / kWarp) {
        for (int p = rowptr[i0 + i] + lane; p < rowptr[i0 + i + 1]; p += kWarp) {
            int64_t j = col[p] - i0;
            if (j >= 0 && j < nb) S[i][j] = val32[p];
        }
    }
    __syncthreads();
    // right-looking Cholesky of the lower triangle; the trailing update visits only the
    // (BJ - j - 1)^2 square below and right of the pivot
    for (int j = 0; j < BJ; ++j) {
        if (threadIdx.x == 0) {
            float d = S[j][j];
            if (!(d > 0.0f)) { atomicOr(bad, 1); d = 1.0f; }
            S[j][j] = sqrtf(d);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < BJ; i += blockDim.x) S[i][j] /= S[j][j];
        __syncthreads();
        const int w = BJ - j - 1;
        for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
            const int i = j + 1 + t / w, k = j + 1 + t % w;
            if (k <= i) S[i][k] -= S[i][j] * S[k][j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double ld = 0.0;
        for (int i = 0; i < nb; ++i) ld += log((double)S[i][i]);
        logdet_blk[b] = 2.0 * ld;
    }
    // V = L^{-1} in place, columns from the last to the first: V L = I gives V_jj = 1 / L_jj and
    // V_ij = -(sum_{k=j+1..i} V_ik L_kj) / L_jj, which needs only the columns of V to the right of
    // j (already in place) and column j of L (saved in tmp first).
    for (int j = BJ - 1; j >= 0; --j) {
        for (int k = j + threadIdx.x; k < BJ; k += blockDim.x) tmp[k] = S[k][j];
        __syncthreads();
        const float ljj = tmp[j];
        for (int i = j + 1 + threadIdx.x; i < BJ; i += blockDim.x) {
            float s = 0.0f;
            for (int k = j + 1; k <= i; ++k) s = fmaf(S[i][k], tmp[k], s);
            S[i][j] = -s / ljj;
        }
        if (threadIdx.x == 0) S[j][j] = 1.0f / ljj;
        __syncthreads();
    }
    float *Mb = Minv32 + b * BJ * BJ;
    for (int t = threadIdx.x; t < BJ * BJ; t += blockDim.x) {
        int i = t / BJ, j = t % BJ;
        // (L^{-T} L^{-1})_ij = sum_k V[k][i] V[k][j], k >= max(i, j)
        float s = 0.0f;
        for (int k = i > j ? i : j; k < BJ; ++k) s = fmaf(S[k][i], S[k][j], s);
        Mb[t] = s;
    }
}

// Out (BJ x m, row stride m) = Mat (BJ x BJ, given transposed in shared memory: MT[k][i] =
// Mat[i][k]) x In (BJ x m in shared memory).  Each thread owns 4 x 4 output tiles.
template <int BJ, class Fn>
__device__ __forceinline__ void bj_tile_mm(const float *__restrict__ MT, const float *__restrict__ In, int m, Fn &&emit)
{
    const int cgroups = m / 4;
    const int tiles = (BJ / 4) * cgroups;
    for (int tt = threadIdx.x; tt < tiles; tt += blockDim.x) {
        const int rg = tt / cgroups, cg = tt - rg * cgroups;
        const int i0 = rg * 4, c0 = cg * 4;
        // row pairs (0,1), (2,3) accumulate with packed FP32x2 FMAs (each half rounds like fmaf)
        float2 acc2[2][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc2[a][q] = make_float2(0.0f, 0.0f);
#pragma unroll 8
        for (int k = 0; k < BJ; ++k) {
            const float4 mv = *reinterpret_cast<const float4 *>(MT + k * BJ + i0);
            const float4 iv = *reinterpret_cast<const float4 *>(In + k * m + c0);
            const float2 mp[2] = {make_float2(mv.x, mv.y), make_float2(mv.z, mv.w)};
            const float ia[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 iq = make_float2(ia[q], ia[q]);
#pragma unroll
                for (int a = 0; a < 2; ++a) acc2[a][q] = __ffma2_rn(mp[a], iq, acc2[a][q]);
            }
        }
        float acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[0][q] = acc2[0][q].x;
            acc[1][q] = acc2[0][q].y;
            acc[2][q] = acc2[1][q].x;
            acc[3][q] = acc2[1][q].y;
        }
        emit(i0, c0, acc);
    }
}

// Fused PCG step on BJ-row blocks.  INIT: x = 0, r = rhs, z = M^{-1} r, p = z.  UPDATE:
// r -= alpha q, z = M^{-1} r (the probe group's x += alpha p is done by the direction kernel; the
// y column's here).  RESTART (a CG column switching to PCG): x and r kept,
// z = M^{-1} r, p = z.  All emit per-CTA partial dots r^T z and r^T r per column.
// CTAs [0, gz) work on the probe group (n x m), CTAs [gz, gridDim) on the y column.
// REPLACE (y column only): r = rhs (the true residual), x = 0, z = M^{-1} r; p is kept (a reliable
// update of the y column's recursion).
enum { PC_INIT = 0, PC_UPDATE = 1, PC_RESTART = 2, PC_REPLACE = 3 };
template <int MODE, int BJ>
__global__ void __launch_bounds__(kPCThreads, 3)
k_pc_step(int64_t n, int m, int64_t nblk, int gz, const float *__restrict__ Minv32, float *__restrict__ xz,
          float *__restrict__ rz, float *__restrict__ pz, const float *__restrict__ qz, float *__restrict__ zz,
          float *__restrict__ xy, float *__restrict__ ry, float *__restrict__ py, const float *__restrict__ qy,
          float *__restrict__ zy, const double *__restrict__ rhs_y, const double *__restrict__ sc,
          double *__restrict__ part_rz, double *__restrict__ part_rr, int pstride, int wy)
{
    constexpr bool SETP = MODE == PC_INIT || MODE == PC_RESTART;   // p = z
    extern __shared__ __align__(16) float pc_sh[];
    if ((int)blockIdx.x < gz) {
        float *MT = pc_sh;                       // M^{-1} (symmetric, so no transpose)
        float *R = pc_sh + BJ * BJ;              // BJ x m residual block
        float *Pd = R + BJ * m;                  // (BJ / 4) x m partial dot rows (r^T z)
        // wy (UPDATE only): the y column's update rides along on the staged M^{-1} block, its
        // residual block staged after Pd; threads [0, BJ) own its rows in the elementwise phase and
        // the last BJ threads form z_y = M^{-1} r_y beside the probes' product
        float *Ry = Pd + (BJ / 4) * m;
        double yrr = 0.0, yrz = 0.0;
        const double alpha_y = (MODE == PC_UPDATE && wy) ? sc[S_ALPHA] : 0.0;
        const int yu = (int)threadIdx.x - ((int)blockDim.x - BJ);
        double acc_rz = 0.0, acc_rr = 0.0;       // thread c < m: this CTA's column sums
        // elementwise phase: thread t owns the 4 columns 4 (t % cgs) .. +3 of rows t / cgs + k rps
        const int cgs = m / 4;
        const int rps = kPCThreads / cgs;
        const int ecg = threadIdx.x % cgs, er0 = threadIdx.x / cgs;
        const bool eth = er0 < rps;
        float a4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            a4[q] = MODE == PC_UPDATE ? (float)sc[(ecg * 4 + q + 1) * kScal + S_ALPHA] : 0.0f;
        for (int64_t b = blockIdx.x; b < nblk; b += gz) {
            const int64_t i0 = b * BJ;
            const int nb = (int)(n - i0 < BJ ? n - i0 : BJ);
            const float4 *Mg = reinterpret_cast<const float4 *>(Minv32 + b * BJ * BJ);
            for (int t = threadIdx.x; t < BJ * BJ / 4; t += blockDim.x) reinterpret_cast<float4 *>(MT)[t] = __ldcs(Mg + t);
            if (eth) {
                for (int i = er0; i < BJ; i += rps) {
                    float r4[4] = {0.f, 0.f, 0.f, 0.f};
                    if (i < nb) {
                        const int64_t e = (i0 + i) * m + ecg * 4;
                        load_k<float, 4>(rz + e, r4);
                        if (MODE == PC_INIT) {
                            const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
                            store_k<float, 4>(xz + e, zero4);   // the right-hand side was written into r
                        } else if (MODE == PC_UPDATE) {
                            // r -= alpha q (x += alpha p is left to the direction kernel, which
                            // reads p anyway)
                            float q4[4];
                            load_k<float, 4>(qz + e, q4);
#pragma unroll
                            for (int q = 0; q < 4; ++q) r4[q] = r4[q] - a4[q] * q4[q];
                            store_k<float, 4>(rz + e, r4);
                        }
                    }
                    *reinterpret_cast<float4 *>(R + i * m + ecg * 4) = make_float4(r4[0], r4[1], r4[2], r4[3]);
                }
            }
            if (MODE == PC_UPDATE && wy && (int)threadIdx.x < BJ) {
                const int i = threadIdx.x;
                float r = 0.0f;
                if (i < nb) {
                    const int64_t e = i0 + i;
                    r = ry[e];
                    if (alpha_y != 0.0) {
                        const float a = (float)alpha_y;
                        xy[e] = xy[e] + a * py[e];
                        r = r - a * qy[e];
                        ry[e] = r;
                    }
                    yrr = fma((double)r, (double)r, yrr);
                }
                Ry[i] = r;
            }
            __syncthreads();
            // z = M^{-1} r, written with the partial dots of this block
            bj_tile_mm<BJ>(MT, R, m, [&](int it, int c0, float (&acc)[4][4]) {
                float drz[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (it + a >= nb) continue;
                    const int64_t e = (i0 + it + a) * m + c0;
                    *reinterpret_cast<float4 *>(zz + e) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
                    if (SETP)
                        *reinterpret_cast<float4 *>(pz + e) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) drz[q] = fmaf(R[(it + a) * m + c0 + q], acc[a][q], drz[q]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) Pd[(it / 4) * m + c0 + q] = drz[q];
            });
            if (MODE == PC_UPDATE && wy && yu >= 0) {
                // z_y[u] = sum_k M^{-1}[k][u] r_y[k] (the y column's own step sums the same way)
                float z = 0.0f;
#pragma unroll 8
                for (int k = 0; k < BJ; ++k) z = fmaf(MT[k * BJ + yu], Ry[k], z);
                if (yu < nb) {
                    zy[i0 + yu] = z;
                    yrz = fma((double)Ry[yu], (double)z, yrz);
                }
            }
            __syncthreads();
            if ((int)threadIdx.x < m) {
                float srz = 0.0f, srr = 0.0f;
                for (int g = 0; g < BJ / 4; ++g) srz += Pd[g * m + threadIdx.x];
                for (int i = 0; i < nb; ++i) {
                    const float rv = R[i * m + threadIdx.x];
                    srr = fmaf(rv, rv, srr);
                }
                acc_rz += (double)srz;
                acc_rr += (double)srr;
            }
            __syncthreads();
        }
        if ((int)threadIdx.x < m) {
            part_rz[(int64_t)(threadIdx.x + 1) * pstride + blockIdx.x] = acc_rz;
            part_rr[(int64_t)(threadIdx.x + 1) * pstride + blockIdx.x] = acc_rr;
        }
        if (MODE == PC_UPDATE && wy) {
            // the y column's partials of this CTA: warp sums, then the warps in order
            __shared__ double yred[2][kPCThreads / kWarp];
            double v1 = yrz, v2 = yrr;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                v2 += __shfl_xor_sync(0xffffffffu, v2, o);
            }
            if ((threadIdx.x & 31) == 0) {
                yred[0][threadIdx.x >> 5] = v1;
                yred[1][threadIdx.x >> 5] = v2;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double s1 = 0.0, s2 = 0.0;
                for (int w = 0; w < (int)(blockDim.x / kWarp); ++w) { s1 += yred[0][w]; s2 += yred[1][w]; }
                part_rz[blockIdx.x] = s1;
                part_rr[blockIdx.x] = s2;
            }
        }
    } else {
        // y column: the CTA's BJ-thread groups each take one block; thread i of a group owns
        // row i and forms z_i = sum_k Minv[k][i] r_k (coalesced rows of the symmetric M^{-1})
        constexpr int G = kPCThreads / BJ;
        float *R = pc_sh;                         // G x BJ
        __shared__ double red[2][kPCThreads / kWarp];
        const int gy = gridDim.x - gz;
        const int cb = blockIdx.x - gz;
        const int sub = threadIdx.x / BJ;
        double arz = 0.0, arr = 0.0;
        const double alpha = MODE == PC_UPDATE ? sc[S_ALPHA] : 0.0;
        const float a = (float)alpha;
        for (int64_t bg = cb; bg * G < nblk; bg += gy) {
            const int64_t b = bg * G + sub;
            const bool live = b < nblk;
            const int64_t i0 = b * BJ;
            const int nb = live ? (int)(n - i0 < BJ ? n - i0 : BJ) : 0;
            {
                const int i = threadIdx.x % BJ;
                float r = 0.0f;
                if (i < nb) {
                    const int64_t e = i0 + i;
                    if (MODE == PC_INIT || MODE == PC_REPLACE) {
                        r = (float)rhs_y[e];
                        ry[e] = r;
                        xy[e] = 0.0f;
                    } else if (MODE == PC_RESTART) {
                        r = ry[e];
                    } else {
                        r = ry[e];
                        if (alpha != 0.0) {
                            xy[e] = xy[e] + a * py[e];
                            r = r - a * qy[e];
                            ry[e] = r;
                        }
                    }
                }
                R[sub * BJ + i] = r;
            }
            __syncthreads();
            if (live) {
                const int i = threadIdx.x % BJ;
                float z = 0.0f;
                const float *Mb = Minv32 + b * BJ * BJ;
                const float *Rb = R + sub * BJ;
#pragma unroll 8
                for (int k = 0; k < BJ; ++k) z = fmaf(__ldcs(Mb + k * BJ + i), Rb[k], z);
                if (i < nb) {
                    zy[i0 + i] = z;
                    if (SETP) py[i0 + i] = z;
                    arz = fma((double)Rb[i], (double)z, arz);
                    arr = fma((double)Rb[i], (double)Rb[i], arr);
                }
            }
            __syncthreads();
        }
        double v1 = arz, v2 = arr;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = v1;
            red[1][threadIdx.x >> 5] = v2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s1 = 0.0, s2 = 0.0;
            for (int w = 0; w < kPCThreads / kWarp; ++w) { s1 += red[0][w]; s2 += red[1][w]; }
            part_rz[cb] = s1;
            part_rr[cb] = s2;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Probe-group PCG update with the bulk-copy engine: r -= alpha q, z = M^{-1} r and the partial
// dots r^T z, r^T r on BJ-row blocks (x += alpha p is done by the direction kernel).  One
// persistent CTA per SM takes blocks b = blockIdx.x + k gridDim.x; two shared-memory stages hold
// M^{-1}_b (BJ x BJ) and r_b (BJ x m, contiguous in the row-major probe block), filled by
// cp.async.bulk copies that one thread issues for block k + 2 as soon as block k has released the
// stage, so the HBM reads of later blocks run under the product of the current one.  q of the
// next block is prefetched into registers.  Every wait on a stage's mbarrier is bounded: after
// about a second without the copy completing the kernel sets err and returns.
// ---------------------------------------------------------------------------------------------
constexpr int kPPThreads = 512;

// two stages of (M^{-1} block, residual block), the y column's two staged residual blocks and its
// split products (WY), the two mbarriers
template <int BJ, int SB, int M>
size_t pp_smem()
{
    return sizeof(float) * (2 * ((size_t)BJ * SB + (size_t)BJ * M) + 2 * (size_t)BJ + 4 * (size_t)BJ) + 64;
}

// WY: the y column's PCG update rides along on the same staged M^{-1} blocks (when it uses the
// probes' factors): x_y += alpha_y p_y, r_y -= alpha_y q_y by the producers, z_y = M^{-1} r_y by the
// consumers (each half of them sums half of the block's columns), partial dots in column 0 of
// part_rz / part_rr.  This saves the y column's own pass over all of M^{-1} per iteration.
// Stages of BJ = 128 rows; the block-Jacobi blocks are SB = 128 or 64 rows (a stage then holds two
// consecutive 64 x 64 blocks of M^{-1}, contiguous in memory, and each tile multiplies within its
// own block).
template <int BJ, int SB, int M, bool WY>
__global__ void __launch_bounds__(kPPThreads, 1)
k_pc_probe(int64_t n, int64_t nblk, const float *__restrict__ Minv32, float *__restrict__ rz,
           const float *__restrict__ qz, float *__restrict__ zz, const double *__restrict__ sc,
           double *__restrict__ part_rz, double *__restrict__ part_rr, int pstride, int *__restrict__ err,
           float *__restrict__ xy, float *__restrict__ ry, const float *__restrict__ py, const float *__restrict__ qy,
           float *__restrict__ zy)
{
    // Warp-specialised: warps 8..15 (producers) turn the staged r of block k into r - alpha q and
    // hand the stage over through named barrier 1 + (k & 1); warps 0..7 (consumers) take it, form
    // z = M^{-1} r with 8 x 4 register tiles (one tile per thread), then release the stage, and
    // thread 0 refills it with block k + 2.  The producers' elementwise work of block k + 1
    // overlaps the consumers' product of block k.
    constexpr int NT = kPPThreads / 2;         // threads per role
    constexpr int CG = M / 4;                  // column groups of four
    constexpr int NF4 = BJ * M / 4;            // float4 per residual block
    constexpr int PER = NF4 / NT;              // float4 per producer thread
    constexpr int TR = 8;                      // tile rows per consumer thread
    constexpr int NTILE = (BJ / TR) * CG;      // consumer tiles (<= NT; the rest of the consumers idle)
    static_assert(NF4 % NT == 0 && NT % CG == 0 && NTILE <= NT, "block shape");
    static_assert(BJ % SB == 0 && SB % TR == 0, "tiles within one block-Jacobi block");
    static_assert(!WY || NT == 2 * BJ, "the y product splits each block's columns over two halves of the consumers");
    constexpr int MS = BJ * SB;                // floats of M^{-1} per stage (BJ / SB blocks of SB x SB)
    extern __shared__ __align__(128) unsigned char pp_sh[];
    float *stage0 = reinterpret_cast<float *>(pp_sh);
    float *stage1 = stage0 + MS + BJ * M;
    float *ys = stage1 + MS + BJ * M;          // 2 x BJ: the y column's residual blocks
    float *yp = ys + 2 * BJ;                   // 2 x 2 x BJ: halves of z_y = M^{-1} r_y
    uint64_t *bar = reinterpret_cast<uint64_t *>(yp + 4 * BJ);
    const int tid = threadIdx.x;
    const bool producer = tid >= NT;
    const int t = producer ? tid - NT : tid;
    const int cg = t % CG;                     // this thread's four columns, in either role
    double dacc[4] = {0.0, 0.0, 0.0, 0.0};     // r^T r (producers) or r^T z (consumers)
    double ydacc = 0.0;                        // the y column's r^T r (producers) or r^T z (consumers)
    const int64_t nmine = (int64_t)blockIdx.x < nblk ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    const int64_t nsub = (n + SB - 1) / SB;    // block-Jacobi blocks of the matrix
    auto issue = [&](int64_t k) {
        const int64_t b = blockIdx.x + k * gridDim.x;
        float *st = (k & 1) ? stage1 : stage0;
        const int64_t i0 = b * BJ;
        const int nb = (int)(n - i0 < BJ ? n - i0 : BJ);
        // the stage's blocks of M^{-1} that exist (the matrix's last stage may hold fewer)
        const int64_t s0 = b * (BJ / SB);
        const int ns = (int)(nsub - s0 < BJ / SB ? nsub - s0 : BJ / SB);
        const uint32_t mb = sizeof(float) * SB * SB * (uint32_t)ns, rb = sizeof(float) * (uint32_t)nb * M;
        mbar_expect_tx(&bar[k & 1], mb + rb);
        bulk_copy_g2s(st, Minv32 + s0 * SB * SB, mb, &bar[k & 1]);
        bulk_copy_g2s(st + MS, rz + i0 * M, rb, &bar[k & 1]);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        if (nmine > 0) issue(0);
        if (nmine > 1) issue(1);
    }
    if (producer) {
        float a4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a4[q] = (float)sc[(cg * 4 + q + 1) * kScal + S_ALPHA];
        const double alpha_y = WY ? sc[S_ALPHA] : 0.0;
        const float ay = (float)alpha_y;
        bool ok = true;
        for (int64_t k = 0; k < nmine; ++k) {
            float *R = ((k & 1) ? stage1 : stage0) + MS;
            const int64_t i0 = (blockIdx.x + k * gridDim.x) * BJ;
            const int nb = (int)(n - i0 < BJ ? n - i0 : BJ);
            float4 q4[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int e = t + j * NT;
                q4[j] = e / CG < nb ? reinterpret_cast<const float4 *>(qz + i0 * M)[e] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // the y column's row i0 + t (the same arithmetic as the y column's own PCG step)
            float yr = 0.0f, yq = 0.0f, yx = 0.0f, ypv = 0.0f;
            const bool yrow = WY && t < nb;
            if (yrow) {
                yr = ry[i0 + t];
                if (alpha_y != 0.0) {
                    yq = qy[i0 + t];
                    yx = xy[i0 + t];
                    ypv = py[i0 + t];
                }
            }
            // a copy that never lands is reported; the stage is handed over all the same so that
            // the consumers never wait on a barrier nobody arrives at
            if (ok && !mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1))) {
                ok = false;
                atomicExch(err, 1);
            }
            float srr[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int e = t + j * NT;
                float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (e / CG < nb) {
                    r4 = reinterpret_cast<const float4 *>(R)[e];
                    r4.x = r4.x - a4[0] * q4[j].x;
                    r4.y = r4.y - a4[1] * q4[j].y;
                    r4.z = r4.z - a4[2] * q4[j].z;
                    r4.w = r4.w - a4[3] * q4[j].w;
                    reinterpret_cast<float4 *>(rz + i0 * M)[e] = r4;
                    srr[0] = fmaf(r4.x, r4.x, srr[0]);
                    srr[1] = fmaf(r4.y, r4.y, srr[1]);
                    srr[2] = fmaf(r4.z, r4.z, srr[2]);
                    srr[3] = fmaf(r4.w, r4.w, srr[3]);
                }
                reinterpret_cast<float4 *>(R)[e] = r4;   // rows past the matrix are zero
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) dacc[q] += (double)srr[q];
            if (WY && t < BJ) {
                // after the stage's wait: the consumers are done with the block two back
                if (yrow && alpha_y != 0.0) {
                    xy[i0 + t] = yx + ay * ypv;
                    yr = yr - ay * yq;
                    ry[i0 + t] = yr;
                }
                if (yrow) ydacc = fma((double)yr, (double)yr, ydacc);
                ys[(k & 1) * BJ + t] = yr;
            }
            asm volatile("bar.arrive %0, %1;" ::"r"(1 + (int)(k & 1)), "r"(kPPThreads) : "memory");
        }
        if (!ok && t == 0) {
            // give copies still in flight a bounded chance to land before the CTA leaves
            for (int b = 0; b < 2; ++b)
                for (uint32_t par = 0; par < 2; ++par) mbar_wait_bounded(&bar[b], par);
        }
    } else {
        const int rg = t / CG;                 // rows TR rg .. TR rg + TR - 1, columns 4 cg .. 4 cg + 3
        const int i0t = rg * TR, c0 = cg * 4;
        const bool has_tile = t < NTILE;
        for (int64_t k = 0; k < nmine; ++k) {
            const float *MT = (k & 1) ? stage1 : stage0;
            const float *R = MT + MS;
            const int64_t i0 = (blockIdx.x + k * gridDim.x) * BJ;
            const int nb = (int)(n - i0 < BJ ? n - i0 : BJ);
            asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(k & 1)), "r"(kPPThreads) : "memory");
            if (has_tile) {
            // z = M^{-1} r (symmetric M^{-1}: row kk of the stage is column kk), rows in pairs with
            // packed FP32x2 FMAs (each half rounds like fmaf)
            float2 acc[TR / 2][4];
#pragma unroll
            for (int a = 0; a < TR / 2; ++a)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[a][q] = make_float2(0.f, 0.f);
            // the tile's rows lie in block sb of the stage: M^{-1}_sb (SB x SB, symmetric) times
            // the block's SB residual rows
            const int sb = i0t / SB;
            const float *MB = MT + sb * SB * SB + (i0t - sb * SB);
            const float *RB = R + sb * SB * M + c0;
#pragma unroll 4
            for (int kk = 0; kk < SB; ++kk) {
                const float4 m0 = *reinterpret_cast<const float4 *>(MB + kk * SB);
                const float4 m1 = *reinterpret_cast<const float4 *>(MB + kk * SB + 4);
                const float4 rv = *reinterpret_cast<const float4 *>(RB + kk * M);
                const float2 mp[4] = {make_float2(m0.x, m0.y), make_float2(m0.z, m0.w), make_float2(m1.x, m1.y),
                                      make_float2(m1.z, m1.w)};
                const float ra[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 rq = make_float2(ra[q], ra[q]);
#pragma unroll
                    for (int a = 0; a < TR / 2; ++a) acc[a][q] = __ffma2_rn(mp[a], rq, acc[a][q]);
                }
            }
            float srz[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < TR; ++a) {
                const int i = i0t + a;
                if (i >= nb) continue;
                const float z[4] = {(a & 1) ? acc[a / 2][0].y : acc[a / 2][0].x, (a & 1) ? acc[a / 2][1].y : acc[a / 2][1].x,
                                    (a & 1) ? acc[a / 2][2].y : acc[a / 2][2].x, (a & 1) ? acc[a / 2][3].y : acc[a / 2][3].x};
                *reinterpret_cast<float4 *>(zz + (i0 + i) * M + c0) = make_float4(z[0], z[1], z[2], z[3]);
                const float4 rv = *reinterpret_cast<const float4 *>(R + i * M + c0);
                srz[0] = fmaf(rv.x, z[0], srz[0]);
                srz[1] = fmaf(rv.y, z[1], srz[1]);
                srz[2] = fmaf(rv.z, z[2], srz[2]);
                srz[3] = fmaf(rv.w, z[3], srz[3]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) dacc[q] += (double)srz[q];
            }
            float yri = 0.0f;
            if (WY) {
                // half h = t / BJ of z_y[i] = sum_kk M^{-1}_sb[kk][i] r_y[kk] over row i's block sb,
                // kk in [h SB/2, (h+1) SB/2)
                const int i = t % BJ, h = t / BJ;
                const int sb = i / SB, il = i - sb * SB;
                const float *yrs = ys + (k & 1) * BJ + sb * SB;
                const float *MB = MT + sb * SB * SB + il;
                float zp = 0.0f;
#pragma unroll 8
                for (int kk = h * (SB / 2); kk < (h + 1) * (SB / 2); ++kk) zp = fmaf(MB[kk * SB], yrs[kk], zp);
                yp[((k & 1) * 2 + h) * BJ + i] = zp;
                if (t < BJ) yri = ys[(k & 1) * BJ + t];
            }
            // every consumer is done with the stage: refill it with block k + 2
            asm volatile("bar.sync 3, %0;" ::"r"(NT) : "memory");
            if (t == 0 && k + 2 < nmine) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(k + 2);
            }
            if (WY && t < nb) {
                const float z = yp[((k & 1) * 2) * BJ + t] + yp[((k & 1) * 2 + 1) * BJ + t];
                zy[i0 + t] = z;
                ydacc = fma((double)yri, (double)z, ydacc);
            }
        }
    }
    __syncthreads();
    // per-column partials of this CTA in thread order: r^T z from the consumers, r^T r from the producers
    double *red = reinterpret_cast<double *>(stage0);
#pragma unroll
    for (int q = 0; q < 4; ++q) red[(size_t)tid * 4 + q] = dacc[q];
    __syncthreads();
    if (tid < M) {
        const int g = tid / 4, q = tid % 4;
        double s1 = 0.0, s2 = 0.0;
        for (int u = g; u < NT; u += CG) {
            s1 += red[(size_t)u * 4 + q];
            s2 += red[(size_t)(NT + u) * 4 + q];
        }
        part_rz[(int64_t)(tid + 1) * pstride + blockIdx.x] = s1;
        part_rr[(int64_t)(tid + 1) * pstride + blockIdx.x] = s2;
    }
    if (WY) {
        // the y column's partials: consumers' r^T z, then producers' r^T r, each in thread order
        __syncthreads();
        red[tid] = ydacc;
        __syncthreads();
        if (tid == 0) {
            double s1 = 0.0, s2 = 0.0;
            for (int u = 0; u < NT; ++u) {
                s1 += red[u];
                s2 += red[NT + u];
            }
            part_rz[blockIdx.x] = s1;
            part_rr[blockIdx.x] = s2;
        }
    }
}

// Dynamic shared memory of k_pc_step: the probe group stages the block's M^{-1} (BJ x BJ), the
// BJ x m residual block and the (BJ / 4) x m partial dots; the y column stages kPCThreads
// residuals (kPCThreads / BJ blocks of BJ rows).  The launch covers both.
size_t pc_smem(int m, int bj)
{
    const size_t z = m > 0 ? (size_t)bj * bj + (size_t)bj * m + (size_t)(bj / 4) * m + bj : 0;
    const size_t y = (size_t)kPCThreads;
    return sizeof(float) * (z > y ? z : y) + 64;
}

// Block size of the block-Jacobi preconditioner: opts.bj_block when set, else 128 rows for
// matrices with at least 64 stored entries per row and enough rows to give every SM six blocks
// (there the larger blocks cut the iteration count by about a fifth, which outweighs the dearer
// step), else 64 (with fewer entries per row 64-row blocks already capture the neighbourhoods,
// and a small problem needs the finer blocks to fill the GPU).  The probe columns and the y
// column can use different sizes (two sets of factors); the automatic choice gives both the same.
int bj_block_size(const gp2s_ctx *c)
{
    const int req = c->A.opts.bj_block;
    if (req == 64 || req == 128) return req;
    const bool dense_rows = c->A.nnz >= 64 * c->A.n;
    const bool many_rows = c->A.n >= (int64_t)128 * 6 * c->num_sms;
    return dense_rows && many_rows ? 128 : 64;
}

// Build one set of block-Jacobi factors (FP32 M^{-1}) with blocks of bj rows.
static gp2s_status build_bj_set(gp2s_ctx *c, int bj, DevBuf &minv, double *logdet)
{
    const int64_t n = c->A.n;
    const int64_t nblk = ceil_div(n, bj);
    GP2S_TRY(ensure(c, minv, sizeof(float) * (size_t)nblk * bj * bj));
    GP2S_TRY(ensure(c, c->bj_ld, sizeof(double) * (size_t)nblk + 64));
    GP2S_TRY(ensure(c, c->counters, 256));
    int *bad = reinterpret_cast<int *>(c->counters.as<char>() + 208);
    GP2S_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    const size_t smem = sizeof(float) * ((size_t)bj * (bj + 1) + bj);
    if (bj == 128) {
        GP2S_TRY(smem_attr(c, (const void *)k_bj_build<128>, smem));
        k_bj_build<128><<<(unsigned)nblk, kPCThreads, smem, c->stream>>>(
            c->rowptr.as<int32_t>(), c->col.as<int32_t>(), c->val32.as<float>(), n, minv.as<float>(),
            c->bj_ld.as<double>(), bad);
    } else {
        GP2S_TRY(smem_attr(c, (const void *)k_bj_build<64>, smem));
        k_bj_build<64><<<(unsigned)nblk, kPCThreads, smem, c->stream>>>(
            c->rowptr.as<int32_t>(), c->col.as<int32_t>(), c->val32.as<float>(), n, minv.as<float>(),
            c->bj_ld.as<double>(), bad);
    }
    GP2S_LAUNCH(c);
    // log|M| = sum of the block log-determinants (fixed-order host sum)
    std::vector<double> ld((size_t)nblk);
    int hbad = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(ld.data(), c->bj_ld.p, sizeof(double) * nblk, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hbad) return set_err(c, GP2S_ENOTPD, "block-Jacobi: a diagonal block is not positive definite");
    double s = 0.0;
    for (double v : ld) s += v;
    *logdet = s;
    return GP2S_OK;
}

// Build the block-Jacobi factors of the current matrix: one set for the probe columns and, when
// the y column uses another block size, a second set for it.
gp2s_status build_block_jacobi(gp2s_ctx *c)
{
    const int bjz = bj_block_size(c), bjy = bjz;
    GP2S_TRY(build_bj_set(c, bjz, c->bj_Minv, &c->bj_logdet));
    if (bjy != bjz) {
        double ldy = 0.0;
        GP2S_TRY(build_bj_set(c, bjy, c->bj_Minv_y, &ldy));
    }
    c->bj_size = bjz;
    c->bj_size_y = bjy;
    c->bj_valid = true;
    return GP2S_OK;
}

// Build the RB8 copy of the FP32 matrix (count -> scan -> fill) and its per-CTA block ranges.
gp2s_status build_rb8(gp2s_ctx *c)
{
    const Assembled &A = c->A;
    const int64_t n = A.n;
    const int64_t nblk = ceil_div(n, kRB);
    const unsigned gb = (unsigned)std::min<int64_t>(ceil_div(nblk * 32, 256), 152 * 16);
    int64_t nu = c->rb_entries;
    if (!c->rb_pattern_valid) {
        // the union structure depends on the pattern only: counted once per pattern
        GP2S_TRY(ensure(c, c->rb_cnt, sizeof(int32_t) * (size_t)(nblk + 1)));
        GP2S_TRY(ensure(c, c->rb_ptr, sizeof(int32_t) * (size_t)(nblk + 1)));
        k_rb_build<false><<<gb, 256, 0, c->stream>>>(c->rowptr.as<int32_t>(), c->col.as<int32_t>(),
                                                     c->val32.as<float>(), n, nblk, c->rb_cnt.as<int32_t>(), nullptr,
                                                     nullptr, nullptr);
        GP2S_LAUNCH(c);
        GP2S_TRY(scan_counts_i32(c, c->rb_cnt.as<int32_t>(), c->rb_ptr.as<int32_t>(), nblk, &nu));
    }
    GP2S_TRY(ensure(c, c->rb_col, sizeof(int32_t) * (size_t)(nu + 1)));
    GP2S_TRY(ensure(c, c->rb_val, sizeof(float) * kRB * (size_t)(nu + 1)));
    k_rb_build<true><<<gb, 256, 0, c->stream>>>(c->rowptr.as<int32_t>(), c->col.as<int32_t>(), c->val32.as<float>(),
                                                n, nblk, nullptr, c->rb_ptr.as<int32_t>(), c->rb_col.as<int32_t>(),
                                                c->rb_val.as<float>());
    GP2S_LAUNCH(c);
    // the SpMM's tile and segment counters start at zero (each launch leaves them there)
    GP2S_TRY(ensure(c, c->counters, 256));
    GP2S_CUDA(c, cudaMemsetAsync(c->counters.as<char>() + kRBWorkOffset, 0, sizeof(RBWork), c->stream));
    GP2S_TRY(ensure(c, c->rb_seg, sizeof(int) * kMaxPartBlocks));
    GP2S_CUDA(c, cudaMemsetAsync(c->rb_seg.p, 0, sizeof(int) * kMaxPartBlocks, c->stream));
    c->rb_entries = nu;
    c->rb_valid = true;
    c->rb_pattern_valid = true;
    return GP2S_OK;
}

// A captured run of CG iterations (CUDA graph) for one column set, with the work counters of
// one replay so that the launch / SpMM accounting stays exact.
struct GraphRun {
    gp2s_ctx *c;
    cudaGraphExec_t exec = nullptr;
    int mc = -1;
    bool pcz = false;
    int64_t launches = 0, spmm_launches = 0;
    double spmm_bytes = 0.0;
    explicit GraphRun(gp2s_ctx *cc) : c(cc) {}
    ~GraphRun() { if (exec) cudaGraphExecDestroy(exec); }
    bool matches(int m_, bool p_) const { return exec && mc == m_ && pcz == p_; }
    template <class F>
    gp2s_status capture(int m_, bool p_, int iters, F &&body)
    {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        const int64_t l0 = c->launches, s0 = c->spmm_launches;
        const double b0 = c->spmm_bytes;
        // capture on the context's private stream (the caller's stream may be the legacy default
        // stream, which cannot be captured); the graph is then launched on the caller's stream
        if (!c->capture_stream) GP2S_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
        cudaStream_t user = c->stream;
        c->stream = c->capture_stream;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c->stream = user;
            return cuda_err(c, e, "cudaStreamBeginCapture");
        }
        gp2s_status st = GP2S_OK;
        for (int r = 0; r < iters && st == GP2S_OK; ++r) st = body();
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->stream, &g);
        c->stream = user;
        // nothing ran while capturing: take the counts back, and add them per replay
        launches = c->launches - l0;
        spmm_launches = c->spmm_launches - s0;
        spmm_bytes = c->spmm_bytes - b0;
        c->launches = l0;
        c->spmm_launches = s0;
        c->spmm_bytes = b0;
        if (st != GP2S_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            exec = nullptr;
            return cuda_err(c, e, "cudaGraphInstantiate");
        }
        mc = m_;
        pcz = p_;
        return GP2S_OK;
    }
    gp2s_status launch()
    {
        GP2S_CUDA(c, cudaGraphLaunch(exec, c->stream));
        c->launches += launches;
        c->spmm_launches += spmm_launches;
        c->spmm_bytes += spmm_bytes;
        return GP2S_OK;
    }
};

// Reliable updates of the y column (FP32 block-Jacobi PCG): its recursive FP32 residual drifts
// from the true one at about 1e-5 relative, so instead of a restarted FP64 refinement solve the
// column's x is folded into the FP64 accumulator xh and its residual replaced by the true FP64
// residual b - Ah xh each time the recursion has gained the factor delta (the column stops on the
// device, the host replaces at the next convergence check).  The search direction p is kept, so
// the column goes on from its Krylov space and reaches tol_refine while the probe columns still
// run (Sleijpen & van der Vorst's reliable-update scheme).
}  // namespace
gp2s_status y_residual(gp2s_ctx *c, const double *y_sorted_dev, double *relres);
namespace {

struct ReliableY {
    const double *y_sorted;   // original-order y, sorted (for the original-space residual)
    double tol_refine, delta;
    bool done = false;        // the true residual met tol_refine
    double relres = 0.0;
    int replacements = 0;
};

// One CG run (x0 = 0) on columns [y | probes]; the probe right-hand sides must already be in rz.
template <class T, class V>
gp2s_status cg_run(gp2s_ctx *c, int m, const V *val, const CGBuffers &B, const double *rhs_y, double tol_y,
                   double tol_z, int kmin_probe, int ksteps, double *rec, int max_iter, int *iters_y,
                   int *iters_z, bool *breakdown, ReliableY *ru = nullptr)
{
    const Assembled &A = c->A;
    const int64_t n = A.n;
    const int k = 1 + m;
    const int nb = std::max(1, std::min(kMaxPartBlocks, c->num_sms));   // one SpMM CTA per SM
    const int pstride = kMaxPartBlocks;
    GP2S_TRY(ensure(c, c->rsplit, sizeof(int32_t) * (size_t)(nb + 1)));
    k_row_split<<<1, 1024, 0, c->stream>>>(c->rowptr.as<int32_t>(), n, nb, c->rsplit.as<int32_t>());
    GP2S_LAUNCH(c);
    const int32_t *rsplit = c->rsplit.as<int32_t>();
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
    int *flags = active + kMaxCols;   // [0] breakdown, [1] active columns, [2] active probe columns
    GP2S_CUDA(c, cudaMemsetAsync(flags, 0, sizeof(int) * 4, c->stream));

    // Block-Jacobi PCG (FP32 vectors, when the preconditioner is built) or plain CG on Ah.  The y
    // column is preconditioned from the start; the probe columns only when no SLQ records are
    // wanted, otherwise they run kmin_probe plain CG steps (Ah's Lanczos coefficients) and are
    // then restarted as PCG.
    const bool pc_avail = std::is_same<T, float>::value && c->bj_valid;
    bool pcy = pc_avail;
    bool pcz = pc_avail && kmin_probe == 0;
    // probe group: bjz-row blocks, one block per CTA step, ~6 CTAs per SM; y column: bjy-row
    // blocks, kPCThreads / bjy blocks per CTA step
    const int bjz = c->bj_size, bjy = c->bj_size_y;
    const int64_t nblkz = ceil_div(n, bjz), nblky = ceil_div(n, bjy);
    const int pgz = m > 0 ? (int)std::min<int64_t>((int64_t)c->num_sms * 6, nblkz) : 0;
    const int pgy = (int)std::min<int64_t>(kMaxPartBlocks, ceil_div(nblky, kPCThreads / bjy));
    GP2S_TRY(ensure(c, c->partials, sizeof(double) * (size_t)pstride * kMaxCols * 2));
    part = c->partials.as<double>();
    double *part_rr = part + (size_t)pstride * kMaxCols;
    const float *Minvz = pc_avail ? c->bj_Minv.as<float>() : nullptr;
    const float *Minvy = pc_avail ? (bjy == bjz ? c->bj_Minv.as<float>() : c->bj_Minv_y.as<float>()) : nullptr;
    if (pc_avail) {
        const size_t smem = pc_smem(m, bjz);
        if (bjz == 128) {
            GP2S_TRY(smem_attr(c, (const void *)k_pc_step<PC_INIT, 128>, smem));
            GP2S_TRY(smem_attr(c, (const void *)k_pc_step<PC_UPDATE, 128>, smem));
            GP2S_TRY(smem_attr(c, (const void *)k_pc_step<PC_RESTART, 128>, smem));
        } else {
            GP2S_TRY(smem_attr(c, (const void *)k_pc_step<PC_INIT, 64>, smem));
            GP2S_TRY(smem_attr(c, (const void *)k_pc_step<PC_UPDATE, 64>, smem));
            GP2S_TRY(smem_attr(c, (const void *)k_pc_step<PC_RESTART, 64>, smem));
        }
    }
    // probe group (bjz-row blocks) and y column (bjy-row blocks) launches
#define GP2S_PCZ_BJ(MODE, BJ, MM, WY)                                                                               \
    k_pc_step<MODE, BJ><<<pgz, kPCThreads, pc_smem(MM, BJ), c->stream>>>(                                          \
        n, MM, nblkz, pgz, Minvz, (float *)B.xz, (float *)B.rz, (float *)B.pz, (const float *)B.qz, (float *)B.zz, \
        (float *)B.xy, (float *)B.ry, (float *)B.py, (const float *)B.qy, (float *)B.zy, rhs_y, sc, part, part_rr,  \
        pstride, WY)
#define GP2S_PCZ_WY(MODE, MM, WY)                                                                                   \
    do {                                                                                                            \
        if (bjz == 128) GP2S_PCZ_BJ(MODE, 128, MM, WY);                                                             \
        else GP2S_PCZ_BJ(MODE, 64, MM, WY);                                                                         \
    } while (0)
#define GP2S_PCZ(MODE, MM) GP2S_PCZ_WY(MODE, MM, 0)
#define GP2S_PCY_BJ(MODE, BJ)                                                                                       \
    k_pc_step<MODE, BJ><<<pgy, kPCThreads, pc_smem(0, BJ), c->stream>>>(                                           \
        n, 0, nblky, 0, Minvy, (float *)B.xz, (float *)B.rz, (float *)B.pz, (const float *)B.qz, (float *)B.zz,    \
        (float *)B.xy, (float *)B.ry, (float *)B.py, (const float *)B.qy, (float *)B.zy, rhs_y, sc, part, part_rr, \
        pstride, 0)
#define GP2S_PCY(MODE)                                                                                              \
    do {                                                                                                            \
        if (bjy == 128) GP2S_PCY_BJ(MODE, 128);                                                                     \
        else GP2S_PCY_BJ(MODE, 64);                                                                                 \
    } while (0)
    // the probe group's UPDATE step on the warp-specialised bulk-copy kernel (FP32, m = 32 or 64, the
    // instantiated widths; 128-row stages holding one 128-row or two 64-row block-Jacobi blocks):
    // one CTA per SM, x updated by the direction kernel.  Against the staged kernel at several CTAs
    // per SM: clusters_3d at N = 1M 1.66 against 1.84 s, sphere_4d at N = 10M 1.78 against 1.86 s.
    const bool pc_async = pc_avail && c->pc_async && (m == 32 || m == 64) &&
                          (bjz == 128 || (bjz == 64 && c->pc_async64));
    const int64_t nstage = ceil_div(n, (int64_t)128);   // the bulk-copy kernel's 128-row stages
    const int pga = (int)std::min<int64_t>(c->num_sms, nstage);
    int *dev_err = flags + 3;
    // the y column's PCG update joins the probe group's step when both use the same factors
    const bool pc_fuse_y = pcy && bjy == bjz && c->pc_fuse_y;
    // the probe group's plain-CG steps on the vectorised update (x += alpha p in the direction kernel)
    const bool upd4 = std::is_same<T, float>::value && m % 4 == 0 && m > 0;
#define GP2S_PP_ATTR(SB_, M_, WY_) \
    GP2S_TRY(smem_attr(c, (const void *)k_pc_probe<128, SB_, M_, WY_>, pp_smem<128, SB_, M_>()))
    if (pc_async) {
        if (bjz == 128) {
            GP2S_PP_ATTR(128, 64, false); GP2S_PP_ATTR(128, 32, false);
            GP2S_PP_ATTR(128, 64, true); GP2S_PP_ATTR(128, 32, true);
        } else {
            GP2S_PP_ATTR(64, 64, false); GP2S_PP_ATTR(64, 32, false);
            GP2S_PP_ATTR(64, 64, true); GP2S_PP_ATTR(64, 32, true);
        }
    }
#undef GP2S_PP_ATTR
    auto launch_pc_probe = [&](int mm, bool wy) -> gp2s_status {
        float *rzp = (float *)B.rz, *zzp = (float *)B.zz;
        const float *qzp = (const float *)B.qz;
#define GP2S_PP(SB_, M_, WY_)                                                                                \
    k_pc_probe<128, SB_, M_, WY_><<<pga, kPPThreads, pp_smem<128, SB_, M_>(), c->stream>>>(                  \
        n, nstage, Minvz, rzp, qzp, zzp, sc, part, part_rr, pstride, dev_err, (float *)B.xy, (float *)B.ry, \
        (const float *)B.py, (const float *)B.qy, (float *)B.zy)
        if (bjz == 128) {
            if (mm == 64) {
                if (wy) GP2S_PP(128, 64, true);
                else GP2S_PP(128, 64, false);
            } else {
                if (wy) GP2S_PP(128, 32, true);
                else GP2S_PP(128, 32, false);
            }
        } else {
            if (mm == 64) {
                if (wy) GP2S_PP(64, 64, true);
                else GP2S_PP(64, 64, false);
            } else {
                if (wy) GP2S_PP(64, 32, true);
                else GP2S_PP(64, 32, false);
            }
        }
#undef GP2S_PP
        return GP2S_OK;
    };
    // initial state: probe group then y column
    if (m > 0) {
        if (pcz) GP2S_PCZ(PC_INIT, m);
        else k_cg_init<T><<<nbz, ut, 0, c->stream>>>(n, m, rhs_y, (T *)B.xz, (T *)B.rz, (T *)B.pz, (T *)B.xy,
                                                      (T *)B.ry, (T *)B.py, part, pstride, nbz);
        GP2S_LAUNCH(c);
    }
    if (pcy) GP2S_PCY(PC_INIT);
    else k_cg_init<T><<<nby, ut, 0, c->stream>>>(n, m > 0 ? m : 1, rhs_y, (T *)B.xz, (T *)B.rz, (T *)B.pz,
                                                  (T *)B.xy, (T *)B.ry, (T *)B.py, part, pstride, 0);
    GP2S_LAUNCH(c);
    // reliable updates need the y column's block-Jacobi step (REPLACE mode)
    ReliableY *rel = (ru && pcy) ? ru : nullptr;
    k_scal_init<<<k, 256, 0, c->stream>>>(part, part_rr, pstride, pcy ? pgy : nby, pcz ? pgz : nbz, sc, active,
                                          rel ? rel->delta : tol_y, tol_z, pcy, pcz);
    GP2S_LAUNCH(c);

    // squared relative residual at the rounding level of the vector precision
    const double lucky = std::is_same<T, float>::value ? 1e-12 : 1e-26;
    const int check_every = 8;
    int it = 0;
    int *hcount = reinterpret_cast<int *>(c->hbuf.p);
    int mc = m;          // probe columns still iterated; 0 once every probe column has stopped
    // one CG / PCG iteration on the active columns (every argument is fixed for given mc, pcz:
    // the scalars live in device memory), so runs of iterations can be captured into a graph
    auto one_iter = [&]() -> gp2s_status {
        const int kc = 1 + mc;
        int np = nb;
        GP2S_TRY((launch_spmm<T, V>(c, mc, true, val, B, part, pstride, nb, rsplit, active, &np, dev_err)));
        k_scal_alpha<<<kc, 256, 0, c->stream>>>(part, pstride, np, sc, active, flags, rec, ksteps, lucky);
        GP2S_LAUNCH(c);
        GP2S_CUDA(c, cudaMemsetAsync(flags + 1, 0, sizeof(int) * 2, c->stream));
        const bool fused_y = mc > 0 && pcz && pc_fuse_y;
        if (mc > 0) {
            if (pcz && pc_async) GP2S_TRY(launch_pc_probe(mc, fused_y));
            else if (pcz) GP2S_PCZ_WY(PC_UPDATE, mc, fused_y ? 1 : 0);
            else if (upd4) k_update_z4<<<nbz, 256, 0, c->stream>>>(n, m, (float *)B.rz, (const float *)B.qz, sc,
                                                                    part, pstride);
            else k_update<T><<<nbz, ut, 0, c->stream>>>(n, m, (T *)B.xz, (T *)B.rz, (const T *)B.pz, (const T *)B.qz,
                                                         (T *)B.xy, (T *)B.ry, (const T *)B.py, (const T *)B.qy, sc,
                                                         part, pstride, nbz);
            GP2S_LAUNCH(c);
        }
        if (!fused_y) {
            if (pcy) GP2S_PCY(PC_UPDATE);
            else k_update<T><<<nby, ut, 0, c->stream>>>(n, m > 0 ? m : 1, (T *)B.xz, (T *)B.rz, (const T *)B.pz,
                                                         (const T *)B.qz, (T *)B.xy, (T *)B.ry, (const T *)B.py,
                                                         (const T *)B.qy, sc, part, pstride, 0);
            GP2S_LAUNCH(c);
        }
        k_scal_beta<<<kc, 256, 0, c->stream>>>(part, part_rr, pstride, fused_y ? (pc_async ? pga : pgz) : pcy ? pgy : nby,
                                               pcz ? (pc_async ? pga : pgz) : nbz, sc, active, flags + 1, rec, ksteps,
                                               kmin_probe, pcy, pcz, lucky);
        GP2S_LAUNCH(c);
        {
            // direction: p = z + beta p (z = M^{-1} r for a preconditioned group, z = r otherwise)
            const int cgs = mc / 4;
            const int dthreads = mc > 0 ? cgs * std::max(1, 256 / cgs) : 256;
            const int dgz = mc > 0 ? (int)std::min<int64_t>(152 * 8, ceil_div(n, dthreads / cgs)) : 0;
            const int dgy = (int)std::min<int64_t>(152 * 2, ceil_div(n, dthreads));
            const T *zzp = pcz ? (const T *)B.zz : (const T *)B.rz;
            const T *zyp = pcy ? (const T *)B.zy : (const T *)B.ry;
            k_direction<T><<<dgz + dgy, dthreads, 0, c->stream>>>(n, mc, zzp, (T *)B.pz, zyp, (T *)B.py, sc, active,
                                                                 dgz, (T *)B.xz, ((pcz && pc_avail) || (!pcz && upd4)) ? 1 : 0);
            GP2S_LAUNCH(c);
        }
        return GP2S_OK;
    };
    // The y column has stopped (its recursion gained the factor delta, or reached its rounding
    // level): fold x_y into xh, form the true residual in FP64; done at tol_refine, else restart the
    // recursion from the true residual with p kept.
    auto replace_y = [&]() -> gp2s_status {
        double *b64v = c->vec64.as<double>();
        double *xh = b64v + n, *r64 = b64v + 2 * n;
        const unsigned gbn = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
        k_accum64<float><<<gbn, 256, 0, c->stream>>>(n, (const float *)B.xy, xh);
        GP2S_LAUNCH(c);
        GP2S_CUDA(c, cudaMemsetAsync(B.xy, 0, sizeof(float) * (size_t)n, c->stream));
        double relres = 0.0;
        GP2S_TRY(y_residual(c, rel->y_sorted, &relres));
        rel->relres = relres;
        ++rel->replacements;
        if (!(relres > rel->tol_refine)) {
            rel->done = true;
            return GP2S_OK;
        }
        if (bjy == 128)
            k_pc_step<PC_REPLACE, 128><<<pgy, kPCThreads, pc_smem(0, 128), c->stream>>>(
                n, 0, nblky, 0, Minvy, (float *)B.xz, (float *)B.rz, (float *)B.pz, (const float *)B.qz,
                (float *)B.zz, (float *)B.xy, (float *)B.ry, (float *)B.py, (const float *)B.qy, (float *)B.zy, r64,
                sc, part, part_rr, pstride, 0);
        else
            k_pc_step<PC_REPLACE, 64><<<pgy, kPCThreads, pc_smem(0, 64), c->stream>>>(
                n, 0, nblky, 0, Minvy, (float *)B.xz, (float *)B.rz, (float *)B.pz, (const float *)B.qz,
                (float *)B.zz, (float *)B.xy, (float *)B.ry, (float *)B.py, (const float *)B.qy, (float *)B.zy, r64,
                sc, part, part_rr, pstride, 0);
        GP2S_LAUNCH(c);
        k_scal_replace<<<1, 256, 0, c->stream>>>(part, part_rr, pgy, sc, active, rel->delta);
        GP2S_LAUNCH(c);
        // the step's pending direction update, p = z' + beta p (y column only)
        const int dgy = (int)std::min<int64_t>(152 * 2, ceil_div(n, 256));
        k_direction<float><<<dgy, 256, 0, c->stream>>>(n, 0, (const float *)B.zz, (float *)B.pz, (const float *)B.zy,
                                                       (float *)B.py, sc, active, 0, (float *)B.xz, 0);
        GP2S_LAUNCH(c);
        return GP2S_OK;
    };
    // Runs of check_every iterations between two convergence checks are captured once into a CUDA
    // graph and replayed while the column set (mc, pcz) stays the same: one launch instead of
    // about seven per iteration.  The first run (it allocates the per-launch scratch), the run
    // holding the probes' PCG restart, a shortened last run and profiled calls go eagerly.
    GraphRun gr(c);
    while (it < max_iter) {
        const int len = std::min(check_every, max_iter - it);
        const bool restart_in_run = pc_avail && !pcz && mc > 0 && kmin_probe >= it && kmin_probe < it + len;
        if (c->use_graphs && !c->profile && it > 0 && len == check_every && !restart_in_run) {
            if (!gr.matches(mc, pcz)) GP2S_TRY(gr.capture(mc, pcz, check_every, one_iter));
            GP2S_TRY(gr.launch());
            it += len;
        } else {
            for (int r = 0; r < len; ++r, ++it) {
                if (pc_avail && !pcz && mc > 0 && it == kmin_probe) {
                    // the SLQ steps are recorded: their quadratures go to the side stream, and the
                    // probe columns restart as PCG from their iterates
                    if (rec && c->slq_async) GP2S_TRY(slq_start_async(c, m, ksteps));
                    GP2S_PCZ(PC_RESTART, mc);
                    GP2S_LAUNCH(c);
                    k_scal_restart<<<mc, 256, 0, c->stream>>>(part, pstride, pgz, sc, active);
                    GP2S_LAUNCH(c);
                    pcz = true;
                }
                GP2S_TRY(one_iter());
            }
        }
        GP2S_CUDA(c, cudaMemcpyAsync(hcount, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
        if (rel) GP2S_CUDA(c, cudaMemcpyAsync(hcount + 4, active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
        GP2S_TRY(flush_profile(c));
        if (hcount[3]) {
            // a warp that gave up left its tiles undone: clear the SpMM's counters for the next solve
            GP2S_CUDA(c, cudaMemsetAsync(c->counters.as<char>() + kRBWorkOffset, 0, sizeof(RBWork), c->stream));
            if (c->rb_seg.p) GP2S_CUDA(c, cudaMemsetAsync(c->rb_seg.p, 0, sizeof(int) * kMaxPartBlocks, c->stream));
            GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
            return set_err(c, GP2S_ETIMEOUT, "a bulk copy (block-Jacobi stage or SpMM row gather) did not complete "
                                             "(bounded wait gave up)");
        }
        bool y_back = false;
        if (rel && !rel->done && hcount[4] == 0 && !hcount[0]) {
            GP2S_TRY(replace_y());
            y_back = !rel->done;
        }
        if (hcount[1] == 0 && !y_back) break;
        if (mc > 0 && hcount[2] == 0) mc = 0;   // only the y column is left: y-only kernels
    }
#undef GP2S_PCZ
#undef GP2S_PCZ_BJ
#undef GP2S_PCY
#undef GP2S_PCY_BJ
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

// Layout of the Krylov vectors in c->vec: probe group x, r, p, q (n x m each), y group x, r, p, q
// (n each), then z of the y column and z of the probe group (block-Jacobi PCG).
static gp2s_status cg_layout(gp2s_ctx *c, int mm, CGBuffers *B)
{
    const int64_t n = c->A.n;
    const size_t es = c->A.precision == GP2S_PREC_MIXED ? sizeof(float) : sizeof(double);
    GP2S_TRY(ensure(c, c->vec, es * (size_t)n * (5 + 5 * (size_t)mm) + 256));
    char *base = c->vec.as<char>();
    size_t nz = es * (size_t)n * mm;
    B->xz = base; B->rz = base + nz; B->pz = base + 2 * nz; B->qz = base + 3 * nz;
    char *yb = base + 4 * nz;
    B->xy = yb; B->ry = yb + es * n; B->py = yb + 2 * es * n; B->qy = yb + 3 * es * n;
    B->zz = yb + 4 * es * n;
    B->zy = (char *)B->zz + nz;
    return GP2S_OK;
}

gp2s_status krylov_columns_buffers(gp2s_ctx *c, int m, void **rz, void **xz)
{
    CGBuffers B;
    GP2S_TRY(cg_layout(c, m, &B));
    *rz = B.rz;
    *xz = B.xz;
    return GP2S_OK;
}

gp2s_status krylov_columns_solve(gp2s_ctx *c, int m, double tol, int *iters)
{
    Assembled &A = c->A;
    const int64_t n = A.n;
    const bool mixed = A.precision == GP2S_PREC_MIXED;
    CGBuffers B;
    GP2S_TRY(cg_layout(c, m, &B));
    if (mixed && A.opts.precond == 2 && !c->bj_valid) GP2S_TRY(build_block_jacobi(c));
    if (mixed && !c->rb_valid) GP2S_TRY(build_rb8(c));
    GP2S_TRY(ensure_host(c, c->hbuf, 4096));
    // the y column is idle: a zero right-hand side leaves it inactive from the first step
    GP2S_TRY(ensure(c, c->vec64, sizeof(double) * (size_t)n * 4 + 256));
    double *zero = c->vec64.as<double>();   // slot 0 (the refinement's b), free after the solve
    GP2S_CUDA(c, cudaMemsetAsync(zero, 0, sizeof(double) * n, c->stream));
    int iy = 0, iz = 0;
    bool brk = false;
    if (mixed)
        GP2S_TRY((cg_run<float, float>(c, m, c->val32.as<float>(), B, zero, 1.0, tol, 0, 0, nullptr, A.opts.max_iter,
                                       &iy, &iz, &brk)));
    else
        GP2S_TRY((cg_run<double, double>(c, m, c->val64.as<double>(), B, zero, 1.0, tol, 0, 0, nullptr,
                                         A.opts.max_iter, &iy, &iz, &brk)));
    c->have_probes = false;
    *iters = iz;
    if (brk) return set_err(c, GP2S_EBREAKDOWN, "CG breakdown in a posterior-variance solve");
    if (iz >= A.opts.max_iter) return set_err(c, GP2S_ENOCONV, "posterior-variance solve hit max_iter");
    return GP2S_OK;
}

gp2s_status krylov_solve(gp2s_ctx *c, const double *y_sorted_dev, bool with_probes, int m, int ksteps,
                         CGResult *res)
{
    Assembled &A = c->A;
    const int64_t n = A.n;
    if (!with_probes) m = 0;
    const bool mixed = A.precision == GP2S_PREC_MIXED;
    const int mm = m > 0 ? m : 0;
    CGBuffers B;
    GP2S_TRY(cg_layout(c, mm, &B));
    // block-Jacobi preconditioner (FP32 path, opts.precond == 2)
    if (mixed && A.opts.precond == 2 && !c->bj_valid) GP2S_TRY(build_block_jacobi(c));
    // FP64 refinement vectors: b64, xhat64, res64, a64 (solution in sorted order)
    GP2S_TRY(ensure(c, c->vec64, sizeof(double) * (size_t)n * 4 + 256));
    double *b64 = c->vec64.as<double>();
    double *xh = b64 + n, *r64 = b64 + 2 * n, *a64 = b64 + 3 * n;
    GP2S_TRY(ensure_host(c, c->hbuf, 4096));
    // a pending SLQ launch of the previous solve still reads rec and the scalars
    GP2S_TRY(slq_fence(c));
    c->slq_pending = false;
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
    if (mixed && mm > 0 && !c->rb_valid) GP2S_TRY(build_rb8(c));
    const double tol_first = mixed ? o.tol_inner : std::min(o.tol_inner, 0.1 * o.tol_refine);
    // probe columns: the k SLQ steps always; solved to tol_probe only when the gradient needs
    // u_s = A^{-1} D^{1/2} z_s (a relative tolerance of 1 stops them right after the k steps)
    const double tol_z = c->probes_for_grad ? o.tol_probe : 1.0;
    int iy = 0, iz = 0;
    bool brk = false;
    if (o.solver == GP2S_SOLVER_MINRES) {
        // the probe columns run CG beside an idle y column (zero right-hand side) ...
        if (mm > 0) {
            GP2S_CUDA(c, cudaMemsetAsync(r64, 0, sizeof(double) * n, c->stream));
            if (mixed)
                GP2S_TRY((cg_run<float, float>(c, mm, c->val32.as<float>(), B, r64, 1.0, tol_z, ksteps, ksteps, rec,
                                               o.max_iter, &iy, &iz, &brk)));
            else
                GP2S_TRY((cg_run<double, double>(c, mm, c->val64.as<double>(), B, r64, 1.0, tol_z, ksteps, ksteps, rec,
                                                 o.max_iter, &iy, &iz, &brk)));
            if (brk) return set_err(c, GP2S_EBREAKDOWN, "CG breakdown in a probe column");
        }
        // ... and the y column is MINRES's: FP64 on Ah, restarted on the FP64 residual
        int st = 0, total = 0, outer = 0;
        double relres = 0.0;
        GP2S_TRY(minres_solve(c, b64, xh, 0.1 * o.tol_refine, o.max_iter, &st));
        total += st;
        for (;;) {
            GP2S_TRY(y_residual(c, y_sorted_dev, &relres));
            if (!(relres > o.tol_refine) || outer >= o.max_outer) break;
            ++outer;
            GP2S_TRY(minres_solve(c, r64, a64, std::min(0.5, 0.1 * o.tol_refine / relres), o.max_iter, &st));
            total += st;
            k_accum64<double><<<gbn, 256, 0, c->stream>>>(n, a64, xh);
            GP2S_LAUNCH(c);
        }
        k_scale64<<<gbn, 256, 0, c->stream>>>(n, c->s64.as<double>(), xh, a64);
        GP2S_LAUNCH(c);
        res->iters_y = total;
        res->iters_probes = iz;
        res->outer = outer;
        res->relres = relres;
        c->have_solution = true;
        c->have_probes = mm > 0;
        c->solve_iters = total;
        c->solve_outer = outer;
        c->solve_relres = relres;
        c->probe_iters = iz;
        if (relres > o.tol_refine) {
            res->status = GP2S_ENOCONV;
            return set_err(c, GP2S_ENOCONV, "MINRES did not reach tol_refine within max_outer restarts");
        }
        return GP2S_OK;
    }
    // xhat accumulates the y solution in FP64 (the reliable updates fold x_y into it during the run)
    GP2S_CUDA(c, cudaMemsetAsync(xh, 0, sizeof(double) * n, c->stream));
    ReliableY ru;
    ru.y_sorted = y_sorted_dev;
    ru.tol_refine = o.tol_refine;
    ru.delta = c->reliable_delta;
    // Reliable updates pay where iterations are dear: each replacement costs a host synchronisation,
    // about ten launches and up to one check interval of idle y iterations, which a small problem's
    // cheap restarted refinement undercuts (the 256-problem batch, n <= 65,536: 21 problems/s with
    // them against 29 without; at n = 1M and 10M they save 13 % and 10 %).
    const bool reliable = c->reliable_y && n >= c->reliable_min_rows;
    if (mixed)
        GP2S_TRY((cg_run<float, float>(c, mm, c->val32.as<float>(), B, b64, tol_first, tol_z, mm > 0 ? ksteps : 0,
                                       ksteps, rec, o.max_iter, &iy, &iz, &brk, reliable ? &ru : nullptr)));
    else
        GP2S_TRY((cg_run<double, double>(c, mm, c->val64.as<double>(), B, b64, tol_first, tol_z,
                                         mm > 0 ? ksteps : 0, ksteps, rec, o.max_iter, &iy, &iz, &brk)));
    res->iters_probes = iz;
    int total_y = iy;
    if (brk) {
        res->status = GP2S_EBREAKDOWN;
        return set_err(c, GP2S_EBREAKDOWN, "CG breakdown (p^T A p <= 0 or NaN)");
    }
    // xhat += x_y (FP64 accumulate)
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
        // the correction only has to shrink the residual by tol_refine / relres (with a 10x margin)
        const double tol_corr = std::min(0.5, std::max(o.tol_inner, 0.1 * o.tol_refine / relres));
        if (mixed)
            GP2S_TRY((cg_run<float, float>(c, 0, c->val32.as<float>(), B, r64, tol_corr, o.tol_probe, 0, 0, nullptr,
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
