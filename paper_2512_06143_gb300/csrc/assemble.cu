// assemble.cu -- count -> scan -> fill assembly of A = K + sigma^2 I into CSR (Sec. 4.6 redesigned),
// the bump tables (Eq. 7), the Jacobi diagonal, and the FP64 values pass.
//
// One CTA per work item (a run of at most kRowsPerItem rows of one occupied cell).  The CTA finds
// the 3^d neighbour cells by binary search in the sorted cell-key table, orders their point ranges
// by start index, stages chunks of the concatenated candidate points (hi/lo FP32 coordinates, and
// in the fill pass the FP32 bump values and Jacobi scales) in shared memory, and each warp tests
// its rows against the staged chunk with a conservative FP32 guard band; pairs inside the band are
// decided by the exact FP64 test (same operation order as the oracle).  Warp ballots give the row
// counts (count pass) and the ordered, compacted column/value writes (fill pass): candidates are
// visited in ascending sorted index, so columns come out ascending.
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "gp2s_geometry.cuh"
#include "gp2s_kernel_math.cuh"

namespace gp2s {

namespace {

constexpr int kAsmThreads = 128;
constexpr int kAsmWarps = kAsmThreads / kWarp;
constexpr int kRowsPerItem = 64;
constexpr int kChunk = 256;

struct AsmArgs {
    const float4 *Xhi, *Xlo;
    const double4_16a *X64;
    const int4 *items;
    const int32_t *cell_start;
    const uint64_t *cell_key;
    int64_t ncells;
    const float *B32;     // n x L
    const float *s32;     // n
    const double4_16a *Lam;   // Wendland convolution: lambda_k of every sorted point (padded to 4)
    const int32_t *rowptr;
    int32_t *rowcnt;
    int32_t *col;
    float *val;
    unsigned long long *stats;   // [0] candidates, [1] band pairs
};

template <int D>
__device__ __forceinline__ void decode_coarse(uint64_t ck, int cb, int64_t *cc)
{
#pragma unroll
    for (int k = 0; k < D; ++k) cc[k] = 0;
    for (int b = 0; b < cb; ++b)
#pragma unroll
        for (int k = 0; k < D; ++k) cc[k] |= (int64_t)((ck >> (b * D + k)) & 1ull) << b;
}

__device__ __forceinline__ int64_t find_cell(const uint64_t *__restrict__ keys, int64_t n, uint64_t k)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < n && keys[lo] == k) ? lo : -1;
}

// FP32 squared distance from the hi/lo split: Dk = (hi_i - hi_j) + (lo_i - lo_j).
template <int D>
__device__ __forceinline__ float d2_f32(const float4 &hi_i, const float4 &lo_i, const float4 &hi_j,
                                        const float4 &lo_j)
{
    const float hi[4] = {hi_i.x, hi_i.y, hi_i.z, hi_i.w}, lo[4] = {lo_i.x, lo_i.y, lo_i.z, lo_i.w};
    const float hj[4] = {hi_j.x, hi_j.y, hi_j.z, hi_j.w}, lj[4] = {lo_j.x, lo_j.y, lo_j.z, lo_j.w};
    float q = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float dk = __fadd_rn(__fsub_rn(hi[k], hj[k]), __fsub_rn(lo[k], lj[k]));
        q = __fmaf_rn(dk, dk, q);
    }
    return q;
}

// The exact pattern test: ((D0*D0 + D1*D1) + D2*D2) + ... < r*r, FP64, no fused multiply-add.
template <int D>
__device__ __forceinline__ bool exact_in(const double4_16a &a, const double4_16a &b, double r2)
{
    const double xa[4] = {a.x, a.y, a.z, a.w}, xb[4] = {b.x, b.y, b.z, b.w};
    double q = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        double dk = __dsub_rn(xa[k], xb[k]);
        q = __dadd_rn(q, __dmul_rn(dk, dk));
    }
    return q < r2;
}

// Wendland convolution kernel (Eq. 6): the polynomial bump psi_l(x) = (1 - |x - c_l|^2 / rho_l^2)^3,
// the signal field s(x) = w0 + sum_l a_l psi_l(x) and the length-scale field lambda_k(x) =
// ell_k^2 + sum_l G_lk psi_l(x), every operation one FP64 round-to-nearest step in the written
// order (no contraction): the pattern test below depends on lambda bit for bit.
template <int D>
__device__ __forceinline__ double wc_psi(const double *x, const KernelParams &kp, int l)
{
    double q = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const double dk = __dsub_rn(x[k], kp.centers[l * D + k]);
        q = __dadd_rn(q, __dmul_rn(dk, dk));
    }
    const double rho = kp.radii[l];
    const double s = __ddiv_rn(q, __dmul_rn(rho, rho));
    if (!(s < 1.0)) return 0.0;
    const double u = __dsub_rn(1.0, s);
    return __dmul_rn(__dmul_rn(u, u), u);
}

template <int D>
__device__ __forceinline__ void wc_fields(const double *x, const KernelParams &kp, double &sig, double *lam,
                                          double *psi_out)
{
    double sg = 0.0, acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.0;
    for (int l = 0; l < kp.L; ++l) {
        const double ps = wc_psi<D>(x, kp, l);
        if (psi_out) psi_out[l] = ps;
        sg = __dadd_rn(sg, __dmul_rn(kp.amps[l], ps));
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = __dadd_rn(acc[k], __dmul_rn(kp.G[l * D + k], ps));
    }
    sig = __dadd_rn(kp.w0, sg);
#pragma unroll
    for (int k = 0; k < D; ++k) lam[k] = __dadd_rn(__dmul_rn(kp.ell[k], kp.ell[k]), acc[k]);
}

// Q(i, j) = ((D0 D0 / m0 + D1 D1 / m1) + ...), m_k = (lambda_ik + lambda_jk) * 0.5
template <int D>
__device__ __forceinline__ double wc_q(const double4_16a &a, const double4_16a &b, const double4_16a &la,
                                       const double4_16a &lb)
{
    const double xa[4] = {a.x, a.y, a.z, a.w}, xb[4] = {b.x, b.y, b.z, b.w};
    const double ma[4] = {la.x, la.y, la.z, la.w}, mb[4] = {lb.x, lb.y, lb.z, lb.w};
    double q = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const double dk = __dsub_rn(xa[k], xb[k]);
        const double m = __dmul_rn(__dadd_rn(ma[k], mb[k]), 0.5);
        q = __dadd_rn(q, __ddiv_rn(__dmul_rn(dk, dk), m));
    }
    return q;
}

template <int D, bool FILL>
__global__ void __launch_bounds__(kAsmThreads)
k_assemble(AsmArgs a, GridParams g, SupportParams sp, KernelParams kp)
{
    constexpr int NNB = D == 1 ? 3 : D == 2 ? 9 : D == 3 ? 27 : 81;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *c_hi = reinterpret_cast<float4 *>(smem);
    float4 *c_lo = c_hi + kChunk;
    float4 *r_hi = c_lo + kChunk;
    float4 *r_lo = r_hi + kRowsPerItem;
    int *c_j = reinterpret_cast<int *>(r_lo + kRowsPerItem);
    int *r_run = c_j + kChunk;
    int2 *rng = reinterpret_cast<int2 *>(r_run + kRowsPerItem);      // NNB (start, end)
    int2 *rng_sorted = rng + NNB;
    int *pref = reinterpret_cast<int *>(rng_sorted + NNB);           // NNB + 1
    int *nr_sh = pref + NNB + 1;

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int4 item = a.items[blockIdx.x];
    const int cell = item.x, r0 = item.y, r1 = item.z;
    const int nrows = r1 - r0;

    // 1. neighbour cells and their point ranges
    const int cb = g.bits - g.fine_bits;
    if (threadIdx.x < NNB) {
        int64_t cc[D], nc[D];
        decode_coarse<D>(a.cell_key[cell], cb, cc);
        int t = threadIdx.x;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            int o = t % 3 - 1;
            t /= 3;
            nc[k] = cc[k] + o;
            ok = ok && nc[k] >= 0 && nc[k] < g.dims[k];
        }
        int2 rr = make_int2(0, 0);
        if (ok) {
            int64_t f = find_cell(a.cell_key, a.ncells, coarse_key<D>(nc, g));
            if (f >= 0) rr = make_int2(a.cell_start[f], a.cell_start[f + 1]);
        }
        rng[threadIdx.x] = rr;
    }
    // rows of the item
    for (int t = threadIdx.x; t < nrows; t += kAsmThreads) {
        r_hi[t] = a.Xhi[r0 + t];
        r_lo[t] = a.Xlo[r0 + t];
        r_run[t] = 0;
    }
    __syncthreads();
    // 2. order the non-empty ranges by start (ranges of distinct cells are disjoint)
    if (wid == 0) {
        for (int e = lane; e < NNB; e += kWarp) {
            int2 me = rng[e];
            if (me.y > me.x) {
                int rank = 0;
                for (int f = 0; f < NNB; ++f) {
                    int2 o = rng[f];
                    rank += (o.y > o.x && o.x < me.x) ? 1 : 0;
                }
                rng_sorted[rank] = me;
            }
        }
        unsigned cnt = 0;
        for (int e = lane; e < NNB; e += kWarp) cnt += rng[e].y > rng[e].x ? 1u : 0u;
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) {
            int run = 0;
            for (int e = 0; e < (int)cnt; ++e) {
                pref[e] = run;
                run += rng_sorted[e].y - rng_sorted[e].x;
            }
            pref[cnt] = run;
            nr_sh[0] = (int)cnt;
        }
    }
    __syncthreads();
    const int nr = nr_sh[0];
    const int total = pref[nr];
    unsigned long long band = 0;

    // 3. candidate chunks
    for (int base = 0; base < total; base += kChunk) {
        const int cnt = min(kChunk, total - base);
        for (int q = threadIdx.x; q < cnt; q += kAsmThreads) {
            int p = base + q;
            int lo = 0, hi = nr - 1;           // last range with pref <= p
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (pref[mid] <= p) lo = mid; else hi = mid - 1;
            }
            int j = rng_sorted[lo].x + (p - pref[lo]);
            c_j[q] = j;
            c_hi[q] = a.Xhi[j];
            c_lo[q] = a.Xlo[j];
        }
        __syncthreads();
        for (int rs = wid; rs < nrows; rs += kAsmWarps) {
            const int i = r0 + rs;
            const float4 hi_i = r_hi[rs], lo_i = r_lo[rs];
            int run = r_run[rs];
            int64_t obase = FILL ? (int64_t)a.rowptr[i] : 0;
            // the fill pass accepts exactly the count pass's pairs (same arithmetic); the row end
            // is still checked so a mismatch could never write past the row
            const int rowlen = FILL ? a.rowptr[i + 1] - a.rowptr[i] : 0;
            for (int q0 = 0; q0 < cnt; q0 += kWarp) {
                const int q = q0 + lane;
                bool acc = false;
                float d2 = 0.0f;
                int j = -1;
                if (q < cnt) {
                    j = c_j[q];
                    d2 = d2_f32<D>(hi_i, lo_i, c_hi[q], c_lo[q]);
                    if (j == i || d2 < sp.thr_lo) {
                        acc = true;
                    } else if (d2 <= sp.thr_hi) {
                        ++band;
                        // the Wendland convolution's support is Q < r^2; the FP32 band around
                        // the Euclidean bound r sqrt(max lambda) only rejects
                        acc = kp.family == 1 ? wc_q<D>(a.X64[i], a.X64[j], a.Lam[i], a.Lam[j]) < sp.r2
                                             : exact_in<D>(a.X64[i], a.X64[j], sp.r2);
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, acc);
                if (FILL && acc) {
                    // columns only: the values pass evaluates every stored pair in FP64
                    const int pos = run + __popc(bal & ((1u << lane) - 1u));
                    if (pos < rowlen) a.col[obase + pos] = j;
                }
                run += __popc(bal);
            }
            if (lane == 0) r_run[rs] = run;
            __syncwarp();
        }
        __syncthreads();
    }
    if (!FILL) {
        for (int t = threadIdx.x; t < nrows; t += kAsmThreads) a.rowcnt[r0 + t] = r_run[t];
        // statistics: candidates tested and FP64 band tests
        for (int o = 16; o > 0; o >>= 1) band += __shfl_xor_sync(0xffffffffu, band, o);
        if (lane == 0 && band) atomicAdd(&a.stats[1], band);
        if (threadIdx.x == 0) atomicAdd(&a.stats[0], (unsigned long long)total * (unsigned long long)nrows);
    }
}

size_t asm_smem_bytes(int D, bool fill, int L)
{
    int NNB = D == 1 ? 3 : D == 2 ? 9 : D == 3 ? 27 : 81;
    size_t b = sizeof(float4) * (2 * kChunk + 2 * kRowsPerItem) + sizeof(int) * (kChunk + kRowsPerItem) +
               sizeof(int2) * 2 * NNB + sizeof(int) * (NNB + 1 + 4);
    (void)fill;
    (void)L;
    return b + 16;
}

// Bump tables (Eq. 7) in FP64 (+ an FP32 copy), the diagonal D_i = A_ii = (sum_l b_l^2 + w0)
// + sigma^2 and the Jacobi scales s_i = D_i^{-1/2}.
// Wendland convolution (family 1): B64 holds psi_l (the gradient's chain rule needs it), Lam the
// length-scale field, Sig the signal field, and D_i = s(x_i)^2 + sigma^2 (Q = 0 and the
// prefactor is 1 on the diagonal).
template <int D>
__global__ void k_bumps(const double4_16a *__restrict__ X64, int64_t n, KernelParams kp,
                        double *__restrict__ B64, float *__restrict__ B32, double *__restrict__ D64,
                        double *__restrict__ s64, float *__restrict__ s32, int *__restrict__ bad,
                        double4_16a *__restrict__ Lam, double *__restrict__ Sig, uint32_t *__restrict__ ffmask)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double4_16a xv = X64[i];
        const double x[4] = {xv.x, xv.y, xv.z, xv.w};
        if (kp.family == 1) {
            double sig, lam[D];
            wc_fields<D>(x, kp, sig, lam, B64 + i * kp.L);
            double4_16a lv;
            lv.x = lam[0];
            lv.y = D > 1 ? lam[D > 1 ? 1 : 0] : 1.0;
            lv.z = D > 2 ? lam[D > 2 ? 2 : 0] : 1.0;
            lv.w = D > 3 ? lam[D > 3 ? 3 : 0] : 1.0;
            Lam[i] = lv;
            Sig[i] = sig;
            for (int l = 0; l < kp.L; ++l) B32[i * kp.L + l] = (float)B64[i * kp.L + l];
            const double Dii = sig * sig + kp.sigma2;
            D64[i] = Dii;
            if (!(Dii > 0.0) || !isfinite(Dii)) {
                atomicOr(bad, 1);
                s64[i] = 0.0;
                s32[i] = 0.0f;
            } else {
                const double sc = 1.0 / sqrt(Dii);
                s64[i] = sc;
                s32[i] = (float)sc;
            }
            continue;
        }
        double S = 0.0;
        uint32_t mask = 0;
        for (int l = 0; l < kp.L; ++l) {
            double q = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double dk = __dsub_rn(x[k], kp.centers[l * D + k]);
                q = __dadd_rn(q, __dmul_rn(dk, dk));
            }
            double rho = kp.radii[l];
            double s = __ddiv_rn(q, __dmul_rn(rho, rho));
            double e = 0.0;
            if (s < 1.0) {
                e = exp(kp.beta * (1.0 - 1.0 / (1.0 - s)));
                mask |= 1u << l;   // inside bump l (the far-field kernel's pattern)
            }
            double b = kp.amps[l] * e;
            B64[i * kp.L + l] = b;
            B32[i * kp.L + l] = (float)b;
            S = S + b * b;
        }
        if (ffmask) ffmask[i] = mask;
        double Dii = (S + kp.w0) + kp.sigma2;
        D64[i] = Dii;
        if (!(Dii > 0.0) || !isfinite(Dii)) {
            atomicOr(bad, 1);
            s64[i] = 0.0;
            s32[i] = 0.0f;
        } else {
            double sc = 1.0 / sqrt(Dii);
            s64[i] = sc;
            s32[i] = (float)sc;
        }
    }
}

// FP64 values of Ah on the assembled pattern: one warp per row, lanes over the row's entries.
// Every kernel here is symmetric bit for bit in its FP64 evaluation (squared differences, products
// of the two points' factors, the product s_i s_j of the Jacobi scales), and so is the pattern: row
// i evaluates only its pairs j >= i and writes each value also into row j, at the position of
// column i that a binary search of row j's ascending columns finds.  Half the FP64 evaluations,
// the same matrix.  A row j without column i (never, for a symmetric pattern) sets bit 0 of *bad.
template <int D>
__global__ void __launch_bounds__(256)
k_values64(const double4_16a *__restrict__ X64, const int32_t *__restrict__ rowptr,
           const int32_t *__restrict__ col, int64_t n, KernelParams kp, const double *__restrict__ B64,
           const double *__restrict__ s64, double *__restrict__ val64, float *__restrict__ val32,
           const double4_16a *__restrict__ Lam, const double *__restrict__ Sig, int *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int L = kp.L;
    for (int64_t i = warp0; i < n; i += nwarps) {
        const double4_16a xi = X64[i];
        const double si = s64[i];
        const int p0 = rowptr[i], p1 = rowptr[i + 1];
        // first entry with column >= i (the diagonal is stored): a search over the row's columns
        int lo = p0, hi = p1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col[mid] < (int32_t)i) lo = mid + 1; else hi = mid;
        }
        for (int p = lo + lane; p < p1; p += kWarp) {
            const int j = col[p];
            double v;
            if (j == i) {
                v = 1.0;
            } else if (kp.family == 2) {
                // Sec. 4.5: w0 phi(|D| / r) inside the ball + kappa(|D|) sum_l b_l(x_i) b_l(x_j)
                const double4_16a xj = X64[j];
                const double a[4] = {xi.x, xi.y, xi.z, xi.w}, b[4] = {xj.x, xj.y, xj.z, xj.w};
                double q = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    double dk = __dsub_rn(a[k], b[k]);
                    q = __dadd_rn(q, __dmul_rn(dk, dk));
                }
                double S = 0.0;
                for (int l = 0; l < L; ++l) S = fma(B64[i * L + l], B64[(int64_t)j * L + l], S);
                const double loc = q < kp.r * kp.r ? kp.w0 * wendland<double>(kp.kind, D, sqrt(q) * kp.inv_r) : 0.0;
                const double kap = exp(-q / (2.0 * kp.ell[0] * kp.ell[0]));
                v = (loc + kap * S) * (si * s64[j]);
            } else if (kp.family == 1) {
                // Eq. 6: s_i s_j prod_k (l_ik l_jk)^(1/4) / ((l_ik + l_jk) / 2)^(1/2) phi(sqrt(Q) / r)
                const double4_16a li = Lam[i], lj = Lam[j];
                const double q = wc_q<D>(xi, X64[j], li, lj);
                const double ai[4] = {li.x, li.y, li.z, li.w}, aj[4] = {lj.x, lj.y, lj.z, lj.w};
                double pref = 1.0;
#pragma unroll
                for (int k = 0; k < D; ++k) pref = pref * (sqrt(sqrt(ai[k] * aj[k])) / sqrt((ai[k] + aj[k]) * 0.5));
                const double phi = wendland<double>(kp.kind, D, sqrt(q) * kp.inv_r);
                v = (Sig[i] * Sig[j] * pref * phi) * (si * s64[j]);
            } else {
                const double4_16a xj = X64[j];
                const double a[4] = {xi.x, xi.y, xi.z, xi.w}, b[4] = {xj.x, xj.y, xj.z, xj.w};
                double q = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    double dk = __dsub_rn(a[k], b[k]);
                    q = __dadd_rn(q, __dmul_rn(dk, dk));
                }
                double t = sqrt(q) * kp.inv_r;
                double phi = wendland<double>(kp.kind, D, t);
                double S = 0.0;
                for (int l = 0; l < L; ++l) S = fma(B64[i * L + l], B64[(int64_t)j * L + l], S);
                v = (phi * (S + kp.w0)) * (si * s64[j]);
            }
            val64[p] = v;
            if (val32) val32[p] = (float)v;   // the FP32 copy is the FP64 value rounded once
            if (j != i) {
                int a = rowptr[j], e = rowptr[j + 1];
                while (a < e) {
                    const int mid = (a + e) >> 1;
                    if (col[mid] < (int32_t)i) a = mid + 1; else e = mid;
                }
                if (a < rowptr[j + 1] && col[a] == (int32_t)i) {
                    val64[a] = v;
                    if (val32) val32[a] = (float)v;
                } else {
                    atomicOr(bad, 1);
                }
            }
        }
    }
}

// Far-field kernel: bump l's members (points strictly inside it, ascending sorted index).
__global__ void k_ff_flags(const uint32_t *__restrict__ mask, int64_t n, int l, int32_t *__restrict__ flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (int32_t)((mask[i] >> l) & 1u);
}

__global__ void k_ff_members(const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int64_t n,
                             int32_t *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = (int32_t)i;
}

// Row i of the far-field pattern: the union of its Euclidean row and the member lists of the bumps
// it lies in, by a warp merge with the list heads in lanes (lane 0: the Euclidean row, lane 1 + l:
// bump l).  COUNT writes the union's length, FILL its columns (ascending, each once).
template <bool FILL>
__global__ void __launch_bounds__(256)
k_ff_union(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, const uint32_t *__restrict__ mask,
           const int32_t *__restrict__ mptr, const int32_t *__restrict__ mcol, int64_t n,
           const int32_t *__restrict__ uptr, int32_t *__restrict__ ucnt, int32_t *__restrict__ ucol)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const uint32_t mi = mask[i];
        int pos = 0, end = 0;
        if (lane == 0) {
            pos = rowptr[i];
            end = rowptr[i + 1];
        } else if (lane <= 31 && ((mi >> (lane - 1)) & 1u)) {
            pos = mptr[lane - 1];
            end = mptr[lane];
        }
        const int *src = lane == 0 ? col : mcol;
        int head = pos < end ? src[pos] : INT_MAX;
        int64_t out = FILL ? uptr[i] : 0;
        int emitted = 0;
        for (;;) {
            int mn = head;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            if (mn == INT_MAX) break;
            if (FILL && lane == 0) ucol[out + emitted] = mn;
            ++emitted;
            if (head == mn) {
                ++pos;
                head = pos < end ? src[pos] : INT_MAX;
            }
        }
        if (!FILL && lane == 0) ucnt[i] = emitted;
    }
}

// Replace the Euclidean CSR by its union with the bumps' member blocks (far-field kernel).
static gp2s_status far_field_union(gp2s_ctx *c, int64_t n, int L, int64_t *nnz)
{
    const unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    // member lists: one scan per bump
    GP2S_TRY(ensure(c, c->ff_flag, sizeof(int32_t) * (size_t)(n + 1) * 2));
    int32_t *flag = c->ff_flag.as<int32_t>(), *pos = flag + n + 1;
    std::vector<int32_t> hptr(L + 1, 0);
    std::vector<int64_t> cnt(L, 0);
    for (int l = 0; l < L; ++l) {
        k_ff_flags<<<gb, 256, 0, c->stream>>>(c->ff_mask.as<uint32_t>(), n, l, flag);
        GP2S_LAUNCH(c);
        GP2S_TRY(scan_counts_i32(c, flag, pos, n, &cnt[l]));
        hptr[l + 1] = hptr[l] + (int32_t)cnt[l];
    }
    GP2S_TRY(ensure(c, c->ff_mptr, sizeof(int32_t) * (size_t)(L + 1)));
    GP2S_TRY(ensure(c, c->ff_mcol, sizeof(int32_t) * (size_t)(hptr[L] > 0 ? hptr[L] : 1)));
    GP2S_CUDA(c, cudaMemcpyAsync(c->ff_mptr.p, hptr.data(), sizeof(int32_t) * (L + 1), cudaMemcpyHostToDevice, c->stream));
    for (int l = 0; l < L; ++l) {
        if (cnt[l] == 0) continue;
        k_ff_flags<<<gb, 256, 0, c->stream>>>(c->ff_mask.as<uint32_t>(), n, l, flag);
        GP2S_LAUNCH(c);
        int64_t t = 0;
        GP2S_TRY(scan_counts_i32(c, flag, pos, n, &t));
        k_ff_members<<<gb, 256, 0, c->stream>>>(flag, pos, n, c->ff_mcol.as<int32_t>() + hptr[l]);
        GP2S_LAUNCH(c);
    }
    // union count -> scan -> fill
    const unsigned gw = (unsigned)std::min<int64_t>(ceil_div(n * 32, 256), 152 * 32);
    GP2S_TRY(ensure(c, c->ff_ucnt, sizeof(int32_t) * (size_t)(n + 1)));
    GP2S_TRY(ensure(c, c->ff_uptr, sizeof(int32_t) * (size_t)(n + 1)));
    k_ff_union<false><<<gw, 256, 0, c->stream>>>(c->rowptr.as<int32_t>(), c->col.as<int32_t>(), c->ff_mask.as<uint32_t>(),
                                                 c->ff_mptr.as<int32_t>(), c->ff_mcol.as<int32_t>(), n, nullptr,
                                                 c->ff_ucnt.as<int32_t>(), nullptr);
    GP2S_LAUNCH(c);
    int64_t unnz = 0;
    GP2S_TRY(scan_counts_i32(c, c->ff_ucnt.as<int32_t>(), c->ff_uptr.as<int32_t>(), n, &unnz));
    if (unnz > (int64_t)INT32_MAX - 1) return set_err(c, GP2S_EOVERFLOW, "far-field pattern exceeds int32 entries");
    GP2S_TRY(ensure(c, c->ff_ucol, sizeof(int32_t) * (size_t)(unnz > 0 ? unnz : 1)));
    k_ff_union<true><<<gw, 256, 0, c->stream>>>(c->rowptr.as<int32_t>(), c->col.as<int32_t>(), c->ff_mask.as<uint32_t>(),
                                                c->ff_mptr.as<int32_t>(), c->ff_mcol.as<int32_t>(), n,
                                                c->ff_uptr.as<int32_t>(), nullptr, c->ff_ucol.as<int32_t>());
    GP2S_LAUNCH(c);
    std::swap(c->rowptr, c->ff_uptr);
    std::swap(c->col, c->ff_ucol);
    std::swap(c->rowcnt, c->ff_ucnt);
    *nnz = unnz;
    return GP2S_OK;
}

__global__ void k_rowcnt_minmax(const int32_t *__restrict__ cnt, int64_t n, int *__restrict__ mm)
{
    int lo = INT32_MAX, hi = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        lo = min(lo, cnt[i]);
        hi = max(hi, cnt[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

template <int D, bool FILL>
gp2s_status launch_assemble(gp2s_ctx *c, const AsmArgs &a, const GridParams &g, const SupportParams &sp,
                            const KernelParams &kp, int64_t nitems)
{
    size_t smem = asm_smem_bytes(D, FILL, kp.L);
    GP2S_TRY(smem_attr(c, (const void *)k_assemble<D, FILL>, smem));
    k_assemble<D, FILL><<<(unsigned)nitems, kAsmThreads, smem, c->stream>>>(a, g, sp, kp);
    GP2S_LAUNCH(c);
    return GP2S_OK;
}

template <bool FILL>
gp2s_status dispatch_assemble(gp2s_ctx *c, int d, const AsmArgs &a, const GridParams &g,
                              const SupportParams &sp, const KernelParams &kp, int64_t nitems)
{
    switch (d) {
    case 1: return launch_assemble<1, FILL>(c, a, g, sp, kp, nitems);
    case 2: return launch_assemble<2, FILL>(c, a, g, sp, kp, nitems);
    case 3: return launch_assemble<3, FILL>(c, a, g, sp, kp, nitems);
    default: return launch_assemble<4, FILL>(c, a, g, sp, kp, nitems);
    }
}

float round_down_f(double x)
{
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -FLT_MAX);
    return f;
}
float round_up_f(double x)
{
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, FLT_MAX);
    return f;
}

}  // namespace

gp2s_status validate_hyper(gp2s_ctx *c, const gp2s_hyper *h)
{
    if (!h) return set_err(c, GP2S_EINVAL, "hyper is NULL");
    if (h->d < 1 || h->d > kMaxDim) return set_err(c, GP2S_EINVAL, "d must be in 1..4");
    if (h->L < 0 || h->L > kMaxBumps) return set_err(c, GP2S_EINVAL, "L must be in 0..32");
    if (!(h->r > 0.0) || !std::isfinite(h->r)) return set_err(c, GP2S_EINVAL, "r must be finite and > 0");
    if (!(h->sigma2 >= 0.0) || !std::isfinite(h->sigma2)) return set_err(c, GP2S_EINVAL, "sigma2 must be finite and >= 0");
    if (!std::isfinite(h->beta) || !std::isfinite(h->w0)) return set_err(c, GP2S_EINVAL, "beta / w0 must be finite");
    if (h->kind != GP2S_WENDLAND_C2 && h->kind != GP2S_WENDLAND_C6_PAPER) return set_err(c, GP2S_EINVAL, "unknown Wendland kind");
    if (h->kind == GP2S_WENDLAND_C6_PAPER && h->d > 3) return set_err(c, GP2S_EINVAL, "Eq. 3 C6 form is positive definite only for d <= 3");
    if (h->L > 0 && (!h->centers || !h->radii || !h->amps)) return set_err(c, GP2S_EINVAL, "bump arrays are NULL");
    if (h->family != GP2S_KERNEL_PRODUCT && h->family != GP2S_KERNEL_WENDCONV && h->family != GP2S_KERNEL_FARFIELD)
        return set_err(c, GP2S_EINVAL, "unknown kernel family");
    if (h->family == GP2S_KERNEL_FARFIELD) {
        if (!h->ell || !(h->ell[0] > 0.0) || !std::isfinite(h->ell[0]))
            return set_err(c, GP2S_EINVAL, "the far-field core length ell[0] must be finite and > 0");
        if (h->L > 31) return set_err(c, GP2S_EINVAL, "the far-field kernel takes at most 31 bumps");
    }
    if (h->family == GP2S_KERNEL_WENDCONV) {
        if (!h->ell || (h->L > 0 && !h->G)) return set_err(c, GP2S_EINVAL, "ell / G arrays are NULL");
        for (int k = 0; k < h->d; ++k)
            if (!(h->ell[k] > 0.0) || !std::isfinite(h->ell[k])) return set_err(c, GP2S_EINVAL, "ell must be finite and > 0");
        for (int e = 0; e < h->L * h->d; ++e)
            if (!(h->G[e] >= 0.0) || !std::isfinite(h->G[e])) return set_err(c, GP2S_EINVAL, "G must be finite and >= 0");
    }
    for (int l = 0; l < h->L; ++l) {
        if (!(h->radii[l] > 0.0) || !std::isfinite(h->radii[l]) || !std::isfinite(h->amps[l]))
            return set_err(c, GP2S_EINVAL, "bump radius must be > 0 and amplitudes finite");
        for (int k = 0; k < h->d; ++k)
            if (!std::isfinite(h->centers[l * h->d + k])) return set_err(c, GP2S_EINVAL, "bump center not finite");
    }
    return GP2S_OK;
}

KernelParams make_kernel_params(const gp2s_hyper *h)
{
    KernelParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.d = h->d;
    kp.L = h->L;
    kp.kind = h->kind;
    kp.r = h->r;
    kp.inv_r = 1.0 / h->r;
    kp.sigma2 = h->sigma2;
    kp.beta = h->beta;
    kp.w0 = h->w0;
    kp.family = h->family;
    for (int l = 0; l < h->L; ++l) {
        for (int k = 0; k < h->d; ++k) kp.centers[l * h->d + k] = h->centers[l * h->d + k];
        kp.radii[l] = h->radii[l];
        kp.amps[l] = h->amps[l];
    }
    if (h->family == GP2S_KERNEL_WENDCONV) {
        for (int k = 0; k < h->d; ++k) kp.ell[k] = h->ell[k];
        for (int e = 0; e < h->L * h->d; ++e) kp.G[e] = h->G[e];
    }
    if (h->family == GP2S_KERNEL_FARFIELD) kp.ell[0] = h->ell[0];
    return kp;
}

// Largest lambda_k(x_i) of the Wendland convolution's length-scale field over the points (per-CTA
// maxima): the cell edge must cover r sqrt(max lambda), the farthest a stored pair can reach.
template <int D>
__global__ void k_wc_lammax(const double *__restrict__ X, int64_t n, KernelParams kp, double *__restrict__ part)
{
    __shared__ double sh[256];
    double mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x[D], sig, lam[D];
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = X[i * D + k];
        wc_fields<D>(x, kp, sig, lam, nullptr);
#pragma unroll
        for (int k = 0; k < D; ++k) mx = fmax(mx, lam[k]);
    }
    sh[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

static gp2s_status wc_lambda_max(gp2s_ctx *c, const double *X, int64_t n, const KernelParams &kp, double *lmax)
{
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)c->num_sms * 2));
    GP2S_TRY(ensure(c, c->bbox_part, sizeof(double) * (size_t)(nb > 2 * kMaxDim * 304 ? nb : 2 * kMaxDim * 304) + 64));
    double *part = c->bbox_part.as<double>();
    switch (kp.d) {
    case 1: k_wc_lammax<1><<<nb, 256, 0, c->stream>>>(X, n, kp, part); break;
    case 2: k_wc_lammax<2><<<nb, 256, 0, c->stream>>>(X, n, kp, part); break;
    case 3: k_wc_lammax<3><<<nb, 256, 0, c->stream>>>(X, n, kp, part); break;
    default: k_wc_lammax<4><<<nb, 256, 0, c->stream>>>(X, n, kp, part); break;
    }
    GP2S_LAUNCH(c);
    std::vector<double> h(nb);
    GP2S_CUDA(c, cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    double m = 0.0;
    for (double v : h) m = std::fmax(m, v);
    *lmax = m;
    return GP2S_OK;
}

// Order-independent 64-bit fingerprint of X (n x d FP64): the sum over elements of a SplitMix64-style
// mix of (bits, position), so equal inputs give equal hashes whatever the thread schedule.
__global__ void k_hash_x(const double *__restrict__ X, int64_t cnt, unsigned long long *__restrict__ out)
{
    unsigned long long acc = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)__double_as_longlong(X[e]) + 0x9E3779B97F4A7C15ull * (unsigned long long)(e + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        acc += z ^ (z >> 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

static gp2s_status hash_x(gp2s_ctx *c, const double *X, int64_t cnt, uint64_t *hash)
{
    GP2S_TRY(ensure(c, c->counters, 256));
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(c->counters.as<char>() + 160);
    GP2S_CUDA(c, cudaMemsetAsync(acc, 0, sizeof(unsigned long long), c->stream));
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cnt, 256), (int64_t)c->num_sms * 8));
    k_hash_x<<<gb, 256, 0, c->stream>>>(X, cnt, acc);
    GP2S_LAUNCH(c);
    unsigned long long h = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    *hash = h;
    return GP2S_OK;
}

template <int D>
static void launch_bumps(gp2s_ctx *c, int64_t n, const KernelParams &kp, int *dbad)
{
    const unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 16);
    k_bumps<D><<<gb, 256, 0, c->stream>>>(c->Xs64.as<double4_16a>(), n, kp, c->B64.as<double>(), c->B32.as<float>(),
                                          c->D64.as<double>(), c->s64.as<double>(), c->s32.as<float>(), dbad,
                                          c->wc_lam.as<double4_16a>(), c->wc_sig.as<double>(),
                                          kp.family == 2 ? c->ff_mask.as<uint32_t>() : nullptr);
}

template <int D>
static void launch_values(gp2s_ctx *c, int64_t n, const KernelParams &kp, bool mixed, int *vbad)
{
    const unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n * 32, 256), 152 * 32);
    k_values64<D><<<gb, 256, 0, c->stream>>>(c->Xs64.as<double4_16a>(), c->rowptr.as<int32_t>(), c->col.as<int32_t>(), n,
                                             kp, c->B64.as<double>(), c->s64.as<double>(), c->val64.as<double>(),
                                             mixed ? c->val32.as<float>() : nullptr, c->wc_lam.as<double4_16a>(),
                                             c->wc_sig.as<double>(), vbad);
}

// Bump tables (FP64 and FP32), the diagonal and the Jacobi scales of the current points.
static gp2s_status bumps_and_checks(gp2s_ctx *c, int64_t n, int d, const KernelParams &kp, int *dbad)
{
    switch (d) {
    case 1: launch_bumps<1>(c, n, kp, dbad); break;
    case 2: launch_bumps<2>(c, n, kp, dbad); break;
    case 3: launch_bumps<3>(c, n, kp, dbad); break;
    default: launch_bumps<4>(c, n, kp, dbad); break;
    }
    GP2S_LAUNCH(c);
    return GP2S_OK;
}

// The values of every stored pair of the current pattern (synchronises the stream: the mirror
// check is read back).
static gp2s_status values_pass(gp2s_ctx *c, int64_t n, int d, const KernelParams &kp, bool mixed)
{
    GP2S_TRY(ensure(c, c->counters, 256));
    int *vbad = reinterpret_cast<int *>(c->counters.as<char>() + 32);
    GP2S_CUDA(c, cudaMemsetAsync(vbad, 0, sizeof(int), c->stream));
    switch (d) {
    case 1: launch_values<1>(c, n, kp, mixed, vbad); break;
    case 2: launch_values<2>(c, n, kp, mixed, vbad); break;
    case 3: launch_values<3>(c, n, kp, mixed, vbad); break;
    default: launch_values<4>(c, n, kp, mixed, vbad); break;
    }
    GP2S_LAUNCH(c);
    int hv = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&hv, vbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hv) return set_err(c, GP2S_EINVAL, "internal: the assembled pattern is not symmetric");
    return GP2S_OK;
}

// Same points and the same r as the last assembly: the pattern (and the sorted points, the cell
// table and the CSR structure) depend on nothing else, so only the bump tables, the diagonal and
// the values are recomputed for the new hyperparameters (the "pattern cached" evaluation).
static gp2s_status refresh_values(gp2s_ctx *c, const gp2s_hyper *h, const gp2s_opts *o)
{
    Assembled &A = c->A;
    const int64_t n = A.n;
    const int d = A.d;
    cudaEvent_t ev[2];
    for (int k = 0; k < 2; ++k) GP2S_CUDA(c, cudaEventCreate(&ev[k]));
    struct EvGuard { cudaEvent_t *e; ~EvGuard() { for (int k = 0; k < 2; ++k) cudaEventDestroy(e[k]); } } guard{ev};
    GP2S_CUDA(c, cudaEventRecord(ev[0], c->stream));
    const KernelParams kp = make_kernel_params(h);
    GP2S_TRY(ensure(c, c->counters, 256));
    int *dbad = c->counters.as<int>();
    GP2S_CUDA(c, cudaMemsetAsync(dbad, 0, sizeof(int), c->stream));
    GP2S_TRY(bumps_and_checks(c, n, d, kp, dbad));
    GP2S_TRY(values_pass(c, n, d, kp, o->precision == GP2S_PREC_MIXED));
    GP2S_CUDA(c, cudaEventRecord(ev[1], c->stream));
    int hbad = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hbad) {
        c->pat_valid = false;
        return set_err(c, GP2S_ENOTPD, "a diagonal entry of A is zero (sigma2 = 0 and the point lies outside every bump, w0 = 0)");
    }
    gp2s_assemble_info &info = A.info;
    info.ms_geometry = info.ms_count = info.ms_fill = 0.0f;
    cudaEventElapsedTime(&info.ms_values64, ev[0], ev[1]);
    info.pattern_reused = 1;
    A.kp = kp;
    A.opts = *o;
    A.valid = true;
    return GP2S_OK;
}

gp2s_status assemble_problem(gp2s_ctx *c, int64_t n, const double *X_dev, const gp2s_hyper *h,
                             const gp2s_opts *o)
{
    Assembled &A = c->A;
    A.valid = false;
    c->have_solution = false;
    c->have_probes = false;
    c->have_exact = false;
    c->rb_valid = false;
    c->bj_valid = false;
    const int d = h->d;
    uint64_t xhash = 0;
    GP2S_TRY(hash_x(c, X_dev, n * d, &xhash));
    if (o->pattern_cache == 0 && h->family == GP2S_KERNEL_PRODUCT && c->pat_valid && c->pat_n == n && c->pat_d == d &&
        std::memcmp(&c->pat_r, &h->r, sizeof(double)) == 0 && c->pat_exact == o->exact_support &&
        c->pat_precision == o->precision && c->pat_hash == xhash)
        return refresh_values(c, h, o);
    c->pat_valid = false;
    c->rb_pattern_valid = false;
    cudaEvent_t ev[5];
    for (int k = 0; k < 5; ++k) GP2S_CUDA(c, cudaEventCreate(&ev[k]));
    struct EvGuard { cudaEvent_t *e; ~EvGuard() { for (int k = 0; k < 5; ++k) cudaEventDestroy(e[k]); } } guard{ev};
    GP2S_CUDA(c, cudaEventRecord(ev[0], c->stream));

    // ---- bounding box, grid, guard band (host arithmetic in FP64, no contraction) ----
    double box[2 * kMaxDim + 1];
    GP2S_TRY(geom_bbox(c, X_dev, n, d, box));
    int bad = 0;
    std::memcpy(&bad, &box[2 * kMaxDim], sizeof(int));
    if (bad) return set_err(c, GP2S_EINVAL, "X contains NaN or infinity");
    GridParams g;
    std::memset(&g, 0, sizeof(g));
    g.d = d;
    // the farthest a stored pair reaches: r (product kernel), r sqrt(max lambda) (convolution)
    double r_eff = h->r;
    if (h->family == GP2S_KERNEL_WENDCONV) {
        double lmax = 0.0;
        GP2S_TRY(ensure(c, c->wc_lam, sizeof(double4_16a) * (size_t)n));
        GP2S_TRY(ensure(c, c->wc_sig, sizeof(double) * (size_t)n));
        GP2S_TRY(wc_lambda_max(c, X_dev, n, make_kernel_params(h), &lmax));
        if (!(lmax > 0.0) || !std::isfinite(lmax)) return set_err(c, GP2S_EINVAL, "length-scale field not finite");
        r_eff = h->r * std::sqrt(lmax) * (1.0 + std::ldexp(1.0, -30));
        A.wc_lmax = lmax;
    }
    double h_cell = r_eff * (1.0 + std::ldexp(1.0, -20));
    double M = 0.0;
    for (int k = 0; k < d; ++k) {
        M = std::fmax(M, std::fmax(std::fabs(box[k]), std::fabs(box[kMaxDim + k])));
        g.origin[k] = box[k];
    }
    const int max_bits = d == 1 ? 30 : 64 / d;
    int fine = 2;
    for (;;) {
        double inv_h = 1.0 / h_cell;
        int cb = 1;
        for (int k = 0; k < d; ++k) {
            double ext = (box[kMaxDim + k] - box[k]) * inv_h;
            int64_t dims = (int64_t)std::floor(ext) + 1;
            g.dims[k] = dims;
            while ((int64_t(1) << cb) < dims) ++cb;
        }
        if (cb + fine > max_bits) fine = std::max(0, max_bits - cb);
        if (cb + fine <= max_bits) {
            g.inv_h = inv_h;
            g.h = h_cell;
            g.fine_bits = fine;
            g.bits = cb + fine;
            break;
        }
        h_cell *= 2.0;   // grid too fine for the key width: coarser cells are still correct
    }
    SupportParams sp;
    sp.r2 = h->r * h->r;
    const double re2 = r_eff * r_eff;
    const double u = std::ldexp(1.0, -24);
    const double ratio = M / r_eff;
    bool exact = o->exact_support != 0 || ratio > 1e6 || re2 < 1e-30 || M > 1e18;
    double delta = 32.0 * u + 16.0 * d * u * u * ratio;
    if (exact) {
        sp.thr_lo = -1.0f;
        sp.thr_hi = FLT_MAX;
        delta = INFINITY;
    } else {
        sp.thr_lo = round_down_f(re2 * (1.0 - delta));
        sp.thr_hi = round_up_f(re2 * (1.0 + delta));
    }
    if (h->family == GP2S_KERNEL_WENDCONV) sp.thr_lo = -1.0f;   // the FP32 test only rejects

    // ---- sort, permute, cells ----
    GP2S_TRY(geom_sort(c, X_dev, n, g));
    GP2S_TRY(geom_permute(c, X_dev, n, d));
    int64_t ncells = 0, nitems = 0;
    GP2S_TRY(geom_cells(c, n, g, kRowsPerItem, &ncells, &nitems));
    KernelParams kp = make_kernel_params(h);

    // ---- bumps, diagonal, Jacobi scales ----
    const int L = h->L;
    GP2S_TRY(ensure(c, c->B64, sizeof(double) * (size_t)n * (L > 0 ? L : 1)));
    GP2S_TRY(ensure(c, c->B32, sizeof(float) * (size_t)n * (L > 0 ? L : 1)));
    if (h->family == GP2S_KERNEL_FARFIELD) GP2S_TRY(ensure(c, c->ff_mask, sizeof(uint32_t) * (size_t)n));
    GP2S_TRY(ensure(c, c->D64, sizeof(double) * n));
    GP2S_TRY(ensure(c, c->s64, sizeof(double) * n));
    GP2S_TRY(ensure(c, c->s32, sizeof(float) * n));
    GP2S_TRY(ensure(c, c->counters, 256));
    int *dbad = c->counters.as<int>();
    unsigned long long *stats = reinterpret_cast<unsigned long long *>(c->counters.as<char>() + 64);
    int *mm = reinterpret_cast<int *>(c->counters.as<char>() + 128);
    GP2S_CUDA(c, cudaMemsetAsync(c->counters.p, 0, 256, c->stream));
    GP2S_TRY(bumps_and_checks(c, n, d, kp, dbad));
    GP2S_CUDA(c, cudaEventRecord(ev[1], c->stream));

    // ---- count -> scan ----
    GP2S_TRY(ensure(c, c->rowcnt, sizeof(int32_t) * (n + 1)));
    GP2S_TRY(ensure(c, c->rowptr, sizeof(int32_t) * (n + 1)));
    AsmArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Xhi = c->Xhi.as<float4>();
    a.Xlo = c->Xlo.as<float4>();
    a.X64 = c->Xs64.as<double4_16a>();
    a.items = c->items.as<int4>();
    a.cell_start = c->cell_start.as<int32_t>();
    a.cell_key = cell_keys_ptr(c, ncells);
    a.ncells = ncells;
    a.B32 = c->B32.as<float>();
    a.s32 = c->s32.as<float>();
    a.Lam = c->wc_lam.as<double4_16a>();
    a.rowcnt = c->rowcnt.as<int32_t>();
    a.stats = stats;
    if (nitems > 0) GP2S_TRY(dispatch_assemble<false>(c, d, a, g, sp, kp, nitems));
    GP2S_CUDA(c, cudaEventRecord(ev[2], c->stream));
    int64_t nnz = 0;
    GP2S_TRY(scan_counts_i32(c, c->rowcnt.as<int32_t>(), c->rowptr.as<int32_t>(), n, &nnz));
    int hbad = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hbad) return set_err(c, GP2S_ENOTPD, "a diagonal entry of A is zero (sigma2 = 0 and the point lies outside every bump, w0 = 0)");

    // ---- fill ----
    const bool mixed = o->precision == GP2S_PREC_MIXED;
    GP2S_TRY(ensure(c, c->col, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)));
    if (mixed) GP2S_TRY(ensure(c, c->val32, sizeof(float) * (size_t)(nnz > 0 ? nnz : 1)));
    GP2S_TRY(ensure(c, c->val64, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1)));
    a.rowptr = c->rowptr.as<int32_t>();
    a.col = c->col.as<int32_t>();
    if (nitems > 0) GP2S_TRY(dispatch_assemble<true>(c, d, a, g, sp, kp, nitems));
    if (h->family == GP2S_KERNEL_FARFIELD) {
        GP2S_TRY(far_field_union(c, n, L, &nnz));
        if (mixed) GP2S_TRY(ensure(c, c->val32, sizeof(float) * (size_t)(nnz > 0 ? nnz : 1)));
        GP2S_TRY(ensure(c, c->val64, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1)));
    }
    GP2S_CUDA(c, cudaEventRecord(ev[3], c->stream));

    // ---- values: every stored pair in FP64 (and its FP32 rounding in MIXED precision) ----
    GP2S_TRY(values_pass(c, n, d, kp, mixed));
    GP2S_CUDA(c, cudaEventRecord(ev[4], c->stream));
    {
        int init[2] = {INT32_MAX, 0};
        GP2S_CUDA(c, cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
        unsigned gb = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 4);
        k_rowcnt_minmax<<<gb, 256, 0, c->stream>>>(c->rowcnt.as<int32_t>(), n, mm);
        GP2S_LAUNCH(c);
    }
    unsigned long long hstats[2];
    int hmm[2];
    GP2S_CUDA(c, cudaMemcpyAsync(hstats, stats, sizeof(hstats), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));

    gp2s_assemble_info &info = A.info;
    std::memset(&info, 0, sizeof(info));
    info.n = n;
    info.nnz = nnz;
    info.candidates = (int64_t)hstats[0];
    info.band_pairs = (int64_t)hstats[1];
    info.ncells = ncells;
    info.nnz_row_min = hmm[0];
    info.nnz_row_max = hmm[1];
    info.guard_delta = delta;
    info.cell_h = g.h;
    cudaEventElapsedTime(&info.ms_geometry, ev[0], ev[1]);
    cudaEventElapsedTime(&info.ms_count, ev[1], ev[2]);
    cudaEventElapsedTime(&info.ms_fill, ev[2], ev[3]);
    cudaEventElapsedTime(&info.ms_values64, ev[3], ev[4]);

    A.n = n;
    A.nnz = nnz;
    A.ncells = ncells;
    A.nitems = nitems;
    A.d = d;
    A.L = L;
    A.precision = o->precision;
    A.kp = kp;
    A.gp = g;
    A.sp = sp;
    A.opts = *o;
    A.valid = true;
    c->pat_valid = true;
    c->pat_n = n;
    c->pat_d = d;
    c->pat_r = h->r;
    c->pat_exact = o->exact_support;
    c->pat_precision = o->precision;
    c->pat_hash = xhash;
    return GP2S_OK;
}

}  // namespace gp2s
