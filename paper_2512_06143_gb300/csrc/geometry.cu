// geometry.cu -- bounding box, Morton keys of a uniform cell grid, point permutation, cell table.
//
// This replaces the paper's all-pairs block decomposition (Sec. 4.6, App. B.7: every block of the
// n x n covariance is evaluated because the non-zeros are not known in advance).  The kernel of
// Sec. 4.1 carries the Wendland factor phi(|xi - xj| / r), which is zero for |xi - xj| >= r, so a
// uniform grid of cells with edge h >= r puts every stored pair into two cells whose integer
// coordinates differ by at most one per dimension.  Sorting the points along a Morton curve of a
// finer grid (2^F sub-cells per cell edge) keeps each cell contiguous and orders the points inside a
// cell spatially, which is what the SpMM's cache reuse relies on.
#include "gp2s_geometry.cuh"

namespace gp2s {

namespace {

constexpr int kBoxThreads = 256;

__global__ void __launch_bounds__(kBoxThreads)
k_bbox_partial(const double *__restrict__ X, int64_t n, int d, double *__restrict__ part,
               int *__restrict__ bad)
{
    double lo[kMaxDim], hi[kMaxDim];
    for (int k = 0; k < kMaxDim; ++k) { lo[k] = 1.0 / 0.0; hi[k] = -1.0 / 0.0; }
    int nonfinite = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < d; ++k) {
            double v = X[i * d + k];
            if (!isfinite(v)) nonfinite = 1;
            lo[k] = fmin(lo[k], v);
            hi[k] = fmax(hi[k], v);
        }
    }
    __shared__ double slo[kMaxDim][kBoxThreads], shi[kMaxDim][kBoxThreads];
    for (int k = 0; k < kMaxDim; ++k) { slo[k][threadIdx.x] = lo[k]; shi[k][threadIdx.x] = hi[k]; }
    if (nonfinite) atomicOr(bad, 1);
    __syncthreads();
    for (int s = kBoxThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < kMaxDim; ++k) {
                slo[k][threadIdx.x] = fmin(slo[k][threadIdx.x], slo[k][threadIdx.x + s]);
                shi[k][threadIdx.x] = fmax(shi[k][threadIdx.x], shi[k][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < kMaxDim; ++k) {
            part[blockIdx.x * 2 * kMaxDim + k] = slo[k][0];
            part[blockIdx.x * 2 * kMaxDim + kMaxDim + k] = shi[k][0];
        }
}

__global__ void k_bbox_final(const double *__restrict__ part, int nparts, double *__restrict__ box)
{
    // one thread per (lo/hi, dim): a short serial reduction in a fixed order
    int t = threadIdx.x;
    if (t >= 2 * kMaxDim) return;
    bool is_lo = t < kMaxDim;
    double v = is_lo ? 1.0 / 0.0 : -1.0 / 0.0;
    for (int p = 0; p < nparts; ++p) {
        double w = part[p * 2 * kMaxDim + t];
        v = is_lo ? fmin(v, w) : fmax(v, w);
    }
    box[t] = v;
}

// Spread the low `bits` bits of v so that bit b lands at position b * D + k.
template <int D>
__device__ __forceinline__ uint64_t morton(const uint64_t *f, int bits)
{
    uint64_t key = 0;
    for (int b = 0; b < bits; ++b)
#pragma unroll
        for (int k = 0; k < D; ++k) key |= ((f[k] >> b) & 1ull) << (b * D + k);
    return key;
}

template <int D>
__global__ void k_morton(const double *__restrict__ X, int64_t n, GridParams g,
                         uint64_t *__restrict__ keys, int32_t *__restrict__ idx)
{
    const double scale = (double)(1ll << g.fine_bits);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t f[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double y = __dmul_rn(__dsub_rn(X[i * D + k], g.origin[k]), g.inv_h);   // cell units
            double fy = floor(__dmul_rn(y, scale));                                // exact scaling
            int64_t fi = (int64_t)fy;
            int64_t fmax_ = (g.dims[k] << g.fine_bits) - 1;
            fi = fi < 0 ? 0 : (fi > fmax_ ? fmax_ : fi);
            f[k] = (uint64_t)fi;
        }
        keys[i] = morton<D>(f, g.bits);
        idx[i] = (int32_t)i;
    }
}

template <int D>
__global__ void k_permute(const double *__restrict__ X, const int32_t *__restrict__ perm, int64_t n,
                          double4_16a *__restrict__ Xs64, float4 *__restrict__ Xhi, float4 *__restrict__ Xlo,
                          int32_t *__restrict__ iperm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = perm[i];
        double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = X[o * D + k];
        float h[4], l[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            h[k] = __double2float_rn(v[k]);
            l[k] = __double2float_rn(__dsub_rn(v[k], (double)h[k]));   // v - hi is exact in FP64
        }
        Xs64[i] = make_double4_16a(v[0], v[1], v[2], v[3]);
        Xhi[i] = make_float4(h[0], h[1], h[2], h[3]);
        Xlo[i] = make_float4(l[0], l[1], l[2], l[3]);
        iperm[o] = (int32_t)i;
    }
}

__global__ void k_cell_flags(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             int32_t *__restrict__ flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift)) ? 1 : 0;
}

__global__ void k_cell_starts(const uint64_t *__restrict__ keys, const int32_t *__restrict__ flag,
                              const int32_t *__restrict__ cidx, int64_t n, int shift,
                              int32_t *__restrict__ cell_start, uint64_t *__restrict__ cell_key,
                              int64_t ncells)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            int32_t c = cidx[i];
            cell_start[c] = (int32_t)i;
            cell_key[c] = keys[i] >> shift;
        }
        if (i == 0) cell_start[ncells] = (int32_t)n;
    }
}

// Work items: each occupied cell is split into chunks of at most kRowsPerItem rows.
__global__ void k_item_counts(const int32_t *__restrict__ cell_start, int64_t ncells, int rpi,
                              int32_t *__restrict__ cnt)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int pop = cell_start[c + 1] - cell_start[c];
        cnt[c] = (pop + rpi - 1) / rpi;
    }
}

__global__ void k_item_fill(const int32_t *__restrict__ cell_start, const int32_t *__restrict__ ioff,
                            int64_t ncells, int rpi, int4 *__restrict__ items)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int s = cell_start[c], e = cell_start[c + 1];
        int k = ioff[c];
        for (int r = s; r < e; r += rpi, ++k) items[k] = make_int4((int)c, r, min(e, r + rpi), 0);
    }
}

inline unsigned grid_for(int64_t n, int threads, int cap = 152 * 16)
{
    int64_t b = ceil_div(n, threads);
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

gp2s_status geom_bbox(gp2s_ctx *c, const double *X, int64_t n, int d, double *box_host)
{
    const int nparts = 152 * 2;
    GP2S_TRY(ensure(c, c->bbox_part, sizeof(double) * 2 * kMaxDim * nparts + 64));
    GP2S_TRY(ensure(c, c->bbox, sizeof(double) * 2 * kMaxDim + 64));
    double *part = c->bbox_part.as<double>();
    int *bad = reinterpret_cast<int *>(c->bbox.as<char>() + sizeof(double) * 2 * kMaxDim);
    GP2S_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    k_bbox_partial<<<nparts, kBoxThreads, 0, c->stream>>>(X, n, d, part, bad);
    GP2S_LAUNCH(c);
    k_bbox_final<<<1, 32, 0, c->stream>>>(part, nparts, c->bbox.as<double>());
    GP2S_LAUNCH(c);
    GP2S_CUDA(c, cudaMemcpyAsync(box_host, c->bbox.p, sizeof(double) * 2 * kMaxDim + sizeof(int),
                                 cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    return GP2S_OK;
}

gp2s_status geom_sort(gp2s_ctx *c, const double *X, int64_t n, const GridParams &g)
{
    GP2S_TRY(ensure(c, c->keys, sizeof(uint64_t) * n));
    GP2S_TRY(ensure(c, c->keys2, sizeof(uint64_t) * n));
    GP2S_TRY(ensure(c, c->idx, sizeof(int32_t) * n));
    GP2S_TRY(ensure(c, c->idx2, sizeof(int32_t) * n));
    unsigned gb = grid_for(n, 256);
    switch (g.d) {
    case 1: k_morton<1><<<gb, 256, 0, c->stream>>>(X, n, g, c->keys.as<uint64_t>(), c->idx.as<int32_t>()); break;
    case 2: k_morton<2><<<gb, 256, 0, c->stream>>>(X, n, g, c->keys.as<uint64_t>(), c->idx.as<int32_t>()); break;
    case 3: k_morton<3><<<gb, 256, 0, c->stream>>>(X, n, g, c->keys.as<uint64_t>(), c->idx.as<int32_t>()); break;
    default: k_morton<4><<<gb, 256, 0, c->stream>>>(X, n, g, c->keys.as<uint64_t>(), c->idx.as<int32_t>()); break;
    }
    GP2S_LAUNCH(c);
    return radix_sort_pairs(c, c->keys.as<uint64_t>(), c->keys2.as<uint64_t>(), c->idx.as<int32_t>(),
                            c->idx2.as<int32_t>(), n, g.d * g.bits);
}

gp2s_status geom_permute(gp2s_ctx *c, const double *X, int64_t n, int d)
{
    GP2S_TRY(ensure(c, c->Xs64, sizeof(double4_16a) * n));
    GP2S_TRY(ensure(c, c->Xhi, sizeof(float4) * n));
    GP2S_TRY(ensure(c, c->Xlo, sizeof(float4) * n));
    GP2S_TRY(ensure(c, c->iperm, sizeof(int32_t) * n));
    GP2S_TRY(ensure(c, c->perm, sizeof(int32_t) * n));
    GP2S_CUDA(c, cudaMemcpyAsync(c->perm.p, c->idx.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
    unsigned gb = grid_for(n, 256);
    const int32_t *perm = c->perm.as<int32_t>();
    double4_16a *x64 = c->Xs64.as<double4_16a>();
    float4 *hi = c->Xhi.as<float4>(), *lo = c->Xlo.as<float4>();
    int32_t *ip = c->iperm.as<int32_t>();
    switch (d) {
    case 1: k_permute<1><<<gb, 256, 0, c->stream>>>(X, perm, n, x64, hi, lo, ip); break;
    case 2: k_permute<2><<<gb, 256, 0, c->stream>>>(X, perm, n, x64, hi, lo, ip); break;
    case 3: k_permute<3><<<gb, 256, 0, c->stream>>>(X, perm, n, x64, hi, lo, ip); break;
    default: k_permute<4><<<gb, 256, 0, c->stream>>>(X, perm, n, x64, hi, lo, ip); break;
    }
    GP2S_LAUNCH(c);
    return GP2S_OK;
}

gp2s_status geom_cells(gp2s_ctx *c, int64_t n, const GridParams &g, int rows_per_item,
                       int64_t *ncells_out, int64_t *nitems_out)
{
    int shift = g.d * g.fine_bits;
    GP2S_TRY(ensure(c, c->cell_flag, sizeof(int32_t) * (n + 1) * 2));
    int32_t *flag = c->cell_flag.as<int32_t>();
    int32_t *cidx = flag + n + 1;
    unsigned gb = grid_for(n, 256);
    k_cell_flags<<<gb, 256, 0, c->stream>>>(c->keys.as<uint64_t>(), n, shift, flag);
    GP2S_LAUNCH(c);
    int64_t ncells = 0;
    GP2S_TRY(scan_counts_i32(c, flag, cidx, n, &ncells));
    // cell_start (ncells + 1 int32) followed by the cell keys (ncells uint64, 8-byte aligned)
    size_t off_keys = ((sizeof(int32_t) * (ncells + 1) + 15) / 16) * 16;
    GP2S_TRY(ensure(c, c->cell_start, off_keys + sizeof(uint64_t) * ncells + 16));
    int32_t *cs = c->cell_start.as<int32_t>();
    uint64_t *ck = reinterpret_cast<uint64_t *>(c->cell_start.as<char>() + off_keys);
    k_cell_starts<<<gb, 256, 0, c->stream>>>(c->keys.as<uint64_t>(), flag, cidx, n, shift, cs, ck, ncells);
    GP2S_LAUNCH(c);
    // work items
    GP2S_TRY(ensure(c, c->item_cnt, sizeof(int32_t) * (ncells + 1) * 2));
    int32_t *icnt = c->item_cnt.as<int32_t>();
    int32_t *ioff = icnt + ncells + 1;
    unsigned gc = grid_for(ncells, 256);
    k_item_counts<<<gc, 256, 0, c->stream>>>(cs, ncells, rows_per_item, icnt);
    GP2S_LAUNCH(c);
    int64_t nitems = 0;
    GP2S_TRY(scan_counts_i32(c, icnt, ioff, ncells, &nitems));
    GP2S_TRY(ensure(c, c->items, sizeof(int4) * (nitems + 1)));
    k_item_fill<<<gc, 256, 0, c->stream>>>(cs, ioff, ncells, rows_per_item, c->items.as<int4>());
    GP2S_LAUNCH(c);
    *ncells_out = ncells;
    *nitems_out = nitems;
    return GP2S_OK;
}

const uint64_t *cell_keys_ptr(gp2s_ctx *c, int64_t ncells)
{
    size_t off_keys = ((sizeof(int32_t) * (ncells + 1) + 15) / 16) * 16;
    return reinterpret_cast<const uint64_t *>(c->cell_start.as<char>() + off_keys);
}

}  // namespace gp2s
