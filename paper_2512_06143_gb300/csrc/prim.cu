// prim.cu -- device primitives: exclusive scan (reduce-then-scan) and a stable LSD radix sort.
// Both are plain multi-launch algorithms: no inter-CTA waits, no atomics across CTAs.
#include <cstdio>

#include "gp2s_internal.cuh"

namespace gp2s {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048 elements per CTA

// Block-wide exclusive scan of one int64 per thread; returns the thread's exclusive prefix and
// writes the block total to *total.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t warp_sums[kScanThreads / kWarp];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kScanThreads / kWarp ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / kWarp) warp_sums[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    int64_t warp_off = wid > 0 ? warp_sums[wid - 1] : 0;
    *total = warp_sums[kScanThreads / kWarp - 1];
    __syncthreads();
    return warp_off + x - v;
}

template <class TIn>
__global__ void k_scan_reduce(const TIn *__restrict__ in, int64_t n, int64_t *__restrict__ bsum)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) s += (int64_t)in[i];
    }
    int64_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Exclusive scan of a tile with a per-CTA offset.  When `last_total` is non-null the CTA that
// owns element n-1 also writes out[n] = grand total.
template <class TIn, class TOut>
__global__ void k_scan_down(const TIn *__restrict__ in, int64_t n, const int64_t *__restrict__ boff,
                            TOut *__restrict__ out, int write_total)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? (int64_t)in[i] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t pre = block_exclusive_scan(s, &total) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = (TOut)pre;
        pre += v[k];
        if (write_total && i == n - 1) out[n] = (TOut)pre;
    }
}

// Generic exclusive scan with an int64 total (recursive over the per-CTA sums).
template <class TIn, class TOut>
gp2s_status scan_impl(gp2s_ctx *c, const TIn *in, TOut *out, int64_t n, int64_t *total_dev_slot,
                      int depth)
{
    if (n <= 0) return GP2S_OK;
    int64_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        k_scan_down<TIn, TOut><<<1, kScanThreads, 0, c->stream>>>(in, n, nullptr, out, 1);
        GP2S_LAUNCH(c);
        return GP2S_OK;
    }
    // scratch for the block sums of this level: two int64 arrays of nb (+1) entries
    DevBuf &tmp = depth == 0 ? c->scan_tmp : c->scan_tmp2;
    size_t need = sizeof(int64_t) * (size_t)(2 * nb + 2);
    if (depth > 1) return set_err(c, GP2S_EINVAL, "scan: input too large");
    GP2S_TRY(ensure(c, tmp, need));
    int64_t *bsum = tmp.as<int64_t>();
    int64_t *boff = bsum + nb + 1;
    k_scan_reduce<TIn><<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, bsum);
    GP2S_LAUNCH(c);
    GP2S_TRY((scan_impl<int64_t, int64_t>(c, bsum, boff, nb, nullptr, depth + 1)));
    k_scan_down<TIn, TOut><<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, boff, out, 1);
    GP2S_LAUNCH(c);
    (void)total_dev_slot;
    return GP2S_OK;
}

}  // namespace

gp2s_status scan_counts_i32(gp2s_ctx *c, const int32_t *in, int32_t *out, int64_t n, int64_t *total_host)
{
    // Scan in int64 into a temporary int64 array first when the total may overflow int32: we
    // compute the int64 total of the per-CTA sums and refuse if it exceeds 2^31 - 1.
    if (n <= 0) {
        if (total_host) *total_host = 0;
        GP2S_CUDA(c, cudaMemsetAsync(out, 0, sizeof(int32_t), c->stream));
        return GP2S_OK;
    }
    int64_t nb = ceil_div(n, kScanTile);
    GP2S_TRY(ensure(c, c->scan_tmp, sizeof(int64_t) * (size_t)(2 * nb + 2)));
    int64_t *bsum = c->scan_tmp.as<int64_t>();
    int64_t *boff = bsum + nb + 1;
    k_scan_reduce<int32_t><<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, bsum);
    GP2S_LAUNCH(c);
    if (nb > 1) {
        GP2S_TRY((scan_impl<int64_t, int64_t>(c, bsum, boff, nb, nullptr, 1)));
    } else {
        GP2S_CUDA(c, cudaMemsetAsync(boff, 0, sizeof(int64_t) * 2, c->stream));
        GP2S_CUDA(c, cudaMemcpyAsync(boff + 1, bsum, sizeof(int64_t), cudaMemcpyDeviceToDevice, c->stream));
    }
    int64_t tot = 0;
    GP2S_CUDA(c, cudaMemcpyAsync(&tot, boff + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    if (total_host) *total_host = tot;
    if (tot > (int64_t)INT32_MAX) return set_err(c, GP2S_EOVERFLOW, "nnz exceeds 2^31-1");
    k_scan_down<int32_t, int32_t><<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, boff, out, 1);
    GP2S_LAUNCH(c);
    return GP2S_OK;
}

gp2s_status scan_counts_i64(gp2s_ctx *c, const int32_t *in, int64_t *out, int64_t n, int64_t *total_host)
{
    if (n <= 0) {
        if (total_host) *total_host = 0;
        GP2S_CUDA(c, cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream));
        return GP2S_OK;
    }
    GP2S_TRY((scan_impl<int32_t, int64_t>(c, in, out, n, nullptr, 0)));
    if (total_host) {
        GP2S_CUDA(c, cudaMemcpyAsync(total_host, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        GP2S_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return GP2S_OK;
}

// ---------------------------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Per pass: per-tile digit histograms (digit-major
// layout), one exclusive scan, and a scatter that ranks keys stably inside each tile with
// warp match masks.  A tile is 8 warps x 16 rounds x 32 lanes = 4096 keys.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / kWarp;
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;

__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ hist,
             int64_t ntiles)
{
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)wid * (kRadixRounds * kWarp);
#pragma unroll 4
    for (int r = 0; r < kRadixRounds; ++r) {
        int64_t i = base + r * kWarp + lane;
        if (i < n) atomicAdd(&cnt[(int)((keys[i] >> shift) & 255u)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin,
                uint64_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n, int shift,
                const int32_t *__restrict__ offsets, int64_t ntiles)
{
    __shared__ int32_t wcnt[kRadixWarps][257];
    __shared__ int32_t toff[256];
    for (int t = threadIdx.x; t < kRadixWarps * 257; t += kRadixThreads) (&wcnt[0][0])[t] = 0;
    toff[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)wid * (kRadixRounds * kWarp);
    uint64_t key[kRadixRounds];
    int32_t val[kRadixRounds];
    int32_t rank[kRadixRounds];
    int16_t dig[kRadixRounds];
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        int64_t i = base + r * kWarp + lane;
        bool ok = i < n;
        key[r] = ok ? kin[i] : 0ull;
        val[r] = ok ? vin[i] : 0;
        int dg = ok ? (int)((key[r] >> shift) & 255u) : 256;
        dig[r] = (int16_t)dg;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        int before = __popc(peers & lt);
        int cur = wcnt[wid][dg];
        rank[r] = cur + before;
        __syncwarp();
        if (before == 0) wcnt[wid][dg] = cur + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // exclusive prefix of the per-warp counts for digit threadIdx.x
        int d = threadIdx.x;
        int run = 0;
        for (int w = 0; w < kRadixWarps; ++w) {
            int t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        int dg = dig[r];
        if (dg < 256) {
            int64_t pos = (int64_t)toff[dg] + wcnt[wid][dg] + rank[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

}  // namespace

gp2s_status radix_sort_pairs(gp2s_ctx *c, uint64_t *keys, uint64_t *keys_alt, int32_t *vals,
                             int32_t *vals_alt, int64_t n, int bits)
{
    if (n <= 1 || bits <= 0) return GP2S_OK;
    int passes = (bits + 7) / 8;
    int64_t ntiles = ceil_div(n, kRadixTile);
    int64_t nh = ntiles * 256;
    GP2S_TRY(ensure(c, c->hist, sizeof(int32_t) * (size_t)(2 * nh + 2)));
    int32_t *hist = c->hist.as<int32_t>();
    int32_t *off = hist + nh + 1;
    uint64_t *ka = keys, *kb = keys_alt;
    int32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix_hist<<<(unsigned)ntiles, kRadixThreads, 0, c->stream>>>(ka, n, shift, hist, ntiles);
        GP2S_LAUNCH(c);
        GP2S_TRY((scan_impl<int32_t, int32_t>(c, hist, off, nh, nullptr, 0)));
        k_radix_scatter<<<(unsigned)ntiles, kRadixThreads, 0, c->stream>>>(ka, va, kb, vb, n, shift, off, ntiles);
        GP2S_LAUNCH(c);
        uint64_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        GP2S_CUDA(c, cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
        GP2S_CUDA(c, cudaMemcpyAsync(vals, va, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
    }
    return GP2S_OK;
}

}  // namespace gp2s
