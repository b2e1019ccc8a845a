// gp2s_geometry.cuh -- launchers of the geometry stage (geometry.cu) and the device-side helpers
// the assembly kernels share with it (cell coordinates <-> Morton keys).
#pragma once

#include "gp2s_internal.cuh"

namespace gp2s {

// Bounding box of X (n x d FP64) -> box_host[0..3] = lo, box_host[4..7] = hi, and the int right
// after the 8 doubles is non-zero if X holds a NaN or an infinity.  Synchronises the stream.
gp2s_status geom_bbox(gp2s_ctx *c, const double *X, int64_t n, int d, double *box_host);
// Morton keys of the fine grid + stable radix sort: c->keys (sorted keys), c->idx (sorted ->
// original index).
gp2s_status geom_sort(gp2s_ctx *c, const double *X, int64_t n, const GridParams &g);
// Gather the sorted points: c->Xs64 (double4 per point), c->Xhi / c->Xlo (float4 hi/lo split),
// c->perm (sorted -> original), c->iperm (original -> sorted).
gp2s_status geom_permute(gp2s_ctx *c, const double *X, int64_t n, int d);
// Occupied-cell table (c->cell_start: ncells + 1 starts, then the cell keys) and work items
// (c->items: int4 {cell, row begin, row end, 0}, at most rows_per_item rows each).
gp2s_status geom_cells(gp2s_ctx *c, int64_t n, const GridParams &g, int rows_per_item,
                       int64_t *ncells_out, int64_t *nitems_out);
const uint64_t *cell_keys_ptr(gp2s_ctx *c, int64_t ncells);

// Coarse cell coordinates from a fine Morton key (bits per dimension = g.bits, the low
// g.fine_bits of each coordinate are the sub-cell position).
template <int D>
__device__ __forceinline__ void decode_cell(uint64_t key, const GridParams &g, int64_t *cc)
{
#pragma unroll
    for (int k = 0; k < D; ++k) cc[k] = 0;
    for (int b = 0; b < g.bits; ++b)
#pragma unroll
        for (int k = 0; k < D; ++k) cc[k] |= (int64_t)((key >> (b * D + k)) & 1ull) << b;
#pragma unroll
    for (int k = 0; k < D; ++k) cc[k] >>= g.fine_bits;
}

// Coarse Morton key (the fine key shifted right by D * fine_bits) of integer cell coordinates.
template <int D>
__device__ __forceinline__ uint64_t coarse_key(const int64_t *cc, const GridParams &g)
{
    uint64_t key = 0;
    const int cb = g.bits - g.fine_bits;
    for (int b = 0; b < cb; ++b)
#pragma unroll
        for (int k = 0; k < D; ++k) key |= (((uint64_t)cc[k] >> b) & 1ull) << (b * D + k);
    return key;
}

}  // namespace gp2s
