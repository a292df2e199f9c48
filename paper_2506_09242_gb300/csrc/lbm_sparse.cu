// lbm_sparse.cu -- the fluid-node list for lattices that are mostly wall
// (porous media): compaction of the fluid nodes in x-fastest order, and the
// per-row fluid bitmask table from which the compact step finds the list
// position of each neighbour (CompactMap, lbm_internal.cuh).
//
// Construction (once per lbm_set_tags): a per-row count of fluid nodes, an
// exclusive prefix sum of the counts (the re-indexing use of scans, Sec. 2.2),
// then a scatter in which each warp ranks its row's fluid nodes with a ballot;
// the ballot of 32 x positions is one word of the bitmask table, and the
// running count before it is the word's list position.
#include "lbm_kernels.cuh"

namespace lbm {

// One warp per row (z * ny + y).
__global__ void k_row_fluid_count(Grid g, const uint8_t *__restrict__ tags, int *__restrict__ count)
{
    const long long rows = (long long)g.nz * g.ny;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    if (warp >= rows) return;
    const uint8_t *row = tags + warp * g.px;
    int c = 0;
    for (int x0 = 0; x0 < g.nx; x0 += 32) {
        const int x = x0 + (int)lane;
        const bool fluid = x < g.nx && !is_wall_tag(row[x] & kTagMask);
        c += __popc(__ballot_sync(0xffffffffu, fluid));
    }
    if (lane == 0) count[warp] = c;
}

// List entries (offset | kListForced) and the bitmask table of one row per
// warp; the table covers the padded row (px = 32 nw), whose padding is never
// fluid.
__global__ void k_row_fluid_scatter(Grid g, const uint8_t *__restrict__ tags, const int *__restrict__ start,
                                    uint32_t *__restrict__ list, uint2 *__restrict__ words)
{
    const long long rows = (long long)g.nz * g.ny;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    if (warp >= rows) return;
    const int nw = g.px / 32;
    int pos = start[warp];
    for (int w = 0; w < nw; ++w) {
        const int x = 32 * w + (int)lane;
        const unsigned t = x < g.nx ? (tags[warp * g.px + x] & kTagMask) : (unsigned)LBM_TAG_SOLID;
        const bool fluid = !is_wall_tag(t);
        const unsigned ball = __ballot_sync(0xffffffffu, fluid);
        if (fluid) {
            const uint32_t off = (uint32_t)(warp * g.px + x);
            list[pos + __popc(ball & ((1u << lane) - 1u))] = off | (t == LBM_TAG_FORCED ? kListForced : 0u);
        }
        if (lane == 0) words[warp * nw + w] = make_uint2(ball, (unsigned)pos);
        pos += __popc(ball);
    }
}

cudaError_t launch_fluid_count(const Grid &g, const uint8_t *tags, int *count, cudaStream_t s)
{
    const long long rows = (long long)g.nz * g.ny;
    const long long blocks = (rows * 32 + 255) / 256;
    k_row_fluid_count<<<(unsigned)blocks, 256, 0, s>>>(g, tags, count);
    return cudaGetLastError();
}

cudaError_t launch_fluid_scatter(const Grid &g, const uint8_t *tags, const int *start, uint32_t *list, uint2 *words,
                                 cudaStream_t s)
{
    const long long rows = (long long)g.nz * g.ny;
    const long long blocks = (rows * 32 + 255) / 256;
    k_row_fluid_scatter<<<(unsigned)blocks, 256, 0, s>>>(g, tags, start, list, words);
    return cudaGetLastError();
}

}  // namespace lbm

namespace lbm {

// Compact fluid-only storage (a copy of the state used while stepping a
// mostly-wall lattice): populations Ac[Q][nfp] in list order.
template <typename S>
__global__ void k_gather_compact(int Q, const S *__restrict__ A, long long sN, const uint32_t *__restrict__ list,
                                 long long n, long long nfp, S *__restrict__ Ac)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const uint32_t off = list[k] & kListOffset;
        for (int i = 0; i < Q; ++i) Ac[(long long)i * nfp + k] = A[(long long)i * sN + off];
    }
}

template <typename S>
__global__ void k_scatter_compact(int Q, const S *__restrict__ Ac, long long nfp, const uint32_t *__restrict__ list,
                                  long long n, long long sN, S *__restrict__ A)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const uint32_t off = list[k] & kListOffset;
        for (int i = 0; i < Q; ++i) A[(long long)i * sN + off] = Ac[(long long)i * nfp + k];
    }
}

static unsigned grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

cudaError_t launch_compact_copy(lbm_dtype dtype, int Q, bool to_compact, const void *src, void *dst, long long sN,
                                const uint32_t *list, long long n, long long nfp, cudaStream_t s)
{
#define LBM_COMPACT_CASE(T)                                                                                     \
    if (to_compact)                                                                                            \
        k_gather_compact<T><<<grid_for(n), 256, 0, s>>>(Q, (const T *)src, sN, list, n, nfp, (T *)dst);        \
    else                                                                                                       \
        k_scatter_compact<T><<<grid_for(n), 256, 0, s>>>(Q, (const T *)src, nfp, list, n, sN, (T *)dst);
    switch (dtype) {
    case LBM_F64: LBM_COMPACT_CASE(double) break;
    case LBM_F32: LBM_COMPACT_CASE(float) break;
    default: LBM_COMPACT_CASE(uint16_t) break;  // both 16-bit types move as raw bits
    }
#undef LBM_COMPACT_CASE
    return cudaGetLastError();
}

}  // namespace lbm
