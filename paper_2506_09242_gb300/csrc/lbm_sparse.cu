// lbm_sparse.cu -- the fluid-node list for lattices that are mostly wall
// (porous media): compaction of the fluid nodes in x-fastest order and one
// bounce-back link mask per fluid node.  The collide kernel that walks the
// list is k_collide_stream_list (lbm_kernels.cuh).
//
// Construction (once per lbm_set_tags): a per-row count of fluid nodes, an
// exclusive prefix sum of the counts (the re-indexing use of scans, Sec. 2.2),
// then a scatter in which each warp ranks its row's fluid nodes with a ballot.
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

template <int Q>
__global__ void k_row_fluid_scatter(Grid g, const uint8_t *__restrict__ tags, const int *__restrict__ start,
                                    int *__restrict__ list, uint32_t *__restrict__ mask)
{
    const long long rows = (long long)g.nz * g.ny;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = threadIdx.x & 31u;
    if (warp >= rows) return;
    const int y = (int)(warp % g.ny), z = (int)(warp / g.ny);
    int pos = start[warp];
    for (int x0 = 0; x0 < g.nx; x0 += 32) {
        const int x = x0 + (int)lane;
        const unsigned t = x < g.nx ? (tags[warp * g.px + x] & kTagMask) : (unsigned)LBM_TAG_SOLID;
        const bool fluid = !is_wall_tag(t);
        const unsigned ball = __ballot_sync(0xffffffffu, fluid);
        if (fluid) {
            Nbr nb;
            nb.init(g, x, y, z);
            uint32_t m = 0;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const unsigned ts = tags[nb.src(i)] & kTagMask;
                if (is_wall_tag(ts)) m |= 1u << i;
                if (ts >= LBM_TAG_WALL0 && ts < LBM_NTAGS) m |= kListAnyWall;
            }
            if (t == LBM_TAG_FORCED) m |= kListForced;
            const int k = pos + __popc(ball & ((1u << lane) - 1u));
            list[k] = nb.self;
            mask[k] = m;
        }
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

cudaError_t launch_fluid_scatter(int Q, const Grid &g, const uint8_t *tags, const int *start, int *list,
                                 uint32_t *mask, cudaStream_t s)
{
    const long long rows = (long long)g.nz * g.ny;
    const long long blocks = (rows * 32 + 255) / 256;
    if (Q == 19)
        k_row_fluid_scatter<19><<<(unsigned)blocks, 256, 0, s>>>(g, tags, start, list, mask);
    else
        k_row_fluid_scatter<27><<<(unsigned)blocks, 256, 0, s>>>(g, tags, start, list, mask);
    return cudaGetLastError();
}

}  // namespace lbm

namespace lbm {

// Compact fluid-only storage (a copy of the state used while stepping a
// mostly-wall lattice): populations Ac[Q][nfp] in list order, and the
// neighbour index nbr[i-1][k] of the pull source of direction i of listed node
// k: its list position if it is fluid, -1 for a SOLID source (bounce-back),
// -2 - w for a source on moving wall w (Ladd).
__global__ void k_fill_index(const int *__restrict__ list, long long n, int *__restrict__ index)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        index[list[k]] = (int)k;
}

template <int Q>
__global__ void k_build_neighbours(Grid g, const uint8_t *__restrict__ tags, const int *__restrict__ list,
                                   const int *__restrict__ index, long long n, long long nfp, int *__restrict__ nbr)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int off = list[k];
        const int r = off / g.px;
        Nbr nb;
        nb.init(g, off - r * g.px, r % g.ny, r / g.ny);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int s = nb.src(i);
            const unsigned ts = tags[s] & kTagMask;
            int v;
            if (ts == LBM_TAG_SOLID)
                v = -1;
            else if (is_wall_tag(ts))
                v = -2 - (int)(ts - LBM_TAG_WALL0);
            else
                v = index[s];
            nbr[(long long)(i - 1) * nfp + k] = v;
        }
    }
}

template <typename S>
__global__ void k_gather_compact(int Q, const S *__restrict__ A, long long sN, const int *__restrict__ list, long long n,
                                 long long nfp, S *__restrict__ Ac)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int off = list[k];
        for (int i = 0; i < Q; ++i) Ac[(long long)i * nfp + k] = A[(long long)i * sN + off];
    }
}

template <typename S>
__global__ void k_scatter_compact(int Q, const S *__restrict__ Ac, long long nfp, const int *__restrict__ list,
                                  long long n, long long sN, S *__restrict__ A)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int off = list[k];
        for (int i = 0; i < Q; ++i) A[(long long)i * sN + off] = Ac[(long long)i * nfp + k];
    }
}

static unsigned grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

cudaError_t launch_build_neighbours(int Q, const Grid &g, const uint8_t *tags, const int *list, long long n,
                                    long long nfp, int *index, int *nbr, cudaStream_t s)
{
    k_fill_index<<<grid_for(n), 256, 0, s>>>(list, n, index);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (Q == 19)
        k_build_neighbours<19><<<grid_for(n), 256, 0, s>>>(g, tags, list, index, n, nfp, nbr);
    else
        k_build_neighbours<27><<<grid_for(n), 256, 0, s>>>(g, tags, list, index, n, nfp, nbr);
    return cudaGetLastError();
}

cudaError_t launch_compact_copy(lbm_dtype dtype, int Q, bool to_compact, const void *src, void *dst, long long sN,
                                const int *list, long long n, long long nfp, cudaStream_t s)
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
