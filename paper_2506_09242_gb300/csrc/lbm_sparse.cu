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
