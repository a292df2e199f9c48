// lbm_mlp_tma.cuh -- the collide-and-stream step with the learned closure,
// fed by the Tensor Memory Accelerator (TMA).
//
// The learned closure adds about 530 instructions per node to the BGK step
// (the network on the warp-level tensor-core tile, its activations and the
// relaxation with the corrected time), so a warp spends most of its time
// computing, and in a one-node-per-thread kernel its population loads are
// not in flight while it does.  Here the loads run ahead on their own:
//
//  - persistent blocks of 128 threads walk tiles of 128 x-consecutive nodes
//    of one row; the block holds the packed network for its whole life;
//  - for every tile, one thread issues Q TMA copies, one per population: the
//    row of the tile's pull sources of direction i, i.e. the 128 nodes
//    shifted by -c_i in y and z (wrapped on the host side of the copy) and
//    widened by kTmaHalo elements on each side in x, so that the +-1 x shift
//    of the pull is an offset into shared memory;
//  - the copies of the next tiles are in flight while the current tile is
//    computed (kStages buffers, an mbarrier each, completed by the copies'
//    transaction bytes);
//  - only the periodic x seam (x = 0 and x = nx - 1) and bounced links of
//    nodes next to a wall read global memory directly.
//
// Roles are split by warp: one lane of a fifth warp issues the copies, the
// four computing warps wait only for their data (a "full" mbarrier per
// buffer, completed by the copies' bytes) and release a buffer as soon as
// they have read it (an "empty" mbarrier per buffer with one arrival per
// warp), so no warp waits for another at the end of a tile.
//
// Same arithmetic, node for node, as k_collide_stream_mlp, so the two
// kernels give the same bits.  A/B pattern only (the AA steps keep the
// one-node-per-thread kernel).  Every wait is bounded: one that runs out (it
// never should) turns the block's remaining nodes to NaN, which the
// reductions report, and the copy warp waits (bounded) for its copies in
// flight before the block exits.
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; the map is encoded on the host)

#include "lbm_mlp.cuh"

namespace lbm {

constexpr int kTmaHalo = 8;                     // x elements on each side: 16 bytes at 16-bit storage
constexpr int kTmaRow = kTileM + 2 * kTmaHalo;  // elements per population row of a tile

// Elements between consecutive population rows in shared memory: every copy
// starts on a 128-byte boundary.
template <typename S> constexpr int tma_pitch() { return (int)(((kTmaRow * sizeof(S) + 127) / 128) * 128 / sizeof(S)); }
// Bytes one tile's Q copies deliver (the mbarrier's transaction count).
template <int Q, typename S> constexpr uint32_t tma_tile_bytes() { return (uint32_t)(Q * kTmaRow * sizeof(S)); }
template <int Q, typename S> constexpr size_t tma_stage_bytes() { return (size_t)Q * tma_pitch<S>() * sizeof(S); }
// Three buffers while a tile's rows fit in 16 KB, else two.
template <int Q, typename S> constexpr int tma_stages() { return tma_stage_bytes<Q, S>() > 16384u ? 2 : 3; }
// Dynamic shared memory of the kernel: the buffers and 128 bytes of room to
// align their start.
template <int Q, typename S> constexpr size_t tma_smem_bytes()
{
    return (size_t)tma_stages<Q, S>() * tma_stage_bytes<Q, S>() + 128;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Makes mbarrier initialisation visible to the copy engine.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Tiled copy of one box of a 4D tensor (x, y, z, population) into shared
// memory, completing on bar with its byte count.  c0 * element size must be
// a multiple of 16 bytes (x starts on 16-byte boundaries); c0 may be
// negative or run past the end (those elements read as zero).
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// Tile index -> (x0, y, z).
struct TileCoord {
    int x0, y, z;
};
__device__ __forceinline__ TileCoord tile_coord(long long tile, int ntx, int ny)
{
    const long long row = tile / ntx;
    return TileCoord{(int)(tile - row * ntx) * kTileM, (int)(row % ny), (int)(row / ny)};
}

// Thread 0: the Q copies of one tile into stage buffer buf.
template <int Q, typename S>
__device__ __forceinline__ void tma_issue_tile(const CUtensorMap *map, S *buf, uint64_t *bar, const Grid &g,
                                               const TileCoord &c)
{
    mbar_expect_tx(bar, tma_tile_bytes<Q, S>());
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cy = cvel(i, 1), cz = cvel(i, 2);
        int ys = c.y - cy, zs = c.z - cz;
        ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
        zs = zs < 0 ? zs + g.nz : (zs >= g.nz ? zs - g.nz : zs);
        tma_load_4d(buf + i * tma_pitch<S>(), map, c.x0 - kTmaHalo, ys, zs, i, bar);
    }
}

// Arrival of one thread on an mbarrier (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Threads of a block: kTileM computing threads (four warps, one node each)
// and one copy warp, of which one lane issues the copies.
constexpr int kTmaThreads = kTileM + 32;

template <int Q, typename S, bool GENERAL>
__global__ void __launch_bounds__(kTmaThreads, 4)
    k_collide_stream_mlp_tma(const __grid_constant__ CUtensorMap tmap, const S *__restrict__ A, S *__restrict__ B,
                             const uint8_t *__restrict__ tags, Grid g, KParams<typename Store<S>::T> p,
                             const MlpSmem *__restrict__ mlp_image, int ntx, long long ntiles)
{
    using T = typename Store<S>::T;
    using St = Store<S>;
    constexpr int NS = tma_stages<Q, S>();
    constexpr int kWarps = kTileM / 32;
    extern __shared__ __align__(128) uint8_t tma_dyn[];
    const uint32_t pad = (128u - (smem_addr(tma_dyn) & 127u)) & 127u;
    S *stage = reinterpret_cast<S *>(tma_dyn + pad);  // [NS][Q][tma_pitch], 128-byte aligned
    constexpr int kStageElems = Q * tma_pitch<S>();
    __shared__ MlpSmem W;
    __shared__ uint32_t frag[kWarps][32 * 8];
    __shared__ __align__(8) uint64_t full[NS];   // copies of a tile landed (one arrival + bytes)
    __shared__ __align__(8) uint64_t empty[NS];  // every computing warp is done with the buffer
    __shared__ volatile int failed;              // a bounded wait ran out somewhere in the block
    const int tid = threadIdx.x;
    copy_mlp_image(mlp_image, W, tid, kTmaThreads);
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kWarps);
        }
        failed = 0;
        fence_mbar_init();
    }
    __syncthreads();  // the last block-wide barrier: from here the warps run on their own
    const long long first = blockIdx.x, step = gridDim.x;

    if (tid >= kTileM) {
        // Copy warp.  Tile k goes to buffer k % NS once the computing warps
        // have released the buffer's previous tile.
        if (tid != kTileM) return;
        int k = 0;  // tiles issued
        for (long long tile = first; tile < ntiles; tile += step, ++k) {
            const int s = k % NS;
            if (k >= NS && !mbar_wait(&empty[s], (uint32_t)(k / NS - 1) & 1u)) failed = 1;
            if (failed) break;
            tma_issue_tile<Q, S>(&tmap, stage + s * kStageElems, &full[s], g, tile_coord(tile, ntx, g.ny));
        }
        // The shared memory is released when the last thread exits: let every
        // copy land first (immediate when its tile was consumed).  The last
        // copies issued are those of tiles k - NS .. k - 1.
        for (int j = k - NS < 0 ? 0 : k - NS; j < k; ++j) mbar_wait(&full[j % NS], (uint32_t)(j / NS) & 1u);
        return;
    }

    const unsigned lane = (unsigned)tid & 31u;
    int k = 0;
    for (long long tile = first; tile < ntiles; tile += step, ++k) {
        const int s = k % NS;
        bool ok = !failed;
        if (ok) {
            ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)(k / NS) & 1u));  // warp-uniform
            if (!ok) failed = 1;
        }
        const TileCoord c = tile_coord(tile, ntx, g.ny);
        const int x = c.x0 + tid;
        const bool inx = x < g.nx;
        const int self = (c.z * g.ny + c.y) * g.px + x;
        unsigned t = 0;
        bool active = inx;
        if (GENERAL && inx) {
            t = tags[self];
            active = !is_wall_tag(t & kTagMask);
        }
        if (!ok) {  // the copy never completed: mark the tile's nodes for the reductions
            if (active)
#pragma unroll
                for (int i = 0; i < Q; ++i) St::st(B + (long long)i * g.sN + self, T(__int_as_float(0x7fc00000)));
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            continue;
        }
        const S *buf = stage + s * kStageElems;
        T h[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            h[i] = active ? St::ldc(buf + i * tma_pitch<S>() + kTmaHalo + tid - cvel(i, 0)) : T(0);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp's reads of the buffer are done
        const bool seam = inx && (x == 0 || x == g.nx - 1);
        if (seam || (GENERAL && active && (t & kNearWall))) {
            Nbr nb;
            nb.init(g, x, c.y, c.z);
            if (seam)  // periodic in x: the wrapped source is not in the copied row
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (cvel(i, 0) != 0) h[i] = St::ld(A + step_load_off<kPatAB>(i, g, nb));
            if (GENERAL && active && (t & kNearWall)) apply_walls<Q, S, kPatAB>(h, A, tags, g, nb, p);
        }
        const bool forced = GENERAL && (t & kTagMask) == LBM_TAG_FORCED;
        const Macro<T> m = node_macros<Q, T>(h, forced, p);
        T pi[6];
        pi_neq<Q, T>(h, m, pi);
        const float xf[kMlpIn] = {(float)pi[0], (float)pi[1], (float)pi[2], (float)pi[3],
                                  (float)pi[4], (float)pi[5], (float)m.rho};
        const float dtau = mlp_warp_dtau(W, frag[tid >> 5], xf, lane);
        relax<Q, T>(h, m, T(1) / (p.tau + T(dtau)), forced);
        if (active)
#pragma unroll
            for (int i = 0; i < Q; ++i) St::st(B + (long long)i * g.sN + self, h[i]);
    }
}

}  // namespace lbm
