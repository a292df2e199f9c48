// lbm_mlp.cuh -- the learned relaxation-time closure on the GPU (no text in
// the paper; an addition of this library).
//
// Network: x (7 features: Pi^neq xx, yy, zz, xy, xz, yz, rho) -> normalise
// -> 32 -> SiLU -> 32 -> SiLU -> y -> dtau = out_scale * softplus(y).
// Precision: normalised inputs, first-layer weights and activations and
// second-layer weights in BF16 (round to nearest even), products accumulated
// in FP32 on the tensor cores; biases, the second activations and the last
// layer in FP32.
//
// Parameter layout (LBM_MLP_NPARAM = 1345 floats): W1[32][7], b1[32],
// W2[32][32], b2[32], w3[32], b3.  Normalisation (LBM_MLP_NNORM = 16):
// mean[7], std[7], out_scale, unused.
#pragma once

#include <cstddef>

#include "lbm_internal.cuh"

namespace lbm {

// Shared-memory copy of the network, packed for the mma fragments: BF16
// pairs (k, k+1) of each output row, inputs padded from 7 to 16.  Layers 1
// and 2 hold W/2 and b/2 (exact: a power-of-two scale commutes with BF16 and
// FP32 rounding), so that their accumulators hold z/2 and
// SiLU(z) = (z/2)(1 + tanh(z/2)) costs one tanh and one FMA.
struct __align__(16) MlpSmem {
    uint32_t W1p[kMlpH][8];   // row n: pairs of W1[n][0..15] (cols 7..15 zero)
    uint32_t W2p[kMlpH][16];  // row n: pairs of W2[n][0..31]
    float b1[kMlpH], b2[kMlpH], w3[kMlpH];
    float b3, out_scale;
    float mean[kMlpIn], inv_std[kMlpIn];
};
static_assert(sizeof(MlpSmem) % 16 == 0, "the packed network is copied in 16-byte words");

// Copies a packed network (built once by load_mlp_smem into global memory)
// into shared memory with 16-byte loads.  All threads call it; the caller
// synchronises after.
__device__ __forceinline__ void copy_mlp_image(const MlpSmem *__restrict__ img, MlpSmem &sm, int tid, int nthreads)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(img);
    uint4 *dst = reinterpret_cast<uint4 *>(&sm);
    for (int e = tid; e < (int)(sizeof(MlpSmem) / 16); e += nthreads) dst[e] = __ldg(src + e);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Block-cooperative load of FP32 parameters into the packed shared layout.
// Every thread of the block must call it; the caller synchronises after.
__device__ __forceinline__ void load_mlp_smem(const float *__restrict__ P, const float *__restrict__ norm,
                                              MlpSmem &sm, int tid, int nthreads)
{
    const float *W1 = P;
    const float *b1 = W1 + kMlpH * kMlpIn;
    const float *W2 = b1 + kMlpH;
    const float *b2 = W2 + kMlpH * kMlpH;
    const float *w3 = b2 + kMlpH;
    const float *b3 = w3 + kMlpH;
    for (int e = tid; e < kMlpH * 8; e += nthreads) {
        const int n = e / 8, k = 2 * (e % 8);
        const float lo = k < kMlpIn ? 0.5f * W1[n * kMlpIn + k] : 0.f;
        const float hi = k + 1 < kMlpIn ? 0.5f * W1[n * kMlpIn + k + 1] : 0.f;
        sm.W1p[n][e % 8] = pack_bf16(lo, hi);
    }
    for (int e = tid; e < kMlpH * 16; e += nthreads) {
        const int n = e / 16, k = 2 * (e % 16);
        sm.W2p[n][e % 16] = pack_bf16(0.5f * W2[n * kMlpH + k], 0.5f * W2[n * kMlpH + k + 1]);
    }
    for (int e = tid; e < kMlpH; e += nthreads) {
        sm.b1[e] = 0.5f * b1[e];
        sm.b2[e] = 0.5f * b2[e];
        sm.w3[e] = w3[e];
    }
    if (tid == 0) {
        sm.b3 = b3[0];
        sm.out_scale = norm[2 * kMlpIn];
    }
    for (int e = tid; e < kMlpIn; e += nthreads) {
        sm.mean[e] = norm[e];
        sm.inv_std[e] = 1.f / norm[kMlpIn + e];
    }
}

// D = A (16x16, row) * B (16x8, col) + C on the tensor cores, BF16 inputs,
// FP32 accumulate (PTX mma.sync.m16n8k16).  Fragment layouts, with
// g = lane / 4 and q = lane % 4: a0 = A[g][2q..2q+1], a1 = A[g+8][2q..],
// a2 = A[g][8+2q..], a3 = A[g+8][8+2q..]; b0 = B[2q..2q+1][g],
// b1 = B[8+2q..][g]; c0,c1 = C[g][2q..2q+1], c2,c3 = C[g+8][2q..].
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// SiLU(z) = z sigmoid(z) = (z/2) (1 + tanh(z/2)), with the hardware tanh
// approximation (one MUFU operation; relative error about 2^-11, below the
// BF16 rounding that follows in the first layer).
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu_f(float z)
{
    const float hz = 0.5f * z;
    return fmaf(hz, tanh_approx(hz), hz);
}
// SiLU of two pre-activations given halved (hz = z/2) as hz + hz tanh(hz);
// the two FMAs are one FP32x2 FMA, whose lanes round as fmaf does, so the
// result is bit-identical to silu_f of the full pre-activations.
__device__ __forceinline__ float2 silu2_half(float hz0, float hz1)
{
    const float2 h = make_float2(hz0, hz1);
    return __ffma2_rn(h, make_float2(tanh_approx(hz0), tanh_approx(hz1)), h);
}
__device__ __forceinline__ float softplus_f(float y) { return y > 20.f ? y : log1pf(__expf(y)); }

// The network on 32 nodes at once, one per lane (a warp-collective call:
// all 32 lanes must take part).  stage: 32 x 8 words of per-warp shared
// memory.  Returns this lane's dtau.  The 32 nodes form two 16-row tiles that
// share every weight fragment: layer 1 is 4 mma per tile (N = 32 hidden in 4
// tiles of 8, K = 16 padded inputs), layer 2 is 8 mma per tile (K = 32 in 2
// steps, the layer-1 results re-packed in registers as the A fragments),
// layer 3 a dot product reduced over each lane quad.  Accumulators start at
// the (halved) biases and end at z/2.
__device__ __forceinline__ float mlp_warp_dtau(const MlpSmem &W, uint32_t *stage, const float (&x)[kMlpIn],
                                               unsigned lane)
{
    float xn[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xn[k] = (x[k] - W.mean[k]) * W.inv_std[k];
    uint32_t *row = stage + lane * 8;
    row[0] = pack_bf16(xn[0], xn[1]);
    row[1] = pack_bf16(xn[2], xn[3]);
    row[2] = pack_bf16(xn[4], xn[5]);
    row[3] = pack_bf16(xn[6], 0.f);
    __syncwarp();
    const unsigned g = lane >> 2, q = lane & 3;
    // A fragments of the inputs for both tiles (columns 8..15 are zero).
    uint32_t a0[2], a1[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        a0[t] = stage[(16 * t + g) * 8 + q];
        a1[t] = stage[(16 * t + g + 8) * 8 + q];
    }
    // Layer 1, re-packed as layer-2 A fragments a2[t][k-step][4].
    uint32_t a2[2][2][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t b0 = W.W1p[8 * j + g][q], b1 = W.W1p[8 * j + g][4 + q];
        const int col = 8 * j + 2 * q;
        const float bias0 = W.b1[col], bias1 = W.b1[col + 1];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            float c[4] = {bias0, bias1, bias0, bias1};
            mma_bf16(c, a0[t], a1[t], 0u, 0u, b0, b1);
            const float2 s01 = silu2_half(c[0], c[1]), s23 = silu2_half(c[2], c[3]);
            a2[t][j >> 1][(j & 1) * 2] = pack_bf16(s01.x, s01.y);
            a2[t][j >> 1][(j & 1) * 2 + 1] = pack_bf16(s23.x, s23.y);
        }
    }
    // Layer 2 and the output dot product.
    float pg[2] = {0.f, 0.f}, pg8[2] = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = 8 * j + 2 * q;
        const float bias0 = W.b2[col], bias1 = W.b2[col + 1];
        const float w0 = W.w3[col], w1 = W.w3[col + 1];
        float c[2][4];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            c[t][0] = c[t][2] = bias0;
            c[t][1] = c[t][3] = bias1;
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const uint32_t b0 = W.W2p[8 * j + g][8 * s + q], b1 = W.W2p[8 * j + g][8 * s + 4 + q];
#pragma unroll
            for (int t = 0; t < 2; ++t) mma_bf16(c[t], a2[t][s][0], a2[t][s][1], a2[t][s][2], a2[t][s][3], b0, b1);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const float2 s01 = silu2_half(c[t][0], c[t][1]), s23 = silu2_half(c[t][2], c[t][3]);
            pg[t] = fmaf(s01.x, w0, fmaf(s01.y, w1, pg[t]));
            pg8[t] = fmaf(s23.x, w0, fmaf(s23.y, w1, pg8[t]));
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        pg[t] += __shfl_xor_sync(0xffffffffu, pg[t], 1);
        pg[t] += __shfl_xor_sync(0xffffffffu, pg[t], 2);
        pg8[t] += __shfl_xor_sync(0xffffffffu, pg8[t], 1);
        pg8[t] += __shfl_xor_sync(0xffffffffu, pg8[t], 2);
    }
    // Row r of tile t lives in lane quad (r mod 8); hand it to lane 16 t + r.
    const unsigned r = lane & 15, src = 4 * (r & 7);
    const float v00 = __shfl_sync(0xffffffffu, pg[0], src), v01 = __shfl_sync(0xffffffffu, pg8[0], src);
    const float v10 = __shfl_sync(0xffffffffu, pg[1], src), v11 = __shfl_sync(0xffffffffu, pg8[1], src);
    const float y = (lane < 16 ? (r < 8 ? v00 : v01) : (r < 8 ? v10 : v11)) + W.b3;
    __syncwarp();  // stage may be rewritten by the caller after this
    return W.out_scale * softplus_f(y);
}


// ===========================================================================
// Batch inference on the 5th-generation tensor cores (tcgen05), for
// lbm_mlp_forward: a block's 128 samples are the M = 128 rows of one tile,
// the 32 hidden units its N, the (padded) inputs and first activations its
// K.  One thread issues the MMAs from shared-memory operands, the FP32
// results collect in tensor memory (TMEM), and tcgen05.ld hands every thread
// its own row back (warp w reads TMEM lanes 32w .. 32w+31).  Same roundings
// as the warp tile above; only the FP32 accumulation order differs.
//
// The collide kernel keeps the warp tile: inside a memory-streaming stencil
// the network's 1,280 MACs per node keep the tensor pipe a few percent busy
// either way, and the CTA-level tile's block barriers, MMA round trips and
// TMEM set-up per 128 nodes cost more than the warp tile's fragment traffic
// (measured at 512^3: 19.5 against 25.3 GLUPS; persistent blocks 7.6).
// ===========================================================================
constexpr int kTileM = 128;  // nodes per tile = threads per block of the step kernels

// Byte offset of element (r, k) of a K-major BF16 operand in the tensor
// cores' no-swizzle layout: core matrices of 8 rows x 16 bytes (8 values)
// stored as 128 contiguous bytes, K-adjacent core matrices 128 bytes apart,
// each group of 8 rows kcores x 128 bytes after the previous one.
__host__ __device__ constexpr uint32_t tc_kmajor_off(int r, int k, int kcores)
{
    return (uint32_t)(r / 8) * (128u * (uint32_t)kcores) + (uint32_t)(k / 8) * 128u + (uint32_t)(r % 8) * 16u +
           (uint32_t)(k % 8) * 2u;
}

// The network for the tensor-core tile.  W1 (N = 32, K = 16: the 7 inputs
// and 9 zero columns) and W2 (N = 32, K = 32) are the B operands of the two
// layers, BF16 bits in the layout above.
struct __align__(128) MlpTcNet {
    uint16_t W1u[kMlpH * 16];
    uint16_t W2u[kMlpH * kMlpH];
    float b1[kMlpH], b2[kMlpH], w3[kMlpH];
    float b3, out_scale;
    float mean[kMlpIn], inv_std[kMlpIn];
};
static_assert(offsetof(MlpTcNet, W2u) % 128 == 0, "tensor-core operands start on 128-byte boundaries");

// Per-block operands and bookkeeping of the tile.
struct __align__(128) MlpTile {
    uint16_t a1[kTileM * 16];     // normalised inputs, K = 16 (2 core matrices per 8 rows)
    uint16_t a2[kTileM * kMlpH];  // first activations, K = 32 (4 per 8 rows)
    uint64_t mbar;                // completion of the MMAs (phase 0: layer 1, 1: layer 2)
    uint32_t tmem;                // TMEM base: 32 columns, layer 1 then layer 2
};
// Layer 2 reuses layer 1's columns: every thread has read its layer-1 row
// (tcgen05.wait::ld) before the barrier that precedes the layer-2 MMAs.
// 32 columns a block lets 16 blocks share an SM's 512.
constexpr int kTmemCols = 32;

__device__ __forceinline__ uint16_t bf16_bits(float v)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t *>(&b);
}

// Block-cooperative load of FP32 parameters into the tensor-core layout.
// Every thread of the block must call it; the caller synchronises after.
__device__ __forceinline__ void load_mlp_tc(const float *__restrict__ P, const float *__restrict__ norm,
                                            MlpTcNet &sm, int tid, int nthreads)
{
    const float *W1 = P;
    const float *b1 = W1 + kMlpH * kMlpIn;
    const float *W2 = b1 + kMlpH;
    const float *b2 = W2 + kMlpH * kMlpH;
    const float *w3 = b2 + kMlpH;
    const float *b3 = w3 + kMlpH;
    for (int e = tid; e < kMlpH * 16; e += nthreads) {
        const int n = e / 16, k = e % 16;
        sm.W1u[tc_kmajor_off(n, k, 2) / 2] = bf16_bits(k < kMlpIn ? W1[n * kMlpIn + k] : 0.f);
    }
    for (int e = tid; e < kMlpH * kMlpH; e += nthreads) {
        const int n = e / kMlpH, k = e % kMlpH;
        sm.W2u[tc_kmajor_off(n, k, 4) / 2] = bf16_bits(W2[n * kMlpH + k]);
    }
    for (int e = tid; e < kMlpH; e += nthreads) {
        sm.b1[e] = b1[e];
        sm.b2[e] = b2[e];
        sm.w3[e] = w3[e];
    }
    if (tid == 0) {
        sm.b3 = b3[0];
        sm.out_scale = norm[2 * kMlpIn];
    }
    for (int e = tid; e < kMlpIn; e += nthreads) {
        sm.mean[e] = norm[e];
        sm.inv_std[e] = 1.f / norm[kMlpIn + e];
    }
}

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier primitives (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, byte distance of
// K-adjacent core matrices (lbo) and of 8-row groups (sbo), no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// BF16 A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kMlpH >> 3) << 17) |
                              ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Makes this thread's shared-memory writes visible to the tensor cores.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Whole-warp calls.
__device__ __forceinline__ void tc_alloc(uint32_t *dst, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// D (TMEM) = A * B^T (+ D when accumulate), issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, bool accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"((uint32_t)accumulate)
        : "memory");
}
// The mbarrier completes a phase once the MMAs issued so far are done.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// Waits for phase `parity` of the mbarrier, giving up after a bounded number
// of polls (each poll may itself suspend the thread for a short while).
// Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane (whole-warp call:
// warp w reads lanes 32w + lane).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}


// Sets up the tile: TMEM columns (warp 0) and the mbarrier.  Every thread of
// the block calls it, before any other use of T.
__device__ __forceinline__ void mlp_tile_open(MlpTile &T, int tid)
{
    if (tid < 32) tc_alloc(&T.tmem, kTmemCols);
    if (tid == 0) mbar_init(&T.mbar, 1);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Releases the TMEM columns.  Every thread calls it, after its last use of
// the tile.
__device__ __forceinline__ void mlp_tile_close(MlpTile &T, int tid)
{
    tc_fence_before();
    __syncthreads();
    if (tid < 32) tc_dealloc(T.tmem, kTmemCols);
}

// The network on the block's 128 nodes, one per thread (row tid of the tile;
// rows of inactive threads carry any finite features).  A block-collective
// call: every thread of the block takes part in every step.  A completion
// wait that runs out sets *err (when given) and makes the result NaN, so the
// node turns non-finite and the reductions report it.
__device__ __forceinline__ float mlp_block_dtau(const MlpTcNet &W, MlpTile &T, const float (&x)[kMlpIn], int tid,
                                                int *err)
{
    // Layer-1 operand: this node's normalised inputs, 7 values and 9 zeros.
    float xn[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xn[k] = (x[k] - W.mean[k]) * W.inv_std[k];
    uint8_t *a1 = reinterpret_cast<uint8_t *>(T.a1);
    *reinterpret_cast<uint4 *>(a1 + tc_kmajor_off(tid, 0, 2)) =
        make_uint4(pack_bf16(xn[0], xn[1]), pack_bf16(xn[2], xn[3]), pack_bf16(xn[4], xn[5]), pack_bf16(xn[6], 0.f));
    *reinterpret_cast<uint4 *>(a1 + tc_kmajor_off(tid, 8, 2)) = make_uint4(0u, 0u, 0u, 0u);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        tc_mma(T.tmem, tc_smem_desc(smem_addr(T.a1), 128, 256), tc_smem_desc(smem_addr(W.W1u), 128, 256), false);
        tc_commit(&T.mbar);
    }
    bool ok = mbar_wait(&T.mbar, 0);
    tc_fence_after();

    // Layer 1 back from TMEM: bias, SiLU, BF16 into the layer-2 operand.
    const uint32_t lanes = (uint32_t)(tid & ~31) << 16;
    uint8_t *a2 = reinterpret_cast<uint8_t *>(T.a2);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float v[16];
        tc_ld16(T.tmem + lanes + 16 * half, v);
        uint32_t p[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            p[c] = pack_bf16(silu_f(v[2 * c] + W.b1[16 * half + 2 * c]),
                             silu_f(v[2 * c + 1] + W.b1[16 * half + 2 * c + 1]));
        *reinterpret_cast<uint4 *>(a2 + tc_kmajor_off(tid, 16 * half, 4)) = make_uint4(p[0], p[1], p[2], p[3]);
        *reinterpret_cast<uint4 *>(a2 + tc_kmajor_off(tid, 16 * half + 8, 4)) = make_uint4(p[4], p[5], p[6], p[7]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        const uint32_t a = smem_addr(T.a2), b = smem_addr(W.W2u);
        tc_mma(T.tmem, tc_smem_desc(a, 128, 512), tc_smem_desc(b, 128, 512), false);
        tc_mma(T.tmem, tc_smem_desc(a + 256, 128, 512), tc_smem_desc(b + 256, 128, 512), true);
        tc_commit(&T.mbar);
    }
    ok = mbar_wait(&T.mbar, 1) && ok;
    tc_fence_after();

    // Layer 2 back from TMEM: bias, SiLU and the output layer in FP32.
    float y = W.b3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float v[16];
        tc_ld16(T.tmem + lanes + 16 * half, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) y = fmaf(W.w3[16 * half + c], silu_f(v[c] + W.b2[16 * half + c]), y);
    }
    if (!ok) {
        if (err) atomicExch(err, 1);
        return __int_as_float(0x7fc00000);
    }
    return W.out_scale * softplus_f(y);
}

}  // namespace lbm
