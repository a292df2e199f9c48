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

#include "lbm_internal.cuh"

namespace lbm {

// Shared-memory copy of the network, packed for the mma fragments: BF16
// pairs (k, k+1) of each output row, inputs padded from 7 to 16.
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
        const float lo = k < kMlpIn ? W1[n * kMlpIn + k] : 0.f;
        const float hi = k + 1 < kMlpIn ? W1[n * kMlpIn + k + 1] : 0.f;
        sm.W1p[n][e % 8] = pack_bf16(lo, hi);
    }
    for (int e = tid; e < kMlpH * 16; e += nthreads) {
        const int n = e / 16, k = 2 * (e % 16);
        sm.W2p[n][e % 16] = pack_bf16(W2[n * kMlpH + k], W2[n * kMlpH + k + 1]);
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
__device__ __forceinline__ float softplus_f(float y) { return y > 20.f ? y : log1pf(__expf(y)); }

// The network on 32 nodes at once, one per lane (a warp-collective call:
// all 32 lanes must take part).  stage: 32 x 8 words of per-warp shared
// memory.  Returns this lane's dtau.  The 32 nodes form two 16-row tiles that
// share every weight fragment: layer 1 is 4 mma per tile (N = 32 hidden in 4
// tiles of 8, K = 16 padded inputs), layer 2 is 8 mma per tile (K = 32 in 2
// steps, the layer-1 results re-packed in registers as the A fragments),
// layer 3 a dot product reduced over each lane quad.  Accumulators start at
// the biases.
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
            a2[t][j >> 1][(j & 1) * 2] = pack_bf16(silu_f(c[0]), silu_f(c[1]));
            a2[t][j >> 1][(j & 1) * 2 + 1] = pack_bf16(silu_f(c[2]), silu_f(c[3]));
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
            pg[t] = fmaf(silu_f(c[t][0]), w0, fmaf(silu_f(c[t][1]), w1, pg[t]));
            pg8[t] = fmaf(silu_f(c[t][2]), w0, fmaf(silu_f(c[t][3]), w1, pg8[t]));
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

}  // namespace lbm
