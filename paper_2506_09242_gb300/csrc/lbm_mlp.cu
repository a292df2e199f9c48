// lbm_mlp.cu -- training-side kernels of the learned closure and their C
// ABI: batch inference (the same tensor-core tile as the collide kernel),
// the loss gradient, Adam, and the training samples built from a fine field.
// No text in the paper; an addition of this library.
#include <math.h>
#include <stdio.h>

#include "lbm_kernels.cuh"

namespace lbm {
void set_last_error_global(const char *msg);  // defined in lbm_api.cu
}

using namespace lbm;

namespace {

lbm_status fail(lbm_status s, const char *msg)
{
    set_last_error_global(msg);
    return s;
}

lbm_status launched(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return LBM_OK;
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return fail(LBM_ERR_CUDA, buf);
}

constexpr int kTrainThreads = 128;        // samples per block
constexpr int kGradSlots = kMlpNParam + 1;  // gradient + squared-error sum
constexpr int kPitch = kMlpH + 1;         // padded row of per-sample activations

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = sigm(z);
    return s * (1.f + z * (1.f - s));
}

// Batch inference with the tcgen05 tile, 128 samples per block.  A tile
// wait that runs out leaves NaN in that block's outputs.
__global__ void __launch_bounds__(kTileM) k_mlp_forward(const float *__restrict__ P, const float *__restrict__ norm,
                                                       const float *__restrict__ X, int n, float *__restrict__ dtau)
{
    __shared__ MlpTcNet W;
    __shared__ MlpTile tile;
    load_mlp_tc(P, norm, W, threadIdx.x, blockDim.x);
    mlp_tile_open(tile, threadIdx.x);  // synchronises the block
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float x[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = s < n ? X[s * kMlpIn + k] : W.mean[k];
    const float d = mlp_block_dtau(W, tile, x, threadIdx.x, nullptr);
    mlp_tile_close(tile, threadIdx.x);
    if (s < n) dtau[s] = d;
}

// Loss gradient, stage 1: every block runs forward and backward for its 128
// samples (one per thread, FP32 with the BF16 roundings of the inference
// path, straight-through gradients), then sums every parameter's gradient
// over its samples in a fixed order and writes one partial row.
__global__ void __launch_bounds__(kTrainThreads)
    k_mlp_grad(const float *__restrict__ P, const float *__restrict__ norm, const float *__restrict__ X,
               const float *__restrict__ target, int n, float *__restrict__ partials)
{
    extern __shared__ float smem[];
    float *W1r = smem;                         // 224
    float *b1 = W1r + kMlpH * kMlpIn;          // 32
    float *W2r = b1 + kMlpH;                   // 1024
    float *b2 = W2r + kMlpH * kMlpH;           // 32
    float *w3 = b2 + kMlpH;                    // 32
    float *misc = w3 + kMlpH;                  // b3, scale, mean[7], inv_std[7]  (16)
    float *xn = misc + 16;                     // [128][8]
    float *z1 = xn + kTrainThreads * 8;        // [128][33], becomes dz1
    float *h1 = z1 + kTrainThreads * kPitch;   // [128][33]
    float *z2 = h1 + kTrainThreads * kPitch;   // [128][33], becomes dz2
    float *h2 = z2 + kTrainThreads * kPitch;   // [128][33]
    float *dy = h2 + kTrainThreads * kPitch;   // [128]
    float *e2 = dy + kTrainThreads;            // [128]
    const int t = threadIdx.x;
    for (int e = t; e < kMlpH * kMlpIn; e += kTrainThreads) W1r[e] = bf16r(P[e]);
    for (int e = t; e < kMlpH * kMlpH; e += kTrainThreads) W2r[e] = bf16r(P[kMlpH * kMlpIn + kMlpH + e]);
    for (int e = t; e < kMlpH; e += kTrainThreads) {
        b1[e] = P[kMlpH * kMlpIn + e];
        b2[e] = P[kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + e];
        w3[e] = P[kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH + e];
    }
    if (t == 0) {
        misc[0] = P[kMlpNParam - 1];
        misc[1] = norm[2 * kMlpIn];
    }
    if (t < kMlpIn) {
        misc[2 + t] = norm[t];
        misc[9 + t] = 1.f / norm[kMlpIn + t];
    }
    __syncthreads();

    const long long s = blockIdx.x * (long long)kTrainThreads + t;
    const bool valid = s < n;
    float *xr = xn + t * 8;
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xr[k] = valid ? bf16r((X[s * kMlpIn + k] - misc[2 + k]) * misc[9 + k]) : 0.f;
    float *z1r = z1 + t * kPitch, *h1r = h1 + t * kPitch, *z2r = z2 + t * kPitch, *h2r = h2 + t * kPitch;
    for (int j = 0; j < kMlpH; ++j) {
        float z = b1[j];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) z = fmaf(W1r[j * kMlpIn + k], xr[k], z);
        z1r[j] = z;
        h1r[j] = bf16r(z * sigm(z));
    }
    float y = misc[0];
    for (int j = 0; j < kMlpH; ++j) {
        float z = b2[j];
        for (int k = 0; k < kMlpH; ++k) z = fmaf(W2r[j * kMlpH + k], h1r[k], z);
        z2r[j] = z;
        h2r[j] = z * sigm(z);
        y = fmaf(w3[j], h2r[j], y);
    }
    const float scale = misc[1];
    const float dt = scale * (y > 20.f ? y : log1pf(__expf(y)));
    const float err = valid ? dt - target[s] : 0.f;
    e2[t] = err * err;
    const float dyv = valid ? (2.f / (float)n) * err * scale * sigm(y) : 0.f;
    dy[t] = dyv;
    for (int j = 0; j < kMlpH; ++j) z2r[j] = dyv * w3[j] * dsilu(z2r[j]);  // dz2
    for (int k = 0; k < kMlpH; ++k) {
        float a = 0.f;
        for (int j = 0; j < kMlpH; ++j) a = fmaf(z2r[j], W2r[j * kMlpH + k], a);
        z1r[k] = a * dsilu(z1r[k]);  // dz1
    }
    __syncthreads();

    // Per-parameter sums over the block's samples, in sample order.
    float *out = partials + (long long)blockIdx.x * kGradSlots;
    for (int q = t; q < kGradSlots; q += kTrainThreads) {
        float acc = 0.f;
        if (q < kMlpH * kMlpIn) {  // dW1[j][k] = sum dz1[s][j] xn[s][k]
            const int j = q / kMlpIn, k = q % kMlpIn;
            for (int i = 0; i < kTrainThreads; ++i) acc = fmaf(z1[i * kPitch + j], xn[i * 8 + k], acc);
        } else if (q < kMlpH * kMlpIn + kMlpH) {  // db1
            const int j = q - kMlpH * kMlpIn;
            for (int i = 0; i < kTrainThreads; ++i) acc += z1[i * kPitch + j];
        } else if (q < kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH) {  // dW2[j][k] = sum dz2[s][j] h1[s][k]
            const int r = q - (kMlpH * kMlpIn + kMlpH), j = r / kMlpH, k = r % kMlpH;
            for (int i = 0; i < kTrainThreads; ++i) acc = fmaf(z2[i * kPitch + j], h1[i * kPitch + k], acc);
        } else if (q < kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH) {  // db2
            const int j = q - (kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH);
            for (int i = 0; i < kTrainThreads; ++i) acc += z2[i * kPitch + j];
        } else if (q < kMlpNParam - 1) {  // dw3[j] = sum dy[s] h2[s][j]
            const int j = q - (kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH);
            for (int i = 0; i < kTrainThreads; ++i) acc = fmaf(dy[i], h2[i * kPitch + j], acc);
        } else if (q == kMlpNParam - 1) {  // db3
            for (int i = 0; i < kTrainThreads; ++i) acc += dy[i];
        } else {  // squared errors
            for (int i = 0; i < kTrainThreads; ++i) acc += e2[i];
        }
        out[q] = acc;
    }
}

constexpr size_t kGradSmemBytes =
    sizeof(float) * (kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + 2 * kMlpH + 16 + kTrainThreads * 8 +
                     4 * kTrainThreads * kPitch + 2 * kTrainThreads);

// Stage 2: partial rows added in block order.
__global__ void k_mlp_grad_final(const float *__restrict__ partials, int nblocks, int n, float *__restrict__ grad,
                                 float *__restrict__ loss)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kGradSlots; q += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < nblocks; ++b) acc += partials[(long long)b * kGradSlots + q];
        if (q < kMlpNParam)
            grad[q] = acc;
        else if (loss)
            *loss = acc / (float)n;
    }
}

__global__ void k_mlp_adam(float *__restrict__ P, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ g, int np, float lr, float b1, float b2, float eps, float c1,
                           float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    P[q] -= lr * (mq * c1) / (sqrtf(vq * c2) + eps);
}

// Training samples from a fine field: one thread per coarse cell.  Box means
// of rho, u and u_a u_b over f^3 fine nodes, the coarse strain from
// second-order central differences of the box-mean velocity (periodic), the
// eddy viscosity nu_t = max(0, -tau_dev : S / (2 S : S)) of the subgrid
// stress tau = mean(uu) - mean(u) mean(u), target 3 nu_t, and features
// Pi = -(2/3) rho tau0 S (Chapman-Enskog) and rho.
__device__ __forceinline__ void box_u(const double *__restrict__ u, long long N, int nx, int ny, int f, int cx,
                                      int cy, int cz, double (&ub)[3])
{
    ub[0] = ub[1] = ub[2] = 0.0;
    for (int dz = 0; dz < f; ++dz)
        for (int dy = 0; dy < f; ++dy)
            for (int dx = 0; dx < f; ++dx) {
                const long long n = (cx * f + dx) + (long long)nx * ((cy * f + dy) + (long long)ny * (cz * f + dz));
                ub[0] += u[n];
                ub[1] += u[N + n];
                ub[2] += u[2 * N + n];
            }
    const double inv = 1.0 / ((double)f * f * f);
    ub[0] *= inv;
    ub[1] *= inv;
    ub[2] *= inv;
}

__global__ void k_coarse_samples(const double *__restrict__ rho, const double *__restrict__ u, int nx, int ny, int nz,
                                 int f, double tau0, float *__restrict__ X, float *__restrict__ target)
{
    const int cnx = nx / f, cny = ny / f, cnz = nz / f;
    const long long Nc = (long long)cnx * cny * cnz, N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < Nc; c += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(c % cnx), cy = (int)((c / cnx) % cny), cz = (int)(c / ((long long)cnx * cny));
        double rb = 0.0, uu[6] = {0, 0, 0, 0, 0, 0}, ub[3] = {0, 0, 0};
        for (int dz = 0; dz < f; ++dz)
            for (int dy = 0; dy < f; ++dy)
                for (int dx = 0; dx < f; ++dx) {
                    const long long n = (cx * f + dx) + (long long)nx * ((cy * f + dy) + (long long)ny * (cz * f + dz));
                    const double a = u[n], b = u[N + n], d = u[2 * N + n];
                    rb += rho[n];
                    ub[0] += a;
                    ub[1] += b;
                    ub[2] += d;
                    uu[0] += a * a;
                    uu[1] += b * b;
                    uu[2] += d * d;
                    uu[3] += a * b;
                    uu[4] += a * d;
                    uu[5] += b * d;
                }
        const double inv = 1.0 / ((double)f * f * f);
        rb *= inv;
        for (int k = 0; k < 3; ++k) ub[k] *= inv;
        for (int k = 0; k < 6; ++k) uu[k] *= inv;
        // g[a][b] = d_a u_b from the neighbouring coarse cells
        double g[3][3];
        const int cxs[2] = {cx == cnx - 1 ? 0 : cx + 1, cx == 0 ? cnx - 1 : cx - 1};
        const int cys[2] = {cy == cny - 1 ? 0 : cy + 1, cy == 0 ? cny - 1 : cy - 1};
        const int czs[2] = {cz == cnz - 1 ? 0 : cz + 1, cz == 0 ? cnz - 1 : cz - 1};
        double up[3], um[3];
        box_u(u, N, nx, ny, f, cxs[0], cy, cz, up);
        box_u(u, N, nx, ny, f, cxs[1], cy, cz, um);
        for (int b = 0; b < 3; ++b) g[0][b] = 0.5 * (up[b] - um[b]);
        box_u(u, N, nx, ny, f, cx, cys[0], cz, up);
        box_u(u, N, nx, ny, f, cx, cys[1], cz, um);
        for (int b = 0; b < 3; ++b) g[1][b] = 0.5 * (up[b] - um[b]);
        box_u(u, N, nx, ny, f, cx, cy, czs[0], up);
        box_u(u, N, nx, ny, f, cx, cy, czs[1], um);
        for (int b = 0; b < 3; ++b) g[2][b] = 0.5 * (up[b] - um[b]);
        const double S[6] = {g[0][0], g[1][1], g[2][2], 0.5 * (g[0][1] + g[1][0]), 0.5 * (g[0][2] + g[2][0]),
                             0.5 * (g[1][2] + g[2][1])};
        const double tau[6] = {uu[0] - ub[0] * ub[0], uu[1] - ub[1] * ub[1], uu[2] - ub[2] * ub[2],
                               uu[3] - ub[0] * ub[1], uu[4] - ub[0] * ub[2], uu[5] - ub[1] * ub[2]};
        const double tr = (tau[0] + tau[1] + tau[2]) / 3.0;
        const double num = -((tau[0] - tr) * S[0] + (tau[1] - tr) * S[1] + (tau[2] - tr) * S[2] +
                             2.0 * (tau[3] * S[3] + tau[4] * S[4] + tau[5] * S[5]));
        const double den = 2.0 * (S[0] * S[0] + S[1] * S[1] + S[2] * S[2] + 2.0 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5]));
        const double nu = den > 0.0 ? fmax(num / den, 0.0) : 0.0;
        target[c] = (float)(3.0 * nu);
        for (int k = 0; k < 6; ++k) X[c * kMlpIn + k] = (float)(-(2.0 / 3.0) * rb * tau0 * S[k]);
        X[c * kMlpIn + 6] = (float)rb;
    }
}

// Box filter: out[c][coarse cell] = mean of in[c] over its f^3 fine nodes.
__global__ void k_box_filter(const double *__restrict__ in, int ncomp, int nx, int ny, int nz, int f,
                             double *__restrict__ out)
{
    const int cnx = nx / f, cny = ny / f, cnz = nz / f;
    const long long Nc = (long long)cnx * cny * cnz, N = (long long)nx * ny * nz;
    const double inv = 1.0 / ((double)f * f * f);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < Nc * ncomp;
         e += (long long)gridDim.x * blockDim.x) {
        const long long comp = e / Nc, c = e % Nc;
        const int cx = (int)(c % cnx), cy = (int)((c / cnx) % cny), cz = (int)(c / ((long long)cnx * cny));
        double acc = 0.0;
        for (int dz = 0; dz < f; ++dz)
            for (int dy = 0; dy < f; ++dy)
                for (int dx = 0; dx < f; ++dx)
                    acc += in[comp * N + (cx * f + dx) + (long long)nx * ((cy * f + dy) + (long long)ny * (cz * f + dz))];
        out[comp * Nc + c] = acc * inv;
    }
}

// Packs FP32 parameters once into the shared-memory image the collide kernel
// copies (one block).
__global__ void k_mlp_pack(const float *__restrict__ P, const float *__restrict__ norm, MlpSmem *__restrict__ img)
{
    load_mlp_smem(P, norm, *img, threadIdx.x, blockDim.x);
}

}  // namespace

namespace lbm {
size_t mlp_image_bytes() { return sizeof(MlpSmem); }
cudaError_t launch_mlp_pack(const float *params, const float *norm, void *image, cudaStream_t s)
{
    k_mlp_pack<<<1, 128, 0, s>>>(params, norm, (MlpSmem *)image);
    return cudaGetLastError();
}
}  // namespace lbm

extern "C" {

lbm_status lbm_box_filter(const double *in, int ncomp, int nx, int ny, int nz, int factor, double *out, void *stream)
{
    if (!in || !out) return fail(LBM_ERR_ARG, "lbm_box_filter: NULL argument");
    if (ncomp < 1 || factor < 1 || nx < factor || ny < factor || nz < factor || nx % factor || ny % factor ||
        nz % factor)
        return fail(LBM_ERR_ARG, "lbm_box_filter: sizes must be positive multiples of factor, ncomp >= 1");
    const long long work = (long long)(nx / factor) * (ny / factor) * (nz / factor) * ncomp;
    long long blocks = (work + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_box_filter<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(in, ncomp, nx, ny, nz, factor, out);
    return launched("lbm_box_filter");
}

lbm_status lbm_mlp_forward(const float *params, const float *norm, const float *x, int n, float *dtau, void *stream)
{
    if (!params || !norm || (n > 0 && (!x || !dtau))) return fail(LBM_ERR_ARG, "lbm_mlp_forward: NULL argument");
    if (n < 0) return fail(LBM_ERR_ARG, "lbm_mlp_forward: n must be >= 0");
    if (n == 0) return LBM_OK;
    const int blocks = (n + 127) / 128;
    k_mlp_forward<<<blocks, kTileM, 0, (cudaStream_t)stream>>>(params, norm, x, n, dtau);
    return launched("lbm_mlp_forward");
}

size_t lbm_mlp_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    return sizeof(float) * (size_t)kGradSlots * (size_t)((n + kTrainThreads - 1) / kTrainThreads);
}

lbm_status lbm_mlp_loss_grad(const float *params, const float *norm, const float *x, const float *target, int n,
                             float *grad, float *loss, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!params || !norm || !x || !target || !grad || !workspace) return fail(LBM_ERR_ARG, "lbm_mlp_loss_grad: NULL argument");
    if (n <= 0) return fail(LBM_ERR_ARG, "lbm_mlp_loss_grad: n must be >= 1");
    if (workspace_bytes < lbm_mlp_workspace_bytes(n))
        return fail(LBM_ERR_ARG, "lbm_mlp_loss_grad: workspace smaller than lbm_mlp_workspace_bytes(n)");
    static_assert(kGradSmemBytes < 200 * 1024, "training tile exceeds shared memory");
    if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmemBytes) != cudaSuccess)
        return launched("lbm_mlp_loss_grad: shared memory attribute");
    const int blocks = (n + kTrainThreads - 1) / kTrainThreads;
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_grad<<<blocks, kTrainThreads, kGradSmemBytes, s>>>(params, norm, x, target, n, (float *)workspace);
    lbm_status st = launched("lbm_mlp_loss_grad");
    if (st != LBM_OK) return st;
    k_mlp_grad_final<<<(kGradSlots + 255) / 256, 256, 0, s>>>((const float *)workspace, blocks, n, grad, loss);
    return launched("lbm_mlp_loss_grad: final");
}

lbm_status lbm_mlp_adam(float *params, float *m, float *v, const float *grad, int n_params, int t, float lr,
                        float beta1, float beta2, float eps, void *stream)
{
    if (!params || !m || !v || !grad) return fail(LBM_ERR_ARG, "lbm_mlp_adam: NULL argument");
    if (n_params <= 0 || t < 1) return fail(LBM_ERR_ARG, "lbm_mlp_adam: n_params >= 1 and t >= 1 required");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f))
        return fail(LBM_ERR_ARG, "lbm_mlp_adam: bad hyper-parameters");
    const double c1 = 1.0 / (1.0 - pow((double)beta1, t)), c2 = 1.0 / (1.0 - pow((double)beta2, t));
    k_mlp_adam<<<(n_params + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, n_params, lr, beta1, beta2,
                                                                         eps, (float)c1, (float)c2);
    return launched("lbm_mlp_adam");
}

lbm_status lbm_coarse_samples(const double *rho, const double *u, int nx, int ny, int nz, int factor, double tau0,
                              float *x, float *target, void *stream)
{
    if (!rho || !u || !x || !target) return fail(LBM_ERR_ARG, "lbm_coarse_samples: NULL argument");
    if (factor < 1 || nx < factor || ny < factor || nz < factor || nx % factor || ny % factor || nz % factor)
        return fail(LBM_ERR_ARG, "lbm_coarse_samples: sizes must be positive multiples of factor");
    if (!(tau0 > 0.5)) return fail(LBM_ERR_ARG, "lbm_coarse_samples: tau0 must be > 1/2");
    const long long Nc = (long long)(nx / factor) * (ny / factor) * (nz / factor);
    long long blocks = (Nc + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_coarse_samples<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(rho, u, nx, ny, nz, factor, tau0, x, target);
    return launched("lbm_coarse_samples");
}

}  // extern "C"
