// lbm_diag.cu -- kernels of the porous-medium generator and of the enstrophy
// diagnostic (storage-type independent; the host side is in lbm_api.cu).
#include <stdio.h>

#include "lbm_kernels.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Random overlapping spheres (stand-in for the Berea CT volume, Sec. 3.3).
//
// The medium is defined sequentially: spheres are added in list order until
// the pore fraction drops to the target.  In parallel: every voxel records the
// index of the first sphere that covers it (atomicMin over spheres), a
// histogram of those indices gives the pore fraction after any number of
// spheres, and the host scans it for the stopping count.  The result is the
// sequential one exactly.
// ---------------------------------------------------------------------------
constexpr uint32_t kNoSphere = 0xffffffffu;

__device__ __forceinline__ long long wrapll(long long a, long long n) { return ((a % n) + n) % n; }

__device__ __forceinline__ long long min_image(long long d, long long n)
{
    d = wrapll(d, n);
    return 2 * d > n ? d - n : d;
}

// One block per sphere (grid-stride over spheres); threads walk the bounding
// cube [-R, R]^3, R = ceil(r).  An offset counts only if it is the voxel's
// minimum-image offset, so each voxel is tested once per sphere even when the
// cube wraps around a small lattice.
__global__ void __launch_bounds__(256)
    k_sphere_cover(int nx, int ny, int nz, const int *__restrict__ centres, const double *__restrict__ radii, int n,
                   uint32_t *__restrict__ cover)
{
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        const long long cx = centres[3 * s], cy = centres[3 * s + 1], cz = centres[3 * s + 2];
        const double r = radii[s];
        const double r2 = r * r;
        const long long R = (long long)ceil(r);
        const long long side = 2 * R + 1;
        const long long count = side * side * side;
        for (long long k = threadIdx.x; k < count; k += blockDim.x) {
            const long long dx = k % side - R, dy = (k / side) % side - R, dz = k / (side * side) - R;
            const long long x = wrapll(cx + dx, nx), y = wrapll(cy + dy, ny), z = wrapll(cz + dz, nz);
            if (min_image(x - cx, nx) != dx || min_image(y - cy, ny) != dy || min_image(z - cz, nz) != dz) continue;
            const double d2 = (double)(dx * dx + dy * dy + dz * dz);
            if (d2 <= r2) atomicMin(&cover[x + (long long)nx * (y + (long long)ny * z)], (uint32_t)s);
        }
    }
}

__global__ void k_sphere_histogram(long long N, const uint32_t *__restrict__ cover, uint32_t *__restrict__ count)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
        const uint32_t s = cover[v];
        if (s != kNoSphere) atomicAdd(&count[s], 1u);
    }
}

__global__ void k_sphere_tags(long long N, const uint32_t *__restrict__ cover, uint32_t used, uint8_t pore_tag,
                              uint8_t *__restrict__ tags)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
        tags[v] = cover[v] < used ? (uint8_t)LBM_TAG_SOLID : pore_tag;
}

cudaError_t launch_sphere_cover(int nx, int ny, int nz, const int *centres, const double *radii, int n,
                                uint32_t *cover, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int blocks = n < 152 * 16 ? n : 152 * 16;
    k_sphere_cover<<<blocks, 256, 0, s>>>(nx, ny, nz, centres, radii, n, cover);
    return cudaGetLastError();
}

cudaError_t launch_sphere_histogram(long long N, const uint32_t *cover, uint32_t *count, cudaStream_t s)
{
    k_sphere_histogram<<<152 * 8, 256, 0, s>>>(N, cover, count);
    return cudaGetLastError();
}

cudaError_t launch_sphere_tags(long long N, const uint32_t *cover, uint32_t used, uint8_t pore_tag, uint8_t *tags,
                               cudaStream_t s)
{
    k_sphere_tags<<<152 * 8, 256, 0, s>>>(N, cover, used, pore_tag, tags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Enstrophy: eps = (1/N) sum |curl u|^2 / 2 over all nodes, with the
// eighth-order centred first derivative (Sec. 3.1), periodic in every
// direction.  u is the unpadded [3][N] FP64 field of lbm_moments (zero on
// solid and wall nodes).  Arithmetic in T; per-block partial in slot 0 of
// the reduction layout.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T d8(const double *__restrict__ q, long long base, long long stride, int pos, int n)
{
    // a_m (q[pos+m] - q[pos-m]), m = 1..4, with a = 4/5, -1/5, 4/105, -1/280
    const T a[4] = {T(4) / T(5), T(-1) / T(5), T(4) / T(105), T(-1) / T(280)};
    T s = T(0);
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
        int p = pos + m, q_ = pos - m;
        p = p >= n ? p - n : p;
        q_ = q_ < 0 ? q_ + n : q_;
        p = p >= n ? p % n : p;  // lattices shorter than 5 nodes
        q_ = q_ < 0 ? ((q_ % n) + n) % n : q_;
        s += a[m - 1] * (T)(q[base + stride * p] - q[base + stride * q_]);
    }
    return s;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_enstrophy(int nx, int ny, int nz, const double *__restrict__ u, double *__restrict__ partials)
{
    Acc<T> acc;
    const long long N = (long long)nx * ny * nz;
    const double *ux = u, *uy = u + N, *uz = u + 2 * N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx);
        const int y = (int)((n / nx) % ny);
        const int z = (int)(n / ((long long)nx * ny));
        const long long bx = n - x, by = n - (long long)y * nx, bz = n - (long long)z * nx * ny;
        const long long sy = nx, sz = (long long)nx * ny;
        const T wx = d8<T>(uz, by, sy, y, ny) - d8<T>(uy, bz, sz, z, nz);
        const T wy = d8<T>(ux, bz, sz, z, nz) - d8<T>(uz, bx, 1, x, nx);
        const T wz = d8<T>(uy, bx, 1, x, nx) - d8<T>(ux, by, sy, y, ny);
        acc.add(T(0.5) * (wx * wx + wy * wy + wz * wz));
    }
    double slots[kRedSlots] = {acc.get(), 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    block_reduce_slots(slots);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) partials[(long long)blockIdx.x * kRedSlots + k] = slots[k];
}

cudaError_t launch_enstrophy(bool fp64, int nx, int ny, int nz, const double *u, double *partials, int nblocks,
                             double *out, cudaStream_t s)
{
    if (fp64)
        k_enstrophy<double><<<nblocks, kRedThreads, 0, s>>>(nx, ny, nz, u, partials);
    else
        k_enstrophy<float><<<nblocks, kRedThreads, 0, s>>>(nx, ny, nz, u, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, kRedThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 arithmetic roof: the rate of independent FP64 fused multiply-adds on
// every SM (the step on FP64 storage runs all of its arithmetic in FP64).
// Each thread advances kFmaChains independent recurrences a <- a * b + c,
// so the FMA pipe, not latency, sets the time.
// ---------------------------------------------------------------------------
namespace {
constexpr int kFmaChains = 8;
constexpr int kFmaIters = 2048;
constexpr int kFmaThreads = 256;

__global__ void __launch_bounds__(kFmaThreads) k_fp64_fma(double b, double c, double *__restrict__ sink)
{
    double a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < kFmaIters; ++it)
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
    if (threadIdx.x == 0) sink[blockIdx.x] = s;  // keeps the chains live
}
}  // namespace

void set_last_error_global(const char *msg);  // defined in lbm_api.cu

}  // namespace lbm

extern "C" lbm_status lbm_fp64_fma_rate(void *stream, double *flops)
{
    using namespace lbm;
    if (!flops) {
        set_last_error_global("lbm_fp64_fma_rate: NULL output");
        return LBM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *sink = nullptr;
    float ms = 0.f;
    const int blocks_per_sm = 8;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * blocks_per_sm;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double) * (size_t)blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fp64_fma<<<blocks, kFmaThreads, 0, s>>>(0.999999, 1e-7, sink);  // warm-up
        cudaEventRecord(e0, s);
        k_fp64_fma<<<blocks, kFmaThreads, 0, s>>>(0.999999, 1e-7, sink);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof buf, "lbm_fp64_fma_rate: %s", cudaGetErrorString(e));
        set_last_error_global(buf);
        return LBM_ERR_CUDA;
    }
    *flops = 2.0 * kFmaChains * (double)kFmaIters * kFmaThreads * blocks / (ms * 1e-3);
    return LBM_OK;
}
