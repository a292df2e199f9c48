// lbm_internal.cuh -- shared definitions of the CUDA library (not part of the
// C ABI): lattice tables, storage traits, kernel argument structs and the
// launcher declarations implemented once per storage type.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Lattice tables.  Order as documented in lbm.h; weights from |c|^2:
// D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216.  Called with
// compile-time indices inside unrolled loops, so every entry folds to an
// immediate.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cvel(int i, int a)
{
    constexpr int t[27 * 3] = {0,  0,  0,                                          //
                               1,  0,  0,  -1, 0,  0,  0,  1,  0,  0,  -1, 0,  0,  0,  1,  0,  0,  -1,  //
                               1,  1,  0,  -1, -1, 0,  1,  -1, 0,  -1, 1,  0,                         //
                               1,  0,  1,  -1, 0,  -1, 1,  0,  -1, -1, 0,  1,                         //
                               0,  1,  1,  0,  -1, -1, 0,  1,  -1, 0,  -1, 1,                         //
                               1,  1,  1,  -1, -1, -1, 1,  1,  -1, -1, -1, 1,                         //
                               1,  -1, 1,  -1, 1,  -1, -1, 1,  1,  1,  -1, -1};
    return t[3 * i + a];
}

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

__host__ __device__ constexpr int cnorm2(int i)
{
    return cvel(i, 0) * cvel(i, 0) + cvel(i, 1) * cvel(i, 1) + cvel(i, 2) * cvel(i, 2);
}

template <typename T>
__host__ __device__ constexpr T wgt(int Q, int i)
{
    return Q == 19 ? (cnorm2(i) == 0 ? T(1) / T(3) : cnorm2(i) == 1 ? T(1) / T(18) : T(1) / T(36))
                   : (cnorm2(i) == 0   ? T(8) / T(27)
                      : cnorm2(i) == 1 ? T(2) / T(27)
                      : cnorm2(i) == 2 ? T(1) / T(54)
                                       : T(1) / T(216));
}

// ---------------------------------------------------------------------------
// Storage traits: load h = f - w into the compute type, store rounded.
// ld goes through the read-only data path (arrays a kernel only reads); ldc
// is a plain coherent load, for arrays the kernel also writes.
// ---------------------------------------------------------------------------
template <typename S> struct Store;
template <> struct Store<double> {
    using T = double;
    static __device__ __forceinline__ T ld(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ T ldc(const double *p) { return *p; }
    static __device__ __forceinline__ void st(double *p, T v) { *p = v; }
    static __device__ __forceinline__ double from_f64(double v) { return v; }
    static __device__ __forceinline__ T rt(T v) { return v; }  // value as stored
};
template <> struct Store<float> {
    using T = float;
    static __device__ __forceinline__ T ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ T ldc(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, T v) { *p = v; }
    static __device__ __forceinline__ float from_f64(double v) { return (float)v; }
    static __device__ __forceinline__ T rt(T v) { return v; }
};
template <> struct Store<__half> {
    using T = float;
    static __device__ __forceinline__ T ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ T ldc(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, T v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ __half from_f64(double v) { return __float2half_rn((float)v); }
    static __device__ __forceinline__ T rt(T v) { return __half2float(__float2half_rn(v)); }
};
template <> struct Store<__nv_bfloat16> {
    using T = float;
    static __device__ __forceinline__ T ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ T ldc(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, T v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_f64(double v) { return __float2bfloat16_rn((float)v); }
    static __device__ __forceinline__ T rt(T v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

// FP16 of h * 2^12 (LBM_F16_SCALED).  Power-of-two scaling is exact in FP32,
// so the stored value is the FP16 rounding of the scaled deviation.
struct h16s {
    __half v;
};
constexpr float kF16sUp = 4096.0f, kF16sDown = 1.0f / 4096.0f;
template <> struct Store<h16s> {
    using T = float;
    static __device__ __forceinline__ T ld(const h16s *p) { return __half2float(__ldg(&p->v)) * kF16sDown; }
    static __device__ __forceinline__ T ldc(const h16s *p) { return __half2float(p->v) * kF16sDown; }
    static __device__ __forceinline__ void st(h16s *p, T v) { p->v = __float2half_rn(v * kF16sUp); }
    static __device__ __forceinline__ h16s from_f64(double v) { return h16s{__float2half_rn((float)v * kF16sUp)}; }
    static __device__ __forceinline__ T rt(T v) { return __half2float(__float2half_rn(v * kF16sUp)) * kF16sDown; }
};

// Fluid-node list (lattices that are mostly wall): one 32-bit entry per
// listed node, its padded offset (z ny + y) px + x with bit 31 set when the
// node carries the body force (offsets stay below 2^31 - 256).
constexpr uint32_t kListForced = 1u << 31;
constexpr uint32_t kListOffset = kListForced - 1u;
constexpr double kListWallFraction = 0.3;  // use the list above this wall fraction

// Division by a divisor fixed at launch (Granlund & Montgomery, "Division by
// invariant integers using multiplication", 1994, Sec. 4): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, the quotient of
// n < 2^31 is (umulhi(m, n) + n) >> l (the sum stays below 2^32).
struct FastDiv {
    uint32_t d = 1, m = 1;
    int l = 0;
    FastDiv() = default;
    explicit FastDiv(uint32_t div) : d(div)
    {
        l = 0;
        while ((1ull << l) < div) ++l;
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1ull);
    }
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const
    {
#ifdef __CUDA_ARCH__
        return (__umulhi(m, n) + n) >> l;
#else
        return (uint32_t)((((uint64_t)m * n >> 32) + n) >> l);
#endif
    }
};

// Addressing of the compact fluid-only storage without a stored neighbour
// index: per row of the padded lattice and per 32 x positions one entry
// {fluid bits, list position of the word's first fluid node}, so the list
// position of a fluid node (xs, row) is
//   words[row nw + xs/32].y + popc(words[..].x & ((1 << xs%32) - 1)).
// The table holds 8 bytes per 32 nodes (16 MB for 400^3); the step reads it
// through L2, and from HBM only the populations and one list entry per node.
struct CompactMap {
    const uint2 *words;     // [rows][nw]
    const uint32_t *list;   // [n_list]: offset | kListForced
    const uint8_t *tags;    // internal padded tags (read for moving-wall sources)
    int nx, ny, nz, nw;     // nw = px / 32 words per row
    FastDiv by_nw, by_ny;   // row = (offset / 32) / nw, z = row / ny
};

// Internal tag byte: the user tag in the low 7 bits, bit 7 set on fluid
// nodes that have a SOLID or WALL node among their Q neighbours.
constexpr uint8_t kNearWall = 0x80;
constexpr uint8_t kTagMask = 0x7f;

__host__ __device__ constexpr bool is_wall_tag(unsigned t) { return t >= LBM_TAG_SOLID && t < LBM_NTAGS; }

// Lattice geometry as the kernels see it: x padded to px, planes of sN.
struct Grid {
    int nx, ny, nz, px;
    long long sN;   // elements per population plane (>= nz*ny*px)
    long long N;    // nx*ny*nz (unpadded count)
};

// Parameters in the compute type.
template <typename T> struct KParams {
    T omega;                      // 1 / tau
    T omega_minus;                // TRT: 1 / tau_minus
    T tau;                        // tau
    T force[3];                   // g
    T smag18;                     // 18 Cs^2
    T wall6[LBM_NWALLS][3];       // 6 rho_wall u_wall (Ladd term = w_i c_i . wall6); 6 u_wall when wall_local
    int wall_local;               // rho_wall = the node's density after streaming
};

// Number of FP64 slots of one reduction partial.
constexpr int kRedSlots = 12;  // dmass, mom[3], vel[3], ke, ke_rho, umax, n_fluid, nonfinite
constexpr int kRedBlocks = 1216;  // 152 SMs x 8
constexpr int kRedThreads = 256;

// MLP closure parameters as the collide kernel reads them (device memory).
constexpr int kMlpIn = 7;
constexpr int kMlpH = 32;
constexpr int kMlpNParam = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 1345

// Launch arguments common to the per-dtype launchers.
struct Launch {
    int Q;
    Grid g;
    const void *A;
    void *B;
    const uint8_t *tags;      // internal padded tags
    bool general;             // tags present (not all FLUID)
    int closure;
    const void *mlp_image;    // device packed closure network (MlpSmem, closure 2)
    const CUtensorMap *tma_A; // TMA descriptor of the populations at A (host memory), or NULL
    CompactMap cmap;          // compact fluid-only storage (mostly-wall lattices)
    long long n_list;         // number of listed fluid nodes
    bool moving_walls;        // some node carries a moving-wall tag
    cudaStream_t stream;
    bool aa = false;    // AA pattern: one array, A == B
    bool aa_p = false;  // AA state in layout P (the next step is an even one)
};

// Per-storage-type launchers (one translation unit per type; each entry
// point hands AA launches (L.aa) to its _aa counterpart, which lives in the
// type's AA translation unit).
template <typename S> cudaError_t launch_step(const Launch &L, const lbm_params &p);
// One step that also writes per-block FP32 reduction partials of the new
// state, kRedSlots floats per block (cudaErrorNotSupported for FP64 storage
// and for closures without a fused variant).
template <typename S> cudaError_t launch_step_reduce(const Launch &L, const lbm_params &p, float *partials);
// One step on compact storage; with partials (FP32 compute; BGK,
// Smagorinsky, TRT) it also writes the block reduction partials of the new
// state, kRedSlots floats per block of kStepThreads listed nodes.
template <typename S>
cudaError_t launch_step_compact(const Launch &L, const lbm_params &p, const void *Ac, void *Bc, long long nfp,
                                float *partials);
// The domain reduction over the compact copy of the state.
template <typename S>
cudaError_t launch_reduce_compact(const Launch &L, const lbm_params &p, const void *Ac, long long nfp,
                                  double *partials, int nblocks, double *out);
template <typename S>
cudaError_t launch_reduce(const Launch &L, const lbm_params &p, double *partials, int nblocks, double *out);
template <typename S>
cudaError_t launch_moments(const Launch &L, const lbm_params &p, double *rho, double *u);
template <typename S>
cudaError_t launch_init(const Launch &L, const double *rho, const double *u);
template <typename S> cudaError_t launch_get_pop(const Launch &L, int i, double *f_plane);
template <typename S> cudaError_t launch_step_aa(const Launch &L, const lbm_params &p);
template <typename S> cudaError_t launch_step_reduce_aa(const Launch &L, const lbm_params &p, float *partials);
template <typename S>
cudaError_t launch_step_compact_aa(const Launch &L, const lbm_params &p, const void *Ac, void *Bc, long long nfp,
                                   float *partials);
template <typename S>
cudaError_t launch_reduce_compact_aa(const Launch &L, const lbm_params &p, const void *Ac, long long nfp,
                                     double *partials, int nblocks, double *out);
template <typename S>
cudaError_t launch_reduce_aa(const Launch &L, const lbm_params &p, double *partials, int nblocks, double *out);
template <typename S> cudaError_t launch_moments_aa(const Launch &L, const lbm_params &p, double *rho, double *u);
template <typename S> cudaError_t launch_get_pop_aa(const Launch &L, int i, double *f_plane);
// The learned closure's inputs of every node for the next step, x[N][7].
template <typename S> cudaError_t launch_closure_features(const Launch &L, const lbm_params &p, float *x);
template <typename S> cudaError_t launch_closure_features_aa(const Launch &L, const lbm_params &p, float *x);
template <typename S> cudaError_t launch_set_pop(const Launch &L, int i, const double *f_plane);

// Storage-type independent kernels (lbm_api.cu).
cudaError_t launch_prepare_tags(int Q, const Grid &g, const uint8_t *user_tags, uint8_t *tags,
                                unsigned long long *census, cudaStream_t s);
cudaError_t launch_gather_tags(const Grid &g, const uint8_t *tags, uint8_t *out, cudaStream_t s);
// Adds n FP32 block partials in FP64, in a fixed order (kRedChunkBlocks
// chunks into chunks[], then one block), into out[kRedSlots].
constexpr int kRedChunkBlocks = 304;  // 152 SMs x 2; <= kRedBlocks
cudaError_t launch_reduce_partials(const float *partials, long long n, double *chunks, double *out, cudaStream_t s);

// Fluid-node list (lbm_sparse.cu).
cudaError_t launch_fluid_count(const Grid &g, const uint8_t *tags, int *count, cudaStream_t s);
cudaError_t launch_fluid_scatter(const Grid &g, const uint8_t *tags, const int *start, uint32_t *list, uint2 *words,
                                 cudaStream_t s);
cudaError_t launch_compact_copy(lbm_dtype dtype, int Q, bool to_compact, const void *src, void *dst, long long sN,
                                const uint32_t *list, long long n, long long nfp, cudaStream_t s);

// Porous-medium generator and enstrophy diagnostic (lbm_diag.cu).
cudaError_t launch_sphere_cover(int nx, int ny, int nz, const int *centres, const double *radii, int n,
                                uint32_t *cover, cudaStream_t s);
cudaError_t launch_sphere_histogram(long long N, const uint32_t *cover, uint32_t *count, cudaStream_t s);
cudaError_t launch_sphere_tags(long long N, const uint32_t *cover, uint32_t used, uint8_t pore_tag, uint8_t *tags,
                               cudaStream_t s);
cudaError_t launch_mlp_pack(const float *params, const float *norm, void *image, cudaStream_t s);
size_t mlp_image_bytes();
cudaError_t launch_enstrophy(bool fp64, int nx, int ny, int nz, const double *u, double *partials, int nblocks,
                             double *out, cudaStream_t s);

}  // namespace lbm
