// lbm_api.cu -- the C ABI of lbm.h: context, validation, memory, dispatch to
// the per-storage-type launchers, and the storage-independent kernels (tag
// preparation, reduction second pass).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lbm_kernels.cuh"

using namespace lbm;

struct lbm_ctx {
    int nx = 0, ny = 0, nz = 0, px = 0, Q = 0;
    lbm_dtype dtype = LBM_F32;
    Grid g{};
    size_t elem = 4;            // bytes per stored population value
    size_t pop_bytes = 0;       // bytes of one population array (Q planes)
    void *A = nullptr, *B = nullptr;
    uint8_t *tags = nullptr;    // internal padded tags
    double *partials = nullptr; // kRedBlocks x kRedSlots reduction scratch
    double *red_out = nullptr;  // kRedSlots final sums
    unsigned long long *census_dev = nullptr;  // LBM_NTAGS + 1 counters
    float *mlp_params = nullptr;  // closure weights (LBM_MLP_NPARAM) + normalisation (LBM_MLP_NNORM)
    void *mlp_image = nullptr;    // the network packed for the collide kernel
    uint32_t *fluid_list = nullptr;  // fluid-node list (mostly-wall lattices), else NULL
    uint2 *cwords = nullptr;         // its per-row fluid bitmask table (rows x px/32)
    long long n_list = 0;
    // Compact fluid-only copy of the state used while stepping with the list:
    // populations cA/cB [Q][nfp] in list order.
    void *cA = nullptr, *cB = nullptr;
    long long nfp = 0;
    bool compact_valid = false;  // cA holds the current state
    bool dense_stale = false;    // A lacks the current state (it is in cA)
    // AA pattern: one array (B and cB stay NULL), updated in place; aa_p is
    // set while the state is in layout P (after an odd step; the next step
    // is an even one).
    bool aa = false;
    bool aa_p = false;
    // CUDA graphs of two steps (X -> Y, Y -> X), replayed on a private stream
    // ordered after / before the caller's stream by events.  One graph per
    // kernel path (dense, compact) and array orientation; any change of
    // parameters or tags bumps `version` and invalidates them.
    bool use_graphs = true;
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        const void *first = nullptr;  // the array the graph reads first
        int path = -1;                // 0 dense, 1 compact
        unsigned long long version = 0;
    } graphs[4];
    unsigned long long version = 1;
    // TMA descriptors of the two population arrays (A/B pattern), used by the
    // learned-closure step; tma_ok is false when they could not be encoded.
    CUtensorMap tmap[2];
    const void *tmap_base[2] = {nullptr, nullptr};
    bool tma_ok = false;
    float *fpart = nullptr;   // per-block FP32 partials of fused step-and-reduce launches
    long long fpart_cap = 0;
    cudaStream_t stream = nullptr;
    lbm_allocator alloc{};
    bool has_alloc = false;
    lbm_params params{};
    long long census[LBM_NTAGS] = {};
    bool general = false;
    long long steps = 0;
    std::string err;
};

namespace {

thread_local std::string g_err;  // errors of calls without a context

lbm_status fail(lbm_ctx *ctx, lbm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    (ctx ? ctx->err : g_err) = buf;
    return s;
}

lbm_status cuda_fail(lbm_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CUDA_TRY(ctx, expr, what)                          \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

void *dev_alloc(lbm_ctx *ctx, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (ctx->has_alloc) return ctx->alloc.alloc(bytes, (void *)ctx->stream, ctx->alloc.user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lbm_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (ctx->has_alloc)
        ctx->alloc.free(p, bytes, (void *)ctx->stream, ctx->alloc.user);
    else
        cudaFree(p);
}

// RAII temporary device buffer.
struct Tmp {
    lbm_ctx *ctx;
    void *p = nullptr;
    size_t bytes = 0;
    Tmp(lbm_ctx *c, size_t b) : ctx(c), bytes(b) { p = b ? dev_alloc(c, b) : nullptr; }
    ~Tmp() { dev_free(ctx, p, bytes); }
};

Launch make_launch(lbm_ctx *ctx)
{
    Launch L;
    L.Q = ctx->Q;
    L.g = ctx->g;
    L.A = ctx->A;
    L.B = ctx->aa ? ctx->A : ctx->B;
    L.tags = ctx->tags;
    L.general = ctx->general;
    L.closure = ctx->params.closure;
    L.mlp_image = ctx->mlp_image;
    L.tma_A = nullptr;
    for (int k = 0; k < 2; ++k)
        if (ctx->tma_ok && ctx->tmap_base[k] == ctx->A) L.tma_A = &ctx->tmap[k];
    L.cmap.words = ctx->cwords;
    L.cmap.list = ctx->fluid_list;
    L.cmap.tags = ctx->tags;
    L.cmap.nx = ctx->g.nx;
    L.cmap.ny = ctx->g.ny;
    L.cmap.nz = ctx->g.nz;
    L.cmap.nw = ctx->g.px / 32;
    L.cmap.by_nw = FastDiv((uint32_t)(ctx->g.px / 32));
    L.cmap.by_ny = FastDiv((uint32_t)ctx->g.ny);
    L.n_list = ctx->n_list;
    L.moving_walls = false;
    for (int k = LBM_TAG_WALL0; k < LBM_NTAGS; ++k)
        if (ctx->census[k]) L.moving_walls = true;
    L.stream = ctx->stream;
    L.aa = ctx->aa;
    L.aa_p = ctx->aa_p;
    return L;
}

template <typename F> cudaError_t by_dtype(lbm_dtype d, F &&f)
{
    switch (d) {
    case LBM_F64: return f((double *)nullptr);
    case LBM_F32: return f((float *)nullptr);
    case LBM_F16_SHIFTED: return f((__half *)nullptr);
    case LBM_BF16_SHIFTED: return f((__nv_bfloat16 *)nullptr);
    case LBM_F16_SCALED: return f((h16s *)nullptr);
    }
    return cudaErrorInvalidValue;
}

lbm_status wait_stream(lbm_ctx *ctx, int timeout_ms)
{
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) return LBM_OK;
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "stream");
        if (timeout_ms >= 0) {
            const auto ms =
                std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms) return fail(ctx, LBM_ERR_TIMEOUT, "stream still busy after %d ms", timeout_ms);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Synchronizing calls wait without limit: a kernel of this library always
// terminates, so only a fault can end the wait early.
lbm_status sync(lbm_ctx *ctx) { return wait_stream(ctx, -1); }

bool valid_params(const lbm_params *p, std::string &why)
{
    if (!(p->tau > 0.5) || !isfinite(p->tau)) return why = "tau must be finite and > 1/2", false;
    if (p->closure < LBM_CLOSURE_BGK || p->closure > LBM_CLOSURE_TRT) return why = "unknown closure", false;
    if (p->closure == LBM_CLOSURE_TRT && !(p->trt_magic > 0.0 && isfinite(p->trt_magic)))
        return why = "TRT needs a finite trt_magic > 0", false;
    if (!(p->cs_smag >= 0.0) || !isfinite(p->cs_smag)) return why = "cs_smag must be >= 0", false;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(p->force[a])) return why = "force must be finite", false;
    for (int k = 0; k < LBM_NWALLS; ++k)
        for (int a = 0; a < 3; ++a)
            if (!isfinite(p->wall_u[k][a])) return why = "wall velocity must be finite", false;
    if (!isfinite(p->rho_wall)) return why = "rho_wall must be finite", false;
    return true;
}

// cuTensorMapEncodeTiled, looked up through the runtime (no link-time
// dependence on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return (EncodeTiledFn)p;
    }();
    return fn;
}

// TMA descriptor of one population array: a 4D tensor (x over the padded
// pitch, y, z, population) copied in boxes of one row of kTmaRow nodes.
bool encode_population_map(const lbm_ctx *ctx, const void *base, CUtensorMap *map)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn || !base) return false;
    const cuuint64_t e = ctx->elem;
    const CUtensorMapDataType type = e == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                     : e == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                              : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[4] = {(cuuint64_t)ctx->g.px, (cuuint64_t)ctx->g.ny, (cuuint64_t)ctx->g.nz,
                                (cuuint64_t)ctx->Q};
    const cuuint64_t strides[3] = {(cuuint64_t)ctx->g.px * e, (cuuint64_t)ctx->g.px * ctx->g.ny * e,
                                   (cuuint64_t)ctx->g.sN * e};
    const cuuint32_t box[4] = {(cuuint32_t)kTmaRow, 1, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, type, 4, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace lbm {
// Lets entry points without a context (lbm_noalloc.cu) report through
// lbm_last_error(NULL).
void set_last_error_global(const char *msg) { g_err = msg; }
}  // namespace lbm

// ---------------------------------------------------------------------------
// Storage-independent kernels.
// ---------------------------------------------------------------------------
namespace lbm {

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double *__restrict__ partials, int nblocks,
                                                             double *__restrict__ out)
{
    double acc[kRedSlots];
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k)
            acc[k] = (k == 9) ? fmax(acc[k], partials[(long long)b * kRedSlots + k])
                              : acc[k] + partials[(long long)b * kRedSlots + k];
    block_reduce_slots(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) out[k] = acc[k];
}

// First of two fixed-order passes over the FP32 block partials of a fused
// step: block b adds the partials of its contiguous chunk in FP64 and roots
// the maximum of |u|^2 (slot 9) in FP64, as the unfused reduction does.
__global__ void __launch_bounds__(kRedThreads) k_reduce_chunks(const float *__restrict__ partials, long long n,
                                                              double *__restrict__ out)
{
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    double acc[kRedSlots];
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) acc[k] = 0.0;
    for (long long b = lo + threadIdx.x; b < hi; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) {
            const double v = partials[b * kRedSlots + k];
            acc[k] = (k == 9) ? fmax(acc[k], v) : acc[k] + v;
        }
    block_reduce_slots(acc);
    if (threadIdx.x == 0) {
        acc[9] = sqrt(acc[9]);
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) out[(long long)blockIdx.x * kRedSlots + k] = acc[k];
    }
}

cudaError_t launch_reduce_partials(const float *partials, long long n, double *chunks, double *out, cudaStream_t s)
{
    k_reduce_chunks<<<kRedChunkBlocks, kRedThreads, 0, s>>>(partials, n, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, kRedThreads, 0, s>>>(chunks, kRedChunkBlocks, out);
    return cudaGetLastError();
}

// Copies user tags into the padded internal array, flags fluid nodes that
// pull from a SOLID or WALL neighbour, and counts tag values (slot LBM_NTAGS
// counts invalid values).
template <int Q>
__global__ void k_prepare_tags(Grid g, const uint8_t *__restrict__ user, uint8_t *__restrict__ tags,
                               unsigned long long *__restrict__ census)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    Nbr nb;
    nb.init(g, x, y, z);
    const long long n = x + (long long)g.nx * (y + (long long)g.ny * z);
    const unsigned t = user[n];
    if (t >= LBM_NTAGS) {
        atomicAdd(&census[LBM_NTAGS], 1ull);
        return;
    }
    atomicAdd(&census[t], 1ull);
    bool near = false;
    if (!is_wall_tag(t)) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            // source node x - c_i, read from the unpadded user array
            const int xs = nb.xs[1 - cvel(i, 0)];
            const int r = nb.row[1 - cvel(i, 1)][1 - cvel(i, 2)] / g.px;  // z*ny + y of the source
            near |= is_wall_tag(user[xs + (long long)g.nx * r]);
        }
    }
    tags[nb.self] = (uint8_t)(t | (near ? kNearWall : 0));
}

// User view of the internal tags: unpadded, flag bit cleared.
__global__ void k_gather_tags(Grid g, const uint8_t *__restrict__ tags, uint8_t *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    out[x + (long long)g.nx * (y + (long long)g.ny * z)] = tags[(z * g.ny + y) * g.px + x] & kTagMask;
}

cudaError_t launch_gather_tags(const Grid &g, const uint8_t *tags, uint8_t *out, cudaStream_t s)
{
    dim3 grid, block;
    node_launch_shape(g, grid, block);
    k_gather_tags<<<grid, block, 0, s>>>(g, tags, out);
    return cudaGetLastError();
}

cudaError_t launch_prepare_tags(int Q, const Grid &g, const uint8_t *user, uint8_t *tags, unsigned long long *census,
                                cudaStream_t s)
{
    dim3 grid, block;
    node_launch_shape(g, grid, block);
    if (Q == 19)
        k_prepare_tags<19><<<grid, block, 0, s>>>(g, user, tags, census);
    else
        k_prepare_tags<27><<<grid, block, 0, s>>>(g, user, tags, census);
    return cudaGetLastError();
}

}  // namespace lbm

// (Re)builds the fluid-node list after the tags changed, or drops it when the
// lattice is mostly fluid.  Row counts are scanned on the host.
static lbm_status build_fluid_list(lbm_ctx *ctx, bool wanted)
{
    const size_t rows = (size_t)ctx->g.nz * ctx->g.ny;
    const size_t nwords = rows * (size_t)(ctx->g.px / 32);
    dev_free(ctx, ctx->fluid_list, sizeof(uint32_t) * (size_t)ctx->n_list);
    dev_free(ctx, ctx->cwords, sizeof(uint2) * nwords);
    dev_free(ctx, ctx->cA, (size_t)ctx->Q * ctx->nfp * ctx->elem);
    dev_free(ctx, ctx->cB, (size_t)ctx->Q * ctx->nfp * ctx->elem);
    ctx->fluid_list = nullptr;
    ctx->cwords = nullptr;
    ctx->cA = ctx->cB = nullptr;
    ctx->n_list = ctx->nfp = 0;
    ctx->compact_valid = ctx->dense_stale = false;
    if (!wanted) return LBM_OK;
    Tmp count(ctx, sizeof(int) * rows);
    if (!count.p) return fail(ctx, LBM_ERR_OOM, "fluid-list allocation failed");
    CUDA_TRY(ctx, launch_fluid_count(ctx->g, ctx->tags, (int *)count.p, ctx->stream), "fluid count");
    std::vector<int> h(rows);
    CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), count.p, sizeof(int) * rows, cudaMemcpyDeviceToHost, ctx->stream),
             "fluid count copy");
    lbm_status s = sync(ctx);
    if (s != LBM_OK) return s;
    long long total = 0;
    for (size_t r = 0; r < rows; ++r) {  // exclusive prefix sum
        const int c = h[r];
        h[r] = (int)total;
        total += c;
    }
    if (total == 0) return LBM_OK;
    ctx->fluid_list = (uint32_t *)dev_alloc(ctx, sizeof(uint32_t) * (size_t)total);
    ctx->cwords = (uint2 *)dev_alloc(ctx, sizeof(uint2) * nwords);
    ctx->n_list = total;
    if (!ctx->fluid_list || !ctx->cwords) return fail(ctx, LBM_ERR_OOM, "fluid-list allocation failed");
    CUDA_TRY(ctx, cudaMemcpyAsync(count.p, h.data(), sizeof(int) * rows, cudaMemcpyHostToDevice, ctx->stream),
             "fluid start copy");
    CUDA_TRY(ctx, launch_fluid_scatter(ctx->g, ctx->tags, (const int *)count.p, ctx->fluid_list, ctx->cwords,
                                       ctx->stream),
             "fluid scatter");
    // Compact storage of the populations in list order.
    ctx->nfp = (total + 255) / 256 * 256;
    const size_t cbytes = (size_t)ctx->Q * ctx->nfp * ctx->elem;
    ctx->cA = dev_alloc(ctx, cbytes);
    ctx->cB = ctx->aa ? nullptr : dev_alloc(ctx, cbytes);
    if (!ctx->cA || (!ctx->aa && !ctx->cB)) return fail(ctx, LBM_ERR_OOM, "compact storage allocation failed");
    return sync(ctx);
}

// Brings the dense arrays up to date after steps on compact storage.
static lbm_status ensure_dense(lbm_ctx *ctx)
{
    if (!ctx->dense_stale) return LBM_OK;
    CUDA_TRY(ctx, launch_compact_copy(ctx->dtype, ctx->Q, false, ctx->cA, ctx->A, ctx->g.sN, ctx->fluid_list, ctx->n_list,
                                      ctx->nfp, ctx->stream),
             "compact scatter");
    ctx->dense_stale = false;
    return LBM_OK;
}

// The dense state was overwritten: the compact copy no longer holds it.
static void dense_written(lbm_ctx *ctx)
{
    ctx->compact_valid = false;
    ctx->dense_stale = false;
}

#define ENSURE_DENSE(ctx)                           \
    do {                                            \
        lbm_status es_ = ensure_dense(ctx);         \
        if (es_ != LBM_OK) return es_;              \
    } while (0)

// The kRedSlots final sums as an lbm_reduction; UNSTABLE when some fluid
// node had non-finite moments.
static lbm_status fill_reduction(lbm_ctx *ctx, const double *r, lbm_reduction *out)
{
    out->n_fluid = (long long)r[10];
    out->nonfinite = (long long)r[11];
    out->mass = (double)(out->n_fluid - out->nonfinite) + r[0];
    for (int a = 0; a < 3; ++a) {
        out->mom[a] = r[1 + a];
        out->vel[a] = r[4 + a];
    }
    out->ke = r[7];
    out->ke_rho = r[8];
    out->umax = r[9];
    if (out->nonfinite) return fail(ctx, LBM_ERR_UNSTABLE, "%lld fluid nodes have non-finite moments", out->nonfinite);
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------
extern "C" {

const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

lbm_status lbm_destroy(lbm_ctx *ctx)
{
    if (!ctx) return LBM_OK;
    cudaStreamSynchronize(ctx->stream);
    cudaGetLastError();
    for (auto &gr : ctx->graphs)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (ctx->gstream) {
        cudaStreamSynchronize(ctx->gstream);
        cudaStreamDestroy(ctx->gstream);
    }
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    cudaGetLastError();
    dev_free(ctx, ctx->A, ctx->pop_bytes);
    dev_free(ctx, ctx->B, ctx->pop_bytes);
    dev_free(ctx, ctx->tags, (size_t)ctx->g.sN);
    dev_free(ctx, ctx->partials, sizeof(double) * kRedBlocks * kRedSlots);
    dev_free(ctx, ctx->red_out, sizeof(double) * kRedSlots);
    dev_free(ctx, ctx->census_dev, sizeof(unsigned long long) * (LBM_NTAGS + 1));
    dev_free(ctx, ctx->mlp_params, sizeof(float) * (LBM_MLP_NPARAM + LBM_MLP_NNORM));
    dev_free(ctx, ctx->mlp_image, mlp_image_bytes());
    dev_free(ctx, ctx->fluid_list, sizeof(uint32_t) * (size_t)ctx->n_list);
    dev_free(ctx, ctx->cwords, sizeof(uint2) * (size_t)ctx->g.nz * ctx->g.ny * (size_t)(ctx->g.px / 32));
    dev_free(ctx, ctx->cA, (size_t)ctx->Q * ctx->nfp * ctx->elem);
    dev_free(ctx, ctx->cB, (size_t)ctx->Q * ctx->nfp * ctx->elem);
    dev_free(ctx, ctx->fpart, sizeof(float) * kRedSlots * (size_t)ctx->fpart_cap);
    delete ctx;
    return LBM_OK;
}

lbm_status lbm_create(int nx, int ny, int nz, lbm_lattice lattice, lbm_dtype dtype, const lbm_allocator *alloc,
                      void *stream, lbm_ctx **out)
{
    return lbm_create_ex(nx, ny, nz, lattice, dtype, LBM_PATTERN_AB, alloc, stream, out);
}

lbm_status lbm_create_ex(int nx, int ny, int nz, lbm_lattice lattice, lbm_dtype dtype, lbm_pattern pattern,
                         const lbm_allocator *alloc, void *stream, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (pattern != LBM_PATTERN_AB && pattern != LBM_PATTERN_AA)
        return fail(nullptr, LBM_ERR_ARG, "unknown streaming pattern %d", (int)pattern);
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_ERR_ARG, "lattice sizes must be >= 1");
    if (lattice != LBM_D3Q19 && lattice != LBM_D3Q27) return fail(nullptr, LBM_ERR_ARG, "unknown lattice %d", (int)lattice);
    if (dtype < LBM_F64 || dtype > LBM_F16_SCALED) return fail(nullptr, LBM_ERR_ARG, "unknown dtype %d", (int)dtype);
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, LBM_ERR_ARG, "allocator needs alloc and free");
    if (nz > 65535) return fail(nullptr, LBM_ERR_ARG, "nz must be <= 65535");
    const long long px = ((long long)nx + 31) / 32 * 32;
    const long long cells = px * ny * nz;
    if (cells >= (1ll << 31) - 256) return fail(nullptr, LBM_ERR_ARG, "lattice too large (padded nodes >= 2^31)");

    lbm_ctx *ctx = new (std::nothrow) lbm_ctx();
    if (!ctx) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    ctx->nx = nx;
    ctx->ny = ny;
    ctx->nz = nz;
    ctx->px = (int)px;
    ctx->Q = (int)lattice;
    ctx->dtype = dtype;
    ctx->aa = pattern == LBM_PATTERN_AA;
    ctx->elem = dtype == LBM_F64 ? 8 : dtype == LBM_F32 ? 4 : 2;
    ctx->g.nx = nx;
    ctx->g.ny = ny;
    ctx->g.nz = nz;
    ctx->g.px = (int)px;
    ctx->g.sN = (cells + 255) / 256 * 256;  // planes start 512-byte aligned or better
    ctx->g.N = (long long)nx * ny * nz;
    ctx->pop_bytes = (size_t)ctx->Q * (size_t)ctx->g.sN * ctx->elem;
    ctx->stream = (cudaStream_t)stream;
    if (alloc) {
        ctx->alloc = *alloc;
        ctx->has_alloc = true;
    }
    ctx->params.tau = 1.0;
    ctx->params.closure = LBM_CLOSURE_BGK;
    ctx->params.rho_wall = 1.0;
    ctx->params.trt_magic = 3.0 / 16.0;

    ctx->A = dev_alloc(ctx, ctx->pop_bytes);
    ctx->B = ctx->aa ? nullptr : dev_alloc(ctx, ctx->pop_bytes);
    ctx->tags = (uint8_t *)dev_alloc(ctx, (size_t)ctx->g.sN);
    ctx->partials = (double *)dev_alloc(ctx, sizeof(double) * kRedBlocks * kRedSlots);
    ctx->red_out = (double *)dev_alloc(ctx, sizeof(double) * kRedSlots);
    ctx->census_dev = (unsigned long long *)dev_alloc(ctx, sizeof(unsigned long long) * (LBM_NTAGS + 1));
    if (!ctx->A || (!ctx->aa && !ctx->B) || !ctx->tags || !ctx->partials || !ctx->red_out || !ctx->census_dev) {
        const double gb = ((ctx->aa ? 1.0 : 2.0) * ctx->pop_bytes + ctx->g.sN) / 1e9;
        lbm_destroy(ctx);
        return fail(nullptr, LBM_ERR_OOM, "device allocation of %.3f GB failed", gb);
    }
    cudaError_t e = cudaMemsetAsync(ctx->tags, 0, (size_t)ctx->g.sN, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->A, 0, ctx->pop_bytes, ctx->stream);
    if (e == cudaSuccess && ctx->B) e = cudaMemsetAsync(ctx->B, 0, ctx->pop_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        lbm_destroy(ctx);
        return cuda_fail(nullptr, e, "lbm_create");
    }
    ctx->census[LBM_TAG_FLUID] = ctx->g.N;
    if (!ctx->aa) {  // TMA descriptors for the learned-closure step (its older kernel serves without them)
        ctx->tmap_base[0] = ctx->A;
        ctx->tmap_base[1] = ctx->B;
        ctx->tma_ok = encode_population_map(ctx, ctx->A, &ctx->tmap[0]) &&
                      encode_population_map(ctx, ctx->B, &ctx->tmap[1]);
    }
    *out = ctx;
    return LBM_OK;
}

lbm_status lbm_set_params(lbm_ctx *ctx, const lbm_params *p)
{
    if (!ctx || !p) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    std::string why;
    if (!valid_params(p, why)) return fail(ctx, LBM_ERR_ARG, "%s", why.c_str());
    ctx->params = *p;
    ++ctx->version;
    return LBM_OK;
}

lbm_status lbm_set_tags(lbm_ctx *ctx, const uint8_t *tags, int on_device)
{
    if (!ctx || !tags) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (ctx->aa && ctx->aa_p)
        return fail(ctx, LBM_ERR_STATE,
                    "AA state after an odd number of steps holds bounced links for the current tags: step once more "
                    "before changing them");
    ENSURE_DENSE(ctx);
    const size_t n = (size_t)ctx->g.N;
    Tmp user(ctx, n);
    Tmp scratch(ctx, (size_t)ctx->g.sN);
    if (!user.p || !scratch.p) return fail(ctx, LBM_ERR_OOM, "tag staging allocation failed");
    CUDA_TRY(ctx, cudaMemcpyAsync(user.p, tags, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream),
             "tag copy");
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->census_dev, 0, sizeof(unsigned long long) * (LBM_NTAGS + 1), ctx->stream),
             "census reset");
    CUDA_TRY(ctx, cudaMemsetAsync(scratch.p, 0, (size_t)ctx->g.sN, ctx->stream), "tag reset");
    CUDA_TRY(ctx, launch_prepare_tags(ctx->Q, ctx->g, (const uint8_t *)user.p, (uint8_t *)scratch.p, ctx->census_dev, ctx->stream),
             "tag preparation");
    unsigned long long c[LBM_NTAGS + 1];
    CUDA_TRY(ctx, cudaMemcpyAsync(c, ctx->census_dev, sizeof c, cudaMemcpyDeviceToHost, ctx->stream), "census copy");
    lbm_status s = sync(ctx);
    if (s != LBM_OK) return s;
    if (c[LBM_NTAGS] != 0) return fail(ctx, LBM_ERR_ARG, "%llu tag values >= %d", c[LBM_NTAGS], (int)LBM_NTAGS);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->tags, scratch.p, (size_t)ctx->g.sN, cudaMemcpyDeviceToDevice, ctx->stream),
             "tag install");
    bool general = false;
    long long walls = 0;
    for (int k = 0; k < LBM_NTAGS; ++k) {
        ctx->census[k] = (long long)c[k];
        if (k != LBM_TAG_FLUID && c[k]) general = true;
        if (is_wall_tag((unsigned)k)) walls += (long long)c[k];
    }
    ctx->general = general;
    ++ctx->version;
    s = build_fluid_list(ctx, walls > kListWallFraction * (double)ctx->g.N);
    if (s != LBM_OK) return s;
    return sync(ctx);
}

lbm_status lbm_get_tags(lbm_ctx *ctx, uint8_t *tags, int on_device)
{
    if (!ctx || !tags) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    Tmp t(ctx, on_device ? 0 : (size_t)ctx->g.N);
    if (!on_device && !t.p) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    uint8_t *dst = on_device ? tags : (uint8_t *)t.p;
    CUDA_TRY(ctx, launch_gather_tags(ctx->g, ctx->tags, dst, ctx->stream), "tag gather");
    if (!on_device)
        CUDA_TRY(ctx, cudaMemcpyAsync(tags, t.p, (size_t)ctx->g.N, cudaMemcpyDeviceToHost, ctx->stream), "tag copy");
    return sync(ctx);
}

lbm_status lbm_tag_census(lbm_ctx *ctx, long long *counts)
{
    if (!ctx || !counts) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    for (int k = 0; k < LBM_NTAGS; ++k) counts[k] = ctx->census[k];
    return LBM_OK;
}

// The device address of page-locked host memory that the device can read
// directly (pinned by cudaHostAlloc or cudaHostRegister, mapped into the
// device's address space), or NULL for any other pointer.
static const void *device_view_of_pinned(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u, int on_device)
{
    if (!ctx) return fail(ctx, LBM_ERR_ARG, "NULL context");
    const size_t nb = sizeof(double) * (size_t)ctx->g.N;
    Launch L = make_launch(ctx);
    lbm_status s = LBM_OK;
    const double *rho_view = on_device ? nullptr : (const double *)device_view_of_pinned(rho);
    const double *u_view = on_device ? nullptr : (const double *)device_view_of_pinned(u);
    if (!on_device && (rho || u) && (!rho || rho_view) && (!u || u_view)) {
        // Page-locked host fields: the kernel reads them over the host link
        // directly (one pass, no staging buffer, no copy-engine transfer);
        // they must stay valid until the kernel ends, hence the wait.
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_init<S>(L, rho_view, u_view);
                 }),
                 "init");
        s = sync(ctx);
    } else if (on_device || (!rho && !u)) {
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_init<S>(L, rho, u);
                 }),
                 "init");
    } else {
        Tmp r(ctx, rho ? nb : 0), v(ctx, u ? 3 * nb : 0);
        if ((rho && !r.p) || (u && !v.p)) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
        if (rho) CUDA_TRY(ctx, cudaMemcpyAsync(r.p, rho, nb, cudaMemcpyHostToDevice, ctx->stream), "rho copy");
        if (u) CUDA_TRY(ctx, cudaMemcpyAsync(v.p, u, 3 * nb, cudaMemcpyHostToDevice, ctx->stream), "u copy");
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_init<S>(L, rho ? (const double *)r.p : nullptr, u ? (const double *)v.p : nullptr);
                 }),
                 "init");
        s = sync(ctx);
    }
    ctx->steps = 0;
    ctx->aa_p = false;
    dense_written(ctx);
    return s;
}

// One collide-and-stream launch of the current path from X to Y on stream st
// (AA: X == Y, an even step when layout_p, else an odd one).
static cudaError_t launch_one(lbm_ctx *ctx, bool compact, const void *X, void *Y, cudaStream_t st, bool layout_p)
{
    Launch L = make_launch(ctx);
    L.stream = st;
    L.aa_p = ctx->aa && layout_p;
    if (compact)
        return by_dtype(ctx->dtype, [&](auto *tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            return launch_step_compact<S>(L, ctx->params, X, Y, ctx->nfp, nullptr);
        });
    L.A = X;
    L.B = Y;
    L.tma_A = nullptr;
    for (int k = 0; k < 2; ++k)
        if (ctx->tma_ok && ctx->tmap_base[k] == X) L.tma_A = &ctx->tmap[k];
    return by_dtype(ctx->dtype, [&](auto *tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return launch_step<S>(L, ctx->params);
    });
}

// The two-step graph for the current path and orientation, captured on first
// use.  Returns nullptr when graphs cannot be used (capture refused).
static cudaGraphExec_t two_step_graph(lbm_ctx *ctx, bool compact, const void *X, void *Y)
{
    const int path = compact ? 1 : 0;
    lbm_ctx::Graph *slot = nullptr;
    for (auto &gr : ctx->graphs)
        if (gr.exec && gr.path == path && gr.first == X && gr.version == ctx->version) return gr.exec;
    for (auto &gr : ctx->graphs)
        if (!gr.exec || gr.version != ctx->version) {
            slot = &gr;
            break;
        }
    if (!slot) slot = &ctx->graphs[0];
    if (slot->exec) {
        cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
    }
    if (!ctx->gstream) {
        if (cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ctx->use_graphs = false;
            return nullptr;
        }
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        ctx->use_graphs = false;
        return nullptr;
    }
    // AB: X -> Y -> X; AA (X == Y): an odd step, then an even one
    const cudaError_t e1 = launch_one(ctx, compact, X, Y, ctx->gstream, false);
    const cudaError_t e2 = launch_one(ctx, compact, Y, (void *)X, ctx->gstream, ctx->aa);
    const cudaError_t e3 = cudaStreamEndCapture(ctx->gstream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && graph &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        slot->exec = exec;
        slot->first = X;
        slot->path = path;
        slot->version = ctx->version;
    } else {
        exec = nullptr;
        ctx->use_graphs = false;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return exec;
}

// n steps on the current path: pairs of steps as graph replays (when n is
// large enough and graphs are enabled), the remainder as plain launches.
static lbm_status run_steps(lbm_ctx *ctx, int n, bool compact)
{
    if (ctx->aa) {
        // In place: an even step first when the state is in layout P, then
        // (odd, even) pairs, then a final odd step if one is left.
        void *F = compact ? ctx->cA : ctx->A;
        if (ctx->aa_p && n > 0) {
            CUDA_TRY(ctx, launch_one(ctx, compact, F, F, ctx->stream, true), "collide-stream launch");
            ctx->aa_p = false;
            ++ctx->steps;
            --n;
        }
        const int pairs = (ctx->use_graphs && n >= 4) ? n / 2 : 0;
        if (pairs) {
            cudaGraphExec_t exec = two_step_graph(ctx, compact, F, F);
            if (exec) {
                CUDA_TRY(ctx, cudaEventRecord(ctx->ev_in, ctx->stream), "graph order");
                CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0), "graph order");
                for (int r = 0; r < pairs; ++r) CUDA_TRY(ctx, cudaGraphLaunch(exec, ctx->gstream), "graph launch");
                CUDA_TRY(ctx, cudaEventRecord(ctx->ev_out, ctx->gstream), "graph order");
                CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0), "graph order");
                ctx->steps += 2LL * pairs;
                n -= 2 * pairs;
            }
        }
        for (int k = 0; k < n; ++k) {
            CUDA_TRY(ctx, launch_one(ctx, compact, F, F, ctx->stream, ctx->aa_p), "collide-stream launch");
            ctx->aa_p = !ctx->aa_p;
            ++ctx->steps;
        }
        return LBM_OK;
    }
    void **X = compact ? &ctx->cA : &ctx->A;
    void **Y = compact ? &ctx->cB : &ctx->B;
    int pairs = (ctx->use_graphs && n >= 4) ? n / 2 : 0;
    if (pairs) {
        cudaGraphExec_t exec = two_step_graph(ctx, compact, *X, *Y);
        if (exec) {
            CUDA_TRY(ctx, cudaEventRecord(ctx->ev_in, ctx->stream), "graph order");
            CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0), "graph order");
            for (int r = 0; r < pairs; ++r) CUDA_TRY(ctx, cudaGraphLaunch(exec, ctx->gstream), "graph launch");
            CUDA_TRY(ctx, cudaEventRecord(ctx->ev_out, ctx->gstream), "graph order");
            CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0), "graph order");
            ctx->steps += 2LL * pairs;
            n -= 2 * pairs;  // an even number of steps leaves X and Y in place
        }
    }
    for (int k = 0; k < n; ++k) {
        CUDA_TRY(ctx, launch_one(ctx, compact, *X, *Y, ctx->stream, false), "collide-stream launch");
        std::swap(*X, *Y);
        ++ctx->steps;
    }
    return LBM_OK;
}

// Whether steps run on the compact fluid-only copy (mostly-wall lattices;
// the learned closure needs whole warps of x-consecutive nodes and keeps the
// dense sweep).
static bool steps_on_compact(const lbm_ctx *ctx) { return ctx->cA && ctx->params.closure != LBM_CLOSURE_MLP; }

// Makes the compact copy hold the current state before steps on it.
static lbm_status enter_compact(lbm_ctx *ctx)
{
    if (!ctx->compact_valid) {
        CUDA_TRY(ctx, launch_compact_copy(ctx->dtype, ctx->Q, true, ctx->A, ctx->cA, ctx->g.sN, ctx->fluid_list,
                                          ctx->n_list, ctx->nfp, ctx->stream),
                 "compact gather");
        ctx->compact_valid = true;
    }
    ctx->dense_stale = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *ctx, int n)
{
    if (!ctx) return fail(ctx, LBM_ERR_ARG, "NULL context");
    if (n < 0) return fail(ctx, LBM_ERR_ARG, "n must be >= 0");
    if (ctx->params.closure == LBM_CLOSURE_MLP && !ctx->mlp_image)
        return fail(ctx, LBM_ERR_STATE, "MLP closure selected but no weights were set (lbm_set_closure_weights)");
    if (n == 0) return LBM_OK;
    if (steps_on_compact(ctx)) {
        lbm_status st = enter_compact(ctx);
        return st != LBM_OK ? st : run_steps(ctx, n, true);
    }
    ENSURE_DENSE(ctx);
    ctx->compact_valid = false;
    return run_steps(ctx, n, false);
}

lbm_status lbm_step_reduce(lbm_ctx *ctx, int n, lbm_reduction *out)
{
    if (!ctx || !out) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (n < 1) return fail(ctx, LBM_ERR_ARG, "n must be >= 1");
    const bool fusable = ctx->dtype != LBM_F64 && ctx->params.closure != LBM_CLOSURE_MLP &&
                         ctx->params.closure != LBM_CLOSURE_STREAM_ONLY;
    if (!fusable) {  // FP64, learned closure, pure streaming: separate passes
        lbm_status st = lbm_step(ctx, n);
        return st != LBM_OK ? st : lbm_reduce(ctx, out);
    }
    const bool compact = steps_on_compact(ctx);
    lbm_status st;
    if (compact) {
        st = enter_compact(ctx);
        if (st != LBM_OK) return st;
    } else {
        ENSURE_DENSE(ctx);
        ctx->compact_valid = false;
    }
    st = run_steps(ctx, n - 1, compact);
    if (st != LBM_OK) return st;
    Launch L = make_launch(ctx);
    const long long nparts =
        compact ? (ctx->n_list + kStepThreads - 1) / kStepThreads : fused_partials(L, ctx->params, ctx->elem);
    if (nparts > ctx->fpart_cap) {
        dev_free(ctx, ctx->fpart, sizeof(float) * kRedSlots * (size_t)ctx->fpart_cap);
        ctx->fpart = (float *)dev_alloc(ctx, sizeof(float) * kRedSlots * (size_t)nparts);
        ctx->fpart_cap = ctx->fpart ? nparts : 0;
        if (!ctx->fpart) return fail(ctx, LBM_ERR_OOM, "reduction partials allocation failed");
    }
    void **X = compact ? &ctx->cA : &ctx->A;
    void **Y = compact ? (ctx->aa ? &ctx->cA : &ctx->cB) : (ctx->aa ? &ctx->A : &ctx->B);
    CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                 using S = std::remove_pointer_t<decltype(tag)>;
                 if (compact) return launch_step_compact<S>(L, ctx->params, *X, *Y, ctx->nfp, ctx->fpart);
                 return launch_step_reduce<S>(L, ctx->params, ctx->fpart);
             }),
             "fused collide-stream-reduce launch");
    if (ctx->aa)
        ctx->aa_p = !ctx->aa_p;
    else
        std::swap(*X, *Y);
    ++ctx->steps;
    CUDA_TRY(ctx, launch_reduce_partials(ctx->fpart, nparts, ctx->partials, ctx->red_out, ctx->stream), "reduce");
    double r[kRedSlots];
    CUDA_TRY(ctx, cudaMemcpyAsync(r, ctx->red_out, sizeof r, cudaMemcpyDeviceToHost, ctx->stream), "reduce copy");
    st = sync(ctx);
    if (st != LBM_OK) return st;
    return fill_reduction(ctx, r, out);
}

lbm_status lbm_use_graphs(lbm_ctx *ctx, int enable)
{
    if (!ctx) return fail(ctx, LBM_ERR_ARG, "NULL context");
    ctx->use_graphs = enable != 0;
    return LBM_OK;
}

lbm_status lbm_step_count(lbm_ctx *ctx, long long *steps)
{
    if (!ctx || !steps) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    *steps = ctx->steps;
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *u, int on_device)
{
    if (!ctx) return fail(ctx, LBM_ERR_ARG, "NULL context");
    ENSURE_DENSE(ctx);
    if (!rho && !u) return LBM_OK;
    const size_t nb = sizeof(double) * (size_t)ctx->g.N;
    Launch L = make_launch(ctx);
    if (on_device) {
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_moments<S>(L, ctx->params, rho, u);
                 }),
                 "moments");
        return sync(ctx);
    }
    Tmp r(ctx, rho ? nb : 0), v(ctx, u ? 3 * nb : 0);
    if ((rho && !r.p) || (u && !v.p)) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                 using S = std::remove_pointer_t<decltype(tag)>;
                 return launch_moments<S>(L, ctx->params, rho ? (double *)r.p : nullptr, u ? (double *)v.p : nullptr);
             }),
             "moments");
    if (rho) CUDA_TRY(ctx, cudaMemcpyAsync(rho, r.p, nb, cudaMemcpyDeviceToHost, ctx->stream), "rho copy");
    if (u) CUDA_TRY(ctx, cudaMemcpyAsync(u, v.p, 3 * nb, cudaMemcpyDeviceToHost, ctx->stream), "u copy");
    return sync(ctx);
}

lbm_status lbm_reduce(lbm_ctx *ctx, lbm_reduction *out)
{
    if (!ctx || !out) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    Launch L = make_launch(ctx);
    if (ctx->cA && ctx->compact_valid) {
        // The compact copy holds the current state: reduce over the fluid
        // nodes there, without writing the dense arrays back.
        long long nb = (ctx->n_list + kRedThreads - 1) / kRedThreads;
        if (nb > kRedBlocks) nb = kRedBlocks;
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_reduce_compact<S>(L, ctx->params, ctx->cA, ctx->nfp, ctx->partials, (int)nb,
                                                     ctx->red_out);
                 }),
                 "reduce");
    } else {
        ENSURE_DENSE(ctx);
        const long long total = (long long)ctx->g.nz * ctx->g.ny * ctx->g.px;
        long long nb = (total + kRedThreads - 1) / kRedThreads;
        if (nb > kRedBlocks) nb = kRedBlocks;
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_reduce<S>(L, ctx->params, ctx->partials, (int)nb, ctx->red_out);
                 }),
                 "reduce");
    }
    double r[kRedSlots];
    CUDA_TRY(ctx, cudaMemcpyAsync(r, ctx->red_out, sizeof r, cudaMemcpyDeviceToHost, ctx->stream), "reduce copy");
    lbm_status s = sync(ctx);
    if (s != LBM_OK) return s;
    return fill_reduction(ctx, r, out);
}

lbm_status lbm_closure_features(lbm_ctx *ctx, float *x, int on_device)
{
    if (!ctx || !x) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    ENSURE_DENSE(ctx);
    const size_t nb = sizeof(float) * 7 * (size_t)ctx->g.N;
    Tmp t(ctx, on_device ? 0 : nb);
    if (!on_device && !t.p) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    Launch L = make_launch(ctx);
    float *dst = on_device ? x : (float *)t.p;
    CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                 using S = std::remove_pointer_t<decltype(tag)>;
                 return launch_closure_features<S>(L, ctx->params, dst);
             }),
             "closure features");
    if (!on_device) CUDA_TRY(ctx, cudaMemcpyAsync(x, t.p, nb, cudaMemcpyDeviceToHost, ctx->stream), "features copy");
    return sync(ctx);
}

lbm_status lbm_sync(lbm_ctx *ctx, int timeout_ms)
{
    if (!ctx) return fail(ctx, LBM_ERR_ARG, "NULL context");
    return wait_stream(ctx, timeout_ms);
}

lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int on_device)
{
    if (!ctx || !f) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    ENSURE_DENSE(ctx);
    const size_t nb = sizeof(double) * (size_t)ctx->g.N;
    Tmp plane(ctx, on_device ? 0 : nb);
    if (!on_device && !plane.p) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    Launch L = make_launch(ctx);
    for (int i = 0; i < ctx->Q; ++i) {
        double *dst = on_device ? f + (size_t)i * ctx->g.N : (double *)plane.p;
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_get_pop<S>(L, i, dst);
                 }),
                 "population gather");
        if (!on_device) {
            CUDA_TRY(ctx, cudaMemcpyAsync(f + (size_t)i * ctx->g.N, plane.p, nb, cudaMemcpyDeviceToHost, ctx->stream),
                     "population copy");
        }
    }
    return sync(ctx);
}

lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int on_device)
{
    if (!ctx || !f) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    dense_written(ctx);
    ctx->aa_p = false;  // AA: written in layout S
    const size_t nb = sizeof(double) * (size_t)ctx->g.N;
    Tmp plane(ctx, on_device ? 0 : nb);
    if (!on_device && !plane.p) return fail(ctx, LBM_ERR_OOM, "staging allocation failed");
    Launch L = make_launch(ctx);
    for (int i = 0; i < ctx->Q; ++i) {
        const double *src = f + (size_t)i * ctx->g.N;
        if (!on_device) {
            CUDA_TRY(ctx, cudaMemcpyAsync(plane.p, src, nb, cudaMemcpyHostToDevice, ctx->stream), "population copy");
            src = (const double *)plane.p;
        }
        CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                     using S = std::remove_pointer_t<decltype(tag)>;
                     return launch_set_pop<S>(L, i, src);
                 }),
                 "population scatter");
    }
    return on_device ? LBM_OK : sync(ctx);
}

lbm_status lbm_get_state(lbm_ctx *ctx, void *buf, size_t bytes, int *layout, long long *steps, int on_device)
{
    if (!ctx || !buf) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (bytes != ctx->pop_bytes)
        return fail(ctx, LBM_ERR_ARG, "state buffer of %zu bytes, the state has %zu", bytes, ctx->pop_bytes);
    ENSURE_DENSE(ctx);
    CUDA_TRY(ctx,
             cudaMemcpyAsync(buf, ctx->A, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             ctx->stream),
             "state copy");
    lbm_status s = sync(ctx);
    if (s != LBM_OK) return s;
    if (layout) *layout = (ctx->aa && ctx->aa_p) ? 1 : 0;
    if (steps) *steps = ctx->steps;
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx *ctx, const void *buf, size_t bytes, int layout, long long steps, int on_device)
{
    if (!ctx || !buf) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (bytes != ctx->pop_bytes)
        return fail(ctx, LBM_ERR_ARG, "state buffer of %zu bytes, the state has %zu", bytes, ctx->pop_bytes);
    if (layout != 0 && layout != 1) return fail(ctx, LBM_ERR_ARG, "layout must be 0 or 1");
    if (layout == 1 && !ctx->aa) return fail(ctx, LBM_ERR_ARG, "layout 1 exists only with the AA pattern");
    if (steps < 0) return fail(ctx, LBM_ERR_ARG, "steps must be >= 0");
    CUDA_TRY(ctx,
             cudaMemcpyAsync(ctx->A, buf, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             ctx->stream),
             "state copy");
    if (!ctx->aa)
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->B, ctx->A, bytes, cudaMemcpyDeviceToDevice, ctx->stream), "state copy");
    dense_written(ctx);
    ctx->aa_p = layout == 1;
    ctx->steps = steps;
    return sync(ctx);
}

lbm_status lbm_geometry_spheres(lbm_ctx *ctx, const int32_t *centres, const double *radii, int n_spheres,
                                double target_porosity, uint8_t pore_tag, int *n_used, double *porosity)
{
    if (!ctx) return fail(ctx, LBM_ERR_ARG, "NULL context");
    if (n_spheres < 0 || (n_spheres > 0 && (!centres || !radii))) return fail(ctx, LBM_ERR_ARG, "bad sphere list");
    if (pore_tag != LBM_TAG_FLUID && pore_tag != LBM_TAG_FORCED)
        return fail(ctx, LBM_ERR_ARG, "pore_tag must be LBM_TAG_FLUID or LBM_TAG_FORCED");
    if (!isfinite(target_porosity)) return fail(ctx, LBM_ERR_ARG, "target porosity must be finite");
    for (int s = 0; s < n_spheres; ++s)
        if (!(radii[s] >= 0.0) || !(radii[s] <= 1024.0)) return fail(ctx, LBM_ERR_ARG, "radius %d not in [0, 1024]", s);
    const long long N = ctx->g.N;
    const size_t ns = (size_t)n_spheres;
    Tmp dc(ctx, 3 * sizeof(int32_t) * ns), dr(ctx, sizeof(double) * ns), cover(ctx, sizeof(uint32_t) * (size_t)N),
        count(ctx, sizeof(uint32_t) * (ns + 1)), tags(ctx, (size_t)N);
    if ((ns && (!dc.p || !dr.p)) || !cover.p || !count.p || !tags.p)
        return fail(ctx, LBM_ERR_OOM, "geometry staging allocation failed");
    if (ns) {
        CUDA_TRY(ctx, cudaMemcpyAsync(dc.p, centres, 3 * sizeof(int32_t) * ns, cudaMemcpyHostToDevice, ctx->stream), "centres");
        CUDA_TRY(ctx, cudaMemcpyAsync(dr.p, radii, sizeof(double) * ns, cudaMemcpyHostToDevice, ctx->stream), "radii");
    }
    CUDA_TRY(ctx, cudaMemsetAsync(cover.p, 0xff, sizeof(uint32_t) * (size_t)N, ctx->stream), "cover reset");
    CUDA_TRY(ctx, cudaMemsetAsync(count.p, 0, sizeof(uint32_t) * (ns + 1), ctx->stream), "count reset");
    CUDA_TRY(ctx, launch_sphere_cover(ctx->nx, ctx->ny, ctx->nz, (const int *)dc.p, (const double *)dr.p, n_spheres,
                                      (uint32_t *)cover.p, ctx->stream),
             "sphere cover");
    CUDA_TRY(ctx, launch_sphere_histogram(N, (const uint32_t *)cover.p, (uint32_t *)count.p, ctx->stream), "histogram");
    std::vector<uint32_t> hist(ns + 1);
    CUDA_TRY(ctx, cudaMemcpyAsync(hist.data(), count.p, sizeof(uint32_t) * (ns + 1), cudaMemcpyDeviceToHost, ctx->stream),
             "histogram copy");
    lbm_status st = sync(ctx);
    if (st != LBM_OK) return st;
    // Sequential stopping rule: before adding sphere s, stop if the pore
    // fraction is already at or below the target.
    long long solid = 0;
    int used = n_spheres;
    for (int s = 0; s < n_spheres; ++s) {
        if ((double)(N - solid) / (double)N <= target_porosity) {
            used = s;
            break;
        }
        solid += hist[s];
    }
    CUDA_TRY(ctx, launch_sphere_tags(N, (const uint32_t *)cover.p, (uint32_t)used, pore_tag, (uint8_t *)tags.p, ctx->stream),
             "sphere tags");
    st = lbm_set_tags(ctx, (const uint8_t *)tags.p, 1);
    if (st != LBM_OK) return st;
    if (n_used) *n_used = used;
    if (porosity) *porosity = (double)(N - solid) / (double)N;
    return LBM_OK;
}

lbm_status lbm_enstrophy(lbm_ctx *ctx, double *out)
{
    if (!ctx || !out) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    ENSURE_DENSE(ctx);
    const long long N = ctx->g.N;
    Tmp u(ctx, 3 * sizeof(double) * (size_t)N);
    if (!u.p) return fail(ctx, LBM_ERR_OOM, "velocity staging allocation failed");
    Launch L = make_launch(ctx);
    CUDA_TRY(ctx, by_dtype(ctx->dtype, [&](auto *tag) {
                 using S = std::remove_pointer_t<decltype(tag)>;
                 return launch_moments<S>(L, ctx->params, nullptr, (double *)u.p);
             }),
             "moments");
    long long nb = (N + kRedThreads - 1) / kRedThreads;
    if (nb > kRedBlocks) nb = kRedBlocks;
    CUDA_TRY(ctx, launch_enstrophy(ctx->dtype == LBM_F64, ctx->nx, ctx->ny, ctx->nz, (const double *)u.p, ctx->partials,
                                   (int)nb, ctx->red_out, ctx->stream),
             "enstrophy");
    double r[kRedSlots];
    CUDA_TRY(ctx, cudaMemcpyAsync(r, ctx->red_out, sizeof r, cudaMemcpyDeviceToHost, ctx->stream), "enstrophy copy");
    lbm_status st = sync(ctx);
    if (st != LBM_OK) return st;
    *out = r[0] / (double)N;
    return LBM_OK;
}

lbm_status lbm_set_closure_weights(lbm_ctx *ctx, const float *params, const float *norm, int on_device)
{
    if (!ctx || !params || !norm) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    float host[LBM_MLP_NPARAM + LBM_MLP_NNORM];
    const float *src_p = params, *src_n = norm;
    if (on_device) {
        CUDA_TRY(ctx, cudaMemcpyAsync(host, params, sizeof(float) * LBM_MLP_NPARAM, cudaMemcpyDeviceToHost, ctx->stream),
                 "weights copy");
        CUDA_TRY(ctx, cudaMemcpyAsync(host + LBM_MLP_NPARAM, norm, sizeof(float) * LBM_MLP_NNORM, cudaMemcpyDeviceToHost,
                                      ctx->stream),
                 "norm copy");
        lbm_status s = sync(ctx);
        if (s != LBM_OK) return s;
    } else {
        memcpy(host, params, sizeof(float) * LBM_MLP_NPARAM);
        memcpy(host + LBM_MLP_NPARAM, norm, sizeof(float) * LBM_MLP_NNORM);
    }
    src_p = host;
    src_n = host + LBM_MLP_NPARAM;
    for (int k = 0; k < LBM_MLP_NPARAM; ++k)
        if (!isfinite(src_p[k])) return fail(ctx, LBM_ERR_ARG, "closure weight %d is not finite", k);
    for (int k = 0; k < 15; ++k)
        if (!isfinite(src_n[k])) return fail(ctx, LBM_ERR_ARG, "normalisation entry %d is not finite", k);
    for (int k = 7; k < 14; ++k)
        if (!(src_n[k] > 0.f)) return fail(ctx, LBM_ERR_ARG, "normalisation std %d must be > 0", k - 7);
    if (!(src_n[14] >= 0.f)) return fail(ctx, LBM_ERR_ARG, "out_scale must be >= 0");
    if (!ctx->mlp_params) {
        ctx->mlp_params = (float *)dev_alloc(ctx, sizeof(float) * (LBM_MLP_NPARAM + LBM_MLP_NNORM));
        ctx->mlp_image = dev_alloc(ctx, mlp_image_bytes());
        if (!ctx->mlp_params || !ctx->mlp_image) return fail(ctx, LBM_ERR_OOM, "closure weight allocation failed");
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->mlp_params, host, sizeof host, cudaMemcpyHostToDevice, ctx->stream), "weights upload");
    CUDA_TRY(ctx, launch_mlp_pack(ctx->mlp_params, ctx->mlp_params + LBM_MLP_NPARAM, ctx->mlp_image, ctx->stream),
             "weights packing");
    return sync(ctx);
}

lbm_status lbm_info(lbm_ctx *ctx, size_t *population_bytes, int *pitch_x, int *q)
{
    if (!ctx) return fail(ctx, LBM_ERR_ARG, "NULL context");
    if (population_bytes) *population_bytes = ctx->pop_bytes;
    if (pitch_x) *pitch_x = ctx->px;
    if (q) *q = ctx->Q;
    return LBM_OK;
}

}  // extern "C"
