// lbm_noalloc.cu -- the allocation-free variant of the domain reduction.
//
// lbm_reduce needs a context, and lbm_create allocates device memory.  Some
// callers cannot allocate: a host code that owns the whole GPU through its
// own memory pool and forbids any other device allocation (for example an
// in-situ analysis plug-in running inside another solver), or a time loop
// that cannot afford the implicit device synchronisation of cudaMalloc /
// cudaFree.  lbm_reduce_noalloc serves them: the caller passes the
// populations and tags it already holds on the device, and the two-pass
// reduction keeps its per-block partials in the file-scope array below
// instead of in allocated memory.
//
// The array is a static device variable: every GPU that loads this library
// holds it (116,832 bytes) until the process exits.  All calls share it, so
// calls whose work overlaps on the GPU (different streams, or different host
// threads on the same device) race and must be serialised by the caller.
// Each call writes every slot it later reads, so stale contents of an
// earlier call are never used and nothing needs clearing.
#include <stdio.h>

#include <atomic>
#include <chrono>
#include <thread>

#include "lbm_kernels.cuh"

namespace lbm {
void set_last_error_global(const char *msg);  // defined in lbm_api.cu
}

using namespace lbm;

namespace {

// One partial per reduction block plus the final sums.
constexpr size_t kScratchDoubles = (size_t)(kRedBlocks + 1) * kRedSlots;
static __device__ __align__(256) double g_reduce_scratch[kScratchDoubles];
static_assert(sizeof(g_reduce_scratch) == 116832, "the header and the design notes state this size");

// The 32-bit offsets of k_reduce: the last offset a thread forms is below
// N + kRedThreads.
static_assert(LBM_NOALLOC_MAX_NODES + kRedThreads - 1 <= 2147483647LL, "node offsets must fit in int");

constexpr int kMaxDevices = 64;
std::atomic<double *> g_scratch_dev[kMaxDevices];

// Device address of the scratch array on the current device.  In host code
// g_reduce_scratch names a host-side shadow, not device memory, so the address
// must come from cudaGetSymbolAddress with that device current.  Only a
// successful lookup is kept: a lookup that failed (say, during a stream
// capture) is tried again by the next call.  Two threads that race on the
// first lookup store the same address.
cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    double *p = g_scratch_dev[dev].load(std::memory_order_acquire);
    if (!p) {
        void *q = nullptr;
        e = cudaGetSymbolAddress(&q, g_reduce_scratch);
        if (e != cudaSuccess) return e;
        p = (double *)q;
        g_scratch_dev[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

lbm_status fail(lbm_status s, const char *msg)
{
    set_last_error_global(msg);
    return s;
}

lbm_status fail_cuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return fail(LBM_ERR_CUDA, buf);
}

}  // namespace

extern "C" lbm_status lbm_reduce_noalloc(const void *h, lbm_lattice lattice, lbm_dtype dtype, int nx, int ny,
                                         int nz, const uint8_t *tags, const lbm_params *params, void *stream,
                                         lbm_reduction *out)
{
    if (!h || !out) return fail(LBM_ERR_ARG, "lbm_reduce_noalloc: NULL populations or output");
    if (lattice != LBM_D3Q19 && lattice != LBM_D3Q27) return fail(LBM_ERR_ARG, "lbm_reduce_noalloc: unknown lattice");
    if (dtype < LBM_F64 || dtype > LBM_F16_SCALED) return fail(LBM_ERR_ARG, "lbm_reduce_noalloc: unknown dtype");
    if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_ERR_ARG, "lbm_reduce_noalloc: lattice sizes must be >= 1");
    const long long N = (long long)nx * ny * nz;
    if (N > (long long)LBM_NOALLOC_MAX_NODES)
        return fail(LBM_ERR_ARG, "lbm_reduce_noalloc: more than LBM_NOALLOC_MAX_NODES (2^31 - 257) nodes");
    double *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return fail_cuda(e, "lbm_reduce_noalloc: scratch set-up");

    lbm_params p{};
    p.tau = 1.0;
    if (params)
        for (int a = 0; a < 3; ++a) p.force[a] = params->force[a];

    Launch L{};
    L.Q = (int)lattice;
    L.g.nx = nx;
    L.g.ny = ny;
    L.g.nz = nz;
    L.g.px = nx;  // caller layout: unpadded [Q][nz][ny][nx]
    L.g.sN = N;
    L.g.N = N;
    L.A = h;
    L.tags = tags;
    L.general = tags != nullptr;
    L.stream = (cudaStream_t)stream;
    long long nb = (N + kRedThreads - 1) / kRedThreads;
    if (nb > kRedBlocks) nb = kRedBlocks;  // grid-stride: any N fits in kRedBlocks partials
    double *partials = scratch;
    double *sums = scratch + (size_t)kRedBlocks * kRedSlots;
    switch (dtype) {
    case LBM_F64: e = L.Q == 19 ? reduce_q<19, double>(L, p, partials, (int)nb, sums) : reduce_q<27, double>(L, p, partials, (int)nb, sums); break;
    case LBM_F32: e = L.Q == 19 ? reduce_q<19, float>(L, p, partials, (int)nb, sums) : reduce_q<27, float>(L, p, partials, (int)nb, sums); break;
    case LBM_F16_SHIFTED:
        e = L.Q == 19 ? reduce_q<19, __half>(L, p, partials, (int)nb, sums) : reduce_q<27, __half>(L, p, partials, (int)nb, sums);
        break;
    case LBM_F16_SCALED:
        e = L.Q == 19 ? reduce_q<19, h16s>(L, p, partials, (int)nb, sums) : reduce_q<27, h16s>(L, p, partials, (int)nb, sums);
        break;
    default:
        e = L.Q == 19 ? reduce_q<19, __nv_bfloat16>(L, p, partials, (int)nb, sums)
                      : reduce_q<27, __nv_bfloat16>(L, p, partials, (int)nb, sums);
    }
    if (e != cudaSuccess) return fail_cuda(e, "lbm_reduce_noalloc: launch");
    double r[kRedSlots];
    e = cudaMemcpyAsync(r, sums, sizeof r, cudaMemcpyDeviceToHost, L.stream);
    if (e != cudaSuccess) return fail_cuda(e, "lbm_reduce_noalloc: copy");
    for (;;) {  // wait by polling; the reduction kernels always terminate
        e = cudaStreamQuery(L.stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return fail_cuda(e, "lbm_reduce_noalloc: stream");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
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
    if (out->nonfinite) return fail(LBM_ERR_UNSTABLE, "lbm_reduce_noalloc: fluid nodes with non-finite moments");
    return LBM_OK;
}
