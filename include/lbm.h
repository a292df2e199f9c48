/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann hot path.
 *
 * The method is the fused collide-and-stream update of a 3D D3Q19 / D3Q27
 * lattice with structure-of-arrays populations and two-population (A/B)
 * streaming, cell behaviour chosen by an integer tag per node, and the
 * density / velocity / kinetic-energy reductions of Latt & Coreixas,
 * "Multi-GPU Acceleration of PALABOS Fluid Solver using C++ Standard
 * Parallelism" (Sec. 2.3 for the data layout and the tag mechanism, Sec. 3
 * for the collision model, boundary conditions and diagnostics).
 *
 * Conventions shared by every call:
 *  - Every call returns an lbm_status and never aborts the process; the text
 *    of the last failure is available from lbm_last_error().  Kernel faults
 *    surface as LBM_ERR_CUDA at the next call that synchronizes.
 *  - The caller owns every buffer it passes; the library copies in and out.
 *    Arguments called "on_device" say whether a pointer is CUDA device memory
 *    (1) or host memory (0).  Host buffers may be pageable.
 *  - Cell arrays are unpadded and x-fastest: flat index x + nx*(y + ny*z).
 *    Vector fields are [3][N] (component-major), populations [Q][N].
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - All work of a context is issued on the CUDA stream given at creation.
 *    Calls marked "asynchronous" return before the GPU has finished.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument (size, enum, tag value, tau <= 1/2 ...) */
    LBM_ERR_OOM = 2,      /* device allocation failed                              */
    LBM_ERR_CUDA = 3,     /* a CUDA call or kernel failed                          */
    LBM_ERR_STATE = 4,    /* call not valid in the current state                   */
    LBM_ERR_UNSTABLE = 5, /* a reduction met a non-finite density or velocity      */
    LBM_ERR_TIMEOUT = 6   /* lbm_sync gave up waiting                              */
} lbm_status;

/* Velocity sets.  D3Q19 is the paper's lattice (Sec. 3); D3Q27 is the one it
 * names as future work (Sec. 5).  Velocity order: 0 rest; 1..6 = +x -x +y -y
 * +z -z; 7..18 = (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 * (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1); D3Q27 adds 19..26 =
 * (1,1,1) (-1,-1,-1) (1,1,-1) (-1,-1,1) (1,-1,1) (-1,1,-1) (-1,1,1)
 * (1,-1,-1).  Direction i+1 is the opposite of direction i for odd i. */
typedef enum { LBM_D3Q19 = 19, LBM_D3Q27 = 27 } lbm_lattice;

/* Storage type of the populations.  Every type stores the offset-stripped
 * deviation h_i = f_i - w_i (Skordos' shift, Sec. 3); arithmetic runs in FP64
 * for LBM_F64 and in FP32 for the others; reductions accumulate in FP64.
 * The 16-bit types round to nearest-even on store.  LBM_F16_SCALED stores
 * FP16 of h * 2^12: the same 11 significant bits as LBM_F16_SHIFTED, with
 * the subnormal range moved from |h| < 6.1e-5 down to |h| < 1.5e-8 (where
 * a decaying flow's density and velocity deviations end up) and the largest
 * storable |h| at 16 (f lies in [0, rho], so only an unstable state gets
 * there: it becomes infinite and lbm_reduce reports it). */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16_SHIFTED = 2, LBM_BF16_SHIFTED = 3, LBM_F16_SCALED = 4 } lbm_dtype;

/* Streaming pattern (Sec. 2.3.1 names both; the paper's port uses the
 * two-population scheme and leaves the AA pattern to future work).
 *   LBM_PATTERN_AB: two population arrays; each step pulls from one and
 *     writes the other.
 *   LBM_PATTERN_AA: one array updated in place, steps alternating between a
 *     local step (read and write the node's own slots) and a step that reads
 *     from and writes to the neighbours; half the population memory, the
 *     same bytes moved per step and the same results, bit for bit, as AB
 *     (the arithmetic per node is identical). */
typedef enum { LBM_PATTERN_AB = 0, LBM_PATTERN_AA = 1 } lbm_pattern;

/* Node tags (Sec. 2.3.2: one integer per node selects the node's model). */
enum {
    LBM_TAG_FLUID = 0,  /* fluid node, collision only                               */
    LBM_TAG_FORCED = 1, /* fluid node with the body force of lbm_params.force       */
    LBM_TAG_SOLID = 2,  /* resting wall: halfway bounce-back, never updated         */
    LBM_TAG_WALL0 = 3,  /* LBM_TAG_WALL0 + k: moving wall k (Ladd), never updated   */
    LBM_NWALLS = 8,
    LBM_NTAGS = LBM_TAG_WALL0 + LBM_NWALLS
};

/* Collision closures. */
typedef enum {
    LBM_CLOSURE_BGK = 0,         /* BGK with the 2nd-order weighted equilibrium (Sec. 3.1) */
    LBM_CLOSURE_SMAGORINSKY = 1, /* BGK with a Smagorinsky eddy viscosity (Sec. 2.3.2)     */
    LBM_CLOSURE_MLP = 2,         /* BGK with a learned per-cell relaxation-time correction */
    LBM_CLOSURE_STREAM_ONLY = 3, /* no collision: pure streaming, for verification        */
    LBM_CLOSURE_TRT = 4          /* two relaxation times (Sec. 3.3's porous-rock model)    */
} lbm_closure;

/* Optional device allocator.  alloc returns device memory of at least
 * "bytes" bytes usable on "stream" (NULL on failure); free releases it.  A
 * NULL allocator in lbm_create selects cudaMalloc / cudaFree. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} lbm_allocator;

/* Model parameters (lattice units).
 *  tau      BGK relaxation time, tau > 1/2; viscosity nu = (tau - 1/2)/3.
 *  force    body force g applied to LBM_TAG_FORCED nodes with Guo's scheme.
 *  closure  an lbm_closure value.
 *  cs_smag  Smagorinsky constant (closure 1).
 *  wall_u   velocity of moving wall k, used by Ladd's bounce-back
 *           f_i(x) = f*_opp(i)(x) + 6 w_i rho_wall (c_i . wall_u[k]).
 *  rho_wall density in Ladd's wall term (the reference density, 1).
 *  trt_magic TRT's Lambda = (tau - 1/2)(tau_minus - 1/2) > 0, which sets the
 *           relaxation time tau_minus of the part of the populations that is
 *           odd under i -> opp(i); tau relaxes the even part.  Lambda = 3/16
 *           puts halfway bounce-back walls exactly halfway at any tau.
 *  wall_rho_local  1: rho_wall is each node's own density after streaming
 *           (rho_wall is then ignored).  The wall terms are linear in it, so
 *           it is rho0 / (1 - s), with rho0 the node's density with plain
 *           bounce-back and s the sum of 6 w_i (c_i . wall_u) over its
 *           moving-wall links.  0 (default): the constant rho_wall. */
typedef struct {
    double tau;
    double force[3];
    int closure;
    double cs_smag;
    double wall_u[LBM_NWALLS][3];
    double rho_wall;
    double trt_magic;
    int wall_rho_local;
} lbm_params;

/* Sums over fluid nodes (tags FLUID and FORCED), accumulated in FP64 from
 * the stored post-collision populations: rho = sum f_i and
 * u = (sum c_i f_i - rho g / 2) / rho on FORCED nodes (without the g term
 * elsewhere), i.e. the density and velocity that the last collision used. */
typedef struct {
    double mass;         /* sum rho                                   */
    double mom[3];       /* sum rho u                                 */
    double vel[3];       /* sum u                                     */
    double ke;           /* sum |u|^2 / 2   (k of Sec. 3.1 times N)   */
    double ke_rho;       /* sum rho |u|^2 / 2                         */
    double umax;         /* max |u|                                   */
    long long n_fluid;   /* number of fluid nodes                     */
    long long nonfinite; /* fluid nodes with non-finite rho or u      */
} lbm_reduction;

/* Creates a lattice of nx*ny*nz nodes (each >= 1, nx*ny*nz < 2^31 after
 * padding x to a multiple of 32), allocates both population arrays on the
 * device, sets every tag to FLUID, the parameters to tau = 1, no force, BGK,
 * rho_wall = 1, and the state to rest (f = w).  stream: a cudaStream_t, or
 * NULL for the legacy default stream.  On failure *out is NULL and nothing
 * stays allocated.  Errors: ARG, OOM, CUDA. */
lbm_status lbm_create(int nx, int ny, int nz, lbm_lattice lattice, lbm_dtype dtype, const lbm_allocator *alloc,
                      void *stream, lbm_ctx **out);

/* lbm_create with a streaming pattern (lbm_create is LBM_PATTERN_AB).  With
 * LBM_PATTERN_AA one population array is allocated, and after an odd number
 * of steps since the last initialisation the state is held in the
 * neighbour-shifted layout: every call still sees the same state (moments,
 * reductions and lbm_get_populations read either layout), but lbm_set_tags
 * then returns LBM_ERR_STATE, since the bounced links are stored according
 * to the old tags; take one more step first.  The two-nodes-per-thread
 * kernel of 16-bit storage serves A/B steps and the local (even) AA steps;
 * the odd AA steps use one node per thread.
 * Errors: as lbm_create, and ARG for an unknown pattern. */
lbm_status lbm_create_ex(int nx, int ny, int nz, lbm_lattice lattice, lbm_dtype dtype, lbm_pattern pattern,
                         const lbm_allocator *alloc, void *stream, lbm_ctx **out);

/* Waits for the context's stream and frees everything it owns.  NULL is a
 * no-op. */
lbm_status lbm_destroy(lbm_ctx *ctx);

/* Sets the model parameters.  Errors: ARG (tau <= 1/2 or not finite,
 * unknown closure, cs_smag < 0, trt_magic <= 0 with LBM_CLOSURE_TRT). */
lbm_status lbm_set_params(lbm_ctx *ctx, const lbm_params *p);

/* Sets the tag of every node (N bytes, values below LBM_NTAGS), derives the
 * per-node "next to a wall" flag and the tag census used to pick the kernel
 * variant (the analogue of the paper's hand-picked collision kernel,
 * Sec. 2.3.2).  Synchronizes.  Errors: ARG (a tag value >= LBM_NTAGS; the
 * previous tags stay in force), CUDA. */
lbm_status lbm_set_tags(lbm_ctx *ctx, const uint8_t *tags, int on_device);

/* Copies the tags out (N bytes).  Synchronizes. */
lbm_status lbm_get_tags(lbm_ctx *ctx, uint8_t *tags, int on_device);

/* Number of nodes per tag value, counts[LBM_NTAGS]. */
lbm_status lbm_tag_census(lbm_ctx *ctx, long long *counts);

/* Equilibrium initial state (Sec. 3.1, used for the Taylor-Green vortex):
 * f*_i = f_eq_i(rho, u) on every node, written to both population arrays.
 * rho: N values or NULL (uniform 1); u: [3][N] or NULL (rest).  Resets the
 * step counter.  Asynchronous for device inputs.  Host inputs that are
 * page-locked (cudaHostAlloc, cudaHostRegister, torch's pin_memory) are read
 * by the initialisation kernel directly over the host-device link; other
 * host inputs go through a device staging buffer.  Either way the call
 * returns once the host buffers are no longer needed.  Errors: CUDA, OOM. */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u, int on_device);

/* Advances n >= 0 steps of fused pull collide-and-stream (Sec. 2.3.1):
 * f_i(x) = f*_i(x - c_i), with bounce-back from SOLID sources and Ladd's
 * term from WALL sources, then collision on every fluid node, written to the
 * other array.  Asynchronous.  Errors: ARG (n < 0), STATE (MLP closure
 * without weights), CUDA (launch failure). */
lbm_status lbm_step(lbm_ctx *ctx, int n);

/* n >= 1 steps followed by the reduction of lbm_reduce, with the last step
 * computing the reduction partials from the populations it writes, so the
 * new state is not read a second time (the transform-reduce fusion of
 * Sec. 2.2).  Same state as lbm_step(n).  The per-node density and
 * velocity are the ones the last collision used (FP32 storage; lbm_reduce
 * recomputes them from the stored populations, equal up to rounding), or
 * the stored values read back (16-bit storage, as lbm_reduce).  Inside the
 * step every operation is FP32: each block adds its 256 nodes (16-bit
 * storage: 512) by a fixed shuffle tree, about 1e-6 relative on each part;
 * the block partials are then added in FP64 in a fixed order.  FP64
 * storage, lattices stepped on compact storage, the learned closure and
 * pure streaming take the two separate passes (lbm_step, lbm_reduce).
 * The first call allocates 48 bytes of partials per 256 nodes through the
 * context's allocator.  Synchronizes.  Errors: ARG (n < 1), OOM, CUDA,
 * UNSTABLE (as lbm_reduce, *out filled). */
lbm_status lbm_step_reduce(lbm_ctx *ctx, int n, lbm_reduction *out);

/* Enables (default) or disables replaying pairs of steps as CUDA graphs in
 * lbm_step.  With graphs, lbm_step(n >= 4) captures a two-step graph once
 * per kernel path and array orientation (again after lbm_set_params or
 * lbm_set_tags) and replays it on a private stream ordered after and before
 * the context's stream, so results and stream semantics are the same as
 * with one launch per step.  A capture the driver refuses turns graphs off
 * for the context. */
lbm_status lbm_use_graphs(lbm_ctx *ctx, int enable);

/* Number of steps taken since the last initialisation. */
lbm_status lbm_step_count(lbm_ctx *ctx, long long *steps);

/* Density rho[N] and velocity u[3][N] of every node, from the stored
 * post-collision populations (see lbm_reduction).  Solid and wall nodes
 * report 0.  Either pointer may be NULL.  Synchronizes. */
lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *u, int on_device);

/* FP64 domain sums over the fluid nodes (the transform-reduce of Sec. 2.2),
 * deterministic for a given lattice size.  Synchronizes.  Returns
 * LBM_ERR_UNSTABLE, with *out filled, when any fluid node has a non-finite
 * density or velocity. */
lbm_status lbm_reduce(lbm_ctx *ctx, lbm_reduction *out);

/* Waits up to timeout_ms (< 0: no limit) for the context's stream; returns
 * LBM_ERR_TIMEOUT if the work is still running then (the work continues),
 * LBM_ERR_CUDA if it failed. */
lbm_status lbm_sync(lbm_ctx *ctx, int timeout_ms);

/* Unshifted FP64 populations f[Q][N] of the current state (the
 * post-collision set of the last step).  Synchronizes. */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int on_device);

/* Replaces the state by f[Q][N] (unshifted FP64), rounded to the storage
 * type (nearest-even, through FP32 for the 16-bit types), in both arrays.
 * Does not reset the step counter.  Asynchronous for device inputs. */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int on_device);

/* Bit-exact checkpoints (Sec. 2.3.2 mentions checkpointing of serialized
 * data but gives no mechanism).  The FP64 round trip of
 * lbm_get_populations / lbm_set_populations adds and removes the offset w_i,
 * which can round away the smallest stored deviations; these two calls move
 * the stored state itself.
 *
 * lbm_get_state copies the population array byte for byte: the
 * offset-stripped values h_i in the storage type, in the library's padded
 * layout (Q planes of population_bytes / Q bytes each; rows of pitch_x nodes;
 * both from lbm_info).  *layout receives 0 for the local layout, or 1 for the
 * AA pattern's neighbour-shifted layout after an odd number of steps;
 * *steps the step counter (either pointer may be NULL).  bytes must equal
 * lbm_info's population_bytes.  buf is host memory (on_device = 0, pageable
 * is fine) or device memory (1).  Synchronizes.  Errors: ARG (NULL context
 * or buffer, wrong size), CUDA. */
lbm_status lbm_get_state(lbm_ctx *ctx, void *buf, size_t bytes, int *layout, long long *steps, int on_device);

/* Restores a state written by lbm_get_state into a context of the same
 * size, lattice, storage type and pattern (into both arrays with
 * LBM_PATTERN_AB), with its layout word and step counter.  Tags, parameters
 * and closure weights are not part of the state: set them first
 * (lbm_set_tags is refused once layout 1 is restored).  Stepping on then
 * gives, on every fluid node, the same bits as the run that was saved.
 * Synchronizes.  Errors: ARG (NULL context or buffer, wrong size, layout not
 * 0 or 1, layout 1 without the AA pattern, steps < 0), CUDA. */
lbm_status lbm_set_state(lbm_ctx *ctx, const void *buf, size_t bytes, int layout, long long steps, int on_device);

/* Random overlapping spheres as a porous medium: the synthetic stand-in for
 * the Berea sandstone volume of Sec. 3.3.  centres[n][3] (host, integer node
 * coordinates, any value: wrapped periodically) and radii[n] (host, in
 * [0, 1024]) are taken in order; a node is solid when, for some sphere, the
 * squared periodic minimum-image distance to its centre (an integer,
 * compared as a double) is <= r*r.  Spheres are added until the pore
 * fraction is <= target_porosity, checked before each sphere, or the list
 * ends.  Solid nodes get LBM_TAG_SOLID, the others pore_tag (FLUID or
 * FORCED); the tags are then installed as by lbm_set_tags.  *n_used and
 * *porosity (either may be NULL) receive the number of spheres used and the
 * final pore fraction.  Synchronizes.  Errors: ARG, OOM, CUDA. */
lbm_status lbm_geometry_spheres(lbm_ctx *ctx, const int32_t *centres, const double *radii, int n_spheres,
                                double target_porosity, uint8_t pore_tag, int *n_used, double *porosity);

/* Enstrophy average over all N nodes (Sec. 3.1): (1/N) sum |w|^2 / 2 with
 * w = curl u and u from lbm_moments (0 on solid and wall nodes), each
 * derivative the eighth-order centred difference with weights 4/5, -1/5,
 * 4/105, -1/280, periodic in every direction.  Arithmetic in FP64 for FP64
 * storage, FP32 otherwise, accumulated in FP64.  Synchronizes. */
lbm_status lbm_enstrophy(lbm_ctx *ctx, double *out);

/* ---------------------------------------------------------------------------
 * Learned relaxation-time closure (no counterpart in the paper; an addition
 * of this library).  Per fluid node, with Pi^neq the non-equilibrium stress
 * sum_i c_i c_i (f_i - f_eq_i) of the pulled populations:
 *   x   = (Pi_xx, Pi_yy, Pi_zz, Pi_xy, Pi_xz, Pi_yz, rho), normalised as
 *         (x - mean) / std,
 *   y   = w3 . SiLU(W2 SiLU(W1 x_n + b1) + b2) + b3,
 *   tau_eff = tau + out_scale * softplus(y).
 * Normalised inputs, W1, the first activations and W2 are rounded to BF16
 * (nearest even) and multiplied on the tensor cores with FP32 accumulation;
 * biases, the second activations and the last layer are FP32.
 * params[LBM_MLP_NPARAM] = W1[32][7], b1[32], W2[32][32], b2[32], w3[32], b3;
 * norm[LBM_MLP_NNORM]    = mean[7], std[7] (> 0), out_scale (>= 0), unused.
 * ------------------------------------------------------------------------- */
#define LBM_MLP_NPARAM 1345
#define LBM_MLP_NNORM 16

/* Installs the closure weights used by LBM_CLOSURE_MLP (copied; host or
 * device pointers).  Synchronizes.  Errors: ARG (non-finite value, std <= 0,
 * out_scale < 0), OOM, CUDA.  lbm_step with LBM_CLOSURE_MLP and no weights
 * returns LBM_ERR_STATE. */
lbm_status lbm_set_closure_weights(lbm_ctx *ctx, const float *params, const float *norm, int on_device);

/* The closure's inputs for the step that would follow the current state,
 * computed as that step computes them (pull with the boundary rules, in the
 * context's streaming pattern): x[n][7] = (Pi^neq xx, yy, zz, xy, xz, yz,
 * rho) of node n = x + nx (y + ny z), FP32, zeros on solid and wall nodes.
 * The state is not changed.  Training on these a-posteriori features pairs
 * the network with the inputs the solver really produces.  x is caller-owned
 * host memory (N * 7 floats) or device memory (on_device).  Synchronizes.
 * Errors: ARG, OOM, CUDA. */
lbm_status lbm_closure_features(lbm_ctx *ctx, float *x, int on_device);

/* dtau[n] for features x[n][7], batch inference on the 5th-generation
 * tensor cores (tcgen05: 128 samples per MMA tile, FP32 accumulators in
 * tensor memory), with the same BF16 roundings as the collide kernel's warp
 * tile (the FP32 accumulation order may differ).  All pointers are device
 * memory; asynchronous on stream.  A tile whose completion wait runs out
 * leaves NaN in its 128 outputs.  Errors: ARG, CUDA (launch). */
lbm_status lbm_mlp_forward(const float *params, const float *norm, const float *x, int n, float *dtau, void *stream);

/* Bytes of device workspace lbm_mlp_loss_grad needs for n samples. */
size_t lbm_mlp_workspace_bytes(int n);

/* Mean squared error L = (1/n) sum (dtau - target)^2 of the closure on n
 * samples and its gradient grad[LBM_MLP_NPARAM] with respect to params,
 * through the same BF16 roundings as the forward pass (treated as identities
 * for the gradient).  Deterministic: per-block sums over fixed sample sets,
 * added in block order.  All pointers are device memory; loss may be NULL.
 * Asynchronous.  Errors: ARG (n < 1, workspace too small), CUDA. */
lbm_status lbm_mlp_loss_grad(const float *params, const float *norm, const float *x, const float *target, int n,
                             float *grad, float *loss, void *workspace, size_t workspace_bytes, void *stream);

/* One Adam step (Kingma & Ba) on n_params FP32 master weights, step number
 * t >= 1: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * params -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).  Device
 * pointers; asynchronous.  Errors: ARG, CUDA. */
lbm_status lbm_mlp_adam(float *params, float *m, float *v, const float *grad, int n_params, int t, float lr,
                        float beta1, float beta2, float eps, void *stream);

/* Training samples from a fine field (rho[N], u[3][N], device FP64, unpadded
 * x-fastest, periodic): for every coarse cell of a box filter of width
 * factor, the features x[Nc][7] = (-(2/3) rho_bar tau0 S_bar, rho_bar)
 * (Chapman-Enskog estimate of Pi^neq from the filtered strain S_bar, which
 * uses second-order central differences of the filtered velocity on the
 * coarse grid) and the target dtau* = 3 max(0, -tau_dev : S_bar /
 * (2 S_bar : S_bar)) with the subgrid stress tau = mean(u u) - mean(u)
 * mean(u).  Coarse cells in x-fastest order.  Asynchronous.  Errors: ARG
 * (sizes not multiples of factor, tau0 <= 1/2), CUDA. */
lbm_status lbm_coarse_samples(const double *rho, const double *u, int nx, int ny, int nz, int factor, double tau0,
                              float *x, float *target, void *stream);

/* Box filter of ncomp fields in[ncomp][N] (device FP64, unpadded, x-fastest)
 * into out[ncomp][Nc]: the mean over each factor^3 block of nodes, coarse
 * cells in x-fastest order.  Asynchronous.  Errors: ARG, CUDA. */
lbm_status lbm_box_filter(const double *in, int ncomp, int nx, int ny, int nz, int factor, double *out, void *stream);

/* Measurement helper (no counterpart in the paper): the FP64 arithmetic rate
 * of the current device in operations per second (a fused multiply-add
 * counts as two), timed with CUDA events over one launch of independent FP64
 * FMA chains on every SM after a warm-up launch.  It is the arithmetic roof
 * of the step on LBM_F64 storage, whose collision runs in FP64 (on this
 * device's FP64 rate that step is bound by arithmetic, not by memory).
 * stream: cudaStream_t (NULL: legacy default stream).  Allocates and frees
 * a few kilobytes of device memory; synchronizes.  Errors: ARG (NULL
 * output), CUDA. */
lbm_status lbm_fp64_fma_rate(void *stream, double *flops);

/* Library-side sizes: bytes of one population array, x pitch in nodes,
 * number of populations.  Any pointer may be NULL. */
lbm_status lbm_info(lbm_ctx *ctx, size_t *population_bytes, int *pitch_x, int *q);

/* Largest lattice lbm_reduce_noalloc accepts: 2^31 - 257 nodes, the bound
 * lbm_create puts on padded lattices.  The reduction walks node offsets in
 * 32-bit integers, each thread stepping by its block's 256 threads, so the
 * last offset a thread forms is below N + 256 and stays representable. */
#define LBM_NOALLOC_MAX_NODES 2147483391LL

/* Domain reduction that allocates no memory (the paper has no counterpart;
 * it exists for callers that cannot allocate device memory: a host code that
 * owns the whole GPU through its own memory pool and forbids other
 * allocations, such as an analysis plug-in inside another solver, or a time
 * loop that cannot afford the device synchronisation of cudaMalloc).
 *
 * Computes the same sums as lbm_reduce, without a context, over populations
 * the caller already holds on the device:
 *  h       device array of offset-stripped populations h_i = f_i - w_i in the
 *          storage type of dtype (LBM_F16_SCALED: h_i * 2^12), layout
 *          [Q][nz][ny][nx] (x fastest, no padding, plane stride nx*ny*nz);
 *  tags    device array of nx*ny*nz tags (values < LBM_NTAGS), or NULL for
 *          all fluid;
 *  params  only params->force is read (for FORCED nodes); may be NULL;
 *  stream  cudaStream_t to run on (NULL: legacy default stream);
 *  out     host struct, filled on LBM_OK and on LBM_ERR_UNSTABLE.
 * Scratch: the per-block partials live in a file-scope device array of
 * 116,832 bytes (1,217 x 12 doubles) that every GPU loading the library holds
 * until exit; calls never call cudaMalloc, cudaFree or any allocating
 * routine.  The first successful call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it; a failed lookup is not kept,
 * so a later call retries it.  That first call should come before any stream
 * capture.  All calls share the
 * array: calls that overlap on the GPU race and must be serialised by the
 * caller.  Synchronizes the stream.  Errors: ARG (NULL pointer, bad enum,
 * a size < 1, more than LBM_NOALLOC_MAX_NODES nodes), CUDA, UNSTABLE. */
lbm_status lbm_reduce_noalloc(const void *h, lbm_lattice lattice, lbm_dtype dtype, int nx, int ny, int nz,
                              const uint8_t *tags, const lbm_params *params, void *stream, lbm_reduction *out);

/* Text of the last failure of ctx (or of a call without a context, for
 * ctx == NULL).  Never NULL; valid until the next call on the same ctx. */
const char *lbm_last_error(const lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
