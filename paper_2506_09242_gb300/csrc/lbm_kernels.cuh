// lbm_kernels.cuh -- kernel templates of the hot path, instantiated once per
// storage type by lbm_store_*.cu.
//
// Layout in HBM: two population arrays A and B of Q planes each, plane i
// holding h_i = f_i - w_i of every node at offset (z*ny + y)*px + x (x
// fastest, px = nx rounded up to 32); a byte of tag per node in the same
// padded order.  One thread owns one node.
#pragma once

#include "lbm_internal.cuh"
#include "lbm_mlp.cuh"

namespace lbm {

constexpr int kStepThreads = 128;

// Host-side conversion of the parameters to the compute type.
template <typename T> inline KParams<T> make_kparams(int Q, const lbm_params &p)
{
    (void)Q;
    KParams<T> k;
    k.tau = (T)p.tau;
    k.omega = (T)(1.0 / p.tau);
    k.omega_minus = p.trt_magic > 0.0 ? (T)(1.0 / (0.5 + p.trt_magic / (p.tau - 0.5))) : k.omega;
    for (int a = 0; a < 3; ++a) k.force[a] = (T)p.force[a];
    k.smag18 = (T)(18.0 * p.cs_smag * p.cs_smag);
    k.wall_local = p.wall_rho_local != 0;
    const double rw = k.wall_local ? 1.0 : p.rho_wall;
    for (int w = 0; w < LBM_NWALLS; ++w)
        for (int a = 0; a < 3; ++a) k.wall6[w][a] = (T)(6.0 * rw * p.wall_u[w][a]);
    return k;
}

// Neighbour bookkeeping of one node: the three x positions and nine row
// offsets (z, y) of its periodic 3x3x3 neighbourhood.
struct Nbr {
    int xs[3];      // x-1, x, x+1 (wrapped)
    int row[3][3];  // row[dy+1][dz+1] = ((z+dz)*ny + (y+dy)) * px (wrapped)
    int self;
    __device__ __forceinline__ void init(const Grid &g, int x, int y, int z)
    {
        xs[0] = x == 0 ? g.nx - 1 : x - 1;
        xs[1] = x;
        xs[2] = x == g.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
        const int ys[3] = {ym, y, yp};
        const int zs[3] = {zm, z, zp};
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) row[a][b] = (zs[b] * g.ny + ys[a]) * g.px;
        self = row[1][1] + x;
    }
    // Offset of the node x - c_i (the pull source of direction i).
    __device__ __forceinline__ int src(int i) const
    {
        return row[1 - cvel(i, 1)][1 - cvel(i, 2)] + xs[1 - cvel(i, 0)];
    }
    // Offset of the node x + c_i (where direction i streams to).
    __device__ __forceinline__ int dst(int i) const { return src(opp(i)); }
};

// ---------------------------------------------------------------------------
// Streaming patterns.  AB (two arrays): a step pulls from A and writes B at
// the node.  AA (one array F, updated in place; Bailey et al. 2009): steps
// alternate between
//   odd:  h_i = F[opp(i)][x - c_i]  and  f*_i -> F[i][x + c_i],
//   even: h_i = F[i][x]             and  f*_i -> F[opp(i)][x],
// so within a step every location is read and then written by one thread
// only.  Between steps F holds the state f*(x) in one of two layouts:
//   S (after initialisation, set_populations and even steps):
//       F[opp(i)][x] = f*_i(x);
//   P (after odd steps): F[i][x + c_i] = f*_i(x), except where x + c_i is a
//       SOLID or WALL node: there the link's bounce-back is kept in place,
//       F[opp(i)][x] = f*_i(x), and the next even step adds the moving-wall
//       term to it.
// In both layouts F[.][x] belongs to node x alone, so node-by-node copies
// (the compact fluid-only hand-over) keep the layout.
// ---------------------------------------------------------------------------
enum : int { kPatAB = 0, kPatAAOdd = 1, kPatAAEven = 2 };
enum : int { kLayAB = 0, kLayS = 1, kLayP = 2 };

// Step pattern / read layout of a launch.
inline int step_pattern(bool aa, bool layout_p) { return !aa ? kPatAB : layout_p ? kPatAAEven : kPatAAOdd; }
inline int read_layout(bool aa, bool layout_p) { return !aa ? kLayAB : layout_p ? kLayP : kLayS; }

// A population load of a step: the read-only path for AB (A is never
// written by the launch), a coherent load for AA, where the same thread
// later writes the location (through the same pointer).
template <typename S, int PAT> __device__ __forceinline__ typename Store<S>::T pop_ld(const S *p)
{
    if constexpr (PAT == kPatAB)
        return Store<S>::ld(p);
    else
        return Store<S>::ldc(p);
}

// Offset of the value a step reads for direction i from a non-wall source.
template <int PAT>
__device__ __forceinline__ long long step_load_off(int i, const Grid &g, const Nbr &nb)
{
    if (PAT == kPatAB) return (long long)i * g.sN + nb.src(i);
    if (PAT == kPatAAOdd) return (long long)opp(i) * g.sN + nb.src(i);
    return (long long)i * g.sN + nb.self;
}

// Offset a step writes f*_i to; wall: bit j set when the source of direction
// j is a SOLID or WALL node (only the odd AA step looks at it).
template <int PAT>
__device__ __forceinline__ long long step_store_off(int i, const Grid &g, const Nbr &nb, uint32_t wall)
{
    if (PAT == kPatAB) return (long long)i * g.sN + nb.self;
    if (PAT == kPatAAEven) return (long long)opp(i) * g.sN + nb.self;
    return ((wall >> opp(i)) & 1u) ? (long long)opp(i) * g.sN + nb.self : (long long)i * g.sN + nb.dst(i);
}

// ---------------------------------------------------------------------------
// Reduction helpers (FP64 sums over fluid nodes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction of kRedSlots values (slot 9 is a max, the rest sums)
// for blocks of up to 256 threads; thread 0 ends with the result in acc.
// Every thread of the block must call it.
__device__ __forceinline__ void block_reduce_slots(double (&acc)[kRedSlots])
{
    __shared__ double sm[kRedThreads / 32][kRedSlots];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) / 32;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) acc[k] = (k == 9) ? warp_max(acc[k]) : warp_sum(acc[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) sm[warp][k] = acc[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) {
            const double v = lane < nwarps ? sm[lane][k] : 0.0;
            acc[k] = (k == 9) ? warp_max(v) : warp_sum(v);
        }
    }
}

// Per-thread accumulator of the reduction: plain FP64 for FP64 compute; for
// FP32 compute a double-float pair (hi + lo) updated with Knuth's TwoSum,
// which keeps about 44 significant bits while staying off the FP64 pipe
// (GB300 has a low FP64 rate); partials are combined in FP64.
template <typename T> struct Acc {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double get() const { return v; }
};
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float s = hi + x;
        const float bp = s - hi;
        const float e = (hi - (s - bp)) + (x - bp);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// The sums of one thread's fluid nodes, in the slot order of the reduction.
template <typename T> struct RedAcc {
    Acc<T> dm, m[3], v[3], ke, ker;
    T usq_max = T(0);
    unsigned n_fluid = 0, n_bad = 0;
    __device__ __forceinline__ void add(T d, const T (&u)[3])
    {
        const T rho = T(1) + d;
        const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        ++n_fluid;
        if (!isfinite(rho) || !isfinite(usq)) {
            ++n_bad;
            return;
        }
        dm.add(d);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            m[k].add(rho * u[k]);
            v[k].add(u[k]);
        }
        ke.add(T(0.5) * usq);
        ker.add(T(0.5) * rho * usq);
        usq_max = usq > usq_max ? usq : usq_max;
    }
    __device__ __forceinline__ void slots(double (&acc)[kRedSlots]) const
    {
        acc[0] = dm.get();
        for (int k = 0; k < 3; ++k) {
            acc[1 + k] = m[k].get();
            acc[4 + k] = v[k].get();
        }
        acc[7] = ke.get();
        acc[8] = ker.get();
        acc[9] = sqrt((double)usq_max);
        acc[10] = (double)n_fluid;
        acc[11] = (double)n_bad;
    }
};

// Additions and multiplications rounded once each, never contracted.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Density deviation and velocity of one node from its post-collision set as
// it is stored (rounded to the storage type), the same quantities
// node_moments reads back from memory.
template <int Q, typename S>
__device__ __forceinline__ void stored_moments(const typename Store<S>::T (&h)[Q], bool forced,
                                               const KParams<typename Store<S>::T> &p, typename Store<S>::T &drho,
                                               typename Store<S>::T (&u)[3])
{
    // Roundings spelled out as in NodeSums::add.
    using T = typename Store<S>::T;
    T d = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T v = Store<S>::rt(h[i]);
        d = add_rn(d, v);
        if (cvel(i, 0)) jx = add_rn(jx, cvel(i, 0) > 0 ? v : -v);
        if (cvel(i, 1)) jy = add_rn(jy, cvel(i, 1) > 0 ? v : -v);
        if (cvel(i, 2)) jz = add_rn(jz, cvel(i, 2) > 0 ? v : -v);
    }
    const T rho = add_rn(T(1), d);
    if (forced) {
        const T hr = mul_rn(T(-0.5), rho);
        jx = fma(hr, p.force[0], jx);
        jy = fma(hr, p.force[1], jy);
        jz = fma(hr, p.force[2], jz);
    }
    const T inv = T(1) / rho;
    drho = d;
    u[0] = mul_rn(jx, inv);
    u[1] = mul_rn(jy, inv);
    u[2] = mul_rn(jz, inv);
}

// Reduction slots of the nodes one thread owns inside a fused step, in FP32.
// GB300 runs FP64 at 1/64 of the FP32 rate, so a step kernel that did even
// a few dozen FP64 operations per block of 256 nodes would be bound by them;
// here every per-node and per-block operation is FP32, and the block partials
// are added in FP64 by a separate pass over the (small) partial buffer.
struct NodeSums {
    float s[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dmass, mom[3], vel[3], ke, ke_rho
    float usq_max = 0.f;
    unsigned n_fluid = 0, n_bad = 0;
    // Every rounding is spelled out (fused multiply-adds and _rn operations,
    // which the compiler never contracts or splits), so that each kernel
    // that inlines this sums a node with the same bits.
    __device__ __forceinline__ void add(float d, const float (&u)[3])
    {
        const float rho = __fadd_rn(1.f, d);
        const float usq = fmaf(u[2], u[2], fmaf(u[1], u[1], __fmul_rn(u[0], u[0])));
        ++n_fluid;
        if (!isfinite(rho) || !isfinite(usq)) {
            ++n_bad;
            return;
        }
        s[0] = __fadd_rn(s[0], d);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s[1 + k] = fmaf(rho, u[k], s[1 + k]);
            s[4 + k] = __fadd_rn(s[4 + k], u[k]);
        }
        s[7] = fmaf(0.5f, usq, s[7]);
        s[8] = fmaf(__fmul_rn(0.5f, rho), usq, s[8]);
        usq_max = fmaxf(usq_max, usq);
    }
};

// Writes the block's kRedSlots partial (slot 9 = max |u|^2, rooted in FP64
// when the partials are combined) to out[0..kRedSlots).  Lanes are added by a shuffle tree, warps in a fixed
// order by one thread each slot, so the result does not depend on
// scheduling.  Every thread of the block must call it (no early returns).
__device__ __forceinline__ void block_partial_f32(const NodeSums &ns, float *__restrict__ out)
{
    __shared__ float wsum[kStepThreads / 32][kRedSlots];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5, nwarps = (blockDim.x * blockDim.y + 31) / 32;
    float v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = ns.s[k];
    float mx = ns.usq_max;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const unsigned nf = __reduce_add_sync(0xffffffffu, ns.n_fluid);
    const unsigned nb = __reduce_add_sync(0xffffffffu, ns.n_bad);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) wsum[warp][k] = v[k];
        wsum[warp][9] = mx;
        wsum[warp][10] = (float)nf;  // at most 2 x kStepThreads: exact
        wsum[warp][11] = (float)nb;
    }
    __syncthreads();
    if (tid < kRedSlots) {
        float a = wsum[0][tid];
        for (int w = 1; w < nwarps; ++w) a = (tid == 9) ? fmaxf(a, wsum[w][tid]) : a + wsum[w][tid];
        out[tid] = a;
    }
}

__device__ __forceinline__ long long linear_block() { return blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z); }

// ---------------------------------------------------------------------------
// Boundary rules for one fluid node next to a wall (tag bit kNearWall):
// halfway bounce-back from a SOLID source, h_i(x) = h*_opp(i)(x); Ladd's
// moving-wall term from a WALL_k source, + 6 w_i rho_wall (c_i . u_wall_k).
// Where the bounced value sits depends on the pattern: AB reads it from
// A[opp(i)][x], the odd AA step from F[i][x] (layout S), and the even AA step
// has already read it from F[i][x] (layout P) and only adds the wall term.
// Returns the links with a SOLID or WALL source (bit i).  With the
// local-density wall (p.wall_local) the wall terms are added after all links
// are bounced, scaled by the node's density rho0 / (1 - s).
// ---------------------------------------------------------------------------
// c_i . v with only the non-zero terms of c_i (components are 0 or +-1).
// Written as T(c_x) v_x + T(c_y) v_y + T(c_z) v_z, IEEE semantics would keep
// every 0 * v_a as a real operation; here the branches fold at compile time
// once i is a constant of an unrolled loop.
template <typename T> __device__ __forceinline__ T cdot(int i, T vx, T vy, T vz)
{
    const int cx = cvel(i, 0), cy = cvel(i, 1), cz = cvel(i, 2);
    T r;
    if (cx) {
        r = cx > 0 ? vx : -vx;
        if (cy) r = cy > 0 ? r + vy : r - vy;
        if (cz) r = cz > 0 ? r + vz : r - vz;
    } else if (cy) {
        r = cy > 0 ? vy : -vy;
        if (cz) r = cz > 0 ? r + vz : r - vz;
    } else if (cz) {
        r = cz > 0 ? vz : -vz;
    } else {
        r = T(0);
    }
    return r;
}

// Ladd's moving-wall term 6 w_i rho_wall (c_i . u_wall) of the wall whose tag
// is ts (without rho_wall for the local-density wall).
template <int Q, typename T>
__device__ __forceinline__ T wall_term(int i, unsigned ts, const KParams<T> &p)
{
    // select the wall's velocity without indexing the parameter block
    // dynamically (which would copy it to local memory)
    T ux = T(0), uy = T(0), uz = T(0);
#pragma unroll
    for (int k = 0; k < LBM_NWALLS; ++k)
        if (ts == (unsigned)(LBM_TAG_WALL0 + k)) {
            ux = p.wall6[k][0];
            uy = p.wall6[k][1];
            uz = p.wall6[k][2];
        }
    return wgt<T>(Q, i) * cdot<T>(i, ux, uy, uz);
}

// The local wall density: rho0 / (1 - s), rho0 = 1 + sum h (plain bounce-back).
template <int Q, typename T> __device__ __forceinline__ T local_wall_rho(const T (&h)[Q], T s)
{
    T r0 = T(1);
#pragma unroll
    for (int i = 0; i < Q; ++i) r0 += h[i];
    return r0 / (T(1) - s);
}

// LOCAL: the kernel supports the local-density wall (p.wall_local); the
// 16-bit two-node kernel is built without it (the second pass over the
// links costs that kernel about 20 registers) and is not used when it is on.
template <int Q, typename S, int PAT = kPatAB, bool LOCAL = true>
__device__ __forceinline__ uint32_t apply_walls(typename Store<S>::T (&h)[Q], const S *__restrict__ A,
                                                const uint8_t *__restrict__ tags, const Grid &g, const Nbr &nb,
                                                const KParams<typename Store<S>::T> &p)
{
    using T = typename Store<S>::T;
    uint32_t wall = 0;
    T s = T(0);
    bool moving = false;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const unsigned ts = tags[nb.src(i)] & kTagMask;
        if (is_wall_tag(ts)) {
            wall |= 1u << i;
            T v = PAT == kPatAB      ? pop_ld<S, PAT>(A + (long long)opp(i) * g.sN + nb.self)
                  : PAT == kPatAAOdd ? pop_ld<S, PAT>(A + (long long)i * g.sN + nb.self)
                                     : h[i];
            if (ts >= LBM_TAG_WALL0) {
                const T term = wall_term<Q, T>(i, ts, p);
                if (LOCAL && p.wall_local) {
                    s += term;
                    moving = true;
                } else {
                    v += term;
                }
            }
            h[i] = v;
        }
    }
    if (LOCAL && p.wall_local && moving) {
        const T rw = local_wall_rho<Q, T>(h, s);
#pragma unroll
        for (int i = 1; i < Q; ++i)
            if ((wall >> i) & 1u) {
                const unsigned ts = tags[nb.src(i)] & kTagMask;
                if (ts >= LBM_TAG_WALL0) h[i] = fma(rw, wall_term<Q, T>(i, ts, p), h[i]);
            }
    }
    return wall;
}

// ---------------------------------------------------------------------------
// Collision of one node's pulled set (in place), Sec. 3.1 BGK with the
// second-order weighted equilibrium on offset-stripped values, optional Guo
// body force, and the Smagorinsky closure; split into the macroscopic
// moments, the non-equilibrium stress and the relaxation so that the learned
// closure can run between them.
// ---------------------------------------------------------------------------
// sum_i c_ia h_i over the directions with c_ia != 0, in index order, started
// from the first term (no addition of zero).
template <int Q, typename T, int AX> __device__ __forceinline__ T csum(const T (&h)[Q])
{
    T r = T(0);
    bool first = true;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (cvel(i, AX)) {
            const T v = cvel(i, AX) > 0 ? h[i] : -h[i];
            r = first ? v : r + v;
            first = false;
        }
    return r;
}

template <typename T> struct Macro {
    T drho, rho, inv, ux, uy, uz, Gx, Gy, Gz;
};

// rho = 1 + sum h, j = sum c h (+ rho g / 2 on a forced node), u = j / rho;
// every sum starts from its first term (no addition of zero).
template <int Q, typename T>
__device__ __forceinline__ Macro<T> node_macros(const T (&h)[Q], bool forced, const KParams<T> &p)
{
    Macro<T> m;
    T drho = h[0];
    T jx = csum<Q, T, 0>(h), jy = csum<Q, T, 1>(h), jz = csum<Q, T, 2>(h);
#pragma unroll
    for (int i = 1; i < Q; ++i) drho += h[i];
    m.drho = drho;
    m.rho = T(1) + drho;
    m.Gx = m.Gy = m.Gz = T(0);
    if (forced) {
        m.Gx = mul_rn(m.rho, p.force[0]);
        m.Gy = mul_rn(m.rho, p.force[1]);
        m.Gz = mul_rn(m.rho, p.force[2]);
        jx = fma(T(0.5), m.Gx, jx);
        jy = fma(T(0.5), m.Gy, jy);
        jz = fma(T(0.5), m.Gz, jz);
    }
    m.inv = T(1) / m.rho;
    m.ux = mul_rn(jx, m.inv);
    m.uy = mul_rn(jy, m.inv);
    m.uz = mul_rn(jz, m.inv);
    return m;
}

// Pi^neq_ab = sum c_a c_b (f - f_eq) = sum c_a c_b h - rho u_a u_b
//             - (drho / 3) delta_ab   (closed-form equilibrium moments);
// order xx, yy, zz, xy, xz, yz.
template <int Q, typename T>
__device__ __forceinline__ void pi_neq(const T (&h)[Q], const Macro<T> &m, T (&pi)[6])
{
    // second moments, each started from its first term (no addition of zero)
    T sxx = T(0), syy = T(0), szz = T(0), sxy = T(0), sxz = T(0), syz = T(0);
    bool fxx = true, fyy = true, fzz = true, fxy = true, fxz = true, fyz = true;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int cx = cvel(i, 0), cy = cvel(i, 1), cz = cvel(i, 2);
        if (cx) { sxx = fxx ? h[i] : sxx + h[i]; fxx = false; }
        if (cy) { syy = fyy ? h[i] : syy + h[i]; fyy = false; }
        if (cz) { szz = fzz ? h[i] : szz + h[i]; fzz = false; }
        if (cx * cy) { const T v = cx * cy > 0 ? h[i] : -h[i]; sxy = fxy ? v : sxy + v; fxy = false; }
        if (cx * cz) { const T v = cx * cz > 0 ? h[i] : -h[i]; sxz = fxz ? v : sxz + v; fxz = false; }
        if (cy * cz) { const T v = cy * cz > 0 ? h[i] : -h[i]; syz = fyz ? v : syz + v; fyz = false; }
    }
    const T third = T(1) / T(3);
    const T rx = mul_rn(m.rho, m.ux), ry = mul_rn(m.rho, m.uy);
    pi[0] = fma(-m.drho, third, fma(-rx, m.ux, sxx));
    pi[1] = fma(-m.drho, third, fma(-ry, m.uy, syy));
    pi[2] = fma(-m.drho, third, fma(-mul_rn(m.rho, m.uz), m.uz, szz));
    pi[3] = fma(-rx, m.uy, sxy);
    pi[4] = fma(-rx, m.uz, sxz);
    pi[5] = fma(-ry, m.uz, syz);
}

// h_i <- h_i + omega (h_eq_i - h_i) + (1 - omega / 2) F_i, the rest
// population first, then each pair of opposite directions (i, i + 1): their
// equilibria h_eq = S +- A share the even part S = w (drho + rho (4.5 (c.u)^2
// - 1.5 u^2)) and differ in the sign of the odd part A = 3 w rho (c.u), and
// Guo's source F = w [3 (c - u) + 9 (c.u) c] . G splits the same way.
template <int Q, typename T>
__device__ __forceinline__ void relax(T (&h)[Q], const Macro<T> &m, T omega, bool forced)
{
    const T usq15 = mul_rn(T(1.5), fma(m.uz, m.uz, fma(m.uy, m.uy, mul_rn(m.ux, m.ux))));
    const T cf = fma(T(-0.5), omega, T(1));
    const T uG = fma(m.uz, m.Gz, fma(m.uy, m.Gy, mul_rn(m.ux, m.Gx)));
    {
        const T w0 = wgt<T>(Q, 0);
        T h0 = fma(omega, fma(w0, fma(-m.rho, usq15, m.drho), -h[0]), h[0]);
        if (forced) h0 = fma(cf, mul_rn(w0, mul_rn(T(-3), uG)), h0);
        h[0] = h0;
    }
    const T r3 = mul_rn(T(3), m.rho);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const T cu = cdot<T>(i, m.ux, m.uy, m.uz);
        const T w = wgt<T>(Q, i);
        const T X = fma(m.rho, fma(mul_rn(T(4.5), cu), cu, -usq15), m.drho);  // S = w X
        const T A = mul_rn(mul_rn(w, r3), cu);
        T hi = fma(omega, add_rn(fma(w, X, A), -h[i]), h[i]);
        T ho = fma(omega, add_rn(fma(w, X, -A), -h[i + 1]), h[i + 1]);
        if (forced) {
            const T cG = cdot<T>(i, m.Gx, m.Gy, m.Gz);
            const T Y = fma(mul_rn(T(9), cu), cG, mul_rn(T(-3), uG));  // Fs = w Y
            const T Fa = mul_rn(mul_rn(T(3), w), cG);
            hi = fma(cf, fma(w, Y, Fa), hi);
            ho = fma(cf, fma(w, Y, -Fa), ho);
        }
        h[i] = hi;
        h[i + 1] = ho;
    }
}

// TRT (Ginzburg): the parts of h, h_eq and the Guo source that are even and
// odd under i -> opp(i) relax with omega and omega_minus.  With
// h_eq_i = S + A and h_eq_opp(i) = S - A, S = w (drho + rho (4.5 (c.u)^2 -
// 1.5 u^2)), A = 3 w rho (c.u), and the source split the same way.
template <int Q, typename T>
__device__ __forceinline__ void relax_trt(T (&h)[Q], const Macro<T> &m, T wp, T wm, bool forced)
{
    const T usq15 = mul_rn(T(1.5), fma(m.uz, m.uz, fma(m.uy, m.uy, mul_rn(m.ux, m.ux))));
    const T cfp = fma(T(-0.5), wp, T(1)), cfm = fma(T(-0.5), wm, T(1));
    const T uG = fma(m.uz, m.Gz, fma(m.uy, m.Gy, mul_rn(m.ux, m.Gx)));
    {
        const T w0 = wgt<T>(Q, 0);
        T h0 = fma(-wp, fma(-w0, fma(-m.rho, usq15, m.drho), h[0]), h[0]);
        if (forced) h0 = fma(mul_rn(cfp, w0), mul_rn(T(-3), uG), h0);
        h[0] = h0;
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const T cu = cdot<T>(i, m.ux, m.uy, m.uz);
        const T w = wgt<T>(Q, i);
        const T X = fma(m.rho, fma(mul_rn(T(4.5), cu), cu, -usq15), m.drho);  // S = w X
        const T A = mul_rn(mul_rn(mul_rn(T(3), w), m.rho), cu);
        const T P = fma(-w, X, mul_rn(T(0.5), add_rn(h[i], h[i + 1])));  // even part minus S
        const T M = fma(T(0.5), add_rn(h[i], -h[i + 1]), -A);           // odd part minus A
        T hi = fma(-wm, M, fma(-wp, P, h[i])), ho = fma(wm, M, fma(-wp, P, h[i + 1]));
        if (forced) {
            const T cG = cdot<T>(i, m.Gx, m.Gy, m.Gz);
            const T Fs = mul_rn(w, fma(mul_rn(T(9), cu), cG, mul_rn(T(-3), uG)));
            const T Fa = mul_rn(mul_rn(T(3), w), cG);
            hi = fma(cfp, Fs, fma(cfm, Fa, hi));
            ho = fma(cfp, Fs, fma(-cfm, Fa, ho));
        }
        h[i] = hi;
        h[i + 1] = ho;
    }
}

// Returns the density and velocity the collision used (mass and momentum
// invariants of the new state).  Every step kernel collides with this
// function, so the same pulled set gives the same bits in all of them: the
// collision's arithmetic (node_macros, pi_neq, relax, relax_trt and the
// Smagorinsky time) spells out each rounding as fma, add_rn or mul_rn,
// because ptxas may contract a plain multiply and add into an FMA in one
// kernel and not in another.
template <int Q, typename T, int CLOSURE>
__device__ __forceinline__ Macro<T> collide_node(T (&h)[Q], bool forced, const KParams<T> &p)
{
    if (CLOSURE == LBM_CLOSURE_STREAM_ONLY) return Macro<T>{};
    const Macro<T> m = node_macros<Q, T>(h, forced, p);
    if (CLOSURE == LBM_CLOSURE_TRT) {
        relax_trt<Q, T>(h, m, p.omega, p.omega_minus, forced);
        return m;
    }
    T omega = p.omega;
    if (CLOSURE == LBM_CLOSURE_SMAGORINSKY) {
        T pi[6];
        pi_neq<Q, T>(h, m, pi);
        const T diag = fma(pi[2], pi[2], fma(pi[1], pi[1], mul_rn(pi[0], pi[0])));
        const T offd = fma(pi[5], pi[5], fma(pi[4], pi[4], mul_rn(pi[3], pi[3])));
        const T pp = fma(T(2), offd, diag);
        const T te = mul_rn(T(0.5), add_rn(p.tau, sqrt(fma(p.tau, p.tau, mul_rn(mul_rn(p.smag18, sqrt(mul_rn(T(2), pp))), m.inv)))));
        omega = T(1) / te;
    }
    relax<Q, T>(h, m, omega, forced);
    return m;
}

// The work of one node (x, y, z): pull, boundary rules, collision, store.
// Solid and wall nodes are never updated.  With REDUCE (FP32 compute only)
// the node's density deviation and velocity are added to ns: the values the
// collision used where the storage is FP32 (mass and momentum are collision
// invariants), otherwise recomputed from the post-collision set rounded to
// the storage type, which is what a later pass over memory would read.
template <int Q, typename S, bool GENERAL, int CLOSURE, bool REDUCE, int PAT>
__device__ __forceinline__ void collide_stream_node(const S *__restrict__ A, S *__restrict__ B,
                                                    const uint8_t *__restrict__ tags, const Grid &g,
                                                    const KParams<typename Store<S>::T> &p, int x, int y, int z,
                                                    NodeSums &ns)
{
    using T = typename Store<S>::T;
    using St = Store<S>;
    Nbr nb;
    nb.init(g, x, y, z);
    unsigned t = 0;
    if (GENERAL) {
        t = tags[nb.self];
        if (PAT == kPatAB && is_wall_tag(t & kTagMask)) return;
    }

    // Pull: h_i(x) = h*_i(x - c_i).  AA reads through B, the pointer the
    // launch writes, so same-address loads and stores keep program order.
    // The AA steps issue the loads together with the tag's, before it is
    // known whether the node is a wall (a wall node's AA sources are its own
    // slots, which nothing else writes, and it discards what it read): on a
    // 256^3 cavity 0.763 -> 0.788 of the roofline.  A/B keeps the early
    // return, which measured faster there (0.828 against 0.770: loading
    // first costs it 8 registers).
    const S *F = PAT == kPatAB ? A : B;
    T h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = pop_ld<S, PAT>(F + step_load_off<PAT>(i, g, nb));
    if (GENERAL && PAT != kPatAB && is_wall_tag(t & kTagMask)) return;
    uint32_t wall = 0;
    if (GENERAL && (t & kNearWall)) wall = apply_walls<Q, S, PAT>(h, F, tags, g, nb, p);

    const bool forced = GENERAL && (t & kTagMask) == LBM_TAG_FORCED;
    const Macro<T> m = collide_node<Q, T, CLOSURE>(h, forced, p);
    if constexpr (REDUCE) {
        static_assert(sizeof(T) == 4, "fused reductions are FP32-compute only");
        if constexpr (sizeof(S) == sizeof(T)) {
            const float u[3] = {m.ux, m.uy, m.uz};
            ns.add(m.drho, u);
        } else {
            T d, u[3];
            stored_moments<Q, S>(h, forced, p, d, u);
            ns.add(d, u);
        }
    }

#pragma unroll
    for (int i = 0; i < Q; ++i) St::st(B + step_store_off<PAT>(i, g, nb, wall), h[i]);
}

// Fused collide-and-stream, one node per thread.
//   GENERAL: tags are read (bounce-back, Ladd walls, forced nodes); without
//            it every node is a plain fluid node and no tag byte is touched.
//   CLOSURE: LBM_CLOSURE_BGK, _SMAGORINSKY, _STREAM_ONLY or _TRT.
//   REDUCE:  also writes this block's reduction partial of the new state to
//            partials[linear block index][0..kRedSlots).
//   PAT:     kPatAB (A -> B), or an odd or even AA step, in place in B (A is
//            not accessed; no location is touched by two threads).
template <int Q, typename S, bool GENERAL, int CLOSURE, bool REDUCE, int PAT = kPatAB>
__global__ void __launch_bounds__(kStepThreads)
    k_collide_stream(const S *__restrict__ A, S *__restrict__ B, const uint8_t *__restrict__ tags, Grid g,
                     KParams<typename Store<S>::T> p, float *__restrict__ partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    NodeSums ns;
    if (x < g.nx && y < g.ny)
        collide_stream_node<Q, S, GENERAL, CLOSURE, REDUCE, PAT>(A, B, tags, g, p, x, y, z, ns);
    if constexpr (REDUCE) block_partial_f32(ns, partials + linear_block() * kRedSlots);
}

// ---------------------------------------------------------------------------
// Compact fluid-only storage (lattices that are mostly wall, e.g. porous
// media): one thread per listed fluid node t, populations A[Q][nfp] in list
// order.  The list position of each pull source is found from the per-row
// fluid bitmask table (CompactMap): the node's coordinates come from its list
// entry, and the source x - c_i is fluid when its bit is set, at list
// position base + popc(bits below it).  So from HBM a step reads the
// populations and one 4-byte list entry per node; the 8-byte table entries
// (8 bytes per 32 lattice nodes) are shared by the nodes of nine rows and
// stay in L2.
// ---------------------------------------------------------------------------
struct CompactNode {
    int xs[3];          // x - 1, x, x + 1 (wrapped)
    int wx[3];          // their words in a row: xs / 32
    uint32_t bm[3];     // their bits in the word: 1 << (xs % 32)
    int rw[3][3];       // rw[dy+1][dz+1] = row(z + dz, y + dy) * nw (wrapped)
    bool forced;

    __device__ __forceinline__ void init(const CompactMap &cm, uint32_t entry)
    {
        forced = (entry & kListForced) != 0u;
        const uint32_t off = entry & kListOffset;
        const uint32_t row = cm.by_nw.div(off >> 5);
        const int x = (int)(off - row * 32u * (uint32_t)cm.nw);
        const uint32_t z = cm.by_ny.div(row);
        const int y = (int)(row - z * (uint32_t)cm.ny), zi = (int)z;
        xs[0] = x == 0 ? cm.nx - 1 : x - 1;
        xs[1] = x;
        xs[2] = x == cm.nx - 1 ? 0 : x + 1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            wx[k] = xs[k] >> 5;
            bm[k] = 1u << (xs[k] & 31);
        }
        const int ys[3] = {y == 0 ? cm.ny - 1 : y - 1, y, y == cm.ny - 1 ? 0 : y + 1};
        const int zs[3] = {zi == 0 ? cm.nz - 1 : zi - 1, zi, zi == cm.nz - 1 ? 0 : zi + 1};
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) rw[a][b] = (zs[b] * cm.ny + ys[a]) * cm.nw;
    }

    // Code of the pull source x - c_i of direction i: its list position when
    // it is fluid, -1 for a SOLID node, -2 - k for moving wall k (WALLS: the
    // lattice has moving walls, whose tag byte is then read; without them
    // every non-fluid node is SOLID).
    template <bool WALLS>
    __device__ __forceinline__ int code(const CompactMap &cm, int i) const
    {
        const int k = 1 - cvel(i, 0);
        const int r = rw[1 - cvel(i, 1)][1 - cvel(i, 2)];
        const uint2 e = __ldg(cm.words + (uint32_t)(r + wx[k]));
        if (e.x & bm[k]) return (int)(e.y + __popc(e.x & (bm[k] - 1u)));
        if constexpr (!WALLS) {
            return -1;
        } else {
            const unsigned ts = cm.tags[(uint32_t)(r * 32 + xs[k])] & kTagMask;  // row * px = (row * nw) * 32
            return ts == LBM_TAG_SOLID ? -1 : -2 - (int)(ts - LBM_TAG_WALL0);
        }
    }
};

// The local-density wall on compact storage: h holds the bounced links
// without their wall terms; adds rho0 / (1 - s) times each term.  sv: the
// source codes of the node's links.
template <int Q, typename T>
__device__ __forceinline__ void compact_local_wall(T (&h)[Q], const int (&sv)[Q], const KParams<T> &p)
{
    T s = T(0);
    bool any = false;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (sv[i] < -1) {
            s += wall_term<Q, T>(i, (unsigned)(LBM_TAG_WALL0 - 2 - sv[i]), p);
            any = true;
        }
    if (!any) return;
    const T rw = local_wall_rho<Q, T>(h, s);
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (sv[i] < -1) h[i] = fma(rw, wall_term<Q, T>(i, (unsigned)(LBM_TAG_WALL0 - 2 - sv[i]), p), h[i]);
}

// The fused reduction's share of one node (FP32 compute): the density and
// velocity the collision used where the storage is FP32, otherwise those of
// the post-collision set rounded to the storage type.
template <int Q, typename S>
__device__ __forceinline__ void compact_reduce_add(const typename Store<S>::T (&h)[Q],
                                                   const Macro<typename Store<S>::T> &m, bool forced,
                                                   const KParams<typename Store<S>::T> &p, NodeSums &ns)
{
    using T = typename Store<S>::T;
    static_assert(sizeof(T) == 4, "fused reductions are FP32-compute only");
    if constexpr (sizeof(S) == sizeof(T)) {
        const float u[3] = {m.ux, m.uy, m.uz};
        ns.add(m.drho, u);
    } else {
        T d, u[3];
        stored_moments<Q, S>(h, forced, p, d, u);
        ns.add(d, u);
    }
}

// One listed node of the compact step.  I: the index type of the compact
// arrays, uint32_t when Q nfp < 2^32 (one 32-bit multiply-add per address),
// long long otherwise.
//   PAT:    AB (A -> B), or an odd or even AA step in place in B;
//   LOCAL:  the local-density wall (p.wall_local), a separate instantiation
//           since keeping all source codes live costs registers;
//   WALLS:  the lattice has moving walls (their tags are read);
//   REDUCE: add the new state's density and velocity to ns (FP32 compute).
template <int Q, typename S, typename I, int CLOSURE, int PAT, bool LOCAL, bool WALLS, bool REDUCE>
__device__ __forceinline__ void compact_node(const S *__restrict__ A, S *__restrict__ B, const CompactMap &cm, I t,
                                             I nfp, const KParams<typename Store<S>::T> &p, NodeSums &ns)
{
    using T = typename Store<S>::T;
    using St = Store<S>;
    CompactNode nd;
    nd.init(cm, __ldg(cm.list + t));
    T h[Q];
    Macro<T> m;
    if constexpr (PAT == kPatAB && !LOCAL) {
        // AB: h_i = A[i][s_i], a bounced link A[opp(i)][t] (+ Ladd's term).
        // All source codes first, then all population loads: the table
        // loads, then the population loads, are in flight together (measured
        // on a 400^3 porous medium: 1.3x (FP32) to 1.9x (FP16) faster than
        // loading each population right after its code).
        int sv[Q];
        sv[0] = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) sv[i] = nd.code<WALLS>(cm, i);
        h[0] = St::ld(A + t);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int s = sv[i];
            const I a = s >= 0 ? (I)i * nfp + (I)s : (I)opp(i) * nfp + t;
            T v = St::ld(A + a);
            if (WALLS && s < -1) v += wall_term<Q, T>(i, (unsigned)(LBM_TAG_WALL0 - 2 - s), p);
            h[i] = v;
        }
        m = collide_node<Q, T, CLOSURE>(h, nd.forced, p);
        if constexpr (REDUCE) compact_reduce_add<Q, S>(h, m, nd.forced, p, ns);
#pragma unroll
        for (int i = 0; i < Q; ++i) St::st(B + ((I)i * nfp + t), h[i]);
        return;
    }
    const S *F = PAT == kPatAB ? A : B;  // AA: in place through B
    if constexpr (PAT == kPatAAEven) {
        // Local reads (layout P); links from a moving wall add Ladd's term.
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] = St::ldc(F + ((I)i * nfp + t));
        if constexpr (WALLS) {
            int sv[Q];
            sv[0] = 0;
#pragma unroll
            for (int i = 1; i < Q; ++i) sv[i] = nd.code<WALLS>(cm, i);
            if (LOCAL) {
                compact_local_wall<Q, T>(h, sv, p);
            } else {
#pragma unroll
                for (int i = 1; i < Q; ++i)
                    if (sv[i] < -1) h[i] += wall_term<Q, T>(i, (unsigned)(LBM_TAG_WALL0 - 2 - sv[i]), p);
            }
        }
        m = collide_node<Q, T, CLOSURE>(h, nd.forced, p);
        if constexpr (REDUCE) compact_reduce_add<Q, S>(h, m, nd.forced, p, ns);
#pragma unroll
        for (int i = 0; i < Q; ++i) St::st(B + ((I)opp(i) * nfp + t), h[i]);
    } else {
        // AB (local-density wall): h_i = A[i][s_i]; odd AA: h_i = F[opp(i)][s_i]
        // and f*_i goes to F[i][s_opp(i)], the list position of x + c_i.  A
        // bounced link reads (and, in AA, writes back) the node's own slot.
        int sv[Q];
        sv[0] = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) sv[i] = nd.code<WALLS>(cm, i);
        h[0] = pop_ld<S, PAT>(F + t);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int s = sv[i];
            const int slot = PAT == kPatAB ? i : opp(i);
            const I a = s >= 0 ? (I)slot * nfp + (I)s : (I)(PAT == kPatAB ? opp(i) : i) * nfp + t;
            T v = pop_ld<S, PAT>(F + a);
            if (WALLS && s < -1 && !LOCAL) v += wall_term<Q, T>(i, (unsigned)(LBM_TAG_WALL0 - 2 - s), p);
            h[i] = v;
        }
        if (LOCAL && WALLS) compact_local_wall<Q, T>(h, sv, p);
        m = collide_node<Q, T, CLOSURE>(h, nd.forced, p);
        if constexpr (REDUCE) compact_reduce_add<Q, S>(h, m, nd.forced, p, ns);
        if constexpr (PAT == kPatAB) {
#pragma unroll
            for (int i = 0; i < Q; ++i) St::st(B + ((I)i * nfp + t), h[i]);
        } else {
            St::st(B + t, h[0]);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int d = sv[opp(i)];
                St::st(B + (d >= 0 ? (I)i * nfp + (I)d : (I)opp(i) * nfp + t), h[i]);
            }
        }
    }
}

template <int Q, typename S, typename I, int CLOSURE, int PAT, bool LOCAL, bool WALLS, bool REDUCE>
__global__ void __launch_bounds__(kStepThreads)
    k_collide_stream_compact(const S *__restrict__ A, S *__restrict__ B, CompactMap cm, I n, I nfp,
                             KParams<typename Store<S>::T> p, float *__restrict__ partials)
{
    const I t = (I)blockIdx.x * (I)blockDim.x + (I)threadIdx.x;
    NodeSums ns;
    if (t < n) compact_node<Q, S, I, CLOSURE, PAT, LOCAL, WALLS, REDUCE>(A, B, cm, t, nfp, p, ns);
    if constexpr (REDUCE) block_partial_f32(ns, partials + (long long)blockIdx.x * kRedSlots);
}

// The reduction over the compact copy: node t's f*_i sits at A[i][t] (AB),
// A[opp(i)][t] (AA layout S) or, in layout P, at F[i][x + c_i], whose list
// position is the code of direction opp(i) (F[opp(i)][t] where x + c_i is
// a wall).  Same per-block chunking as k_reduce.
template <int Q, typename S, int LAY, bool WALLS>
__global__ void __launch_bounds__(kRedThreads)
    k_reduce_compact(const S *__restrict__ A, CompactMap cm, long long n, long long nfp,
                     KParams<typename Store<S>::T> p, double *__restrict__ partials)
{
    using T = typename Store<S>::T;
    RedAcc<T> ra;
    const long long chunk = ((n + gridDim.x - 1) / gridDim.x + 31) & ~31ll;
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
        const uint32_t entry = __ldg(cm.list + t);
        T h[Q];
        if constexpr (LAY == kLayP) {
            CompactNode nd;
            nd.init(cm, entry);
            h[0] = Store<S>::ld(A + t);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int d = nd.code<WALLS>(cm, opp(i));
                h[i] = Store<S>::ld(A + (d >= 0 ? (long long)i * nfp + d : (long long)opp(i) * nfp + t));
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) h[i] = Store<S>::ld(A + (long long)(LAY == kLayS ? opp(i) : i) * nfp + t);
        }
        T d, u[3];
        stored_moments<Q, S>(h, (entry & kListForced) != 0u, p, d, u);
        ra.add(d, u);
    }
    double acc[kRedSlots];
    ra.slots(acc);
    block_reduce_slots(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) partials[(long long)blockIdx.x * kRedSlots + k] = acc[k];
}

// ---------------------------------------------------------------------------
// The step with the learned closure: tau_eff = tau + dtau(Pi^neq, rho) per
// node, the network evaluated by each warp on its 32 nodes as a BF16
// tensor-core tile (mlp_warp_dtau).  Every lane of a warp takes part in the
// network, so lanes past the row end and solid nodes only skip their loads
// and stores.  Requires blockDim.x to be a multiple of 32.
// ---------------------------------------------------------------------------
template <int Q, typename S, bool GENERAL, int PAT = kPatAB>
__global__ void __launch_bounds__(kStepThreads)
    k_collide_stream_mlp(const S *__restrict__ A, S *__restrict__ B, const uint8_t *__restrict__ tags, Grid g,
                         KParams<typename Store<S>::T> p, const MlpSmem *__restrict__ mlp_image)
{
    using T = typename Store<S>::T;
    using St = Store<S>;
    __shared__ MlpSmem W;
    __shared__ uint32_t stage[kStepThreads / 32][32 * 8];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    copy_mlp_image(mlp_image, W, tid, blockDim.x * blockDim.y);
    __syncthreads();

    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (y >= g.ny) return;  // uniform over the warp: a warp lies in one row
    const bool inx = x < g.nx;
    Nbr nb;
    nb.init(g, inx ? x : 0, y, z);
    unsigned t = 0;
    bool active = inx;
    if (GENERAL && inx) {
        t = tags[nb.self];
        active = !is_wall_tag(t & kTagMask);
    }
    const S *F = PAT == kPatAB ? A : B;  // AA: in place through B
    T h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = active ? pop_ld<S, PAT>(F + step_load_off<PAT>(i, g, nb)) : T(0);
    uint32_t wall = 0;
    if (GENERAL && active && (t & kNearWall)) wall = apply_walls<Q, S, PAT>(h, F, tags, g, nb, p);

    const bool forced = GENERAL && (t & kTagMask) == LBM_TAG_FORCED;
    const Macro<T> m = node_macros<Q, T>(h, forced, p);
    T pi[6];
    pi_neq<Q, T>(h, m, pi);
    const float xf[kMlpIn] = {(float)pi[0], (float)pi[1], (float)pi[2], (float)pi[3],
                              (float)pi[4], (float)pi[5], (float)m.rho};
    const float dtau = mlp_warp_dtau(W, stage[tid >> 5], xf, (unsigned)tid & 31u);
    relax<Q, T>(h, m, T(1) / (p.tau + T(dtau)), forced);
    if (active) {
#pragma unroll
        for (int i = 0; i < Q; ++i) St::st(B + step_store_off<PAT>(i, g, nb, wall), h[i]);
    }
}

// ---------------------------------------------------------------------------
// The same step with two x-adjacent nodes (x0 = 2t, x0 + 1) per thread, for
// 16-bit storage, where one node per thread is instruction-bound: populations
// move as aligned 32-bit pairs with packed conversions, and the +-1 x shift of
// the pull comes from the neighbouring lane's pair by a warp shuffle.  Only
// the first and last lane of a warp, and the nodes at the periodic x seam,
// load their shifted value directly.  Requires blockDim.x to be a multiple of
// 32 so that a warp covers 64 consecutive nodes of one row; every lane takes
// part in the shuffles, lanes past the row end only clamp their addresses.
// ---------------------------------------------------------------------------
template <typename S> struct Pair;
template <> struct Pair<__half> {
    static __device__ __forceinline__ float2 ld(const __half *p)
    {
        const unsigned v = __ldg(reinterpret_cast<const unsigned *>(p));
        return __half22float2(*reinterpret_cast<const __half2 *>(&v));
    }
    static __device__ __forceinline__ float2 ldc(const __half *p)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    static __device__ __forceinline__ void st(__half *p, float a, float b)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
};
template <> struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ float2 ld(const __nv_bfloat16 *p)
    {
        const unsigned v = __ldg(reinterpret_cast<const unsigned *>(p));
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v));
    }
    static __device__ __forceinline__ float2 ldc(const __nv_bfloat16 *p)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float a, float b)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
    }
};
template <> struct Pair<h16s> {
    static __device__ __forceinline__ float2 ld(const h16s *p)
    {
        const unsigned v = __ldg(reinterpret_cast<const unsigned *>(p));
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&v));
        return make_float2(f.x * kF16sDown, f.y * kF16sDown);
    }
    static __device__ __forceinline__ float2 ldc(const h16s *p)
    {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(p));
        return make_float2(f.x * kF16sDown, f.y * kF16sDown);
    }
    static __device__ __forceinline__ void st(h16s *p, float a, float b)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a * kF16sUp, b * kF16sUp);
    }
};
template <> struct Pair<float> {
    static __device__ __forceinline__ float2 ld(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ float2 ldc(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ void st(float *p, float a, float b)
    {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
};

template <int Q, typename S, bool GENERAL, int CLOSURE, bool REDUCE>
__device__ __forceinline__ void collide_stream_pair(const S *__restrict__ A, S *__restrict__ B,
                                                    const uint8_t *__restrict__ tags, const Grid &g,
                                                    const KParams<float> &p, int pair, int y, int z, NodeSums &ns)
{
    using St = Store<S>;
    const unsigned lane = threadIdx.x & 31u;
    const int x0 = 2 * pair;
    const bool va = x0 < g.nx, vb = x0 + 1 < g.nx;
    const int xc = x0 < g.px ? x0 : g.px - 2;  // in-row address for lanes past the end

    int row[3][3];
    {
        const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
        const int ys[3] = {ym, y, yp};
        const int zs[3] = {zm, z, zp};
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) row[a][b] = (zs[b] * g.ny + ys[a]) * g.px;
    }
    const int self = row[1][1] + xc;

    unsigned ta = 0, tb = 0;
    bool act_a = va, act_b = vb;
    if (GENERAL) {
        const unsigned tt = __ldg(reinterpret_cast<const unsigned short *>(tags + self));
        ta = tt & 0xffu;
        tb = tt >> 8;
        act_a = va && !is_wall_tag(ta & kTagMask);
        act_b = vb && !is_wall_tag(tb & kTagMask);
    }

    float2 h[Q];  // .x: node x0, .y: node x0 + 1
    const bool edge_lo = lane == 0 || x0 == 0;               // source x0 - 1 not in lane - 1
    const bool edge_hi = lane == 31 || x0 + 2 >= g.nx;       // source x0 + 2 not in lane + 1
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const S *Ai = A + (long long)i * g.sN + row[1 - cvel(i, 1)][1 - cvel(i, 2)];
        const float2 P = Pair<S>::ld(Ai + xc);
        if (cvel(i, 0) == 0) {
            h[i] = P;
        } else if (cvel(i, 0) > 0) {  // pull from x - 1
            float up = __shfl_up_sync(0xffffffffu, P.y, 1);
            if (edge_lo && va) up = St::ld(Ai + (x0 == 0 ? g.nx - 1 : x0 - 1));
            h[i] = make_float2(up, P.x);
        } else {  // pull from x + 1
            float dn = __shfl_down_sync(0xffffffffu, P.x, 1);
            if (edge_hi && vb) dn = St::ld(Ai + (x0 + 2 == g.nx ? 0 : x0 + 2));
            h[i] = make_float2(vb ? P.y : St::ld(Ai), dn);  // odd nx: the last node wraps to x = 0
        }
    }

    bool fa = false, fb = false;
    if (GENERAL) {
        if (act_a && (ta & kNearWall)) {
            Nbr nb;
            nb.init(g, x0, y, z);
            float t[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) t[i] = h[i].x;
            apply_walls<Q, S, kPatAB, false>(t, A, tags, g, nb, p);
#pragma unroll
            for (int i = 0; i < Q; ++i) h[i].x = t[i];
        }
        if (act_b && (tb & kNearWall)) {
            Nbr nb;
            nb.init(g, x0 + 1, y, z);
            float t[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) t[i] = h[i].y;
            apply_walls<Q, S, kPatAB, false>(t, A, tags, g, nb, p);
#pragma unroll
            for (int i = 0; i < Q; ++i) h[i].y = t[i];
        }
        fa = (ta & kTagMask) == LBM_TAG_FORCED;
        fb = (tb & kTagMask) == LBM_TAG_FORCED;
    }
    {
        // The two nodes collide one after the other in scalar FP32: a packed
        // FP32x2 collision issues fewer instructions but needs about 84
        // registers, and the occupancy it loses costs more than it saves.
        float ta_[Q], tb_[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            ta_[i] = h[i].x;
            tb_[i] = h[i].y;
        }
        collide_node<Q, float, CLOSURE>(ta_, fa, p);
        collide_node<Q, float, CLOSURE>(tb_, fb, p);
        if constexpr (REDUCE) {
            float d, u[3];
            if (act_a) {
                stored_moments<Q, S>(ta_, fa, p, d, u);
                ns.add(d, u);
            }
            if (act_b) {
                stored_moments<Q, S>(tb_, fb, p, d, u);
                ns.add(d, u);
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] = make_float2(ta_[i], tb_[i]);
    }

    if (act_a && act_b) {
#pragma unroll
        for (int i = 0; i < Q; ++i) Pair<S>::st(B + (long long)i * g.sN + self, h[i].x, h[i].y);
    } else if (act_a || act_b) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (act_a) St::st(B + (long long)i * g.sN + self, h[i].x);
            if (act_b) St::st(B + (long long)i * g.sN + self + 1, h[i].y);
        }
    }
}

// The even (local) AA step of two x-adjacent nodes: each reads its own
// slots F[i][x] and writes F[opp(i)][x], so the pair moves as aligned 32-bit
// words with no neighbour access at all; a link whose source is a moving wall
// adds Ladd's term to the bounced value already in place.
template <int Q, typename S, bool GENERAL, int CLOSURE, bool REDUCE>
__device__ __forceinline__ void collide_even_pair(S *__restrict__ F, const uint8_t *__restrict__ tags, const Grid &g,
                                                  const KParams<float> &p, int pair, int y, int z, NodeSums &ns)
{
    using St = Store<S>;
    const int x0 = 2 * pair;
    if (x0 >= g.nx) return;  // no warp-collective work in this step
    const bool vb = x0 + 1 < g.nx;
    const int self = (z * g.ny + y) * g.px + x0;  // even: a 4-byte aligned pair (x0 + 1 < px)
    unsigned ta = 0, tb = 0;
    bool act_a = true, act_b = vb;
    if (GENERAL) {
        const unsigned tt = __ldg(reinterpret_cast<const unsigned short *>(tags + self));
        ta = tt & 0xffu;
        tb = tt >> 8;
        act_a = !is_wall_tag(ta & kTagMask);
        act_b = vb && !is_wall_tag(tb & kTagMask);
    }
    if (!act_a && !act_b) return;
    float ha[Q], hb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float2 v = Pair<S>::ldc(F + (long long)i * g.sN + self);
        ha[i] = v.x;
        hb[i] = v.y;
    }
    bool fa = false, fb = false;
    if (GENERAL) {
        if (act_a && (ta & kNearWall)) {
            Nbr nb;
            nb.init(g, x0, y, z);
            apply_walls<Q, S, kPatAAEven, false>(ha, F, tags, g, nb, p);
        }
        if (act_b && (tb & kNearWall)) {
            Nbr nb;
            nb.init(g, x0 + 1, y, z);
            apply_walls<Q, S, kPatAAEven, false>(hb, F, tags, g, nb, p);
        }
        fa = (ta & kTagMask) == LBM_TAG_FORCED;
        fb = (tb & kTagMask) == LBM_TAG_FORCED;
    }
    collide_node<Q, float, CLOSURE>(ha, fa, p);
    collide_node<Q, float, CLOSURE>(hb, fb, p);
    if constexpr (REDUCE) {
        float d, u[3];
        if (act_a) {
            stored_moments<Q, S>(ha, fa, p, d, u);
            ns.add(d, u);
        }
        if (act_b) {
            stored_moments<Q, S>(hb, fb, p, d, u);
            ns.add(d, u);
        }
    }
    // The store addresses are those of the loads; taking them again from an
    // offset the compiler cannot see through keeps it from holding all Q of
    // them live across the collisions.
    int so = self;
    asm volatile("" : "+r"(so));
    if (act_a && act_b) {
#pragma unroll
        for (int i = 0; i < Q; ++i) Pair<S>::st(F + (long long)opp(i) * g.sN + so, ha[i], hb[i]);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (act_a) St::st(F + (long long)opp(i) * g.sN + so, ha[i]);
            if (act_b) St::st(F + (long long)opp(i) * g.sN + so + 1, hb[i]);
        }
    }
}

// PAT: kPatAB (pull from A, write B) or kPatAAEven (in place in B).
template <int Q, typename S, bool GENERAL, int CLOSURE, bool REDUCE, int PAT>
__device__ __forceinline__ void collide_stream_x2_body(const S *__restrict__ A, S *__restrict__ B,
                                                       const uint8_t *__restrict__ tags, const Grid &g,
                                                       const KParams<float> &p, float *__restrict__ partials)
{
    const int pair = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    NodeSums ns;
    // y >= ny is uniform over a warp (a warp lies in one row), so skipping
    // those warps keeps every shuffle of the node work warp-complete
    if (y < g.ny) {
        if constexpr (PAT == kPatAAEven)
            collide_even_pair<Q, S, GENERAL, CLOSURE, REDUCE>(B, tags, g, p, pair, y, z, ns);
        else
            collide_stream_pair<Q, S, GENERAL, CLOSURE, REDUCE>(A, B, tags, g, p, pair, y, z, ns);
    }
    if constexpr (REDUCE) block_partial_f32(ns, partials + linear_block() * kRedSlots);
}

template <int Q, typename S, bool GENERAL, int CLOSURE, bool REDUCE, int PAT = kPatAB>
__global__ void __launch_bounds__(kStepThreads)
    k_collide_stream_x2(const S *__restrict__ A, S *__restrict__ B, const uint8_t *__restrict__ tags, Grid g,
                        KParams<float> p, float *__restrict__ partials)
{
    collide_stream_x2_body<Q, S, GENERAL, CLOSURE, REDUCE, PAT>(A, B, tags, g, p, partials);
}

// ---------------------------------------------------------------------------
// Per-node density and velocity from the stored post-collision set.
// ---------------------------------------------------------------------------
// Offset of f*_i(x) in read layout LAY (AB, AA layout S or P).  Layout P
// looks at x + c_i: nb must be initialised and near_wall = the node's
// kNearWall bit; AB and S use nb.self only.
template <int LAY>
__device__ __forceinline__ long long fstar_off(int i, const Grid &g, const Nbr &nb, bool near_wall,
                                               const uint8_t *__restrict__ tags)
{
    if (LAY == kLayAB) return (long long)i * g.sN + nb.self;
    if (LAY == kLayS) return (long long)opp(i) * g.sN + nb.self;
    if (i != 0 && near_wall && is_wall_tag(tags[nb.dst(i)] & kTagMask)) return (long long)opp(i) * g.sN + nb.self;
    return (long long)i * g.sN + nb.dst(i);
}

template <int Q, typename S, int LAY>
__device__ __forceinline__ void node_moments(const S *__restrict__ A, const Grid &g, const Nbr &nb, bool near_wall,
                                             const uint8_t *__restrict__ tags, bool forced,
                                             const KParams<typename Store<S>::T> &p, typename Store<S>::T &drho,
                                             typename Store<S>::T (&u)[3])
{
    using T = typename Store<S>::T;
    T d = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T v = Store<S>::ld(A + fstar_off<LAY>(i, g, nb, near_wall, tags));
        d += v;
        if (cvel(i, 0)) jx += cvel(i, 0) > 0 ? v : -v;
        if (cvel(i, 1)) jy += cvel(i, 1) > 0 ? v : -v;
        if (cvel(i, 2)) jz += cvel(i, 2) > 0 ? v : -v;
    }
    const T rho = T(1) + d;
    if (forced) {
        jx -= T(0.5) * rho * p.force[0];
        jy -= T(0.5) * rho * p.force[1];
        jz -= T(0.5) * rho * p.force[2];
    }
    const T inv = T(1) / rho;
    drho = d;
    u[0] = jx * inv;
    u[1] = jy * inv;
    u[2] = jz * inv;
}

// The node (x, y, z) for a read in layout LAY: the full neighbourhood for
// layout P, the node's own offset otherwise.
template <int LAY> __device__ __forceinline__ void read_node(Nbr &nb, const Grid &g, int x, int y, int z)
{
    if (LAY == kLayP)
        nb.init(g, x, y, z);
    else
        nb.self = (z * g.ny + y) * g.px + x;
}

template <int Q, typename S, bool GENERAL, int LAY = kLayAB>
__global__ void __launch_bounds__(kStepThreads)
    k_moments(const S *__restrict__ A, const uint8_t *__restrict__ tags, Grid g, KParams<typename Store<S>::T> p,
              double *__restrict__ rho, double *__restrict__ u)
{
    using T = typename Store<S>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    Nbr nb;
    read_node<LAY>(nb, g, x, y, z);
    const long long n = x + (long long)g.nx * (y + (long long)g.ny * z);
    const unsigned tb = GENERAL ? tags[nb.self] : 0u;
    const unsigned t = tb & kTagMask;
    if (is_wall_tag(t)) {
        if (rho) rho[n] = 0.0;
        if (u) u[n] = u[g.N + n] = u[2 * g.N + n] = 0.0;
        return;
    }
    T d, v[3];
    node_moments<Q, S, LAY>(A, g, nb, (tb & kNearWall) != 0u, tags, t == LBM_TAG_FORCED, p, d, v);
    if (rho) rho[n] = 1.0 + (double)d;
    if (u) {
        u[n] = (double)v[0];
        u[g.N + n] = (double)v[1];
        u[2 * g.N + n] = (double)v[2];
    }
}

// ---------------------------------------------------------------------------
// The learned closure's inputs for the step that would follow, computed as
// that step computes them: each node's pulled set (pattern PAT, boundary
// rules included), its density and non-equilibrium stress;
// x[n][7] = (Pi xx, yy, zz, xy, xz, yz, rho) for n = x + nx (y + ny z), in
// FP32; zeros on solid and wall nodes.  Nothing is written to the lattice.
// ---------------------------------------------------------------------------
template <int Q, typename S, bool GENERAL, int PAT>
__global__ void __launch_bounds__(kStepThreads)
    k_closure_features(const S *__restrict__ A, const uint8_t *__restrict__ tags, Grid g,
                       KParams<typename Store<S>::T> p, float *__restrict__ xout)
{
    using T = typename Store<S>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    float *out = xout + 7 * (x + (long long)g.nx * (y + (long long)g.ny * z));
    Nbr nb;
    nb.init(g, x, y, z);
    const unsigned t = GENERAL ? tags[nb.self] : 0u;
    if (GENERAL && is_wall_tag(t & kTagMask)) {
#pragma unroll
        for (int k = 0; k < 7; ++k) out[k] = 0.f;
        return;
    }
    T h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = Store<S>::ld(A + step_load_off<PAT>(i, g, nb));
    if (GENERAL && (t & kNearWall)) apply_walls<Q, S, PAT>(h, A, tags, g, nb, p);
    const Macro<T> m = node_macros<Q, T>(h, GENERAL && (t & kTagMask) == LBM_TAG_FORCED, p);
    T pi[6];
    pi_neq<Q, T>(h, m, pi);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k] = (float)pi[k];
    out[6] = (float)m.rho;
}

// ---------------------------------------------------------------------------
// Reduction: FP64 sums over fluid nodes.  Pass 1 writes one partial per block
// (a fixed grid of at most one resident wave; block b sweeps one contiguous
// range of the padded node index, its threads side by side), pass 2 adds the
// partials in a fixed order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
template <int Q, typename S, bool GENERAL, int LAY = kLayAB>
__global__ void __launch_bounds__(kRedThreads)
    k_reduce(const S *__restrict__ A, const uint8_t *__restrict__ tags, Grid g, KParams<typename Store<S>::T> p,
             double *__restrict__ partials)
{
    using T = typename Store<S>::T;
    RedAcc<T> ra;
    const long long total = (long long)g.nz * g.ny * g.px;  // < 2^31 - 256
    const long long chunk = ((total + gridDim.x - 1) / gridDim.x + 31) & ~31ll;
    const long long lo = blockIdx.x * chunk;
    const int hi = (int)(lo + chunk < total ? lo + chunk : total);
    if (lo < total) {
        int idx = (int)lo + threadIdx.x;
        int x = idx % g.px;
        for (; idx < hi; idx += blockDim.x) {
            if (x < g.nx) {
                const unsigned tb = GENERAL ? tags[idx] : 0u;
                const unsigned t = tb & kTagMask;
                if (!is_wall_tag(t)) {
                    Nbr nb;
                    if (LAY == kLayP) {
                        const int row = idx / g.px;
                        nb.init(g, x, row % g.ny, row / g.ny);
                    } else {
                        nb.self = idx;
                    }
                    T d, v[3];
                    node_moments<Q, S, LAY>(A, g, nb, (tb & kNearWall) != 0u, tags, t == LBM_TAG_FORCED, p, d, v);
                    ra.add(d, v);
                }
            }
            x += blockDim.x;
            while (x >= g.px) x -= g.px;
        }
    }
    double acc[kRedSlots];
    ra.slots(acc);
    block_reduce_slots(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) partials[(long long)blockIdx.x * kRedSlots + k] = acc[k];
}

// Second pass: one block adds nblocks partials in a fixed order.
__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double *__restrict__ partials, int nblocks,
                                                             double *__restrict__ out);

// ---------------------------------------------------------------------------
// Initialisation and population transfer.
// ---------------------------------------------------------------------------
// With aa, one array in layout S (slot opp(i) of the node); B is unused.
template <int Q, typename S>
__global__ void __launch_bounds__(kStepThreads)
    k_init(S *__restrict__ A, S *__restrict__ B, Grid g, const double *__restrict__ rho, const double *__restrict__ u,
           bool aa)
{
    // h_eq in the compute type (FP32 except for FP64 storage).
    using T = typename Store<S>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int off = (z * g.ny + y) * g.px + x;
    const long long n = x + (long long)g.nx * (y + (long long)g.ny * z);
    const T dr = rho ? (T)(rho[n] - 1.0) : T(0);
    const T r = T(1) + dr;
    const T ux = u ? (T)u[n] : T(0), uy = u ? (T)u[g.N + n] : T(0), uz = u ? (T)u[2 * g.N + n] : T(0);
    const T usq15 = T(1.5) * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T cu = cdot<T>(i, ux, uy, uz);
        const T heq = wgt<T>(Q, i) * (dr + r * (cu * (T(3) + T(4.5) * cu) - usq15));
        S v;
        Store<S>::st(&v, heq);
        if (aa) {
            A[(long long)opp(i) * g.sN + off] = v;
        } else {
            A[(long long)i * g.sN + off] = v;
            B[(long long)i * g.sN + off] = v;
        }
    }
}

template <int Q, typename S, int LAY = kLayAB>
__global__ void k_get_pop(const S *__restrict__ A, const uint8_t *__restrict__ tags, Grid g, int i,
                          double *__restrict__ f)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    Nbr nb;
    read_node<LAY>(nb, g, x, y, z);
    const long long n = x + (long long)g.nx * (y + (long long)g.ny * z);
    double w = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if (k == i) w = wgt<double>(Q, k);
    // layout P: solid and wall nodes keep their (never updated) own slots
    const bool nw = LAY == kLayP && (tags[nb.self] & kNearWall) != 0u;
    const bool solid = LAY == kLayP && is_wall_tag(tags[nb.self] & kTagMask);
    const long long o = solid ? (long long)opp(i) * g.sN + nb.self : fstar_off<LAY>(i, g, nb, nw, tags);
    f[n] = (double)Store<S>::ld(A + o) + w;
}

// With aa, one array in layout S (slot opp(i) of the node); B is unused.
template <int Q, typename S>
__global__ void k_set_pop(S *__restrict__ A, S *__restrict__ B, Grid g, int i, const double *__restrict__ f, bool aa)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int off = (z * g.ny + y) * g.px + x;
    const long long n = x + (long long)g.nx * (y + (long long)g.ny * z);
    double w = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if (k == i) w = wgt<double>(Q, k);
    const S v = Store<S>::from_f64(f[n] - w);
    if (aa) {
        A[(long long)opp(i) * g.sN + off] = v;
    } else {
        A[(long long)i * g.sN + off] = v;
        B[(long long)i * g.sN + off] = v;
    }
}

// Block shape shared by the node-per-thread kernels.
inline void node_launch_shape(const Grid &g, dim3 &grid, dim3 &block)
{
    const int bx = g.px >= 128 ? 128 : g.px;  // px is a multiple of 32
    const int by = kStepThreads / bx;
    block = dim3(bx, by, 1);
    grid = dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz);
}

}  // namespace lbm

// The TMA-fed learned-closure step (uses the node helpers above).
#include "lbm_mlp_tma.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Launchers, defined once per storage type S by LBM_DEFINE_LAUNCHERS(S).
// ---------------------------------------------------------------------------
// Two nodes per thread for 16-bit storage on rows of at least 64 nodes.
template <typename S> constexpr bool use_pairs() { return sizeof(S) == 2; }

inline void pair_launch_shape(const Grid &g, dim3 &grid, dim3 &block)
{
    const int pairs = g.px / 2;                  // px is a multiple of 32
    // whole warps along x; 64 pairs per block row only where rows hold a
    // multiple of 64 pairs (otherwise the last block of a row idles)
    const int bx = pairs % 64 == 0 ? 64 : 32;
    const int by = kStepThreads / bx;
    block = dim3(bx, by, 1);
    grid = dim3((pairs + bx - 1) / bx, (g.ny + by - 1) / by, g.nz);
}

template <int Q, typename S, bool GEN, bool RED, int CLOSURE, int PAT>
void launch_x2(const Launch &L, const KParams<float> &kp, float *partials, dim3 grid, dim3 block)
{
    const S *A = (const S *)L.A;
    S *B = (S *)L.B;
    k_collide_stream_x2<Q, S, GEN, CLOSURE, RED, PAT><<<grid, block, 0, L.stream>>>(A, B, L.tags, L.g, kp, partials);
}

template <int Q, typename S, bool GEN, bool RED, int PAT>
cudaError_t step_closure_x2(const Launch &L, const KParams<float> &kp, float *partials)
{
    dim3 grid, block;
    pair_launch_shape(L.g, grid, block);
    switch (L.closure) {
    case LBM_CLOSURE_BGK: launch_x2<Q, S, GEN, RED, LBM_CLOSURE_BGK, PAT>(L, kp, partials, grid, block); break;
    case LBM_CLOSURE_SMAGORINSKY:
        launch_x2<Q, S, GEN, RED, LBM_CLOSURE_SMAGORINSKY, PAT>(L, kp, partials, grid, block);
        break;
    case LBM_CLOSURE_TRT: launch_x2<Q, S, GEN, RED, LBM_CLOSURE_TRT, PAT>(L, kp, partials, grid, block); break;
    case LBM_CLOSURE_STREAM_ONLY:
        if constexpr (RED) return cudaErrorNotSupported;
        launch_x2<Q, S, GEN, false, LBM_CLOSURE_STREAM_ONLY, PAT>(L, kp, nullptr, grid, block);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The learned-closure step fed by TMA (A/B): persistent blocks, as many as
// fit on the device at once, each walking tiles of 128 nodes of one row.
template <int Q, typename S, bool GEN>
cudaError_t step_mlp_tma(const Launch &L, const KParams<typename Store<S>::T> &kp)
{
    static int wave = 0;  // resident blocks of this instantiation, found on first use
    constexpr size_t dyn = tma_smem_bytes<Q, S>();
    if (wave == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_collide_stream_mlp_tma<Q, S, GEN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_collide_stream_mlp_tma<Q, S, GEN>,
                                                               kTmaThreads, dyn)) != cudaSuccess)
            return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        wave = sms * occ;
    }
    const int ntx = (L.g.nx + kTileM - 1) / kTileM;
    const long long ntiles = (long long)ntx * L.g.ny * L.g.nz;
    const unsigned blocks = (unsigned)(ntiles < wave ? ntiles : wave);
    k_collide_stream_mlp_tma<Q, S, GEN><<<blocks, kTmaThreads, dyn, L.stream>>>(
        *L.tma_A, (const S *)L.A, (S *)L.B, L.tags, L.g, kp, (const MlpSmem *)L.mlp_image, ntx, ntiles);
    return cudaGetLastError();
}

// One dense step launch.  RED: fused step-and-reduce (FP32 compute; BGK,
// Smagorinsky and TRT).  PAT: streaming pattern (the two-nodes-per-thread
// 16-bit kernel serves A/B steps and the local even AA steps; the odd AA
// steps, which read and write the neighbours' slots, take one node per
// thread).
template <int Q, typename S, bool GEN, bool RED, int PAT>
cudaError_t step_closure(const Launch &L, const KParams<typename Store<S>::T> &kp, dim3 grid, dim3 block,
                         float *partials)
{
    if constexpr (RED && sizeof(typename Store<S>::T) != 4) {
        return cudaErrorNotSupported;
    } else {
        const S *A = (const S *)L.A;
        S *B = (S *)L.B;
        if (L.closure == LBM_CLOSURE_MLP) {
            if (RED) return cudaErrorNotSupported;
            if (!L.mlp_image) return cudaErrorInvalidValue;
            if constexpr (PAT == kPatAB)
                if (L.tma_A) return step_mlp_tma<Q, S, GEN>(L, kp);
            k_collide_stream_mlp<Q, S, GEN, PAT>
                <<<grid, block, 0, L.stream>>>(A, B, L.tags, L.g, kp, (const MlpSmem *)L.mlp_image);
            return cudaGetLastError();
        }
        if constexpr (use_pairs<S>() && (PAT == kPatAB || PAT == kPatAAEven)) {
            if (L.g.px >= 64 && !kp.wall_local) return step_closure_x2<Q, S, GEN, RED, PAT>(L, kp, partials);
        }
        switch (L.closure) {
        case LBM_CLOSURE_BGK:
            k_collide_stream<Q, S, GEN, LBM_CLOSURE_BGK, RED, PAT>
                <<<grid, block, 0, L.stream>>>(A, B, L.tags, L.g, kp, partials);
            break;
        case LBM_CLOSURE_SMAGORINSKY:
            k_collide_stream<Q, S, GEN, LBM_CLOSURE_SMAGORINSKY, RED, PAT>
                <<<grid, block, 0, L.stream>>>(A, B, L.tags, L.g, kp, partials);
            break;
        case LBM_CLOSURE_TRT:
            k_collide_stream<Q, S, GEN, LBM_CLOSURE_TRT, RED, PAT>
                <<<grid, block, 0, L.stream>>>(A, B, L.tags, L.g, kp, partials);
            break;
        case LBM_CLOSURE_STREAM_ONLY:
            if constexpr (RED) return cudaErrorNotSupported;
            k_collide_stream<Q, S, GEN, LBM_CLOSURE_STREAM_ONLY, false, PAT>
                <<<grid, block, 0, L.stream>>>(A, B, L.tags, L.g, kp, nullptr);
            break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

// Number of blocks (= partials) a fused step-and-reduce launch writes.
inline long long fused_partials(const Launch &L, const lbm_params &p, size_t elem)
{
    dim3 grid, block;
    if (elem == 2 && (!L.aa || L.aa_p) && L.g.px >= 64 && !p.wall_rho_local)
        pair_launch_shape(L.g, grid, block);
    else
        node_launch_shape(L.g, grid, block);
    return (long long)grid.x * grid.y * grid.z;
}

template <int Q, typename S, int PAT> cudaError_t step_q(const Launch &L, const lbm_params &p)
{
    dim3 grid, block;
    node_launch_shape(L.g, grid, block);
    const auto kp = make_kparams<typename Store<S>::T>(Q, p);
    return L.general ? step_closure<Q, S, true, false, PAT>(L, kp, grid, block, nullptr)
                     : step_closure<Q, S, false, false, PAT>(L, kp, grid, block, nullptr);
}

template <int Q, typename S, int PAT> cudaError_t step_reduce_q(const Launch &L, const lbm_params &p, float *partials)
{
    dim3 grid, block;
    node_launch_shape(L.g, grid, block);
    const auto kp = make_kparams<typename Store<S>::T>(Q, p);
    return L.general ? step_closure<Q, S, true, true, PAT>(L, kp, grid, block, partials)
                     : step_closure<Q, S, false, true, PAT>(L, kp, grid, block, partials);
}

template <int Q, typename S, int CLOSURE, int PAT, bool LOCAL, bool WALLS, bool RED>
cudaError_t compact_launch(const Launch &L, const KParams<typename Store<S>::T> &kp, const void *Ac, void *Bc,
                           long long nfp, float *partials)
{
    const unsigned blocks = (unsigned)((L.n_list + kStepThreads - 1) / kStepThreads);
    if (blocks == 0) return cudaSuccess;
    const S *A = (const S *)Ac;
    S *B = (S *)Bc;
    if ((long long)Q * nfp <= 0xffffffffll)  // 32-bit element indices
        k_collide_stream_compact<Q, S, uint32_t, CLOSURE, PAT, LOCAL, WALLS, RED><<<blocks, kStepThreads, 0, L.stream>>>(
            A, B, L.cmap, (uint32_t)L.n_list, (uint32_t)nfp, kp, partials);
    else
        k_collide_stream_compact<Q, S, long long, CLOSURE, PAT, LOCAL, WALLS, RED>
            <<<blocks, kStepThreads, 0, L.stream>>>(A, B, L.cmap, L.n_list, nfp, kp, partials);
    return cudaGetLastError();
}

template <int Q, typename S, int PAT, bool LOCAL, bool WALLS, bool RED>
cudaError_t step_compact_closure(const Launch &L, const KParams<typename Store<S>::T> &kp, const void *Ac, void *Bc,
                                 long long nfp, float *partials)
{
    if constexpr (RED && sizeof(typename Store<S>::T) != 4) {
        return cudaErrorNotSupported;
    } else {
        switch (L.closure) {
        case LBM_CLOSURE_BGK:
            return compact_launch<Q, S, LBM_CLOSURE_BGK, PAT, LOCAL, WALLS, RED>(L, kp, Ac, Bc, nfp, partials);
        case LBM_CLOSURE_SMAGORINSKY:
            return compact_launch<Q, S, LBM_CLOSURE_SMAGORINSKY, PAT, LOCAL, WALLS, RED>(L, kp, Ac, Bc, nfp, partials);
        case LBM_CLOSURE_TRT:
            return compact_launch<Q, S, LBM_CLOSURE_TRT, PAT, LOCAL, WALLS, RED>(L, kp, Ac, Bc, nfp, partials);
        case LBM_CLOSURE_STREAM_ONLY:
            if constexpr (RED) return cudaErrorNotSupported;
            return compact_launch<Q, S, LBM_CLOSURE_STREAM_ONLY, PAT, LOCAL, WALLS, false>(L, kp, Ac, Bc, nfp,
                                                                                          nullptr);
        default: return cudaErrorInvalidValue;
        }
    }
}

// The local-density wall only matters next to moving walls.
template <int Q, typename S, int PAT>
cudaError_t step_compact_q(const Launch &L, const lbm_params &p, const void *Ac, void *Bc, long long nfp,
                           float *partials)
{
    const auto kp = make_kparams<typename Store<S>::T>(Q, p);
    if (!L.moving_walls)
        return partials ? step_compact_closure<Q, S, PAT, false, false, true>(L, kp, Ac, Bc, nfp, partials)
                        : step_compact_closure<Q, S, PAT, false, false, false>(L, kp, Ac, Bc, nfp, nullptr);
    if (kp.wall_local)
        return partials ? step_compact_closure<Q, S, PAT, true, true, true>(L, kp, Ac, Bc, nfp, partials)
                        : step_compact_closure<Q, S, PAT, true, true, false>(L, kp, Ac, Bc, nfp, nullptr);
    return partials ? step_compact_closure<Q, S, PAT, false, true, true>(L, kp, Ac, Bc, nfp, partials)
                    : step_compact_closure<Q, S, PAT, false, true, false>(L, kp, Ac, Bc, nfp, nullptr);
}

template <int Q, typename S, int LAY>
cudaError_t reduce_compact_q(const Launch &L, const lbm_params &p, const void *Ac, long long nfp, double *partials,
                             int nblocks, double *out)
{
    const auto kp = make_kparams<typename Store<S>::T>(Q, p);
    const S *A = (const S *)Ac;
    if (L.moving_walls)
        k_reduce_compact<Q, S, LAY, true><<<nblocks, kRedThreads, 0, L.stream>>>(A, L.cmap, L.n_list, nfp, kp, partials);
    else
        k_reduce_compact<Q, S, LAY, false><<<nblocks, kRedThreads, 0, L.stream>>>(A, L.cmap, L.n_list, nfp, kp, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, kRedThreads, 0, L.stream>>>(partials, nblocks, out);
    return cudaGetLastError();
}

// Blocks of `threads` threads of `kernel` that fit on the device at once.
template <typename K> int resident_blocks(K kernel, int threads)
{
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess)
        return 0;
    return sms * occ;
}

// nblocks (<= kRedBlocks) is cut to one resident wave: every block then
// sweeps the same number of nodes at the same time, with no second, partly
// filled wave.
template <int Q, typename S, int LAY = kLayAB>
cudaError_t reduce_q(const Launch &L, const lbm_params &p, double *partials, int nblocks, double *out)
{
    const auto kp = make_kparams<typename Store<S>::T>(Q, p);
    const int wave = L.general ? resident_blocks(k_reduce<Q, S, true, LAY>, kRedThreads)
                               : resident_blocks(k_reduce<Q, S, false, LAY>, kRedThreads);
    if (wave > 0 && nblocks > wave) nblocks = wave;
    if (L.general)
        k_reduce<Q, S, true, LAY><<<nblocks, kRedThreads, 0, L.stream>>>((const S *)L.A, L.tags, L.g, kp, partials);
    else
        k_reduce<Q, S, false, LAY><<<nblocks, kRedThreads, 0, L.stream>>>((const S *)L.A, L.tags, L.g, kp, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, kRedThreads, 0, L.stream>>>(partials, nblocks, out);
    return cudaGetLastError();
}

template <int Q, typename S, int LAY>
cudaError_t moments_q(const Launch &L, const lbm_params &p, double *rho, double *u)
{
    dim3 grid, block;
    node_launch_shape(L.g, grid, block);
    const auto kp = make_kparams<typename Store<S>::T>(Q, p);
    if (L.general)
        k_moments<Q, S, true, LAY><<<grid, block, 0, L.stream>>>((const S *)L.A, L.tags, L.g, kp, rho, u);
    else
        k_moments<Q, S, false, LAY><<<grid, block, 0, L.stream>>>((const S *)L.A, L.tags, L.g, kp, rho, u);
    return cudaGetLastError();
}

template <int Q, typename S, int PAT> cudaError_t features_q(const Launch &L, const lbm_params &p, float *x)
{
    dim3 grid, block;
    node_launch_shape(L.g, grid, block);
    const auto kp = make_kparams<typename Store<S>::T>(Q, p);
    if (L.general)
        k_closure_features<Q, S, true, PAT><<<grid, block, 0, L.stream>>>((const S *)L.A, L.tags, L.g, kp, x);
    else
        k_closure_features<Q, S, false, PAT><<<grid, block, 0, L.stream>>>((const S *)L.A, L.tags, L.g, kp, x);
    return cudaGetLastError();
}

template <int Q, typename S, int LAY> cudaError_t get_pop_q(const Launch &L, int i, double *f)
{
    dim3 grid, block;
    node_launch_shape(L.g, grid, block);
    k_get_pop<Q, S, LAY><<<grid, block, 0, L.stream>>>((const S *)L.A, L.tags, L.g, i, f);
    return cudaGetLastError();
}

// The AA instantiations (one array, steps alternating odd / even; reads in
// layout S or P), kept in translation units of their own.
#define LBM_DEFINE_AA_LAUNCHERS(S)                                                                           \
    template <> cudaError_t launch_step_aa<S>(const Launch &L, const lbm_params &p)                          \
    {                                                                                                        \
        if (L.aa_p) return L.Q == 19 ? step_q<19, S, kPatAAEven>(L, p) : step_q<27, S, kPatAAEven>(L, p);    \
        return L.Q == 19 ? step_q<19, S, kPatAAOdd>(L, p) : step_q<27, S, kPatAAOdd>(L, p);                  \
    }                                                                                                        \
    template <> cudaError_t launch_step_reduce_aa<S>(const Launch &L, const lbm_params &p, float *partials)  \
    {                                                                                                        \
        if (L.aa_p)                                                                                          \
            return L.Q == 19 ? step_reduce_q<19, S, kPatAAEven>(L, p, partials)                              \
                             : step_reduce_q<27, S, kPatAAEven>(L, p, partials);                             \
        return L.Q == 19 ? step_reduce_q<19, S, kPatAAOdd>(L, p, partials)                                   \
                         : step_reduce_q<27, S, kPatAAOdd>(L, p, partials);                                  \
    }                                                                                                        \
    template <>                                                                                              \
    cudaError_t launch_step_compact_aa<S>(const Launch &L, const lbm_params &p, const void *Ac, void *Bc,    \
                                          long long nfp, float *partials)                                    \
    {                                                                                                        \
        if (L.aa_p)                                                                                          \
            return L.Q == 19 ? step_compact_q<19, S, kPatAAEven>(L, p, Ac, Bc, nfp, partials)                \
                             : step_compact_q<27, S, kPatAAEven>(L, p, Ac, Bc, nfp, partials);               \
        return L.Q == 19 ? step_compact_q<19, S, kPatAAOdd>(L, p, Ac, Bc, nfp, partials)                     \
                         : step_compact_q<27, S, kPatAAOdd>(L, p, Ac, Bc, nfp, partials);                    \
    }                                                                                                        \
    template <>                                                                                              \
    cudaError_t launch_reduce_compact_aa<S>(const Launch &L, const lbm_params &p, const void *Ac, long long nfp, \
                                            double *partials, int nb, double *out)                           \
    {                                                                                                        \
        if (L.aa_p)                                                                                          \
            return L.Q == 19 ? reduce_compact_q<19, S, kLayP>(L, p, Ac, nfp, partials, nb, out)              \
                             : reduce_compact_q<27, S, kLayP>(L, p, Ac, nfp, partials, nb, out);             \
        return L.Q == 19 ? reduce_compact_q<19, S, kLayS>(L, p, Ac, nfp, partials, nb, out)                  \
                         : reduce_compact_q<27, S, kLayS>(L, p, Ac, nfp, partials, nb, out);                 \
    }                                                                                                        \
    template <>                                                                                              \
    cudaError_t launch_reduce_aa<S>(const Launch &L, const lbm_params &p, double *partials, int nb, double *out) \
    {                                                                                                        \
        if (L.aa_p)                                                                                          \
            return L.Q == 19 ? reduce_q<19, S, kLayP>(L, p, partials, nb, out)                               \
                             : reduce_q<27, S, kLayP>(L, p, partials, nb, out);                              \
        return L.Q == 19 ? reduce_q<19, S, kLayS>(L, p, partials, nb, out)                                   \
                         : reduce_q<27, S, kLayS>(L, p, partials, nb, out);                                  \
    }                                                                                                        \
    template <> cudaError_t launch_moments_aa<S>(const Launch &L, const lbm_params &p, double *rho, double *u) \
    {                                                                                                        \
        if (L.aa_p) return L.Q == 19 ? moments_q<19, S, kLayP>(L, p, rho, u) : moments_q<27, S, kLayP>(L, p, rho, u); \
        return L.Q == 19 ? moments_q<19, S, kLayS>(L, p, rho, u) : moments_q<27, S, kLayS>(L, p, rho, u);    \
    }                                                                                                        \
    template <> cudaError_t launch_closure_features_aa<S>(const Launch &L, const lbm_params &p, float *x)     \
    {                                                                                                        \
        if (L.aa_p) return L.Q == 19 ? features_q<19, S, kPatAAEven>(L, p, x) : features_q<27, S, kPatAAEven>(L, p, x); \
        return L.Q == 19 ? features_q<19, S, kPatAAOdd>(L, p, x) : features_q<27, S, kPatAAOdd>(L, p, x);    \
    }                                                                                                        \
    template <> cudaError_t launch_get_pop_aa<S>(const Launch &L, int i, double *f)                          \
    {                                                                                                        \
        if (L.aa_p) return L.Q == 19 ? get_pop_q<19, S, kLayP>(L, i, f) : get_pop_q<27, S, kLayP>(L, i, f);  \
        return L.Q == 19 ? get_pop_q<19, S, kLayS>(L, i, f) : get_pop_q<27, S, kLayS>(L, i, f);              \
    }

// The A/B instantiations, and the entry points that dispatch AA launches to
// the functions above.
#define LBM_DEFINE_LAUNCHERS(S)                                                                              \
    template <> cudaError_t launch_step_reduce<S>(const Launch &L, const lbm_params &p, float *partials)     \
    {                                                                                                        \
        if (L.aa) return launch_step_reduce_aa<S>(L, p, partials);                                           \
        return L.Q == 19 ? step_reduce_q<19, S, kPatAB>(L, p, partials) : step_reduce_q<27, S, kPatAB>(L, p, partials); \
    }                                                                                                        \
    template <>                                                                                              \
    cudaError_t launch_step_compact<S>(const Launch &L, const lbm_params &p, const void *Ac, void *Bc,       \
                                       long long nfp, float *partials)                                       \
    {                                                                                                        \
        if (L.aa) return launch_step_compact_aa<S>(L, p, Ac, Bc, nfp, partials);                             \
        return L.Q == 19 ? step_compact_q<19, S, kPatAB>(L, p, Ac, Bc, nfp, partials)                        \
                         : step_compact_q<27, S, kPatAB>(L, p, Ac, Bc, nfp, partials);                       \
    }                                                                                                        \
    template <>                                                                                              \
    cudaError_t launch_reduce_compact<S>(const Launch &L, const lbm_params &p, const void *Ac, long long nfp, \
                                         double *partials, int nb, double *out)                              \
    {                                                                                                        \
        if (L.aa) return launch_reduce_compact_aa<S>(L, p, Ac, nfp, partials, nb, out);                      \
        return L.Q == 19 ? reduce_compact_q<19, S, kLayAB>(L, p, Ac, nfp, partials, nb, out)                 \
                         : reduce_compact_q<27, S, kLayAB>(L, p, Ac, nfp, partials, nb, out);                \
    }                                                                                                        \
    template <> cudaError_t launch_step<S>(const Launch &L, const lbm_params &p)                             \
    {                                                                                                        \
        if (L.aa) return launch_step_aa<S>(L, p);                                                            \
        return L.Q == 19 ? step_q<19, S, kPatAB>(L, p) : step_q<27, S, kPatAB>(L, p);                        \
    }                                                                                                        \
    template <>                                                                                              \
    cudaError_t launch_reduce<S>(const Launch &L, const lbm_params &p, double *partials, int nb, double *out) \
    {                                                                                                        \
        if (L.aa) return launch_reduce_aa<S>(L, p, partials, nb, out);                                       \
        return L.Q == 19 ? reduce_q<19, S>(L, p, partials, nb, out) : reduce_q<27, S>(L, p, partials, nb, out); \
    }                                                                                                        \
    template <> cudaError_t launch_moments<S>(const Launch &L, const lbm_params &p, double *rho, double *u)  \
    {                                                                                                        \
        if (L.aa) return launch_moments_aa<S>(L, p, rho, u);                                                 \
        return L.Q == 19 ? moments_q<19, S, kLayAB>(L, p, rho, u) : moments_q<27, S, kLayAB>(L, p, rho, u);  \
    }                                                                                                        \
    template <> cudaError_t launch_init<S>(const Launch &L, const double *rho, const double *u)              \
    {                                                                                                        \
        dim3 grid, block;                                                                                    \
        node_launch_shape(L.g, grid, block);                                                                 \
        if (L.Q == 19)                                                                                       \
            k_init<19, S><<<grid, block, 0, L.stream>>>((S *)L.A, (S *)L.B, L.g, rho, u, L.aa);              \
        else                                                                                                 \
            k_init<27, S><<<grid, block, 0, L.stream>>>((S *)L.A, (S *)L.B, L.g, rho, u, L.aa);              \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    template <> cudaError_t launch_closure_features<S>(const Launch &L, const lbm_params &p, float *x)        \
    {                                                                                                        \
        if (L.aa) return launch_closure_features_aa<S>(L, p, x);                                             \
        return L.Q == 19 ? features_q<19, S, kPatAB>(L, p, x) : features_q<27, S, kPatAB>(L, p, x);          \
    }                                                                                                        \
    template <> cudaError_t launch_get_pop<S>(const Launch &L, int i, double *f)                             \
    {                                                                                                        \
        if (L.aa) return launch_get_pop_aa<S>(L, i, f);                                                      \
        return L.Q == 19 ? get_pop_q<19, S, kLayAB>(L, i, f) : get_pop_q<27, S, kLayAB>(L, i, f);            \
    }                                                                                                        \
    template <> cudaError_t launch_set_pop<S>(const Launch &L, int i, const double *f)                       \
    {                                                                                                        \
        dim3 grid, block;                                                                                    \
        node_launch_shape(L.g, grid, block);                                                                 \
        if (L.Q == 19)                                                                                       \
            k_set_pop<19, S><<<grid, block, 0, L.stream>>>((S *)L.A, (S *)L.B, L.g, i, f, L.aa);            \
        else                                                                                                 \
            k_set_pop<27, S><<<grid, block, 0, L.stream>>>((S *)L.A, (S *)L.B, L.g, i, f, L.aa);            \
        return cudaGetLastError();                                                                           \
    }

}  // namespace lbm
