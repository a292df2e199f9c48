/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the lattice Boltzmann hot path.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This file is the slow, obviously
 * correct restatement of the method against which the CUDA library is checked.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or helper with the
 * CUDA library: every constant below is written out here from the method's
 * definition.
 *
 * What is computed (Latt & Coreixas, "Multi-GPU Acceleration of PALABOS Fluid
 * Solver using C++ Standard Parallelism"):
 *   - D3Q19 / D3Q27 lattices (Sec. 3 uses D3Q19; D3Q27 is named as future
 *     work in Sec. 5), velocity order fixed by the oracle itself (the paper
 *     gives none).
 *   - Two-population collide-and-stream (Sec. 2.3.1): populations are pulled
 *     from the neighbours into local variables, collided, and written to a
 *     second array.  The stored state at step t is the post-collision set
 *     f*(t) at its own cell.
 *   - BGK collision with the second-order weighted equilibrium (Sec. 3.1).
 *   - Standard (halfway) bounce-back for solid nodes and Ladd's modified
 *     bounce-back for moving walls (Sec. 3 opening paragraph).
 *   - Cell behaviour chosen by an integer tag per node (Sec. 2.3.2).
 *   - Body force by Guo, Zheng & Shi (2002) on tagged cells (no text in the
 *     paper; the paper drives its porous flow by boundary conditions).
 *   - TRT collision (the paper's model for the porous rock of Sec. 3.3), two
 *     relaxation rates for the even and odd parts under i -> opp(i).
 *   - Smagorinsky eddy viscosity (cited in Sec. 2.3.2 as a per-node model
 *     with its own parameter) written in closed form for tau_eff.
 *   - A per-cell MLP relaxation-time closure (no counterpart in the paper).
 *   - Kinetic energy and enstrophy averages with an eighth-order centred
 *     vorticity (Sec. 3.1, the equation after the TGV initial condition).
 *   - A random-sphere porous medium standing in for the Berea volume
 *     (Sec. 3.3), with permeability k = u_mean * nu / g (the body-force form
 *     of the Sec. 3.3 permeability equation).
 *   - Storage-precision emulation: populations kept as f - w_i (the offset
 *     stripping of Skordos cited in Sec. 3) and rounded to FP32, FP16 or BF16
 *     after each step, round-to-nearest-even.
 *
 * Layouts: populations f[i][z][y][x] (x fastest, no padding, N = nx*ny*nz),
 * velocities u[a][z][y][x], tags uint8 [z][y][x].  Every boundary is
 * periodic in the indexing; walls are made by tags.
 *
 * Parity pins: tests/test_oracle_*.py check this file against closed forms
 * (lattice isotropy, equilibrium moments, plane Poiseuille and Couette flow,
 * the decay of a 2D Taylor-Green vortex, exact polynomial differentiation,
 * the momentum rho g that Guo's source adds per step, reductions of
 * populations with known moments), conservation invariants, special cases
 * that reduce to BGK (TRT with equal rates, Smagorinsky at Cs = 0, a closure
 * with zero or constant output) and brute force.  The MLP closure step
 * inside orc_step is pinned against the numpy FP64 MLP in oracle/mlp.py,
 * which is itself pinned by finite differences.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ----------------------------------------------------------------------- */
/* Tags (Sec. 2.3.2: one integer per node selects its behaviour).          */
/* ----------------------------------------------------------------------- */
enum {
    ORC_FLUID = 0,  /* BGK (or closure) fluid node                          */
    ORC_FORCED = 1, /* fluid node with the body force applied               */
    ORC_SOLID = 2,  /* resting wall, standard bounce-back                   */
    ORC_WALL0 = 3   /* ORC_WALL0 + k, k = 0..7: moving wall with velocity k */
};
#define ORC_NWALLS 8

static int is_wall_or_solid(unsigned char t) { return t >= ORC_SOLID && t < ORC_WALL0 + ORC_NWALLS; }

/* Closures. */
enum { ORC_BGK = 0, ORC_SMAGORINSKY = 1, ORC_MLP = 2, ORC_STREAM_ONLY = 3, ORC_TRT = 4 };

/* Storage emulation. */
enum { ORC_F64 = 0, ORC_F32 = 1, ORC_F16 = 2, ORC_BF16 = 3, ORC_F16_SCALED = 4 };

/* Number of MLP parameters: W1[32][7] b1[32] W2[32][32] b2[32] w3[32] b3. */
#define ORC_MLP_IN 7
#define ORC_MLP_H 32
#define ORC_MLP_NPARAM (ORC_MLP_H * ORC_MLP_IN + ORC_MLP_H + ORC_MLP_H * ORC_MLP_H + ORC_MLP_H + ORC_MLP_H + 1)

typedef struct {
    double tau;                      /* BGK relaxation time, > 1/2          */
    double force[3];                 /* body force g on ORC_FORCED cells    */
    int closure;                     /* ORC_BGK ... ORC_STREAM_ONLY         */
    double cs_smag;                  /* Smagorinsky constant                */
    double wall_u[ORC_NWALLS][3];    /* velocity of moving wall k           */
    double rho_wall;                 /* density in Ladd's wall term         */
    const double *mlp_params;        /* ORC_MLP_NPARAM values (closure 2)   */
    const double *mlp_norm;          /* mean[7], std[7], out_scale, unused  */
    int mlp_bf16;                    /* 1: round MLP operands to bf16       */
    double trt_magic;                /* TRT: Lambda = (tau+ - 1/2)(tau- - 1/2) */
    int wall_rho_local;              /* 1: rho_wall = the node's own density  */
} orc_params;

typedef struct {
    double mass;        /* sum of rho over fluid cells                      */
    double mom[3];      /* sum of rho*u                                     */
    double vel[3];      /* sum of u                                         */
    double ke;          /* sum of |u|^2 / 2                                 */
    double ke_rho;      /* sum of rho |u|^2 / 2                             */
    double umax;        /* max |u|                                          */
    long long n_fluid;  /* number of fluid cells                            */
    long long nonfinite;/* fluid cells with a non-finite rho or u           */
} orc_reduction;

/* ----------------------------------------------------------------------- */
/* Lattice descriptors.                                                     */
/* ----------------------------------------------------------------------- */
/* D3Q19: rest, 6 faces, 12 edges; D3Q27 adds the 8 corners.  Directions
 * come in opposite pairs (i, i+1) for odd i. */
static const int C27[27][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},
    {1, 1, 1},   {-1, -1, -1},{1, 1, -1},  {-1, -1, 1},
    {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};

/* Weight of a velocity from its squared length, per lattice. */
static double weight_of(int Q, const int *c)
{
    int n2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    if (Q == 19) {
        if (n2 == 0) return 1.0 / 3.0;
        if (n2 == 1) return 1.0 / 18.0;
        return 1.0 / 36.0;
    }
    if (n2 == 0) return 8.0 / 27.0;
    if (n2 == 1) return 2.0 / 27.0;
    if (n2 == 2) return 1.0 / 54.0;
    return 1.0 / 216.0;
}

static int opposite_of(int Q, int i)
{
    for (int k = 0; k < Q; ++k)
        if (C27[k][0] == -C27[i][0] && C27[k][1] == -C27[i][1] && C27[k][2] == -C27[i][2]) return k;
    return -1;
}

/* Exposes the tables (for the isotropy pins).  Returns 0, or -1 for a bad Q. */
int orc_lattice(int Q, int *c, double *w, int *opp)
{
    if (Q != 19 && Q != 27) return -1;
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = C27[i][a];
        w[i] = weight_of(Q, C27[i]);
        opp[i] = opposite_of(Q, i);
    }
    return 0;
}

/* Second-order weighted equilibrium, c_s^2 = 1/3 (Sec. 3.1):
 * f_eq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u). */
void orc_equilibrium(int Q, double rho, const double *u, double *feq)
{
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = C27[i][0] * u[0] + C27[i][1] * u[1] + C27[i][2] * u[2];
        feq[i] = weight_of(Q, C27[i]) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Guo forcing term F_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . G, G = rho g. */
static void guo_source(int Q, const double *u, const double *G, double *F)
{
    for (int i = 0; i < Q; ++i) {
        double cu = C27[i][0] * u[0] + C27[i][1] * u[1] + C27[i][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (3.0 * (C27[i][a] - u[a]) + 9.0 * cu * C27[i][a]) * G[a];
        F[i] = weight_of(Q, C27[i]) * s;
    }
}

/* Smagorinsky: nu_t = Cs^2 |S|, |S| = sqrt(2 S:S), with the strain taken
 * from the non-equilibrium stress, S = -Pi / (2 rho c_s^2 tau_eff).  Since
 * tau_eff = tau0 + 3 nu_t, this is a quadratic in tau_eff whose positive root
 * is tau_eff = (tau0 + sqrt(tau0^2 + 18 Cs^2 sqrt(2 Pi:Pi) / rho)) / 2. */
double orc_tau_smagorinsky(double tau0, double cs, double rho, const double *pi6)
{
    /* pi6 = (xx, yy, zz, xy, xz, yz); the off-diagonal terms count twice. */
    double pp = pi6[0] * pi6[0] + pi6[1] * pi6[1] + pi6[2] * pi6[2] +
                2.0 * (pi6[3] * pi6[3] + pi6[4] * pi6[4] + pi6[5] * pi6[5]);
    return 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * cs * cs * sqrt(2.0 * pp) / rho));
}

/* --- BF16 / FP16 / FP32 rounding, all round-to-nearest-even. ----------- */
static float to_bf16_float(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) == 0x7f800000u) {           /* inf or nan */
        if (b & 0x007fffffu) b |= 0x00400000u;         /* keep nan quiet */
        b &= 0xffff0000u;
    } else {
        uint32_t lsb = (b >> 16) & 1u;
        b += 0x7fffu + lsb;
        b &= 0xffff0000u;
    }
    float y;
    memcpy(&y, &b, 4);
    return y;
}

static double round_to(double h, int dtype)
{
    switch (dtype) {
    case ORC_F32: return (double)(float)h;
    case ORC_F16: return (double)(_Float16)(float)h;
    case ORC_BF16: return (double)to_bf16_float((float)h);
    /* FP16 of h times 2^12: a power-of-two scale is exact in binary floating
     * point, so only the half-precision rounding of the scaled value acts. */
    case ORC_F16_SCALED: return ldexp((double)(_Float16)(float)ldexp(h, 12), -12);
    default: return h;
    }
}

double orc_round_scalar(double h, int dtype) { return round_to(h, dtype); }

/* Keeps every population as w_i + round(f_i - w_i): the emulated storage of
 * offset-stripped populations in a narrower type. */
int orc_round_storage(int Q, long long N, double *f, int dtype)
{
    if (Q != 19 && Q != 27) return -1;
    for (int i = 0; i < Q; ++i) {
        double w = weight_of(Q, C27[i]);
        for (long long n = 0; n < N; ++n) f[(long long)i * N + n] = w + round_to(f[(long long)i * N + n] - w, dtype);
    }
    return 0;
}

/* --- MLP closure: 7 -> 32 -> SiLU -> 32 -> SiLU -> 1 -> softplus. ------- */
static double silu(double z) { return z / (1.0 + exp(-z)); }
static double softplus(double z) { return z > 30.0 ? z : log1p(exp(z)); }

/* Relaxation-time correction dtau >= 0 for one cell's features
 * x = (Pi_xx, Pi_yy, Pi_zz, Pi_xy, Pi_xz, Pi_yz, rho). */
double orc_mlp_dtau(const double *P, const double *norm, int bf16, const double *x)
{
    const double *W1 = P;
    const double *b1 = W1 + ORC_MLP_H * ORC_MLP_IN;
    const double *W2 = b1 + ORC_MLP_H;
    const double *b2 = W2 + ORC_MLP_H * ORC_MLP_H;
    const double *w3 = b2 + ORC_MLP_H;
    const double *b3 = w3 + ORC_MLP_H;
    double xn[ORC_MLP_IN], h1[ORC_MLP_H], h2[ORC_MLP_H];
    for (int k = 0; k < ORC_MLP_IN; ++k) {
        xn[k] = (x[k] - norm[k]) / norm[ORC_MLP_IN + k];
        if (bf16) xn[k] = round_to(xn[k], ORC_BF16);
    }
    for (int j = 0; j < ORC_MLP_H; ++j) {
        double s = 0.0;
        for (int k = 0; k < ORC_MLP_IN; ++k) {
            double w = bf16 ? round_to(W1[j * ORC_MLP_IN + k], ORC_BF16) : W1[j * ORC_MLP_IN + k];
            s += w * xn[k];
        }
        h1[j] = silu(s + b1[j]);
        if (bf16) h1[j] = round_to(h1[j], ORC_BF16);
    }
    for (int j = 0; j < ORC_MLP_H; ++j) {
        double s = 0.0;
        for (int k = 0; k < ORC_MLP_H; ++k) {
            double w = bf16 ? round_to(W2[j * ORC_MLP_H + k], ORC_BF16) : W2[j * ORC_MLP_H + k];
            s += w * h1[k];
        }
        h2[j] = silu(s + b2[j]);
    }
    double y = b3[0];
    for (int k = 0; k < ORC_MLP_H; ++k) y += w3[k] * h2[k];
    return norm[2 * ORC_MLP_IN] * softplus(y);
}

/* Non-equilibrium stress Pi_ab = sum_i c_ia c_ib (f_i - feq_i), components
 * (xx, yy, zz, xy, xz, yz). */
static void nonequilibrium_stress(int Q, const double *f, const double *feq, double *pi6)
{
    for (int k = 0; k < 6; ++k) pi6[k] = 0.0;
    for (int i = 0; i < Q; ++i) {
        double d = f[i] - feq[i];
        const int *c = C27[i];
        pi6[0] += c[0] * c[0] * d;
        pi6[1] += c[1] * c[1] * d;
        pi6[2] += c[2] * c[2] * d;
        pi6[3] += c[0] * c[1] * d;
        pi6[4] += c[0] * c[2] * d;
        pi6[5] += c[1] * c[2] * d;
    }
}

/* --- One cell's collision (Sec. 3.1 BGK, Guo force, closures). ---------- */
static void collide(int Q, const orc_params *p, int forced, const double *f, double *fout)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += C27[i][a] * f[i];
    }
    double G[3] = {0.0, 0.0, 0.0};
    if (forced)
        for (int a = 0; a < 3; ++a) G[a] = rho * p->force[a];
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * G[a]) / rho;

    double feq[27], F[27];
    orc_equilibrium(Q, rho, u, feq);
    guo_source(Q, u, G, F);

    double tau = p->tau;
    if (p->closure == ORC_SMAGORINSKY || p->closure == ORC_MLP) {
        double pi6[6];
        nonequilibrium_stress(Q, f, feq, pi6);
        if (p->closure == ORC_SMAGORINSKY) {
            tau = orc_tau_smagorinsky(p->tau, p->cs_smag, rho, pi6);
        } else {
            double x[7] = {pi6[0], pi6[1], pi6[2], pi6[3], pi6[4], pi6[5], rho};
            tau = p->tau + orc_mlp_dtau(p->mlp_params, p->mlp_norm, p->mlp_bf16, x);
        }
    }
    double omega = 1.0 / tau;
    if (p->closure == ORC_TRT) {
        /* Two relaxation times (Ginzburg): the parts of f, f_eq and F that are
         * even and odd under i -> opp(i) relax with omega+ = 1/tau and
         * omega- from the magic parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2). */
        const double wp = omega;
        const double wm = 1.0 / (0.5 + p->trt_magic / (tau - 0.5));
        for (int i = 0; i < Q; ++i) {
            const int o = opposite_of(Q, i);
            const double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
            const double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
            const double Fp = 0.5 * (F[i] + F[o]), Fm = 0.5 * (F[i] - F[o]);
            fout[i] = f[i] - wp * (fp - ep) - wm * (fm - em) + (1.0 - 0.5 * wp) * Fp + (1.0 - 0.5 * wm) * Fm;
        }
        return;
    }
    for (int i = 0; i < Q; ++i) fout[i] = f[i] - omega * (f[i] - feq[i]) + (1.0 - 0.5 * omega) * F[i];
}

static long long wrap(long long a, long long n) { return ((a % n) + n) % n; }

/* The pulled (pre-collision) set of fluid node (x, y, z), Sec. 2.3.1-2.3.2:
 *   f_i(x) = f*_i(x - c_i) if the source node is fluid,
 *          = f*_{opp i}(x)                                    if it is SOLID,
 *          = f*_{opp i}(x) + 6 w_i rho_wall (c_i . u_wall_k)   if it is WALL_k,
 * with rho_wall = p->rho_wall, or, with wall_rho_local, the node's own
 * density after streaming, rho = sum_i f_i(x).  The wall terms are linear in
 * it: rho = rho0 + rho s, with rho0 the sum without them and s the sum of
 * 6 w_i (c_i . u_wall_k) over the node's wall links, so rho = rho0 / (1 - s). */
static void pull_node(int Q, long long nx, long long ny, long long nz, const unsigned char *tags, const orc_params *p,
                      const double *fin, long long x, long long y, long long z, double *f)
{
    const long long N = nx * ny * nz;
    const long long n = x + nx * (y + ny * z);
    double t_wall[27];
    double s_wall = 0.0;
    for (int i = 0; i < Q; ++i) {
        t_wall[i] = 0.0;
        const long long xs = wrap(x - C27[i][0], nx);
        const long long ys = wrap(y - C27[i][1], ny);
        const long long zs = wrap(z - C27[i][2], nz);
        const long long s = xs + nx * (ys + ny * zs);
        const unsigned char ts = tags ? tags[s] : ORC_FLUID;
        const int o = opposite_of(Q, i);
        if (ts == ORC_SOLID) {
            f[i] = fin[o * N + n];
        } else if (ts >= ORC_WALL0 && ts < ORC_WALL0 + ORC_NWALLS) {
            const double *uw = p->wall_u[ts - ORC_WALL0];
            const double cu = C27[i][0] * uw[0] + C27[i][1] * uw[1] + C27[i][2] * uw[2];
            t_wall[i] = 6.0 * weight_of(Q, C27[i]) * cu;
            s_wall += t_wall[i];
            f[i] = fin[o * N + n];
        } else {
            f[i] = fin[i * N + s];
        }
    }
    double rho_w = p->rho_wall;
    if (p->wall_rho_local) {
        double rho0 = 0.0;
        for (int i = 0; i < Q; ++i) rho0 += f[i];
        rho_w = rho0 / (1.0 - s_wall);
    }
    for (int i = 0; i < Q; ++i) f[i] += rho_w * t_wall[i];
}

/* Worker threads of the z loops below (1 when built without OpenMP).  The
 * test-suite uses the plain build; the timed CPU baseline may use a build
 * with OpenMP, where each node's arithmetic is the same, so the populations
 * are the same bit for bit.  Returns the number of threads now in use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* One collide-and-stream step in pull form (Sec. 2.3.1-2.3.2): every fluid
 * node pulls its pre-collision set (pull_node), collides, and its
 * post-collision set is written to fout.  Solid and wall nodes are not
 * updated (fout = fin there).  Nodes are independent within a step: with
 * OpenMP the z planes are shared out among threads. */
int orc_step(int Q, int nx, int ny, int nz, const unsigned char *tags, const orc_params *p, const double *fin,
             double *fout)
{
    if (Q != 19 && Q != 27) return -1;
    if (nx < 1 || ny < 1 || nz < 1 || !(p->tau > 0.5)) return -1;
    if (p->closure == ORC_TRT && !(p->trt_magic > 0.0)) return -1;
    const long long N = (long long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long long z = 0; z < nz; ++z)
        for (long long y = 0; y < ny; ++y)
            for (long long x = 0; x < nx; ++x) {
                const long long n = x + nx * (y + ny * z);
                const unsigned char t = tags ? tags[n] : ORC_FLUID;
                if (is_wall_or_solid(t)) {
                    for (int i = 0; i < Q; ++i) fout[i * N + n] = fin[i * N + n];
                    continue;
                }
                double f[27];
                pull_node(Q, nx, ny, nz, tags, p, fin, x, y, z, f);
                double fo[27];
                if (p->closure == ORC_STREAM_ONLY) {
                    for (int i = 0; i < Q; ++i) fo[i] = f[i];
                } else {
                    collide(Q, p, t == ORC_FORCED, f, fo);
                }
                for (int i = 0; i < Q; ++i) fout[i * N + n] = fo[i];
            }
    return 0;
}

/* Closure features of every node for the step that would follow: the
 * pulled set's non-equilibrium stress Pi^neq (xx, yy, zz, xy, xz, yz) and
 * density rho, with u from the pulled set (Guo's half-force shift on forced
 * nodes), x[n][7] for node n = x + nx (y + ny z); zeros on solid and wall
 * nodes.  These are the inputs of the learned closure (see orc_mlp_dtau). */
int orc_closure_features(int Q, int nx, int ny, int nz, const unsigned char *tags, const orc_params *p,
                         const double *fin, double *xout)
{
    if (Q != 19 && Q != 27) return -1;
    for (long long z = 0; z < nz; ++z)
        for (long long y = 0; y < ny; ++y)
            for (long long x = 0; x < nx; ++x) {
                const long long n = x + (long long)nx * (y + (long long)ny * z);
                const unsigned char t = tags ? tags[n] : ORC_FLUID;
                double *out = xout + 7 * n;
                for (int k = 0; k < 7; ++k) out[k] = 0.0;
                if (is_wall_or_solid(t)) continue;
                double f[27], feq[27], u[3], j[3] = {0.0, 0.0, 0.0}, rho = 0.0;
                pull_node(Q, nx, ny, nz, tags, p, fin, x, y, z, f);
                for (int i = 0; i < Q; ++i) {
                    rho += f[i];
                    for (int a = 0; a < 3; ++a) j[a] += C27[i][a] * f[i];
                }
                for (int a = 0; a < 3; ++a)
                    u[a] = (j[a] + (t == ORC_FORCED ? 0.5 * rho * p->force[a] : 0.0)) / rho;
                orc_equilibrium(Q, rho, u, feq);
                nonequilibrium_stress(Q, f, feq, out);
                out[6] = rho;
            }
    return 0;
}

/* Equilibrium initial state: f*_i(x) = f_eq_i(rho(x), u(x)).  rho may be NULL
 * (uniform rho0 = 1), u may be NULL (rest). */
int orc_init_equilibrium(int Q, int nx, int ny, int nz, const double *rho, const double *u, double *f)
{
    if (Q != 19 && Q != 27) return -1;
    const long long N = (long long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double r = rho ? rho[n] : 1.0;
        double v[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int a = 0; a < 3; ++a) v[a] = u[a * N + n];
        double feq[27];
        orc_equilibrium(Q, r, v, feq);
        for (int i = 0; i < Q; ++i) f[i * N + n] = feq[i];
    }
    return 0;
}

/* Density and velocity of every cell from the stored post-collision set.
 * Mass and momentum are collision invariants, and the Guo source adds
 * rho*g to the momentum of a forced cell, so the velocity that the
 * collision used is u = (sum_i c_i f*_i - rho g / 2) / rho.  Solid and wall
 * cells report rho = 0 and u = 0. */
int orc_moments(int Q, int nx, int ny, int nz, const unsigned char *tags, const orc_params *p, const double *f,
                double *rho, double *u)
{
    if (Q != 19 && Q != 27) return -1;
    const long long N = (long long)nx * ny * nz;
    for (long long n = 0; n < N; ++n) {
        const unsigned char t = tags ? tags[n] : ORC_FLUID;
        if (is_wall_or_solid(t)) {
            rho[n] = 0.0;
            for (int a = 0; a < 3; ++a) u[a * N + n] = 0.0;
            continue;
        }
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            r += f[i * N + n];
            for (int a = 0; a < 3; ++a) j[a] += C27[i][a] * f[i * N + n];
        }
        if (t == ORC_FORCED && p)
            for (int a = 0; a < 3; ++a) j[a] -= 0.5 * r * p->force[a];
        rho[n] = r;
        for (int a = 0; a < 3; ++a) u[a * N + n] = j[a] / r;
    }
    return 0;
}

/* Domain sums over fluid cells (the transform-reduce of Sec. 2.2, with the
 * kinetic energy k of Sec. 3.1 as its main use). */
int orc_reduce(int Q, int nx, int ny, int nz, const unsigned char *tags, const orc_params *p, const double *f,
               orc_reduction *out)
{
    if (Q != 19 && Q != 27) return -1;
    memset(out, 0, sizeof(*out));
    const long long N = (long long)nx * ny * nz;
    for (long long n = 0; n < N; ++n) {
        const unsigned char t = tags ? tags[n] : ORC_FLUID;
        if (is_wall_or_solid(t)) continue;
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            r += f[i * N + n];
            for (int a = 0; a < 3; ++a) j[a] += C27[i][a] * f[i * N + n];
        }
        if (t == ORC_FORCED && p)
            for (int a = 0; a < 3; ++a) j[a] -= 0.5 * r * p->force[a];
        double v[3] = {j[0] / r, j[1] / r, j[2] / r};
        double usq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        out->n_fluid += 1;
        if (!isfinite(r) || !isfinite(usq)) {
            out->nonfinite += 1;
            continue;
        }
        out->mass += r;
        for (int a = 0; a < 3; ++a) {
            out->mom[a] += r * v[a];
            out->vel[a] += v[a];
        }
        out->ke += 0.5 * usq;
        out->ke_rho += 0.5 * r * usq;
        if (sqrt(usq) > out->umax) out->umax = sqrt(usq);
    }
    return 0;
}

/* Eighth-order centred first derivative on a periodic line of unit spacing:
 * d/dx f(x) ~ sum_{m=1..4} a_m (f(x+m) - f(x-m)), a = 4/5, -1/5, 4/105,
 * -1/280 (exact for polynomials up to degree 8). */
static const double FD8[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};

static double ddx(const double *q, int nx, int ny, int nz, long long x, long long y, long long z, int axis)
{
    double s = 0.0;
    for (int m = 1; m <= 4; ++m) {
        long long xp = x, yp = y, zp = z, xm = x, ym = y, zm = z;
        if (axis == 0) { xp = wrap(x + m, nx); xm = wrap(x - m, nx); }
        if (axis == 1) { yp = wrap(y + m, ny); ym = wrap(y - m, ny); }
        if (axis == 2) { zp = wrap(z + m, nz); zm = wrap(z - m, nz); }
        s += FD8[m - 1] * (q[xp + nx * (yp + ny * zp)] - q[xm + nx * (ym + ny * zm)]);
    }
    return s;
}

/* Vorticity omega = curl u (u[3][N], periodic) and the enstrophy average
 * (1/N) sum |omega|^2 / 2 (Sec. 3.1).  omega may be NULL. */
double orc_enstrophy(int nx, int ny, int nz, const double *u, double *omega)
{
    const long long N = (long long)nx * ny * nz;
    const double *ux = u, *uy = u + N, *uz = u + 2 * N;
    double acc = 0.0;
    for (long long z = 0; z < nz; ++z)
        for (long long y = 0; y < ny; ++y)
            for (long long x = 0; x < nx; ++x) {
                long long n = x + nx * (y + ny * z);
                double wx = ddx(uz, nx, ny, nz, x, y, z, 1) - ddx(uy, nx, ny, nz, x, y, z, 2);
                double wy = ddx(ux, nx, ny, nz, x, y, z, 2) - ddx(uz, nx, ny, nz, x, y, z, 0);
                double wz = ddx(uy, nx, ny, nz, x, y, z, 0) - ddx(ux, nx, ny, nz, x, y, z, 1);
                if (omega) {
                    omega[n] = wx;
                    omega[N + n] = wy;
                    omega[2 * N + n] = wz;
                }
                acc += 0.5 * (wx * wx + wy * wy + wz * wz);
            }
    return acc / (double)N;
}

/* Random overlapping spheres (the porous stand-in of Sec. 3.3).  Spheres are
 * added in the given order; a voxel v becomes solid when, for some sphere
 * (c, r), the squared minimum-image distance |v - c|^2 (an integer, compared
 * as a double) is <= r*r.  Spheres are added until the pore fraction is
 * <= target, or until the list is exhausted.  Solid voxels get solid_tag,
 * the others pore_tag.  Returns the number of spheres used. */
static long long min_image(long long d, long long n)
{
    d = wrap(d, n);
    if (2 * d > n) d -= n;
    return d;
}

int orc_spheres(int nx, int ny, int nz, const int *centres, const double *radii, int nsph, double target,
                unsigned char solid_tag, unsigned char pore_tag, unsigned char *tags, double *porosity_out)
{
    const long long N = (long long)nx * ny * nz;
    for (long long n = 0; n < N; ++n) tags[n] = pore_tag;
    long long nsolid = 0;
    int used = 0;
    for (int s = 0; s < nsph; ++s) {
        if ((double)(N - nsolid) / (double)N <= target) break;
        const long long cx = centres[3 * s], cy = centres[3 * s + 1], cz = centres[3 * s + 2];
        const double r2 = radii[s] * radii[s];
        const long long R = (long long)ceil(radii[s]);
        /* visit every voxel of the lattice whose minimum-image offset lies in
         * the bounding cube; the offsets are distinct voxels when 2R+1 <= n. */
        for (long long dz = -R; dz <= R; ++dz)
            for (long long dy = -R; dy <= R; ++dy)
                for (long long dx = -R; dx <= R; ++dx) {
                    const long long x = wrap(cx + dx, nx), y = wrap(cy + dy, ny), z = wrap(cz + dz, nz);
                    const long long ex = min_image(x - cx, nx), ey = min_image(y - cy, ny), ez = min_image(z - cz, nz);
                    if (ex != dx || ey != dy || ez != dz) continue; /* reached by a shorter offset */
                    const double d2 = (double)(ex * ex + ey * ey + ez * ez);
                    if (d2 <= r2) {
                        const long long n = x + nx * (y + ny * z);
                        if (tags[n] != solid_tag) {
                            tags[n] = solid_tag;
                            ++nsolid;
                        }
                    }
                }
        used = s + 1;
    }
    if (porosity_out) *porosity_out = (double)(N - nsolid) / (double)N;
    return used;
}
