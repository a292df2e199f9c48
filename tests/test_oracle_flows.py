"""Pins of the oracle's collide-and-stream step against closed forms,
invariants and brute force.

- streaming direction and bounce-back: a single marker population moves to
  x + c_i (mod n) and reflects off a solid neighbour (exact);
- mass and momentum invariants to round-off, and the momentum Guo's force
  adds per step (exactly rho g per node, for BGK, TRT and Smagorinsky);
- Smagorinsky at Cs = 0 and the learned closure with a zero output scale or
  a constant output reduce to BGK;
- the reductions against closed-form sums over populations with known
  moments (forced nodes, skipped walls, a non-finite node);
- the z-extruded 2D Taylor-Green vortex, an exact Navier-Stokes solution:
  amplitude ~ exp(-2 nu k^2 t), with second-order convergence of the rate;
- plane Poiseuille flow under the Guo body force between halfway bounce-back
  walls, exact at tau = 1/2 + sqrt(3)/4;
- plane Couette flow with Ladd's moving wall (linear, exact at any tau);
- the slit permeability (discrete sum of the parabola, tending to H^2/12);
- the eighth-order vorticity on the Taylor-Green field (closed-form
  enstrophy) and its h^8 convergence;
- the random-sphere medium against a brute-force numpy definition.
"""
import math

import numpy as np
import pytest

import lbm_inputs as inp
import oracle


def _marker(Q, shape, cell, i):
    f = np.zeros((Q,) + shape)
    f[(i,) + cell] = 1.0
    return f


@pytest.mark.parametrize("Q", [19, 27])
def test_marker_streams_to_x_plus_c(Q):
    c, _, _ = oracle.lattice(Q)
    shape = (5, 6, 7)
    nz, ny, nx = shape
    prob = oracle.Problem(Q, nx, ny, nz, tau=1.0, closure=oracle.STREAM_ONLY)
    for cell in [(0, 0, 0), (4, 5, 6), (2, 3, 1)]:
        for i in range(Q):
            g = prob.step(_marker(Q, shape, cell, i))
            z, y, x = cell
            dest = ((z + c[i, 2]) % nz, (y + c[i, 1]) % ny, (x + c[i, 0]) % nx)
            assert g[(i,) + dest] == 1.0
            assert np.count_nonzero(g) == 1


@pytest.mark.parametrize("Q", [19, 27])
def test_marker_bounces_off_solid_and_wall(Q):
    c, w, opp = oracle.lattice(Q)
    shape = (6, 6, 6)
    cell = (2, 2, 2)
    uw = np.array([0.03, -0.02, 0.01])
    for i in range(1, Q):
        z, y, x = cell
        nb = (z + c[i, 2], y + c[i, 1], x + c[i, 0])
        for tag in (oracle.SOLID, oracle.WALL0 + 1):
            tags = np.zeros(shape, dtype=np.uint8)
            tags[nb] = tag
            walls = [(0, 0, 0), tuple(uw)]
            prob = oracle.Problem(Q, 6, 6, 6, tags, tau=1.0, closure=oracle.STREAM_ONLY, wall_u=walls)
            g = prob.step(_marker(Q, shape, cell, i))
            expect = 1.0
            if tag != oracle.SOLID:
                expect += 6.0 * w[opp[i]] * float(c[opp[i]] @ uw)
            assert g[(opp[i],) + cell] == pytest.approx(expect, abs=1e-15)
            # the moving-wall term also acts on every other link into the wall
            assert np.count_nonzero(g[:, nb[0], nb[1], nb[2]]) == 0


def test_mass_and_momentum_invariants_periodic():
    Q = 19
    _, w, _ = oracle.lattice(Q)
    shape = (8, 9, 10)
    f = inp.random_populations(w, shape, seed=1, amplitude=0.2)
    prob = oracle.Problem(Q, 10, 9, 8, tau=0.6)
    c, _, _ = oracle.lattice(Q)
    m0 = f.sum()
    j0 = np.einsum("ia,izyx->a", c, f)
    g = prob.step(f, 200)
    assert abs(g.sum() - m0) / m0 <= 1e-12
    assert np.allclose(np.einsum("ia,izyx->a", c, g), j0, atol=1e-12)


@pytest.mark.parametrize("Q", [19, 27])
def test_mass_invariant_with_bounce_back_and_force(Q):
    _, w, _ = oracle.lattice(Q)
    shape = (8, 8, 8)
    tags = inp.random_tags(shape, seed=5, p_solid=0.2, p_forced=0.3, p_wall=0.0)
    f = inp.random_populations(w, shape, seed=2, amplitude=0.2)
    prob = oracle.Problem(Q, 8, 8, 8, tags, tau=0.7, force=(1e-4, -2e-4, 3e-5))
    fluid = tags <= oracle.FORCED
    m0 = f[:, fluid].sum()
    g = prob.step(f, 200)
    assert abs(g[:, fluid].sum() - m0) / m0 <= 1e-12
    # solid nodes are never updated
    assert np.array_equal(g[:, ~fluid], f[:, ~fluid])



@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("closure", [oracle.BGK, oracle.TRT, oracle.SMAGORINSKY])
def test_guo_force_adds_rho_g_per_step(Q, closure):
    """With Guo's source every collision adds exactly rho g to a node's
    momentum: the velocity shift u = (j + rho g / 2) / rho relaxes away
    omega rho g / 2 and the source's first moment adds (1 - omega / 2) rho g,
    for each relaxation rate (BGK, both TRT rates, a Smagorinsky tau per
    node).  On a periodic, fully forced box the total momentum is therefore
    J0 + n M g after n steps.  Dropping the half-force velocity shift, the
    (1 - omega/2) factor or a term of the source breaks it."""
    _, w, _ = oracle.lattice(Q)
    c, _, _ = oracle.lattice(Q)
    shape = (6, 7, 8)
    g_vec = np.array([2e-4, -1e-4, 5e-5])
    tags = np.full(shape, oracle.FORCED, np.uint8)
    f = inp.random_populations(w, shape, seed=3, amplitude=0.2)
    prob = oracle.Problem(Q, 8, 7, 6, tags, tau=0.62, force=tuple(g_vec), closure=closure, cs_smag=0.17)
    m0 = f.sum()
    j0 = np.einsum("ia,izyx->a", c, f)
    n = 25
    g = prob.step(f, n)
    assert abs(g.sum() - m0) / m0 <= 1e-12
    j = np.einsum("ia,izyx->a", c, g)
    np.testing.assert_allclose(j - j0, n * m0 * g_vec, rtol=1e-10, atol=0)


@pytest.mark.parametrize("Q", [19, 27])
def test_reduce_closed_form_sums(Q):
    """The reductions (Sec. 3.1's k = <|u|^2 / 2> over fluid nodes, with the
    mass, momentum, velocity sum, rho-weighted energy, max |u| and counts
    beside it) on populations with known moments: f_i = w_i rho (1 + 3 c_i.m)
    has sum rho and first moment rho m by the lattice's isotropy.  Plain
    fluid nodes take m = u.  Forced nodes hold post-collision populations,
    whose first moment is rho (u + g/2) for the velocity u their collision
    used, so m = u + g/2 must report u.  Solid and wall nodes hold NaN and
    are skipped; one fluid node holding a NaN is counted as fluid and as
    non-finite and left out of every sum."""
    c, w, _ = oracle.lattice(Q)
    shape = (5, 6, 7)
    rng = np.random.default_rng(11)
    tags = rng.choice(np.array([oracle.FLUID, oracle.FORCED, oracle.SOLID, oracle.WALL0 + 1], np.uint8),
                      size=shape, p=[0.4, 0.4, 0.1, 0.1])
    fluid = tags <= oracle.FORCED
    bad = tuple(int(i[0]) for i in np.nonzero(fluid))  # first fluid node: non-finite
    g_vec = np.array([3e-3, -2e-3, 1e-3])
    rho = rng.uniform(0.9, 1.1, shape)
    u = rng.uniform(-0.05, 0.05, (3,) + shape)
    m = u + np.where(tags == oracle.FORCED, 1.0, 0.0)[None] * (0.5 * g_vec)[:, None, None, None]
    f = w[:, None, None, None] * rho[None] * (1.0 + 3.0 * np.einsum("ia,azyx->izyx", c, m))
    f[:, ~fluid] = np.nan
    f[(3,) + bad] = np.nan
    prob = oracle.Problem(Q, 7, 6, 5, tags, tau=0.8, force=tuple(g_vec))
    red = prob.reduce(f)

    ok = fluid.copy()
    ok[bad] = False
    usq = np.sum(u * u, axis=0)
    assert red["n_fluid"] == int(fluid.sum()) and red["nonfinite"] == 1
    assert red["mass"] == pytest.approx(rho[ok].sum(), rel=1e-13)
    for a in range(3):
        assert red["mom"][a] == pytest.approx((rho * u[a])[ok].sum(), rel=1e-11, abs=1e-15)
        assert red["vel"][a] == pytest.approx(u[a][ok].sum(), rel=1e-11, abs=1e-15)
    assert red["ke"] == pytest.approx(0.5 * usq[ok].sum(), rel=1e-12)
    assert red["ke_rho"] == pytest.approx(0.5 * (rho * usq)[ok].sum(), rel=1e-12)
    assert red["umax"] == pytest.approx(np.sqrt(usq[ok].max()), rel=1e-12)

def _tgv_amplitude(u, n):
    """Projection of u_x on the mode -cos(kx) sin(ky)."""
    x = np.arange(n)
    k = 2 * np.pi / n
    mode = -np.cos(k * x)[None, None, :] * np.sin(k * x)[None, :, None]
    return float(np.sum(u[0] * mode) / np.sum(mode * mode * np.ones_like(u[0])))


def _tgv_rate(n, nz, tau, u0, steps, every):
    rho, u = inp.tgv2d(n, n, nz, u0)
    prob = oracle.Problem(19, n, n, nz, tau=tau)
    f = prob.init_equilibrium(rho, u)
    ts, amps = [], []
    for t in range(0, steps + 1, every):
        if t:
            f = prob.step(f, every)
        _, uu = prob.moments(f)
        ts.append(t)
        amps.append(_tgv_amplitude(uu, n))
    ts = np.array(ts[1:], float)
    la = np.log(np.array(amps[1:]))
    slope = np.polyfit(ts, la, 1)[0]
    return -slope, amps


def test_tgv2d_decay_rate_and_convergence():
    """Config: 32^3 D3Q19, tau = 0.8 (nu = 0.1), u0 = 0.02, 200 steps.
    Velocity amplitude decays as exp(-2 nu k^2 t); the rate error must drop
    roughly fourfold when the grid is refined twofold (diffusive scaling),
    which shows the remaining gap is discretisation error."""
    nu = (0.8 - 0.5) / 3.0
    rate32, amps = _tgv_rate(32, 32, 0.8, 0.02, 200, 20)
    exact32 = 2 * nu * (2 * np.pi / 32) ** 2
    err32 = abs(rate32 / exact32 - 1.0)
    assert err32 < 0.01
    # u(200)/u0 = exp(-200 * 2 nu k^2) = 0.2139 to the stated digits
    assert math.exp(-200 * exact32) == pytest.approx(0.2139, abs=1e-4)
    assert amps[-1] / amps[0] == pytest.approx(math.exp(-200 * exact32), rel=0.01)
    rate64, _ = _tgv_rate(64, 1, 0.8, 0.01, 800, 80)
    exact64 = 2 * nu * (2 * np.pi / 64) ** 2
    err64 = abs(rate64 / exact64 - 1.0)
    assert 2.5 < err32 / err64 < 6.0


def _channel_run(tau, H, g, steps, moving=None, wall_rho_local=False):
    ny = H + 2
    tags = inp.channel_tags(1, ny, 1, moving_top=moving is not None,
                            fluid_tag=oracle.FORCED if g else oracle.FLUID)
    walls = [tuple(moving)] if moving is not None else None
    prob = oracle.Problem(19, 1, ny, 1, tags, tau=tau, force=(g, 0.0, 0.0), wall_u=walls,
                          wall_rho_local=wall_rho_local)
    f = prob.init_equilibrium()
    f = prob.step(f, steps)
    _, u = prob.moments(f)
    return u[0, 0, :, 0], prob, f


def test_poiseuille_exact_at_magic_tau():
    """Halfway bounce-back walls at y = 1/2 and H + 1/2 (lattice rows 0 and
    H+1 solid): u(y) = g/(2 nu) (y - 1/2)(H + 1/2 - y).  With BGK the wall
    slip vanishes for (tau - 1/2)^2 = 3/16."""
    H, g = 16, 1e-5
    tau = 0.5 + math.sqrt(3.0) / 4.0
    nu = (tau - 0.5) / 3.0
    ux, _, _ = _channel_run(tau, H, g, 20000)
    y = np.arange(1, H + 1, dtype=float)
    exact = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    assert np.max(np.abs(ux[1:H + 1] - exact)) <= 1e-10 * exact.max()
    # away from the magic tau the profile carries a wall slip
    tau2 = 1.2
    nu2 = (tau2 - 0.5) / 3.0
    ux2, _, _ = _channel_run(tau2, H, g, 20000)
    exact2 = g / (2 * nu2) * (y - 0.5) * (H + 0.5 - y)
    slip = np.max(np.abs(ux2[1:H + 1] - exact2)) / exact2.max()
    assert 1e-4 < slip < 0.05


@pytest.mark.parametrize("tau", [0.7, 1.3])
def test_couette_linear_with_ladd_wall(tau):
    H, U = 12, 0.02
    ux, _, _ = _channel_run(tau, H, 0.0, 15000, moving=(U, 0.0, 0.0))
    y = np.arange(1, H + 1, dtype=float)
    exact = U * (y - 0.5) / H
    assert np.max(np.abs(ux[1:H + 1] - exact)) <= 1e-9 * U


@pytest.mark.parametrize("tau", [0.6, 1.3])
def test_couette_linear_with_local_density_wall(tau):
    """A tangential wall moving in its own plane: the wall terms of every
    node cancel in pairs (s = 0), the density stays 1, and Ladd's wall with
    the local density gives the same exact linear profile."""
    H, U = 12, 0.02
    ux, _, _ = _channel_run(tau, H, 0.0, 15000, moving=(U, 0.0, 0.0), wall_rho_local=True)
    y = np.arange(1, H + 1, dtype=float)
    exact = U * (y - 0.5) / H
    assert np.max(np.abs(ux[1:H + 1] - exact)) <= 1e-9 * U


def test_local_wall_density_is_the_node_density():
    """With the local-density wall, the density used in every wall term is
    the node's density after streaming.  Brute force on a tiny lattice of
    random tags and walls moving in all directions: rebuild each fluid node's
    pulled set from the pre-step state with rho_wall = the node's density
    after the step (collision conserves mass), and check that the set sums
    to that density; with rho_wall = 1 it does not."""
    Q = 19
    c, w, _ = oracle.lattice(Q)
    shape = (4, 5, 6)
    nz, ny, nx = shape
    tags = inp.random_tags(shape, seed=91, p_solid=0.1, p_forced=0.0, p_wall=0.25, n_walls=2)
    f0 = 1.04 * inp.random_populations(w, shape, seed=92, amplitude=0.05)
    walls = [(0.05, -0.03, 0.02), (-0.02, 0.04, 0.06)]
    opp = [0] + [i + 1 if i % 2 else i - 1 for i in range(1, Q)]
    checked = 0
    for local in (True, False):
        prob = oracle.Problem(Q, nx, ny, nz, tags, tau=0.7, wall_u=walls, wall_rho_local=local)
        rho1 = prob.step(f0, 1).sum(axis=0)
        worst = 0.0
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    if tags[z, y, x] >= oracle.SOLID:
                        continue
                    pulled, has_term = 0.0, False
                    for i in range(Q):
                        sz, sy, sx = (z - c[i, 2]) % nz, (y - c[i, 1]) % ny, (x - c[i, 0]) % nx
                        ts = tags[sz, sy, sx]
                        if ts < oracle.SOLID:
                            pulled += f0[i, sz, sy, sx]
                        else:
                            pulled += f0[opp[i], z, y, x]
                            if ts >= oracle.WALL0:
                                uw = walls[ts - oracle.WALL0]
                                pulled += 6.0 * w[i] * rho1[z, y, x] * float(np.dot(c[i], uw))
                                has_term = True
                    if has_term:
                        worst = max(worst, abs(pulled - rho1[z, y, x]))
                        checked += local
        if local:
            assert worst <= 1e-13
        else:
            assert worst > 1e-6
    assert checked > 20


def test_slit_permeability_closed_form():
    """k = u_mean nu / g with u_mean over all cells of the period (solid rows
    count as zero).  Averaging the parabola over the H node centres gives
    sum_s s (H - s) = H^3/6 + H/12 (midpoint rule plus its exact quadratic
    correction), so k = H (H^2 + 1/2) / (12 (H + 2)), which tends to the slit
    value H^2/12 times the pore fraction H/(H+2)."""
    H, g = 16, 1e-5
    tau = 0.5 + math.sqrt(3.0) / 4.0
    ux, prob, f = _channel_run(tau, H, g, 20000)
    red = prob.reduce(f)
    n_total = H + 2
    kperm = oracle.permeability(red["vel"][0] / n_total, tau, g)
    assert kperm == pytest.approx(H * (H * H + 0.5) / (12.0 * (H + 2)), rel=1e-9)


def test_enstrophy_of_taylor_green_field():
    """For u = u0 (sin X cos Y cos Z, -cos X sin Y cos Z, 0), X = 2 pi x / n,
    curl u averages to <|w|^2/2> = (3/8) (u0 k)^2, k = 2 pi / n."""
    n, u0 = 48, 0.04
    _, u = inp.tgv3d(n, u0)
    k = 2 * np.pi / n
    e, om = oracle.enstrophy(u, return_omega=True)
    assert e == pytest.approx(3.0 / 8.0 * (u0 * k) ** 2, rel=1e-9)
    # pointwise: w_z = 2 u0 k sin X sin Y cos Z
    x = np.arange(n) * k
    wz = 2 * u0 * k * np.sin(x)[None, None, :] * np.sin(x)[None, :, None] * np.cos(x)[:, None, None]
    assert np.max(np.abs(om[2] - wz)) < 1e-9 * u0 * k
    assert oracle.kinetic_energy_fields(u) == pytest.approx(u0 * u0 / 8.0, rel=1e-12)


def test_vorticity_is_eighth_order():
    errs = []
    for n in (16, 32):
        x = np.arange(n) * 2 * np.pi / n
        u = np.zeros((3, 4, n, 4))
        u[0] = np.sin(x)[None, :, None]  # u_x(y): w_z = -du_x/dy
        _, om = oracle.enstrophy(u, return_omega=True)
        exact = -np.cos(x) * 2 * np.pi / n
        errs.append(np.max(np.abs(om[2, 0, :, 0] - exact)) / (2 * np.pi / n))
    assert 200 < errs[0] / errs[1] < 300  # 2^8 = 256


def _brute_spheres(shape, centres, radii, target):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    solid = np.zeros(shape, bool)
    used = 0
    for (cx, cy, cz), r in zip(centres, radii):
        if (~solid).mean() <= target:
            break

        def mi(d, n):
            d = np.mod(d, n)
            return np.where(2 * d > n, d - n, d)
        d2 = mi(x - cx, nx) ** 2 + mi(y - cy, ny) ** 2 + mi(z - cz, nz) ** 2
        solid |= d2.astype(float) <= r * r
        used += 1
    return solid, used


@pytest.mark.parametrize("target", [0.0, 0.5, 0.8])
def test_spheres_match_brute_force(target):
    shape = (14, 18, 20)
    centres, radii = inp.sphere_list(shape, seed=42, rmin=2.0, rmax=4.0, count=40)
    tags, used, por = oracle.spheres(shape, centres, radii, target)
    solid, used_b = _brute_spheres(shape, centres, radii, target)
    assert used == used_b
    assert np.array_equal(tags == oracle.SOLID, solid)
    assert por == pytest.approx((~solid).mean(), abs=0)


def test_sphere_porosity_follows_boolean_model():
    """Independent overlapping grains: pore fraction ~ exp(-sum V_s / N)."""
    shape = (64, 64, 64)
    centres, radii = inp.sphere_list(shape, seed=2506, rmin=4.0, rmax=10.0, count=200)
    _, used, por = oracle.spheres(shape, centres, radii, 0.0)
    assert used == 200
    vol = 0.0
    for r in radii:
        R = int(math.ceil(r))
        d = np.arange(-R, R + 1)
        dz, dy, dx = np.meshgrid(d, d, d, indexing="ij")
        vol += np.count_nonzero((dx * dx + dy * dy + dz * dz).astype(float) <= r * r)
    expect = math.exp(-vol / np.prod(shape))
    assert por == pytest.approx(expect, abs=0.03)


def test_trt_reduces_to_bgk_when_both_rates_match():
    """Lambda = (tau - 1/2)^2 gives omega- = omega+: TRT is BGK."""
    Q = 19
    _, w, _ = oracle.lattice(Q)
    shape = (6, 7, 8)
    tags = inp.random_tags(shape, seed=2, p_solid=0.2, p_forced=0.3, p_wall=0.0)
    f0 = inp.random_populations(w, shape, seed=3, amplitude=0.1)
    tau = 0.73
    kw = dict(tau=tau, force=(1e-4, 2e-5, 0.0))
    bgk = oracle.Problem(Q, 8, 7, 6, tags, **kw).step(f0, 10)
    trt = oracle.Problem(Q, 8, 7, 6, tags, closure=oracle.TRT, trt_magic=(tau - 0.5) ** 2, **kw).step(f0, 10)
    assert np.max(np.abs(trt - bgk)) <= 1e-15



def test_relaxation_time_closures_reduce_to_bgk():
    """Special cases that reduce to plain BGK: Smagorinsky with Cs = 0, the
    learned closure with a zero output scale (dtau = 0), and the learned
    closure whose last layer has zero weights, so that its output is the
    constant dtau = scale * softplus(b3) at every node: BGK at tau + dtau."""
    Q = 19
    _, w, _ = oracle.lattice(Q)
    shape = (6, 7, 8)
    tags = inp.random_tags(shape, seed=4, p_solid=0.2, p_forced=0.3, p_wall=0.05, n_walls=1)
    f0 = inp.random_populations(w, shape, seed=5, amplitude=0.1)
    tau = 0.71
    kw = dict(force=(1e-4, 2e-5, 0.0), wall_u=[(0.01, 0.0, 0.0)])
    bgk = oracle.Problem(Q, 8, 7, 6, tags, tau=tau, **kw).step(f0, 10)
    smag0 = oracle.Problem(Q, 8, 7, 6, tags, tau=tau, closure=oracle.SMAGORINSKY, cs_smag=0.0, **kw).step(f0, 10)
    assert np.array_equal(smag0, bgk)

    P = inp.mlp_init(6)
    norm = np.concatenate([np.zeros(7), np.ones(7), [0.0, 0.0]])
    mlp0 = oracle.Problem(Q, 8, 7, 6, tags, tau=tau, closure=oracle.MLP, mlp_params=P, mlp_norm=norm, **kw)
    assert np.array_equal(mlp0.step(f0, 10), bgk)

    P = P.copy()
    P[-33:-1] = 0.0  # w3 = 0
    P[-1] = 0.4      # b3
    norm[14] = 0.05  # output scale
    dtau = oracle.mlp_dtau(P, norm, np.ones(7))
    assert dtau == pytest.approx(0.05 * math.log1p(math.exp(0.4)), rel=1e-15)
    const = oracle.Problem(Q, 8, 7, 6, tags, tau=tau, closure=oracle.MLP, mlp_params=P, mlp_norm=norm, **kw)
    shifted = oracle.Problem(Q, 8, 7, 6, tags, tau=tau + dtau, **kw)
    assert np.max(np.abs(const.step(f0, 10) - shifted.step(f0, 10))) <= 1e-15

@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_trt_magic_poiseuille_is_exact_at_any_tau(tau):
    """With Lambda = 3/16 halfway bounce-back is exact for the parabolic
    profile whatever tau is (unlike BGK, exact only at tau = 1/2 + sqrt(3)/4)."""
    H, g = 16, 1e-5
    ny = H + 2
    tags = inp.channel_tags(1, ny, 1)
    prob = oracle.Problem(19, 1, ny, 1, tags, tau=tau, force=(g, 0.0, 0.0), closure=oracle.TRT, trt_magic=3.0 / 16.0)
    f = prob.step(prob.init_equilibrium(), 30000)
    _, u = prob.moments(f)
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, H + 1, dtype=float)
    exact = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    assert np.max(np.abs(u[0, 0, 1:H + 1, 0] - exact)) <= 1e-9 * exact.max()
