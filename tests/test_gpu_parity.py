"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
- FP64 storage: max relative population difference <= 1e-12 after 200 steps;
- FP32 storage: velocity relative L2 <= 1e-5 against the FP64 oracle;
- FP16 / BF16 shifted storage: one step from a storage-representable state
  agrees with the oracle's FP64 step rounded to the same type except where
  FP32 arithmetic flips a rounding: every value within one unit in the last
  place of the storage type plus the absolute FP32 arithmetic error on the
  O(0.1) intermediates (1e-8, which matters only for values near zero, where
  a BF16 ulp is tiny), and at least 99% of them identical;
- pure streaming (closure STREAM_ONLY) and tags: bit-exact.
Sizes span several thread blocks with ragged x, y and z tails.
"""
import math

import numpy as np
import pytest
import torch

import lbm_inputs as inp
import oracle
from paper_2506_09242_gb300 import lbm

pytestmark = pytest.mark.gpu

DT = {"f64": oracle.F64, "f32": oracle.F32, "f16": oracle.F16, "bf16": oracle.BF16, "f16s": oracle.F16_SCALED}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2506_09242_gb300 import _build
    _build.build()
    lbm.load()


def make(shape, Q=19, dtype="f64", tags=None, **params):
    nz, ny, nx = shape
    lat = lbm.Lattice(nx, ny, nz, Q, dtype)
    if tags is not None:
        lat.set_tags(tags)
    lat.set_params(**params)
    return lat


def oracle_problem(shape, Q=19, tags=None, **params):
    nz, ny, nx = shape
    p = dict(params)
    return oracle.Problem(Q, nx, ny, nz, tags, **p)


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


# ---------------------------------------------------------------------------
# FP64: populations to 1e-12 relative
# ---------------------------------------------------------------------------
def test_f64_tgv2d_config_200_steps():
    """D3Q19, FP64, periodic 32^3, z-extruded 2D TGV u0 = 0.02, tau = 0.8."""
    shape = (32, 32, 32)
    rho, u = inp.tgv2d(32, 32, 32, 0.02)
    lat = make(shape, tau=0.8)
    lat.init_equilibrium(rho, u)
    lat.step(200)
    f = lat.get_populations()
    prob = oracle_problem(shape, tau=0.8)
    g = prob.step(prob.init_equilibrium(rho, u), 200)
    assert max_rel(f, g) <= 1e-12
    red = lat.reduce()
    m0 = float(np.sum(rho))
    assert abs(red["mass"] - m0) / m0 <= 1e-12
    ref = prob.reduce(g)
    assert red["ke"] == pytest.approx(ref["ke"], rel=1e-12)
    assert lat.step_count() == 200
    lat.close()


# Wall fractions below and above the 30% at which the step switches from the
# dense sweep to the fluid-node list.
WALL_MIX = {"dense": dict(p_solid=0.15, p_forced=0.3, p_wall=0.06),
            "list": dict(p_solid=0.45, p_forced=0.2, p_wall=0.1)}


@pytest.mark.parametrize("mix", ["dense", "list"])
@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("closure", [lbm.CLOSURE_BGK, lbm.CLOSURE_SMAGORINSKY, lbm.CLOSURE_TRT])
def test_f64_tags_walls_force_ragged(Q, closure, mix):
    shape = (11, 13, 45)  # nx = 45: one full 32-block and a ragged tail; odd y, z
    tags = inp.random_tags(shape, seed=9, n_walls=3, **WALL_MIX[mix])
    walls = [(0.01, 0.0, 0.0), (0.0, -0.02, 0.005), (0.003, 0.004, -0.006)]
    params = dict(tau=0.62, force=(2e-4, -1e-4, 5e-5), closure=closure, cs_smag=0.17, wall_u=walls)
    rho, u = inp.random_velocity_field(shape, seed=4, amplitude=0.04)
    lat = make(shape, Q, "f64", tags, **params)
    lat.init_equilibrium(rho, u)
    lat.step(60)
    f = lat.get_populations()
    prob = oracle_problem(shape, Q, tags, **params)
    g = prob.step(prob.init_equilibrium(rho, u), 60)
    assert max_rel(f, g) <= 1e-12
    # reductions and moments of the same state
    red, ref = lat.reduce(), prob.reduce(g)
    assert red["n_fluid"] == ref["n_fluid"]
    assert red["mass"] == pytest.approx(ref["mass"], rel=1e-13)
    for key in ("ke", "ke_rho", "umax"):
        assert red[key] == pytest.approx(ref[key], rel=1e-11)
    for a in range(3):
        assert red["mom"][a] == pytest.approx(ref["mom"][a], rel=1e-10, abs=1e-15)
        assert red["vel"][a] == pytest.approx(ref["vel"][a], rel=1e-10, abs=1e-15)
    r_gpu, u_gpu = lat.moments()
    r_ref, u_ref = prob.moments(g)
    assert np.max(np.abs(r_gpu - r_ref)) <= 1e-13
    assert np.max(np.abs(u_gpu - u_ref)) <= 1e-13
    lat.close()


@pytest.mark.parametrize("mix", ["dense", "list"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("Q", [19, 27])
def test_f64_local_density_wall(Q, pattern, mix):
    """Ladd's wall with the node's own density (wall_rho_local): walls moving
    in all directions, forced nodes, dense and compact storage, both
    streaming patterns, against the FP64 oracle."""
    shape = (7, 9, 21)
    tags = inp.random_tags(shape, seed=93, n_walls=3, **WALL_MIX[mix])
    walls = [(0.03, -0.02, 0.01), (-0.01, 0.02, 0.04), (0.0, 0.0, -0.03)]
    params = dict(tau=0.72, force=(1e-4, 0.0, -2e-4), wall_u=walls, wall_rho_local=True)
    rho, u = inp.random_velocity_field(shape, seed=94, amplitude=0.04)
    nz, ny, nx = shape
    lat = lbm.Lattice(nx, ny, nz, Q, "f64", pattern=pattern)
    lat.set_tags(tags)
    lat.set_params(**params)
    lat.init_equilibrium(rho, u)
    prob = oracle_problem(shape, Q, tags, **params)
    g = prob.init_equilibrium(rho, u)
    for n in (3, 6):
        lat.step(n)
        g = prob.step(g, n)
        assert max_rel(lat.get_populations(), g) <= 1e-12
    ref = oracle_problem(shape, Q, tags, **dict(params, wall_rho_local=False))
    assert max_rel(ref.step(ref.init_equilibrium(rho, u), 9), g) > 1e-9  # the variant changes the flow
    lat.close()


@pytest.mark.parametrize("p_solid", [0.2, 0.6])
@pytest.mark.parametrize("Q", [19, 27])
def test_stream_only_is_bit_exact_with_bounce_back(Q, p_solid):
    shape = (9, 10, 37)
    _, w, _ = oracle.lattice(Q)
    tags = inp.random_tags(shape, seed=3, p_solid=p_solid, p_forced=0.0, p_wall=0.0)
    f0 = inp.random_populations(w, shape, seed=8, amplitude=0.3)
    lat = make(shape, Q, "f64", tags, tau=1.0, closure=lbm.CLOSURE_STREAM_ONLY)
    lat.set_populations(f0)
    # the library stores f - w: use values whose shift is exact in FP64
    f_in = lat.get_populations()
    lat.step(3)
    f = lat.get_populations()
    prob = oracle_problem(shape, Q, tags, tau=1.0, closure=oracle.STREAM_ONLY)
    g = prob.step(f_in, 3)
    assert np.array_equal(f, g)
    lat.close()


def test_compact_and_dense_paths_hand_over_the_state():
    """Mostly-wall tags step the compact fluid-only copy; accessors and a tag
    change in mid-run must see the state of every step taken so far."""
    shape = (9, 11, 40)
    Q = 19
    tags_a = inp.random_tags(shape, seed=31, **WALL_MIX["list"])
    tags_b = inp.random_tags(shape, seed=32, **WALL_MIX["dense"])
    tags_b[tags_a >= oracle.SOLID] = tags_a[tags_a >= oracle.SOLID]  # keep the walls, open some pores
    walls = [(0.01, 0.0, 0.0), (0.0, -0.01, 0.0), (0.0, 0.0, 0.02)]
    params = dict(tau=0.65, force=(1e-4, 0.0, 0.0), wall_u=walls)
    rho, u = inp.random_velocity_field(shape, seed=33, amplitude=0.04)
    lat = make(shape, Q, "f64", tags_a, **params)
    lat.init_equilibrium(rho, u)
    pa = oracle_problem(shape, Q, tags_a, **params)
    pb = oracle_problem(shape, Q, tags_b, **params)
    g = pa.init_equilibrium(rho, u)
    lat.step(5)
    g = pa.step(g, 5)
    assert lat.reduce()["mass"] == pytest.approx(pa.reduce(g)["mass"], rel=1e-13)
    lat.step(4)
    g = pa.step(g, 4)
    assert max_rel(lat.get_populations(), g) <= 1e-12
    lat.step(3)
    g = pa.step(g, 3)
    lat.set_tags(tags_b)  # mostly fluid now: dense sweep from here
    lat.step(6)
    g = pb.step(g, 6)
    assert max_rel(lat.get_populations(), g) <= 1e-12
    lat.set_tags(tags_a)  # and back to the compact copy
    lat.step(2)
    g = pa.step(g, 2)
    _, ug = lat.moments()
    _, ur = pa.moments(g)
    assert np.max(np.abs(ug - ur)) <= 1e-13
    lat.close()


def test_trt_magic_poiseuille_on_the_gpu():
    """TRT with Lambda = 3/16: the parabolic channel profile is exact at a tau
    where BGK has a wall slip (FP64 storage)."""
    H, g, tau = 16, 1e-5, 1.7
    shape = (1, H + 2, 32)
    tags = inp.channel_tags(32, H + 2, 1)
    lat = make(shape, 19, "f64", tags, tau=tau, force=(g, 0.0, 0.0), closure=lbm.CLOSURE_TRT)
    lat.init_equilibrium()
    lat.step(30000)
    _, u = lat.moments()
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, H + 1, dtype=float)
    exact = g / (2 * nu) * (y - 0.5) * (H + 0.5 - y)
    assert np.max(np.abs(u[0, 0, 1:H + 1, :] - exact[:, None])) <= 1e-9 * exact.max()
    lat.close()


@pytest.mark.parametrize("mix", ["periodic", "dense", "list"])
def test_graph_replay_is_bit_identical(mix):
    """lbm_step replays pairs of steps as CUDA graphs; the result must be the
    one of one launch per step, across odd counts and a parameter change."""
    shape = (10, 9, 70)
    tags = None if mix == "periodic" else inp.random_tags(shape, seed=41, n_walls=2, **WALL_MIX[mix])
    rho, u = inp.random_velocity_field(shape, seed=42, amplitude=0.04)
    out = []
    for graphs in (False, True):
        lat = make(shape, 19, "f32", tags, tau=0.7, force=(1e-4, 0, 0), wall_u=[(0.01, 0, 0), (0, 0.01, 0)])
        lat.use_graphs(graphs)
        lat.init_equilibrium(rho, u)
        for n in (37, 1, 8):
            lat.step(n)
        lat.set_params(0.62, force=(1e-4, 0, 0), wall_u=[(0.01, 0, 0), (0, 0.01, 0)])
        lat.step(9)
        assert lat.step_count() == 55
        out.append(lat.get_populations())
        lat.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 1), (5, 1, 2), (2, 2, 3)])
@pytest.mark.parametrize("Q", [19, 27])
def test_degenerate_lattices(shape, Q):
    """Lattices of one to a few nodes per axis: every neighbour wraps onto the
    node itself or its row, in the scalar, tag and reduction kernels."""
    _, w, _ = oracle.lattice(Q)
    f0 = inp.random_populations(w, shape, seed=51, amplitude=0.1)
    tags = inp.random_tags(shape, seed=52, p_solid=0.2, p_forced=0.3, p_wall=0.1, n_walls=1)
    tags.flat[0] = oracle.FORCED  # keep at least one fluid node
    params = dict(tau=0.8, force=(1e-3, -1e-3, 5e-4), wall_u=[(0.02, 0.01, 0.0)])
    for t in (None, tags):
        lat = make(shape, Q, "f64", t, **params)
        lat.set_populations(f0)
        lat.step(10)
        prob = oracle_problem(shape, Q, t, **params)
        g = prob.step(f0, 10)
        assert max_rel(lat.get_populations(), g) <= 1e-12
        red, ref = lat.reduce(), prob.reduce(g)
        assert red["n_fluid"] == ref["n_fluid"]
        assert red["mass"] == pytest.approx(ref["mass"], rel=1e-13)
        lat.close()


@pytest.mark.parametrize("kind", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("mix", ["periodic", "dense", "list"])
@pytest.mark.parametrize("closure", [lbm.CLOSURE_BGK, lbm.CLOSURE_TRT])
def test_fused_step_reduce_matches_separate_passes(kind, mix, closure):
    """lbm_step_reduce computes the reduction inside the last step: the state
    must be bit-identical to lbm_step and the counts exact.  FP32/FP64 take
    the collision's own density and velocity (equal to the stored moments up
    to rounding), 16-bit storage the stored values (the same per-node moments
    as lbm_reduce); the sums differ in their grouping."""
    shape = (12, 33, 96)  # many blocks: partials pass through both combine stages
    tags = None if mix == "periodic" else inp.random_tags(shape, seed=61, n_walls=2, **WALL_MIX[mix])
    rho, u = inp.random_velocity_field(shape, seed=62, amplitude=0.05)
    params = dict(tau=0.66, force=(2e-4, 0, 0), wall_u=[(0.02, 0, 0), (0, 0, 0.01)], closure=closure)
    outs = []
    for fused in (False, True):
        lat = make(shape, 19, kind, tags, **params)
        lat.init_equilibrium(rho, u)
        if fused:
            red = lat.step_reduce(7)
        else:
            lat.step(7)
            red = lat.reduce()
        outs.append((lat.get_populations(), red))
        lat.close()
    (fa, ra), (fb, rb) = outs
    assert np.array_equal(fa, fb)
    assert ra["n_fluid"] == rb["n_fluid"] and ra["nonfinite"] == rb["nonfinite"] == 0
    # FP64 storage takes the separate passes; 32/16-bit storage adds each
    # block's 256 (16-bit: 512) nodes in FP32 by a shuffle tree (about 1e-6
    # relative on each part, smaller on the total) and the block partials in
    # FP64; FP32 per-node moments differ from the stored ones by FP32 rounding
    rel = 1e-12 if kind == "f64" else 1e-6
    assert rb["umax"] == pytest.approx(ra["umax"], rel=rel)
    if kind in ("f16", "bf16"):
        assert ra["umax"] == rb["umax"]
    for key in ("mass", "ke", "ke_rho"):
        assert rb[key] == pytest.approx(ra[key], rel=rel)
    scale = ra["n_fluid"] * ra["umax"]
    for a in range(3):
        assert abs(rb["mom"][a] - ra["mom"][a]) <= rel * scale
        assert abs(rb["vel"][a] - ra["vel"][a]) <= rel * scale


def test_all_solid_lattice_is_left_alone():
    shape = (4, 5, 40)
    _, w, _ = oracle.lattice(19)
    f0 = inp.random_populations(w, shape, seed=4)
    lat = make(shape, 19, "f32", np.full(shape, lbm.TAG_SOLID, np.uint8), tau=0.7)
    lat.set_populations(f0)
    before = lat.get_populations()
    lat.step(3)
    assert np.array_equal(lat.get_populations(), before)
    assert lat.reduce()["n_fluid"] == 0
    lat.close()


def test_tags_roundtrip_census_and_rejection():
    shape = (7, 9, 33)
    tags = inp.random_tags(shape, seed=1, p_solid=0.2, p_forced=0.2, p_wall=0.1, n_walls=8)
    lat = make(shape, tau=0.7)
    lat.set_tags(tags)
    assert np.array_equal(lat.get_tags(), tags)
    assert np.array_equal(lat.census(), np.bincount(tags.ravel(), minlength=lbm.NTAGS))
    bad = tags.copy()
    bad[3, 4, 5] = 200
    with pytest.raises(lbm.LBMError) as e:
        lat.set_tags(bad)
    assert e.value.status == lbm.ERR_ARG
    assert np.array_equal(lat.get_tags(), tags)  # previous tags stay in force
    dev = torch.from_numpy(tags.ravel()).cuda()
    lat.set_tags(dev)
    assert np.array_equal(lat.get_tags(), tags)
    lat.close()


def test_population_roundtrip_and_device_buffers():
    shape = (5, 6, 40)
    _, w, _ = oracle.lattice(19)
    f0 = inp.random_populations(w, shape, seed=2, amplitude=0.1)
    lat = make(shape, tau=0.9)
    lat.set_populations(f0)
    assert max_rel(lat.get_populations(), f0) <= 1e-15
    dev = torch.empty((19,) + shape, dtype=torch.float64, device="cuda")
    lat.get_populations(dev)
    assert max_rel(dev.cpu().numpy(), f0) <= 1e-15
    rho, u = inp.random_velocity_field(shape, seed=5)
    lat.init_equilibrium(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    r, v = lat.moments()
    assert np.max(np.abs(r - rho)) <= 1e-14
    assert np.max(np.abs(v - u)) <= 1e-14
    lat.close()


# ---------------------------------------------------------------------------
# FP32: velocity relative L2 <= 1e-5 against the FP64 oracle
# ---------------------------------------------------------------------------
def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_f32_tgv3d_velocity_l2():
    n, steps = 40, 150
    rho, u = inp.tgv3d(n, 0.04)
    tau = 0.53
    lat = make((n, n, n), 19, "f32", tau=tau)
    lat.init_equilibrium(rho, u)
    lat.step(steps)
    _, ug = lat.moments()
    prob = oracle_problem((n, n, n), tau=tau)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(rho, u), steps))
    assert rel_l2(ug, ur) <= 1e-5
    lat.close()


def test_f32_cavity_velocity_l2():
    n, steps = 34, 300
    tags = inp.cavity_tags(n)
    tau = 3 * 0.1 * (n - 2) / 100.0 + 0.5  # Re = 100 on the interior width
    params = dict(tau=tau, wall_u=[(0.1, 0.0, 0.0)])
    lat = make((n, n, n), 19, "f32", tags, **params)
    lat.init_equilibrium()
    lat.step(steps)
    _, ug = lat.moments()
    prob = oracle_problem((n, n, n), 19, tags, **params)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(), steps))
    assert rel_l2(ug, ur) <= 1e-5
    lat.close()


def test_f32_porous_forced_velocity_l2():
    shape = (24, 24, 48)
    centres, radii = inp.sphere_list(shape, seed=2506, rmin=2.0, rmax=4.0, count=400)
    tags, used, por = oracle.spheres(shape, centres, radii, 0.45, pore_tag=oracle.FORCED)
    params = dict(tau=1.0, force=(1e-5, 0.0, 0.0))
    lat = make(shape, 19, "f32", tags, **params)
    lat.init_equilibrium()
    lat.step(200)
    _, ug = lat.moments()
    prob = oracle_problem(shape, 19, tags, **params)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(), 200))
    assert rel_l2(ug, ur) <= 1e-5
    lat.close()


@pytest.mark.parametrize("Q", [19, 27])
def test_f32_smagorinsky_velocity_l2(Q):
    n, steps = 24, 100
    rho, u = inp.tgv3d(n, 0.08)
    params = dict(tau=0.505, closure=lbm.CLOSURE_SMAGORINSKY, cs_smag=0.1)
    lat = make((n, n, n), Q, "f32", **params)
    lat.init_equilibrium(rho, u)
    lat.step(steps)
    _, ug = lat.moments()
    prob = oracle_problem((n, n, n), Q, **params)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(rho, u), steps))
    assert rel_l2(ug, ur) <= 1e-5
    lat.close()


# ---------------------------------------------------------------------------
# FP16 / BF16 shifted storage
# ---------------------------------------------------------------------------
def ulp(h, kind):
    """Spacing of the stored values of h: FP16 below 2^-14 and scaled FP16
    (h * 2^12) below 2^-26 have the fixed spacing of their subnormals."""
    mant = 7 if kind == "bf16" else 10
    e = np.floor(np.log2(np.maximum(np.abs(h), 1e-300)))
    if kind == "f16":
        e = np.maximum(e, -14)
    if kind == "f16s":
        e = np.maximum(e, -26)
    return np.exp2(e - mant)


# 16-bit storage runs two nodes per thread when the padded row has >= 64
# nodes: shapes cover odd nx (last node wraps), one and several warps per row,
# a partial last block, and the one-node-per-thread kernel (px = 32).
HALF_SHAPES = [(10, 12, 50), (5, 7, 45), (4, 6, 150), (3, 5, 64), (6, 5, 31)]


@pytest.mark.parametrize("shape", HALF_SHAPES)
@pytest.mark.parametrize("kind", ["f16", "bf16", "f16s"])
@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("mix", ["dense", "list"])
def test_half_storage_one_step(kind, Q, shape, mix):
    _, w, _ = oracle.lattice(Q)
    tags = inp.random_tags(shape, seed=6, n_walls=2, **WALL_MIX[mix])
    walls = [(0.02, 0.0, 0.0), (0.0, 0.01, -0.01)]
    params = dict(tau=0.7, force=(1e-3, 0.0, -5e-4), wall_u=walls)
    rho, u = inp.random_velocity_field(shape, seed=12, amplitude=0.06)
    prob = oracle_problem(shape, Q, tags, **params)
    f0 = oracle.round_storage(prob.init_equilibrium(rho, u), DT[kind])
    lat = make(shape, Q, kind, tags, **params)
    lat.set_populations(f0)
    assert np.array_equal(lat.get_populations(), f0)  # representable state round-trips exactly
    lat.step(1)
    f = lat.get_populations()
    g = oracle.round_storage(prob.step(f0, 1), DT[kind])
    wv = w.reshape(-1, 1, 1, 1)
    hg, hr = f - wv, g - wv
    diff = np.abs(hg - hr)
    excess = diff - (ulp(hr, kind) * 1.0000001 + 1e-8)
    assert np.all(excess <= 0), f"worst excess {excess.max():.3e} at |h| = {abs(hr.ravel()[excess.argmax()]):.3e}"
    assert np.mean(diff == 0) >= 0.99
    lat.close()


@pytest.mark.parametrize("shape", HALF_SHAPES)
@pytest.mark.parametrize("kind", ["f16", "bf16", "f16s"])
@pytest.mark.parametrize("Q,closure", [(19, lbm.CLOSURE_BGK), (27, lbm.CLOSURE_BGK), (19, lbm.CLOSURE_SMAGORINSKY),
                                       (27, lbm.CLOSURE_TRT)])
def test_half_storage_one_step_periodic(kind, Q, closure, shape):
    """All-fluid lattice: the kernel variant that reads no tags."""
    _, w, _ = oracle.lattice(Q)
    params = dict(tau=0.55, closure=closure, cs_smag=0.15)
    rho, u = inp.random_velocity_field(shape, seed=13, amplitude=0.08)
    prob = oracle_problem(shape, Q, None, **params)
    f0 = oracle.round_storage(prob.init_equilibrium(rho, u), DT[kind])
    lat = make(shape, Q, kind, None, **params)
    lat.set_populations(f0)
    lat.step(1)
    f = lat.get_populations()
    g = oracle.round_storage(prob.step(f0, 1), DT[kind])
    wv = w.reshape(-1, 1, 1, 1)
    hg, hr = f - wv, g - wv
    diff = np.abs(hg - hr)
    excess = diff - (ulp(hr, kind) * 1.0000001 + 1e-8)
    assert np.all(excess <= 0), f"worst excess {excess.max():.3e}"
    assert np.mean(diff == 0) >= 0.99
    lat.close()


@pytest.mark.parametrize("kind", ["f16", "bf16", "f16s"])
def test_half_storage_error_after_200_steps_is_bounded(kind):
    """Error statement (not bit parity): 2D TGV config at 32^3 after 200 steps,
    velocity relative L2 against the FP64 oracle; the bound is a sanity limit."""
    n = 32
    rho, u = inp.tgv2d(n, n, n, 0.02)
    lat = make((n, n, n), 19, kind, tau=0.8)
    lat.init_equilibrium(rho, u)
    lat.step(200)
    _, ug = lat.moments()
    prob = oracle_problem((n, n, n), tau=0.8)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(rho, u), 200))
    err = rel_l2(ug, ur)
    print(f"{kind}: velocity rel L2 after 200 steps = {err:.3e}")
    assert err <= (0.5 if kind == "bf16" else 5e-2)
    lat.close()


def test_scaled_fp16_keeps_small_deviations():
    """A 2D TGV of amplitude 2e-4 (|h| ~ 2e-5, inside plain FP16's subnormal
    range): scaled FP16 keeps 11 significant bits there and must cut the
    velocity error against the FP64 oracle well below plain FP16's."""
    n = 32
    rho, u = inp.tgv2d(n, n, n, 2e-4)
    prob = oracle_problem((n, n, n), tau=0.8)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(rho, u), 100))
    err = {}
    for kind in ("f16", "f16s"):
        lat = make((n, n, n), 19, kind, tau=0.8)
        lat.init_equilibrium(rho, u)
        lat.step(100)
        _, ug = lat.moments()
        err[kind] = rel_l2(ug, ur)
        lat.close()
    print(f"velocity rel L2 after 100 steps at u0 = 2e-4: {err}")
    assert err["f16s"] < 0.25 * err["f16"]
    assert err["f16s"] < 2e-2


# ---------------------------------------------------------------------------
# Failure paths (no GPU fault: host-side checks and bounded waits)
# ---------------------------------------------------------------------------
def test_nan_injection_reports_unstable():
    shape = (6, 6, 32)
    _, w, _ = oracle.lattice(19)
    f0 = inp.random_populations(w, shape, seed=2)
    f0[3, 2, 3, 7] = np.nan
    lat = make(shape, tau=0.8)
    lat.set_populations(f0)
    with pytest.raises(lbm.UnstableError) as e:
        lat.reduce()
    assert e.value.status == lbm.ERR_UNSTABLE
    assert e.value.reduction["nonfinite"] == 1
    assert e.value.reduction["n_fluid"] == 6 * 6 * 32
    lat.close()


def test_bad_params_rejected():
    lat = make((4, 4, 32), tau=0.8)
    for kw in (dict(tau=0.5), dict(tau=float("nan")), dict(tau=0.7, closure=9), dict(tau=0.7, cs_smag=-1.0),
               dict(tau=0.7, closure=lbm.CLOSURE_TRT, trt_magic=0.0)):
        with pytest.raises(lbm.LBMError) as e:
            lat.set_params(**kw)
        assert e.value.status == lbm.ERR_ARG
    with pytest.raises(lbm.LBMError):
        lat.step(-1)
    lat.close()


def test_sync_timeout_is_bounded():
    lat = make((4, 4, 32), tau=0.8)
    torch.cuda._sleep(int(2e8))  # a bounded busy kernel on the same stream
    with pytest.raises(lbm.LBMError) as e:
        lat.sync(timeout_ms=1)
    assert e.value.status == lbm.ERR_TIMEOUT
    lat.sync(timeout_ms=60000)
    lat.close()


# ---------------------------------------------------------------------------
# Full-size workloads in the benchmark's launch configuration: sampled nodes
# against the oracle, computed node by node from their 3x3x3 neighbourhood.
# ---------------------------------------------------------------------------
def _neighbourhood(field, z, y, x):
    idx = [np.arange(v - 1, v + 2) % field.shape[-3 + k] for k, v in enumerate((z, y, x))]
    return field[..., idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


def _sampled_check(lat, Q, kind, rho, u, tags, params, cells):
    """One step from an equilibrium state; compares sampled nodes with an
    oracle step of their periodic 3x3x3 neighbourhood (the centre node of a
    3^3 periodic block sees exactly its true neighbours)."""
    N = lat.N
    out = torch.empty((Q, N), dtype=torch.float64, device="cuda")
    lat.get_populations(out)
    z, y, x = cells.T
    flat = torch.from_numpy(x + lat.nx * (y + lat.ny * z)).cuda()
    got = out[:, flat].cpu().numpy()
    del out
    torch.cuda.empty_cache()
    maxdiff = 0.0
    _, w, _ = oracle.lattice(Q)
    for k, (cz, cy, cx) in enumerate(cells):
        r = _neighbourhood(rho, cz, cy, cx) if rho is not None else np.ones((3, 3, 3))
        v = _neighbourhood(u, cz, cy, cx) if u is not None else np.zeros((3, 3, 3, 3))
        t = _neighbourhood(tags, cz, cy, cx) if tags is not None else None
        prob = oracle.Problem(Q, 3, 3, 3, t, **params)
        f0 = oracle.round_storage(prob.init_equilibrium(r, v), DT[kind])
        g = prob.step(f0, 1)[:, 1, 1, 1]
        maxdiff = max(maxdiff, float(np.max(np.abs(got[:, k] - g))))
    return maxdiff


def test_full_size_tgv512_f32_sampled():
    n = 512
    rho, u = inp.tgv3d(n, 0.04)
    tau = 0.5 + 3 * 0.04 * (n / (2 * math.pi)) / 1600.0
    lat = make((n, n, n), 19, "f32", tau=tau)
    lat.init_equilibrium(rho, u)
    m0 = lat.reduce()["mass"]
    lat.step(1)
    rng = np.random.default_rng(0)
    cells = np.stack([rng.integers(0, n, 48), rng.integers(0, n, 48), rng.integers(0, n, 48)], axis=1)
    cells = np.vstack([cells, [[0, 0, 0], [n - 1, n - 1, n - 1], [0, n - 1, 0], [n - 1, 0, n - 1]]])
    d = _sampled_check(lat, 19, "f32", rho, u, None, dict(tau=tau), cells)
    assert d <= 1e-7  # FP32 arithmetic on |h| <= ~0.1
    lat.step(9)
    red = lat.reduce()
    assert abs(red["mass"] - m0) / m0 <= 1e-6
    assert max(abs(v) for v in red["mom"]) <= 1e-6 * n ** 3 * 0.04
    lat.close()


@pytest.mark.parametrize("pattern", ["aa"])
def test_full_size_tgv512_aa_f32_sampled(pattern):
    """The in-place pattern at the bench size: after one (odd) step the state
    is read back from the neighbour-shifted layout, after two from the local
    one; both sampled against the oracle."""
    n = 512
    rho, u = inp.tgv3d(n, 0.04)
    tau = 0.5 + 3 * 0.04 * (n / (2 * math.pi)) / 1600.0
    nz = ny = nx = n
    lat = lbm.Lattice(nx, ny, nz, 19, "f32", pattern=pattern)
    lat.set_params(tau)
    lat.init_equilibrium(rho, u)
    lat.step(1)
    rng = np.random.default_rng(3)
    cells = np.stack([rng.integers(0, n, 40), rng.integers(0, n, 40), rng.integers(0, n, 40)], axis=1)
    cells = np.vstack([cells, [[0, 0, 0], [n - 1, n - 1, n - 1], [0, n - 1, 0], [n - 1, 0, n - 1]]])
    assert _sampled_check(lat, 19, "f32", rho, u, None, dict(tau=tau), cells) <= 1e-7
    m1 = lat.reduce()["mass"]
    lat.step(1)
    red = lat.reduce()
    assert abs(red["mass"] - m1) <= 1e-6 * abs(m1) + 1e-3
    lat.close()


@pytest.mark.parametrize("Q,kind", [(27, "f16"), (19, "f16s")])
def test_full_size_tgv512_half_sampled(Q, kind):
    """16-bit storage at the precision-study size (512^3; D3Q27 FP16 is that
    study's configuration): one step from a storage-rounded equilibrium,
    sampled nodes within half a storage ulp of |h| <~ 0.1 (plus the FP32
    arithmetic) of the oracle's FP64 step."""
    n = 512
    rho, u = inp.tgv3d(n, 0.04)
    tau = 0.5 + 3 * 0.04 * (n / (2 * math.pi)) / 1600.0
    lat = make((n, n, n), Q, kind, tau=tau)
    lat.init_equilibrium(rho, u)
    lat.step(1)
    rng = np.random.default_rng(4)
    cells = np.stack([rng.integers(0, n, 24), rng.integers(0, n, 24), rng.integers(0, n, 24)], axis=1)
    d = _sampled_check(lat, Q, kind, rho, u, None, dict(tau=tau), cells)
    assert d <= 1e-4
    lat.close()


def test_full_size_cavity256_f32_sampled():
    n = 256
    tags = inp.cavity_tags(n)
    tau = 3 * 0.1 * n / 1000.0 + 0.5
    params = dict(tau=tau, wall_u=[(0.1, 0.0, 0.0)])
    lat = make((n, n, n), 19, "f32", tags, **params)
    lat.init_equilibrium()
    lat.step(1)
    rng = np.random.default_rng(1)
    cells = np.stack([np.full(32, n - 2), rng.integers(1, n - 1, 32), rng.integers(1, n - 1, 32)], axis=1)
    cells = np.vstack([cells, [[n - 2, 1, 1], [n - 2, n - 2, n - 2], [1, 1, 1], [n // 2, n // 2, n // 2]]])
    d = _sampled_check(lat, 19, "f32", None, None, tags, params, cells)
    assert d <= 1e-7
    lat.close()


@pytest.mark.parametrize("pattern,closure", [("ab", "trt"), ("aa", "bgk")])
def test_full_size_porous400_f32_sampled(pattern, closure):
    """The porous benchmark workload at its full size (400^3 random-sphere
    medium, 80% wall: stepped on compact fluid-only storage): one step from a
    random equilibrium, sampled pore nodes (among them nodes with solid
    neighbours) against the oracle's step of their 3x3x3 neighbourhood."""
    n = 400
    centres, radii = inp.sphere_list((n, n, n), seed=2506, rmin=4.0, rmax=10.0, count=100_000)
    lat = lbm.Lattice(n, n, n, 19, "f32", pattern=pattern)
    lat.geometry_spheres(centres, radii, 0.2, lbm.TAG_FORCED)
    kind = {"bgk": (lbm.CLOSURE_BGK, oracle.BGK), "trt": (lbm.CLOSURE_TRT, oracle.TRT)}[closure]
    lat.set_params(1.0, force=(1e-6, 0.0, 0.0), closure=kind[0])
    tags = lat.get_tags()
    rho, u = inp.random_velocity_field((n, n, n), seed=41, amplitude=0.05)
    lat.init_equilibrium(rho, u)
    lat.step(1)
    rng = np.random.default_rng(2)
    pore = np.argwhere(tags < oracle.SOLID)
    cells = pore[rng.choice(len(pore), 48, replace=False)]
    near = [c for c in pore[rng.choice(len(pore), 4000, replace=False)]
            if np.any(_neighbourhood(tags, *c) >= oracle.SOLID)][:16]
    assert len(near) == 16
    cells = np.vstack([cells, np.array(near)])
    d = _sampled_check(lat, 19, "f32", rho, u, tags, dict(tau=1.0, force=(1e-6, 0.0, 0.0), closure=kind[1]), cells)
    assert d <= 1e-7
    lat.close()


@pytest.mark.parametrize("kind", ["f64", "f32", "f16"])
def test_init_from_pinned_pageable_and_device_fields_agree(kind):
    """lbm_init_equilibrium reads page-locked host fields directly from the
    kernel, pageable ones through a staging copy and device ones in place:
    the three give the same stored state, bit for bit."""
    shape = (6, 9, 37)
    nz, ny, nx = shape
    rho, u = inp.random_velocity_field(shape, seed=91, amplitude=0.05)
    sources = {"pageable": (rho, u),
               "pinned": (torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory()),
               "device": (torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())}
    states = {}
    for name, (r, v) in sources.items():
        with lbm.Lattice(nx, ny, nz, 19, kind) as lat:
            lat.init_equilibrium(r, v)
            states[name] = lat.get_state()[0]
            lat.init_equilibrium(r, None)  # density only
            states[name + "_rho"] = lat.get_state()[0]
    for name in ("pinned", "device"):
        assert np.array_equal(states[name], states["pageable"]), name
        assert np.array_equal(states[name + "_rho"], states["pageable_rho"]), name
