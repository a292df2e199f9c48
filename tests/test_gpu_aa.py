"""AA-pattern streaming (one population array, updated in place) against the
two-array A/B scheme and the FP64 oracle.

The AA steps run the same per-node arithmetic as the A/B steps and differ
only in where each population is read and written.  The collision spells out
every rounding (no contraction left to the compiler), so the one-node, the
two-nodes-per-thread and the compact kernels give a node the same bits, and
the two patterns must agree bit for bit: populations, moments and
reductions, after odd step counts (the neighbour-shifted layout) and even
ones, through graph replays and fused step-and-reduce calls, on dense and on
compact fluid-only storage, in every storage type.
"""
import numpy as np
import pytest
import torch

import lbm_inputs as inp
import oracle
from paper_2506_09242_gb300 import lbm

pytestmark = pytest.mark.gpu

WALL_MIX = {"dense": dict(p_solid=0.15, p_forced=0.3, p_wall=0.06),
            "list": dict(p_solid=0.45, p_forced=0.2, p_wall=0.1)}
WALLS = [(0.02, 0.0, 0.0), (0.0, 0.0, -0.01), (0.0, 0.015, 0.0)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2506_09242_gb300 import _build
    _build.build()
    lbm.load()


def make(shape, Q, dtype, pattern, tags=None, **params):
    nz, ny, nx = shape
    lat = lbm.Lattice(nx, ny, nz, Q, dtype, pattern=pattern)
    if tags is not None:
        lat.set_tags(tags)
    lat.set_params(**params)
    return lat


def snapshot(lat):
    rho, u = lat.moments()
    return lat.get_populations(), rho, u, lat.reduce()


def assert_same(a, b):
    fa, ra, ua, reda = a
    fb, rb, ub, redb = b
    assert np.array_equal(fa, fb)
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
    for k in ("mass", "ke", "ke_rho", "umax", "n_fluid", "nonfinite"):
        assert reda[k] == redb[k], k
    assert reda["mom"] == redb["mom"] and reda["vel"] == redb["vel"]


def assert_close(a, b, rel):
    """Rounding-level agreement, relative to each quantity's magnitude."""
    fa, ra, ua, reda = a
    fb, rb, ub, redb = b
    for x, y in ((fa, fb), (ra, rb), (ua, ub)):
        assert np.max(np.abs(x - y)) <= rel * np.max(np.abs(y))
    for k in ("mass", "ke", "ke_rho", "umax"):
        assert reda[k] == pytest.approx(redb[k], rel=rel, abs=1e-300), k
    assert reda["n_fluid"] == redb["n_fluid"] and reda["nonfinite"] == redb["nonfinite"]


def run_both(shape, Q, dtype, tags, params, counts, rho=None, u=None, fused=False):
    out = {}
    for pattern in ("ab", "aa"):
        lat = make(shape, Q, dtype, pattern, tags, **params)
        lat.init_equilibrium(rho, u)
        snaps = []
        for n in counts:
            if fused:
                red = lat.step_reduce(n)
                snaps.append((lat.get_populations(), red))
            else:
                lat.step(n)
                snaps.append(snapshot(lat))
        assert lat.step_count() == sum(counts)
        out[pattern] = snaps
        lat.close()
    return out["ab"], out["aa"]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mix", ["periodic", "dense", "list"])
@pytest.mark.parametrize("closure", [lbm.CLOSURE_BGK, lbm.CLOSURE_TRT, lbm.CLOSURE_SMAGORINSKY])
def test_aa_is_bit_identical_to_ab(dtype, mix, closure):
    """Odd and even step counts, graph replays (n >= 4) and single launches;
    "list" tags step the compact fluid-only storage."""
    shape = (9, 13, 70)  # ragged x tail, several blocks
    tags = None if mix == "periodic" else inp.random_tags(shape, seed=71, n_walls=3, **WALL_MIX[mix])
    rho, u = inp.random_velocity_field(shape, seed=72, amplitude=0.04)
    params = dict(tau=0.63, force=(1e-4, -5e-5, 2e-5), wall_u=WALLS, closure=closure)
    ab, aa = run_both(shape, 19, dtype, tags, params, (1, 1, 7, 8, 3), rho, u)
    for a, b in zip(ab, aa):
        assert_same(a, b)


@pytest.mark.parametrize("Q", [19, 27])
def test_aa_d3q27_and_degenerate_rows(Q):
    """Rows of one to a few nodes: the in-place neighbours wrap onto the node
    itself, where reads and writes of one thread meet the same locations."""
    for shape in [(3, 2, 1), (1, 1, 1), (4, 5, 33)]:
        tags = inp.random_tags(shape, seed=73, p_solid=0.2, p_forced=0.3, p_wall=0.1, n_walls=2)
        tags.flat[0] = oracle.FORCED
        params = dict(tau=0.8, force=(1e-3, 0.0, -1e-3), wall_u=WALLS)
        ab, aa = run_both(shape, Q, "f64", tags, params, (1, 2, 5))
        for a, b in zip(ab, aa):
            assert_same(a, b)


@pytest.mark.parametrize("kind", ["f16", "bf16", "f16s"])
@pytest.mark.parametrize("nx", [32, 96])
def test_aa_half_storage(kind, nx):
    """Rows padded to 32 nodes: both patterns take the one-node kernel; 64 or
    more: A/B and the even AA steps pair two nodes per thread, the odd AA
    steps take one node per thread, with the same bits."""
    shape = (6, 7, nx)
    tags = inp.random_tags(shape, seed=74, n_walls=2, **WALL_MIX["dense"])
    rho, u = inp.random_velocity_field(shape, seed=75, amplitude=0.04)
    params = dict(tau=0.7, force=(1e-4, 0, 0), wall_u=WALLS)
    ab, aa = run_both(shape, 19, kind, tags, params, (1, 4), rho, u)
    for a, b in zip(ab, aa):
        assert_same(a, b)


@pytest.mark.parametrize("kind", ["f16", "bf16", "f16s"])
@pytest.mark.parametrize("Q,nx", [(19, 64), (19, 65), (19, 127), (19, 130), (27, 96)])
@pytest.mark.parametrize("closure", [lbm.CLOSURE_BGK, lbm.CLOSURE_TRT])
def test_aa_half_storage_periodic(kind, Q, nx, closure):
    """Periodic lattices without tags on rows of 64 nodes or more (the even
    AA steps and A/B pair nodes, the odd AA steps take one node per thread):
    odd nx, rows whose last block lies partly past the end, two warps per
    block row (128 nodes), odd and even counts."""
    shape = (5, 6, nx)
    rho, u = inp.random_velocity_field(shape, seed=83, amplitude=0.04)
    ab, aa = run_both(shape, Q, kind, None, dict(tau=0.62, closure=closure), (1, 1, 2), rho, u)
    for a, b in zip(ab, aa):
        assert_same(a, b)


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_aa_half_storage_periodic_fused_and_smagorinsky(kind):
    """The fused step-and-reduce ending on an odd and on an even step, and
    the Smagorinsky closure.  The state is the same bits.  An even AA step
    sums its nodes in the same blocks as A/B (two nodes per thread), so the
    sums are the same bits too; an odd one sums one node per thread, the same
    node values grouped in other FP32 block partials."""
    shape = (6, 7, 96)
    rho, u = inp.random_velocity_field(shape, seed=84, amplitude=0.05)
    counts = (1, 2, 1)
    ab, aa = run_both(shape, 19, kind, None, dict(tau=0.55), counts, rho, u, fused=True)
    for n, (fa, ra), (fb, rb) in zip(np.cumsum(counts), ab, aa):
        assert np.array_equal(fa, fb)
        if n % 2 == 0:
            assert ra == rb
        else:
            assert ra["n_fluid"] == rb["n_fluid"] and ra["nonfinite"] == rb["nonfinite"] == 0
            assert ra["umax"] == rb["umax"]
            for k in ("mass", "ke", "ke_rho"):
                assert ra[k] == pytest.approx(rb[k], rel=1e-6), k
    ab, aa = run_both(shape, 19, kind, None, dict(tau=0.52, closure=lbm.CLOSURE_SMAGORINSKY), (1, 2), rho, u)
    for a, b in zip(ab, aa):
        assert_same(a, b)


def test_aa_matches_the_oracle():
    """FP64 AA against the FP64 oracle directly, walls, force and TRT."""
    shape = (8, 10, 37)
    tags = inp.random_tags(shape, seed=76, n_walls=3, **WALL_MIX["dense"])
    rho, u = inp.random_velocity_field(shape, seed=77, amplitude=0.04)
    params = dict(tau=0.7, force=(2e-4, 0, 1e-4), wall_u=WALLS, closure=lbm.CLOSURE_TRT)
    lat = make(shape, 19, "f64", "aa", tags, **params)
    lat.init_equilibrium(rho, u)
    prob = oracle.Problem(19, shape[2], shape[1], shape[0], tags, tau=0.7, force=(2e-4, 0, 1e-4), wall_u=WALLS,
                          closure=oracle.TRT)
    g = prob.init_equilibrium(rho, u)
    for n in (3, 6):
        lat.step(n)
        g = prob.step(g, n)
        f = lat.get_populations()
        assert float(np.max(np.abs(f - g) / np.maximum(np.abs(g), 1e-300))) <= 1e-12
        red, ref = lat.reduce(), prob.reduce(g)
        assert red["mass"] == pytest.approx(ref["mass"], rel=1e-13)
        assert red["ke"] == pytest.approx(ref["ke"], rel=1e-11)
    lat.close()


@pytest.mark.parametrize("mix", ["dense", "list"])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_aa_fused_step_reduce(dtype, mix):
    """The fused last step writes the same state and, with the one-node
    kernel on both sides (or the compact kernel, for "list" tags), the same
    partial sums."""
    shape = (7, 9, 30)  # rows padded to 32: the one-node kernel in both patterns
    tags = inp.random_tags(shape, seed=78, n_walls=2, **WALL_MIX[mix])
    rho, u = inp.random_velocity_field(shape, seed=79, amplitude=0.04)
    params = dict(tau=0.66, force=(1e-4, 0, 0), wall_u=WALLS)
    ab, aa = run_both(shape, 19, dtype, tags, params, (1, 6, 3), rho, u, fused=True)
    for (fa, ra), (fb, rb) in zip(ab, aa):
        assert np.array_equal(fa, fb)
        assert ra == rb


def test_aa_mlp_closure_is_bit_identical():
    shape = (5, 6, 64)
    tags = inp.random_tags(shape, seed=80, n_walls=1, **WALL_MIX["dense"])
    rho, u = inp.random_velocity_field(shape, seed=81, amplitude=0.04)
    P = inp.mlp_init(12)
    X, _ = inp.mlp_samples(512, seed=5)
    std = X.std(axis=0)
    std[std == 0] = 1.0
    norm = np.concatenate([X.mean(axis=0), std, [1e-3, 0.0]])
    out = []
    for pattern in ("ab", "aa"):
        lat = make(shape, 19, "f32", pattern, tags, tau=0.6, wall_u=WALLS, closure=lbm.CLOSURE_MLP)
        lat.set_closure_weights(np.float32(P), np.float32(norm))
        lat.init_equilibrium(rho, u)
        lat.step(3)
        a = lat.get_populations()
        lat.step(6)
        out.append((a, lat.get_populations()))
        lat.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_aa_set_tags_needs_the_local_layout():
    """After an odd number of steps the bounced links are stored for the
    current tags: changing them is refused until one more step."""
    shape = (4, 5, 32)
    tags = inp.random_tags(shape, seed=82, n_walls=1, **WALL_MIX["dense"])
    lat = make(shape, 19, "f32", "aa", tags, tau=0.8, wall_u=WALLS)
    lat.init_equilibrium()
    lat.step(1)
    with pytest.raises(lbm.LBMError) as e:
        lat.set_tags(tags)
    assert e.value.status == lbm.ERR_STATE
    lat.step(1)
    lat.set_tags(np.zeros(shape, np.uint8))  # two steps: allowed
    lat.step(3)
    with pytest.raises(lbm.LBMError):
        lat.set_tags(tags)
    lat.set_populations(lat.get_populations())  # rewritten in the local layout
    lat.set_tags(tags)
    lat.close()


def test_aa_holds_one_population_array():
    shape = (32, 32, 64)
    used = {}
    for pattern in ("ab", "aa"):
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        lat = make(shape, 19, "f32", pattern, tau=0.8)
        torch.cuda.synchronize()
        used[pattern] = torch.cuda.memory_allocated() - before
        info = lat.info()
        lat.close()
    pop = info["population_bytes"]
    assert used["ab"] - used["aa"] == pop
    assert used["aa"] < pop * 1.1
