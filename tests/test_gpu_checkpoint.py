"""Bit-exact checkpoint and resume: a run of n + m steps against n steps,
save_checkpoint, a new lattice from the file and m more steps.  The stored
populations of every fluid node, the reductions and the step counter must
agree bit for bit, for every storage type, both streaming patterns (AA saved
after an odd step count, in its neighbour-shifted layout), dense and compact
fluid-only storage, and the learned closure."""
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


def run_and_resume(tmp_path, shape, Q, dtype, pattern, tags, params, weights=None, n=5, m=8):
    nz, ny, nx = shape
    rho, u = inp.random_velocity_field(shape, seed=91, amplitude=0.04)
    lat = lbm.Lattice(nx, ny, nz, Q, dtype, pattern=pattern)
    if tags is not None:
        lat.set_tags(tags)
    lat.set_params(**params)
    if weights is not None:
        lat.set_closure_weights(*weights)
    lat.init_equilibrium(rho, u)
    lat.step(n)
    path = tmp_path / "state.npz"
    lat.save_checkpoint(path)
    lat.step(m)
    ref = (lat.get_populations(), lat.reduce(), lat.step_count())
    lat.close()

    back = lbm.Lattice.from_checkpoint(path)
    assert back.step_count() == n
    if tags is not None:
        assert np.array_equal(back.get_tags(), tags)
    back.step(m)
    out = (back.get_populations(), back.reduce(), back.step_count())
    back.close()
    fluid = np.ones(shape, bool) if tags is None else tags <= oracle.FORCED
    assert np.array_equal(out[0][:, fluid], ref[0][:, fluid])
    assert out[1] == ref[1]
    assert out[2] == ref[2] == n + m


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16", "bf16", "f16s"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("mix", ["periodic", "dense", "list"])
def test_resume_is_bit_exact(tmp_path, dtype, pattern, mix):
    shape = (7, 9, 70)  # ragged x tail; 16-bit A/B takes the two-node kernel
    tags = None if mix == "periodic" else inp.random_tags(shape, seed=92, n_walls=3, **WALL_MIX[mix])
    params = dict(tau=0.66, force=(1e-4, 0.0, 5e-5), wall_u=WALLS, closure=lbm.CLOSURE_TRT)
    run_and_resume(tmp_path, shape, 19, dtype, pattern, tags, params)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_resume_d3q27_smagorinsky(tmp_path, pattern):
    shape = (6, 8, 33)
    tags = inp.random_tags(shape, seed=93, n_walls=2, **WALL_MIX["dense"])
    params = dict(tau=0.6, force=(0.0, 1e-4, 0.0), wall_u=WALLS, closure=lbm.CLOSURE_SMAGORINSKY, cs_smag=0.17)
    run_and_resume(tmp_path, shape, 27, "f32", pattern, tags, params)


def test_resume_learned_closure(tmp_path):
    shape = (5, 6, 64)
    tags = inp.random_tags(shape, seed=94, n_walls=1, **WALL_MIX["dense"])
    X, _ = inp.mlp_samples(512, seed=5)
    std = X.std(axis=0)
    std[std == 0] = 1.0
    norm = np.concatenate([X.mean(axis=0), std, [1e-3, 0.0]])
    weights = (np.float32(inp.mlp_init(12)), np.float32(norm))
    params = dict(tau=0.6, wall_u=WALLS, closure=lbm.CLOSURE_MLP)
    run_and_resume(tmp_path, shape, 19, "f32", "ab", tags, params, weights=weights)


def test_state_arguments_are_checked():
    lat = lbm.Lattice(32, 4, 3, 19, "f32")
    raw, layout, steps = lat.get_state()
    assert raw.nbytes == lat.info()["population_bytes"] and layout == 0 and steps == 0
    with pytest.raises(lbm.LBMError) as e:
        lat.set_state(raw[:-16])
    assert e.value.status == lbm.ERR_ARG
    with pytest.raises(lbm.LBMError) as e:
        lat.set_state(raw, layout=1)  # the neighbour-shifted layout is AA only
    assert e.value.status == lbm.ERR_ARG
    with pytest.raises(lbm.LBMError):
        lat.set_state(raw, layout=2)
    with pytest.raises(lbm.LBMError):
        lat.set_state(raw, steps=-1)
    lat.set_state(raw, steps=7)
    assert lat.step_count() == 7
    lat.close()
