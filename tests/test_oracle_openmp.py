"""The OpenMP build of the C oracle, which the CPU baseline times, computes
the same populations bit for bit as the plain build the parity tests use:
the threads share out z planes, and each node's arithmetic is unchanged."""
import numpy as np
import pytest

import lbm_inputs as inp
import oracle


@pytest.mark.parametrize("Q,closure", [(19, oracle.BGK), (27, oracle.TRT), (19, oracle.SMAGORINSKY)])
def test_openmp_build_is_bit_identical(Q, closure):
    shape = (7, 6, 9)
    nz, ny, nx = shape
    tags = inp.random_tags(shape, seed=31, p_solid=0.15, p_forced=0.3, p_wall=0.05, n_walls=2)
    kw = dict(tau=0.7, force=(1e-3, 0.0, -5e-4), closure=closure, cs_smag=0.1,
              wall_u=[(0.02, 0.0, 0.0), (0.0, 0.01, 0.0)])
    rho, u = inp.random_velocity_field(shape, seed=32, amplitude=0.05)
    plain = oracle.Problem(Q, nx, ny, nz, tags, **kw)
    threaded = oracle.Problem(Q, nx, ny, nz, tags, openmp=True, **kw)
    assert oracle.set_threads(4) >= 1
    f0 = plain.init_equilibrium(rho, u)
    assert np.array_equal(threaded.init_equilibrium(rho, u), f0)
    assert np.array_equal(threaded.step(f0, 5), plain.step(f0, 5))
