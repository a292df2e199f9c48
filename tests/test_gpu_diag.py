"""GPU parity of the porous-medium generator and the enstrophy diagnostic.

- sphere medium: tags, number of spheres used and pore fraction identical to
  the oracle's sequential construction (integer / exact-compare work, so
  bit-exact), at small sizes and at the full 400^3 workload size;
- enstrophy: FP64 storage within 1e-12 relative of the oracle's eighth-order
  curl of the oracle's velocity; FP32 within 1e-5; the Taylor-Green initial
  field against its closed form (3/8)(u0 k)^2.
"""
import math

import numpy as np
import pytest
import torch

import lbm_inputs as inp
import oracle
from paper_2506_09242_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2506_09242_gb300 import _build
    _build.build()
    lbm.load()


@pytest.mark.parametrize("target", [0.0, 0.5, 0.8, 1.0])
@pytest.mark.parametrize("pore_tag", [lbm.TAG_FLUID, lbm.TAG_FORCED])
def test_spheres_small_bit_exact(target, pore_tag):
    shape = (14, 18, 20)  # cubes of side up to 9 wrap around the 14-node axis
    nz, ny, nx = shape
    centres, radii = inp.sphere_list(shape, seed=42, rmin=2.0, rmax=4.5, count=40)
    centres[3] = (-5, 40, 7)  # out-of-range centres wrap
    with lbm.Lattice(nx, ny, nz, 19, "f32") as lat:
        used, por = lat.geometry_spheres(centres, radii, target, pore_tag)
        tags = lat.get_tags()
    ref, used_ref, por_ref = oracle.spheres(shape, centres, radii, target, pore_tag=pore_tag)
    assert used == used_ref
    assert por == por_ref
    assert np.array_equal(tags, ref)


def test_spheres_tiny_lattice_with_wrapping_cubes():
    shape = (6, 7, 5)  # smaller than a sphere: offsets alias, minimum image decides
    centres, radii = inp.sphere_list(shape, seed=3, rmin=2.0, rmax=5.0, count=6)
    with lbm.Lattice(5, 7, 6, 19, "f64") as lat:
        used, por = lat.geometry_spheres(centres, radii, 0.0)
        tags = lat.get_tags()
    ref, used_ref, por_ref = oracle.spheres(shape, centres, radii, 0.0)
    assert (used, por) == (used_ref, por_ref)
    assert np.array_equal(tags, ref)


def test_spheres_full_size_400():
    """The porous workload: 400^3, radii U[4, 10), seed 2506, target 0.2."""
    n = 400
    shape = (n, n, n)
    centres, radii = inp.sphere_list(shape, seed=2506, rmin=4.0, rmax=10.0, count=100000)
    with lbm.Lattice(n, n, n, 19, "f32") as lat:
        used, por = lat.geometry_spheres(centres, radii, 0.2, lbm.TAG_FORCED)
        tags = lat.get_tags()
        census = lat.census()
    ref, used_ref, por_ref = oracle.spheres(shape, centres, radii, 0.2, pore_tag=oracle.FORCED)
    assert used == used_ref
    assert por == por_ref
    assert np.array_equal(tags, ref)
    assert 0.199 < por <= 0.2
    assert census[lbm.TAG_FORCED] == round(por * n ** 3)
    print(f"400^3 medium: {used} spheres, porosity {por:.6f}")


def test_sphere_argument_checks():
    with lbm.Lattice(8, 8, 8, 19, "f32") as lat:
        with pytest.raises(lbm.LBMError):
            lat.geometry_spheres(np.zeros((1, 3)), [2000.0], 0.5)
        with pytest.raises(lbm.LBMError):
            lat.geometry_spheres(np.zeros((1, 3)), [2.0], 0.5, pore_tag=lbm.TAG_SOLID)


def test_enstrophy_tgv_closed_form_and_f64_parity():
    n, u0 = 32, 0.04
    rho, u = inp.tgv3d(n, u0)
    k = 2 * math.pi / n
    tau = 0.52
    with lbm.Lattice(n, n, n, 19, "f64") as lat:
        lat.set_params(tau)
        lat.init_equilibrium(rho, u)
        e0 = lat.enstrophy()
        lat.step(60)
        e = lat.enstrophy()
    assert e0 == pytest.approx(3.0 / 8.0 * (u0 * k) ** 2, rel=1e-9)
    prob = oracle.Problem(19, n, n, n, tau=tau)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(rho, u), 60))
    assert e == pytest.approx(oracle.enstrophy(ur), rel=1e-12)


@pytest.mark.parametrize("Q", [19, 27])
def test_enstrophy_f32_with_walls(Q):
    n = 24
    tags = inp.cavity_tags(n)
    params = dict(tau=0.6, wall_u=[(0.1, 0.0, 0.0)])
    with lbm.Lattice(n, n, n, Q, "f32") as lat:
        lat.set_tags(tags)
        lat.set_params(**params)
        lat.init_equilibrium()
        lat.step(80)
        e = lat.enstrophy()
    prob = oracle.Problem(Q, n, n, n, tags, **params)
    _, ur = prob.moments(prob.step(prob.init_equilibrium(), 80))
    assert e == pytest.approx(oracle.enstrophy(ur), rel=1e-5)
