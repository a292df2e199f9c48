"""The allocation-free reduction, lbm_reduce_noalloc, against lbm_reduce.

lbm_reduce_noalloc is for callers that cannot allocate device memory (a host
code that owns the whole GPU through its own pool, or a time loop that cannot
pay for cudaMalloc's synchronisation): it reduces populations the caller
already holds, with its scratch in a static device array.  This test hands
it the state of a normal lattice, rebuilt in the caller layout from
lbm_get_populations, and checks two calls in a row against lbm_reduce on the
same state, within the tolerances of the other reduction tests.  It lives in
a file of its own so that it runs after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import lbm_inputs as inp
import oracle
from paper_2506_09242_gb300 import lbm

pytestmark = pytest.mark.gpu

TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16,
            "f16s": torch.float16}
SCALE = {"f16s": 4096.0}  # scaled FP16 stores h * 2^12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2506_09242_gb300 import _build
    _build.build()
    lbm.load()


def _close(a, b, rel):
    return abs(a - b) <= rel * max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("Q,kind", [(19, "f64"), (19, "f32"), (27, "f32"), (19, "f16"), (27, "bf16"), (19, "f16s")])
def test_noalloc_matches_lbm_reduce(Q, kind):
    shape = (14, 18, 45)
    nz, ny, nx = shape
    tags = inp.random_tags(shape, seed=21, p_solid=0.15, p_forced=0.3, p_wall=0.05, n_walls=2)
    force = (3e-4, -1e-4, 2e-4)
    with lbm.Lattice(nx, ny, nz, Q, kind) as lat:
        lat.set_tags(tags)
        lat.set_params(0.7, force=force, wall_u=[(0.02, 0.0, 0.0), (0.0, 0.01, 0.0)])
        rho, u = inp.random_velocity_field(shape, seed=22, amplitude=0.05)
        lat.init_equilibrium(rho, u)
        lat.step(5)
        ref = lat.reduce()
        f = torch.empty((Q,) + shape, dtype=torch.float64, device="cuda")
        lat.get_populations(f)
    _, w, _ = oracle.lattice(Q)
    wd = torch.from_numpy(w).cuda().view(Q, 1, 1, 1)
    h = ((f - wd) * SCALE.get(kind, 1.0)).to(TORCH_DT[kind]).contiguous()
    tg = torch.from_numpy(tags).cuda()
    rel = 1e-12 if kind == "f64" else 1e-9
    outs = [lbm.reduce_noalloc(h, Q, kind, nx, ny, nz, tags=tg, force=force) for _ in range(2)]
    for out in outs:
        assert out["n_fluid"] == ref["n_fluid"]
        assert out["nonfinite"] == 0
        # FP64 storage: f - w rebuilt from f = h + w can differ from the stored h
        # in the last bit, so umax is compared within the same tolerance
        for key in ("mass", "ke", "ke_rho", "umax"):
            assert _close(out[key], ref[key], rel), key
        scale = ref["n_fluid"] * ref["umax"]
        for a in range(3):
            assert abs(out["mom"][a] - ref["mom"][a]) <= rel * scale
            assert abs(out["vel"][a] - ref["vel"][a]) <= rel * scale
    assert outs[0] == outs[1]


def test_noalloc_without_tags_and_size_limit():
    n = 32
    rho, u = inp.tgv3d(n, 0.04)
    with lbm.Lattice(n, n, n, 19, "f32") as lat:
        lat.set_params(0.6)
        lat.init_equilibrium(rho, u)
        ref = lat.reduce()
        f = torch.empty((19, n, n, n), dtype=torch.float64, device="cuda")
        lat.get_populations(f)
    _, w, _ = oracle.lattice(19)
    h = (f - torch.from_numpy(w).cuda().view(19, 1, 1, 1)).float().contiguous()
    for _ in range(2):
        out = lbm.reduce_noalloc(h, 19, "f32", n, n, n)
        assert out["n_fluid"] == n ** 3
        assert _close(out["ke"], ref["ke"], 1e-9)
        assert _close(out["mass"], ref["mass"], 1e-12)
    # sizes beyond the limit (2^31 - 257 nodes) are rejected before any device
    # work: the bound + 1, and far beyond it
    lib = lbm.load()
    r = lbm.Reduction()
    for dims in ((178481, 47 * 256, 1), (2048, 2048, 1024)):
        st = lib.lbm_reduce_noalloc(ctypes.c_void_p(h.data_ptr()), 19, lbm.F32, *dims, None, None, None,
                                    ctypes.byref(r))
        assert st == lbm.ERR_ARG
    assert b"LBM_NOALLOC_MAX_NODES" in lib.lbm_last_error(None)
    assert lib.lbm_reduce_noalloc(None, 19, lbm.F32, 4, 4, 4, None, None, None, ctypes.byref(r)) == lbm.ERR_ARG
