"""GPU parity of the learned closure against the FP64 oracle (oracle/mlp.py,
and the C oracle's closure step), both sides applying the same BF16
roundings of inputs, first-layer weights and activations, and second-layer
weights.

Tolerances:
- forward (tcgen05 batch tile): each sample within the bound that
  tests/mlp_bounds.py derives for it: FP32 sums, the hardware tanh of SiLU
  (about 2^-11 relative, taken as 2^-10) and one BF16 ulp wherever the exact
  value sits within that error of a rounding midpoint; on a hand-computable
  network (all roundings exact, every SiLU at |z| >= 40) within 2^-10
  relative;
- gradient: samples whose BF16 roundings could go either way are left out,
  and every one of the 1,345 components is compared on its own, within the
  FP32 accumulation error of its own sum of term magnitudes;
- Adam: relative 1e-5 (FP32);
- training samples: relative 1e-5 (FP32 output of FP64 arithmetic);
- box filter: the FP64 rounding of a sum of f^3 values, relative to the mean
  of their magnitudes;
- the collide step with the closure: a flipped BF16 rounding changes dtau by
  up to a few 1e-3 relative, hence a population by up to
  omega^2 * dtau * |h - h_eq| times that (about 2e-5 here); 99% of the
  populations must agree to 1e-7 (FP32 arithmetic), all to 2e-5 after one
  step, and the velocity to relative L2 1e-4 after 20 steps.
"""
import numpy as np
import pytest
import torch

import lbm_inputs as inp
import mlp_bounds as mb
import oracle
from oracle import mlp
from paper_2506_09242_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2506_09242_gb300 import _build
    _build.build()
    lbm.load()


def _params(seed=11):
    P = inp.mlp_init(seed)
    rng = np.random.default_rng(seed)
    P[224:256] = rng.normal(0, 0.2, 32)      # b1
    P[1280:1312] = rng.normal(0, 0.2, 32)    # b2
    P[-1] = -0.5
    return P


def _norm(X, out_scale=1e-3):
    std = X.std(axis=0)
    std[std == 0] = 1.0
    return np.concatenate([X.mean(axis=0), std, [out_scale, 0.0]])


def _cuda32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_matches_oracle():
    X, _ = inp.mlp_samples(3037, seed=4)  # ragged last warp and block
    P = _params()
    norm = _norm(X)
    got = lbm.mlp_forward(_cuda32(P), _cuda32(norm), _cuda32(X)).cpu().numpy().astype(np.float64)
    # the oracle sees the FP32 values the GPU sees
    P32, n32, X32 = (np.float32(a).astype(float) for a in (P, norm, X))
    ref, bound, flips = mb.forward_bound(P32, n32, X32)
    ratio = np.abs(got - ref) / bound
    assert np.all(ratio <= 1.0), f"worst sample at {ratio.max():.2f} of its bound"
    # where no rounding is near a tie the difference is the tanh error alone
    assert np.quantile(np.abs(got - ref) / np.abs(ref), 0.5) <= 1e-3


def test_forward_on_hand_computable_network():
    """The network of the oracle's hand-computed pin, on the tensor cores:
    inputs, W1, W2 and the first activations are exact in BF16 and every
    pre-activation has |z| >= 40, so the only inexact operations are the
    SiLUs (hardware tanh, relative error about 2^-11) and the output sum.
    A wiring mistake (a transposed operand, a bias in the wrong column)
    moves the result by orders of magnitude more."""
    import test_oracle_mlp as pins
    P, norm, perm, b1, b2, w3, b3 = pins._hand_network()
    xns = [np.array([40.0 + 4 * k for k in range(7)]), np.array([-100.0, 50, -100, 50, -100, 50, -100]),
           np.array([64.0, -128, 48, -96, 100, -44, 252])]
    X = np.array([2.0 * xn + np.arange(7) for xn in xns] * 50)  # 150 samples: two tiles, ragged
    want = np.array([pins._hand_expected(xn, perm, b1, b2, w3, b3) for xn in xns] * 50)
    got = lbm.mlp_forward(_cuda32(P), _cuda32(norm), _cuda32(X)).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=2.0 ** -10)


def test_gradient_matches_oracle_and_is_deterministic():
    X, t = inp.mlp_samples(1200, seed=5)
    P = _params(12)
    norm = _norm(X)
    P32, n32, X32, t32 = (np.float32(a).astype(float) for a in (P, norm, X, t))
    keep = ~mb.near_ties_grad_kernel(P32, n32, X32)
    X32, t32 = X32[keep], t32[keep]
    assert len(X32) > 5 * 128  # still several blocks and a ragged last one
    loss_ref, g_ref = mlp.loss_and_grad(P32, n32, X32, t32)
    bound = mb.grad_bound(P32, n32, X32, t32)
    args = (_cuda32(P), _cuda32(norm), _cuda32(X32), _cuda32(t32))
    loss1, g1 = lbm.mlp_loss_grad(*args)
    loss2, g2 = lbm.mlp_loss_grad(*args)
    g = g1.cpu().numpy().astype(np.float64)
    blocks = {"W1": (0, 224), "b1": (224, 256), "W2": (256, 1280), "b2": (1280, 1312), "w3": (1312, 1344),
              "b3": (1344, 1345)}
    for name, (lo, hi) in blocks.items():
        d = np.abs(g[lo:hi] - g_ref[lo:hi])
        assert np.all(d <= bound[lo:hi]), f"{name}: worst at {np.max(d / bound[lo:hi]):.2f} of its bound"
    # the loss: FP32 error of dtau (~1e-5 relative) doubled by the square
    assert float(loss1.item()) == pytest.approx(loss_ref, rel=1e-4)
    assert torch.equal(g1, g2) and torch.equal(loss1, loss2)


@pytest.mark.parametrize("f,ncomp,shape", [(2, 3, (6, 10, 14)), (4, 5, (8, 12, 20)), (3, 1, (9, 6, 15)),
                                           (1, 2, (3, 4, 5))])
def test_box_filter_matches_oracle(f, ncomp, shape):
    """lbm_box_filter against the oracle's block mean, element by element on a
    non-cubic lattice: both sum f^3 FP64 values (in different orders) and
    divide by f^3, so they differ by at most about f^3 roundings of the
    magnitudes summed."""
    rng = np.random.default_rng(17 + f)
    q = rng.normal(size=(ncomp,) + shape) + rng.uniform(-3, 3, size=(ncomp, 1, 1, 1))
    got = lbm.box_filter(torch.from_numpy(q).cuda(), f).cpu().numpy()
    ref = mlp.box_filter(q, f)
    mag = mlp.box_filter(np.abs(q), f)
    assert got.shape == ref.shape
    assert np.all(np.abs(got - ref) <= (f ** 3 + 2) * 2.0 ** -52 * mag)
    one = lbm.box_filter(torch.from_numpy(q[0]).cuda(), f).cpu().numpy()  # the 3D form
    assert np.array_equal(one, got[0])


def test_adam_matches_oracle():
    rng = np.random.default_rng(3)
    P = rng.normal(size=lbm.MLP_NPARAM)
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    Pd, md, vd = _cuda32(P), _cuda32(m), _cuda32(v)
    for step in range(1, 6):
        g = rng.normal(size=lbm.MLP_NPARAM)
        P, m, v = mlp.adam(P, m, v, np.float32(g).astype(float), step, lr=1e-2)
        lbm.mlp_adam(Pd, md, vd, _cuda32(g), step, 1e-2)
    assert np.allclose(Pd.cpu().numpy(), P, rtol=1e-5, atol=1e-6)


def test_coarse_samples_match_oracle():
    f = 4
    shape = (16, 12, 20)
    rho, u = inp.random_velocity_field(shape, seed=7, amplitude=0.05)
    # add a smooth large-scale flow so the coarse strain is not pure noise
    _, ut = inp.tgv3d(20, 0.04)
    u += ut[:, :16, :12, :20]
    X, y = lbm.coarse_samples(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(), f, 0.51)
    Xr, yr = mlp.coarse_samples(rho, u, f, 0.51)
    X, y = X.cpu().numpy(), y.cpu().numpy()
    assert np.allclose(X, Xr, rtol=1e-5, atol=1e-12)
    assert np.allclose(y, yr, rtol=1e-5, atol=1e-12)
    assert (yr > 0).mean() > 0.1  # the fit is not trivially clipped


@pytest.mark.parametrize("Q,kind", [(19, "f64"), (19, "f32"), (27, "f32"), (19, "bf16")])
def test_collide_with_mlp_closure_matches_oracle(Q, kind):
    shape = (9, 10, 40)  # ragged x: lanes past the row end still run the network
    tags = inp.random_tags(shape, seed=8, p_solid=0.1, p_forced=0.3, p_wall=0.05, n_walls=2)
    walls = [(0.02, 0.0, 0.0), (0.0, 0.01, 0.0)]
    rho, u = inp.random_velocity_field(shape, seed=9, amplitude=0.05)
    X, _ = inp.mlp_samples(512, seed=10)
    P = _params(13)
    norm = _norm(X, out_scale=1e-2)
    P32, n32 = np.float32(P).astype(float), np.float32(norm).astype(float)
    params = dict(tau=0.6, force=(1e-4, 0.0, 0.0), wall_u=walls)
    prob = oracle.Problem(Q, shape[2], shape[1], shape[0], tags, closure=oracle.MLP, mlp_params=P32,
                          mlp_norm=n32, mlp_bf16=True, **params)
    dt = {"f64": oracle.F64, "f32": oracle.F32, "bf16": oracle.BF16}[kind]
    f0 = oracle.round_storage(prob.init_equilibrium(rho, u), dt)
    with lbm.Lattice(shape[2], shape[1], shape[0], Q, kind) as lat:
        lat.set_tags(tags)
        lat.set_params(closure=lbm.CLOSURE_MLP, **params)
        lat.set_closure_weights(np.float32(P), np.float32(norm))
        lat.set_populations(f0)
        lat.step(1)
        f1 = lat.get_populations()
        lat.step(19)
        _, ug = lat.moments()
    g1 = prob.step(f0, 1)
    if kind == "bf16":
        g1 = oracle.round_storage(g1, dt)
        c, w, _ = oracle.lattice(Q)
        assert np.max(np.abs(f1 - g1)) <= 1e-4  # one BF16 ulp of |h| <~ 0.03
    else:
        d = np.abs(f1 - g1)
        assert np.quantile(d, 0.99) <= 1e-7
        assert d.max() <= 2e-5
        _, ur = prob.moments(prob.step(f0, 20))
        assert np.linalg.norm(ug - ur) <= 1e-4 * np.linalg.norm(ur)


def test_mlp_closure_needs_weights():
    with lbm.Lattice(32, 4, 4, 19, "f32") as lat:
        lat.set_params(0.6, closure=lbm.CLOSURE_MLP)
        with pytest.raises(lbm.LBMError) as e:
            lat.step(1)
        assert e.value.status == lbm.ERR_STATE
        with pytest.raises(lbm.LBMError):
            lat.set_closure_weights(np.zeros(1345, np.float32), np.zeros(16, np.float32))  # std = 0


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("mix", ["dense", "list"])
def test_closure_features_match_oracle(dtype, pattern, mix):
    """The closure inputs of the current state (pulled set's stress and
    density), after odd and even step counts (AA's two layouts), with walls,
    forcing and compact storage, against the FP64 oracle.  FP64: the FP32
    rounding of the oracle's values; FP32: within the FP32 cancellation of
    the stress (1e-8 absolute for h ~ 1e-2)."""
    Q = 19
    shape = (6, 7, 40)
    nz, ny, nx = shape
    mixes = {"dense": dict(p_solid=0.15, p_forced=0.3, p_wall=0.06),
             "list": dict(p_solid=0.45, p_forced=0.2, p_wall=0.1)}
    tags = inp.random_tags(shape, seed=97, n_walls=2, **mixes[mix])
    walls = [(0.02, 0.0, -0.01), (0.0, 0.03, 0.01)]
    params = dict(tau=0.7, force=(2e-4, 0.0, -1e-4), wall_u=walls)
    rho, u = inp.random_velocity_field(shape, seed=98, amplitude=0.05)
    prob = oracle.Problem(Q, nx, ny, nz, tags, **params)
    g = prob.init_equilibrium(rho, u)
    with lbm.Lattice(nx, ny, nz, Q, dtype, pattern=pattern) as lat:
        lat.set_tags(tags)
        lat.set_params(**params)
        lat.init_equilibrium(rho, u)
        for n in (0, 1, 2):
            if n:
                lat.step(n)
                g = prob.step(g, n)
            got = lat.closure_features().reshape(nz, ny, nx, 7).astype(np.float64)
            ref = prob.closure_features(g)
            if dtype == "f64":
                assert np.array_equal(got, np.float32(ref).astype(np.float64)) or \
                    np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)) <= 1.2e-7
            else:
                assert np.max(np.abs(got[..., :6] - ref[..., :6])) <= 1e-8
                assert np.max(np.abs(got[..., 6] - ref[..., 6])) <= 1e-6
            dev = torch.empty((lat.N, 7), dtype=torch.float32, device="cuda")
            lat.closure_features(dev)
            assert np.array_equal(dev.cpu().numpy().reshape(nz, ny, nx, 7), got.astype(np.float32))
