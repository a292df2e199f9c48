"""Pins of the closure oracle (oracle/mlp.py): finite differences of the FP64
loss, Adam's first step in closed form, exact filters and strains on
polynomial fields, the eddy-viscosity fit on a stress made from a known
viscosity, and agreement of the C oracle's per-cell network with numpy."""
import numpy as np
import pytest

import lbm_inputs as inp
import oracle
from oracle import mlp


def _norm():
    return np.concatenate([np.zeros(6), [1.0], np.full(6, 1e-3), [0.01], [1e-3], [0.0]])


def test_gradient_matches_central_differences():
    P = inp.mlp_init(1)
    P[224:256] = 0.05 * np.arange(32) / 32  # non-zero biases
    P[-1] = -0.3
    X, t = inp.mlp_samples(40, seed=2)
    norm = _norm()
    loss, g = mlp.loss_and_grad(P, norm, X, t, bf=False)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 120, replace=False), [224, 1280, 1310, 1344]])
    for k in idx:
        h = 1e-6 * max(1.0, abs(P[k]))
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (mlp.loss_and_grad(Pp, norm, X, t, bf=False)[0] - mlp.loss_and_grad(Pm, norm, X, t, bf=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g).max(), 1e-30) + 1e-6 * abs(g[k]), k


def test_activation_derivatives():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    assert np.allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-9)
    assert np.allclose(mlp.sigmoid(z), (mlp.softplus(z + h) - mlp.softplus(z - h)) / (2 * h), atol=1e-9)


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    P = np.ones(4)
    Pn, m, v = mlp.adam(P, np.zeros(4), np.zeros(4), g, 1, lr=0.01)
    # bias-corrected moments equal g and g^2 after one step
    assert np.allclose(Pn, P - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_matches_library():
    import torch
    x = np.random.default_rng(3).normal(size=5000) * 10.0 ** np.random.default_rng(4).integers(-6, 3, 5000)
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_box_filter_and_strain_exact_on_polynomials():
    n, f = 16, 4
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c = np.full((n, n, n), 2.5)
    assert np.allclose(mlp.box_filter(c, f), 2.5)
    lin = 3.0 * x + 0.5 * y - z
    xb = np.arange(n // f) * f + (f - 1) / 2.0
    zc, yc, xc = np.meshgrid(xb, xb, xb, indexing="ij")
    assert np.allclose(mlp.box_filter(lin, f), 3.0 * xc + 0.5 * yc - zc)
    # linear velocity on a periodic grid: interior central differences are exact
    u = np.stack([0.2 * y, 0.1 * z, -0.3 * x]).astype(float)
    S = mlp.strain(u)
    inner = (slice(1, -1),) * 3
    for comp, val in zip(range(6), [0.0, 0.0, 0.0, 0.1, -0.15, 0.05]):
        assert np.allclose(S[comp][inner], val)


def test_eddy_viscosity_recovers_known_viscosity():
    """tau = -2 nu S + p I with a traceless S: the fit returns nu wherever
    S != 0, whatever the isotropic part p; the opposite sign (backscatter)
    is clipped to 0."""
    rng = np.random.default_rng(5)
    S6 = rng.normal(size=(6, 4, 4, 4))
    S6[:3] -= (S6[0] + S6[1] + S6[2]) / 3.0  # traceless
    nu = 0.0123
    p = rng.normal(size=(4, 4, 4))
    tau6 = -2.0 * nu * S6
    tau6[:3] += p
    assert np.allclose(mlp.eddy_viscosity(tau6, S6), nu, rtol=1e-12)
    assert np.allclose(mlp.eddy_viscosity(-tau6 + 2 * np.concatenate([np.stack([p] * 3), np.zeros((3, 4, 4, 4))]), S6), 0.0)


def test_coarse_samples_of_block_constant_field_have_zero_target():
    n, f = 8, 4
    rng = np.random.default_rng(6)
    ub = rng.normal(size=(3, 2, 2, 2))
    u = np.repeat(np.repeat(np.repeat(ub, f, axis=1), f, axis=2), f, axis=3)
    rho = np.ones((n, n, n))
    X, t = mlp.coarse_samples(rho, u, f, 0.51)
    assert np.allclose(t, 0.0)
    assert X.shape == (8, 7) and np.allclose(X[:, 6], 1.0)


@pytest.mark.parametrize("bf", [False, True])
def test_c_oracle_network_matches_numpy(bf):
    P = inp.mlp_init(7)
    P[-1] = 0.2
    X, _ = inp.mlp_samples(50, seed=8)
    norm = _norm()
    ref, _ = mlp.forward(P, norm, X, bf=bf)
    got = np.array([oracle.mlp_dtau(P, norm, x, bf16=bf) for x in X])
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_closure_features_recomputed_from_the_pulled_set():
    """The closure inputs of a state are the non-equilibrium stress and the
    density of each node's pulled set: recomputed here from a stream-only
    step (which returns the pulled sets) with the equilibrium of their own
    moments, on random tags, walls and forced nodes."""
    Q = 19
    c, w, _ = oracle.lattice(Q)
    shape = (4, 5, 6)
    nz, ny, nx = shape
    tags = inp.random_tags(shape, seed=95, p_solid=0.15, p_forced=0.3, p_wall=0.1, n_walls=2)
    f = inp.random_populations(w, shape, seed=96, amplitude=0.05)
    params = dict(force=(1e-3, -2e-3, 5e-4), wall_u=[(0.02, 0.0, -0.01), (0.0, 0.03, 0.01)])
    feats = oracle.Problem(Q, nx, ny, nz, tags, tau=0.8, **params).closure_features(f)
    pulled = oracle.Problem(Q, nx, ny, nz, tags, tau=0.8, closure=oracle.STREAM_ONLY, **params).step(f, 1)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if tags[z, y, x] >= oracle.SOLID:
                    assert np.all(feats[z, y, x] == 0.0)
                    continue
                p = pulled[:, z, y, x]
                rho = p.sum()
                g = np.array(params["force"]) if tags[z, y, x] == oracle.FORCED else np.zeros(3)
                u = (c.T @ p + 0.5 * rho * g) / rho
                d = p - oracle.equilibrium(Q, rho, u)
                pi = [np.sum(c[:, a] * c[:, b] * d) for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))]
                np.testing.assert_allclose(feats[z, y, x, :6], pi, rtol=0, atol=1e-15)
                assert feats[z, y, x, 6] == pytest.approx(rho, rel=1e-15)


def test_closure_features_closed_forms():
    """A uniform equilibrium has no non-equilibrium stress; steady plane
    Couette flow has the Chapman-Enskog shear stress
    Pi_xy = -2 rho c_s^2 tau S_xy = -rho tau U / (3 H)."""
    Q = 19
    n = 6
    rho = np.full((n, n, n), 1.02)
    u = np.zeros((3, n, n, n))
    u[0], u[1], u[2] = 0.03, -0.01, 0.02
    prob = oracle.Problem(Q, n, n, n, tau=0.9)
    feats = prob.closure_features(prob.init_equilibrium(rho, u))
    assert np.max(np.abs(feats[..., :6])) <= 1e-16
    assert np.allclose(feats[..., 6], 1.02, rtol=1e-15)
    H, U, tau = 12, 0.02, 0.9
    ny = H + 2
    tags = inp.channel_tags(1, ny, 1, moving_top=True, fluid_tag=oracle.FLUID)
    ch = oracle.Problem(Q, 1, ny, 1, tags, tau=tau, wall_u=[(U, 0.0, 0.0)])
    f = ch.step(ch.init_equilibrium(), 15000)
    pxy = ch.closure_features(f)[0, 2:H, 0, 3]
    np.testing.assert_allclose(pxy, -tau * U / (3.0 * H), rtol=2e-3)


def _hand_network():
    """A network whose output follows by hand.  Every pre-activation is an
    integer of magnitude >= 40 (or exactly a large negative value), where
    SiLU(z) = z / (1 + e^-z) equals max(z, 0) to within 1e-16 relative, so
    each layer is a known selection and shift of the previous one:
      normalised input  xn_k = (x_k - k) / 2,
      layer 1           unit 3k+1 receives xn_k (bias 0); unit j otherwise
                        carries only its bias 41 + j,
      layer 2           unit j receives layer-1 unit (5j + 3) mod 32 (a
                        permutation, not symmetric, so a transposed W2 shows),
                        plus bias 40 + j/4,
      output            y = sum_j w3_j h2_j + b3 with w3_j = (j mod 5 + 1)/16,
                        b3 = 3; y > 30, where softplus(y) = y to 1e-13;
      dtau              = out_scale * softplus(y), out_scale = 1/2.
    Integers below 256 and the chosen fractions are exact in BF16 and FP32,
    so the BF16-rounding path gives the same value."""
    W1 = np.zeros((32, 7))
    b1 = 41.0 + np.arange(32)
    for k in range(7):
        W1[3 * k + 1, k] = 1.0
        b1[3 * k + 1] = 0.0
    perm = [(5 * j + 3) % 32 for j in range(32)]
    W2 = np.zeros((32, 32))
    for j in range(32):
        W2[j, perm[j]] = 1.0
    b2 = 40.0 + np.arange(32) / 4.0
    w3 = (np.arange(32) % 5 + 1) / 16.0
    b3 = 3.0
    P = mlp.pack(W1, b1, W2, b2, w3, b3)
    norm = np.concatenate([np.arange(7.0), np.full(7, 2.0), [0.5, 0.0]])
    return P, norm, perm, b1, b2, w3, b3


def _hand_expected(xn, perm, b1, b2, w3, b3):
    """The network's value by the selection rules of _hand_network, with exact
    rational arithmetic."""
    from fractions import Fraction as F
    h1 = [F(b1[j]) for j in range(32)]
    for k in range(7):
        h1[3 * k + 1] = max(F(xn[k]), F(0))
    y = sum(F(w3[j]) * (h1[perm[j]] + F(b2[j])) for j in range(32)) + F(b3)
    return float(F(1, 2) * y)


@pytest.mark.parametrize("bf", [False, True])
def test_network_on_hand_computable_weights(bf):
    """Pins the forward pass's wiring (which weight multiplies which input,
    where each bias goes, the normalisation and output scale) on a network
    whose output is computed by hand, for the numpy oracle and the C oracle."""
    P, norm, perm, b1, b2, w3, b3 = _hand_network()
    xns = [np.array([40.0 + 4 * k for k in range(7)]),               # every input passes
           np.array([-100.0, 50, -100, 50, -100, 50, -100]),           # alternate inputs cut off by SiLU
           np.array([64.0, -128, 48, -96, 100, -44, 252])]
    X = np.array([2.0 * xn + np.arange(7) for xn in xns])             # x_k = 2 xn_k + k
    want = np.array([_hand_expected(xn, perm, b1, b2, w3, b3) for xn in xns])
    got, cache = mlp.forward(P, norm, X, bf=bf)
    np.testing.assert_allclose(cache["xn"], np.array(xns), rtol=0, atol=0)
    np.testing.assert_allclose(got, want, rtol=1e-13)
    got_c = np.array([oracle.mlp_dtau(P, norm, x, bf16=bf) for x in X])
    np.testing.assert_allclose(got_c, want, rtol=1e-13)
    # a plausible wiring mistake moves the result: W2 transposed, or the
    # first layer's rows and columns exchanged (W1 read as [7][32])
    W1, _, W2, _, _, _ = mlp.unpack(P)
    assert abs(mlp.forward(mlp.pack(W1, b1, W2.T, b2, w3, b3), norm, X, bf=bf)[0] - want).max() > 1.0
    W1_swapped = W1.T.reshape(32, 7)
    assert abs(mlp.forward(mlp.pack(W1_swapped, b1, W2, b2, w3, b3), norm, X, bf=bf)[0] - want).max() > 1.0
