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
