"""The error bounds of tests/mlp_bounds.py, used to compare the GPU closure
network with the FP64 oracle, checked on the CPU: they contain an FP32
emulation of the GPU arithmetic (FP32 sums in a shuffled order, a tanh
perturbed by up to 2^-11 relative, sigmoid with perturbed exponentials),
and they are tight enough that a wiring mistake planted in the oracle's
parameters (two biases exchanged, W2 transposed) falls outside them."""
import numpy as np
import pytest

import lbm_inputs as inp
import mlp_bounds as mb
from oracle import mlp

f32 = np.float32


def _params(seed):
    P = inp.mlp_init(seed)
    rng = np.random.default_rng(seed)
    P[224:256] = rng.normal(0, 0.2, 32)
    P[1280:1312] = rng.normal(0, 0.2, 32)
    P[-1] = -0.5
    return np.float32(P).astype(np.float64)


def _norm(X, out_scale=1e-3):
    std = X.std(axis=0)
    std[std == 0] = 1.0
    return np.float32(np.concatenate([X.mean(axis=0), std, [out_scale, 0.0]])).astype(np.float64)


def _bf(a):
    return mlp.bf16(np.asarray(a, dtype=np.float32)).astype(np.float32)


def _sum32(terms, rng):
    """FP32 sum of the last axis in a random order (the tensor core's order is
    not specified)."""
    t = np.asarray(terms, dtype=np.float32)
    order = rng.permutation(t.shape[-1])
    acc = np.zeros(t.shape[:-1], dtype=np.float32)
    for k in order:
        acc = f32(acc + t[..., k])
    return acc


def _silu_tile(z, rng):
    hz = f32(0.5) * z
    t = np.tanh(hz.astype(np.float64)) * (1.0 + rng.uniform(-2.0 ** -11, 2.0 ** -11, size=hz.shape))
    return f32(hz.astype(np.float64) * f32(t) + hz)  # one rounding: an FMA


def emulate_tile(P, norm, X, rng):
    W1, b1, W2, b2, w3, b3 = (np.asarray(a, dtype=np.float32) for a in mlp.unpack(P))
    norm = np.asarray(norm, dtype=np.float32)
    mean, inv = norm[:7], f32(1.0) / norm[7:14]
    xn = _bf(f32(np.asarray(X, np.float32) - mean) * inv)
    W1r, W2r = _bf(W1), _bf(W2)
    z1 = f32(_sum32(xn[:, None, :] * W1r[None, :, :], rng) + b1)
    h1 = _bf(_silu_tile(z1, rng))
    z2 = f32(_sum32(h1[:, None, :] * W2r[None, :, :], rng) + b2)
    h2 = _silu_tile(z2, rng)
    y = np.full(len(X), b3, dtype=np.float32)
    for j in range(32):
        y = f32(w3[j] * h2[:, j] + y)
    sp = np.where(y > 20, y, np.log1p(np.exp(y.astype(np.float64))) * (1 + rng.uniform(-1e-6, 1e-6, y.shape)))
    return f32(norm[14] * f32(sp)).astype(np.float64)


def emulate_grad(P, norm, X, target, rng):
    """The gradient kernel's arithmetic in FP32: per-sample forward and
    backward, per-block sums over 128 samples in order, block sums in
    order."""
    W1, b1, W2, b2, w3, b3 = (np.asarray(a, dtype=np.float32) for a in mlp.unpack(P))
    norm = np.asarray(norm, dtype=np.float32)
    n = len(X)

    def sigm(z):
        e = np.exp(-z.astype(np.float64)) * (1 + rng.uniform(-2e-7, 2e-7, z.shape))
        return f32(f32(1.0) / f32(f32(1.0) + f32(e)))

    xn = _bf(f32(np.asarray(X, np.float32) - norm[:7]) * (f32(1.0) / norm[7:14]))
    W1r, W2r = _bf(W1), _bf(W2)
    z1 = np.tile(b1, (n, 1))
    for k in range(7):
        z1 = f32(W1r[:, k][None, :] * xn[:, k][:, None] + z1)
    h1 = _bf(f32(z1 * sigm(z1)))
    z2 = np.tile(b2, (n, 1))
    for k in range(32):
        z2 = f32(W2r[:, k][None, :] * h1[:, k][:, None] + z2)
    h2 = f32(z2 * sigm(z2))
    y = np.full(n, b3, dtype=np.float32)
    for j in range(32):
        y = f32(w3[j] * h2[:, j] + y)
    scale = norm[14]
    dt = f32(scale * f32(np.where(y > 20, y, np.log1p(np.exp(y.astype(np.float64))))))
    err = f32(dt - np.asarray(target, np.float32))
    dy = f32(f32(f32(f32(2.0) / f32(n)) * err) * scale) * sigm(y)

    def dsilu(z):
        s = sigm(z)
        return f32(s * f32(f32(1.0) + f32(z * f32(f32(1.0) - s))))

    dz2 = f32(f32(dy[:, None] * w3[None, :]) * dsilu(z2))
    a = np.zeros((n, 32), dtype=np.float32)
    for j in range(32):
        a = f32(dz2[:, j][:, None] * W2r[j][None, :] + a)
    dz1 = f32(a * dsilu(z1))
    terms = [np.einsum("sj,sk->sjk", dz1, xn).reshape(n, -1), dz1, np.einsum("sj,sk->sjk", dz2, h1).reshape(n, -1),
             dz2, dy[:, None] * h2, dy[:, None]]
    T = np.concatenate([f32(t) for t in terms], axis=1)  # (n, 1345) per-sample terms
    g = np.zeros(T.shape[1], dtype=np.float32)
    for b0 in range(0, n, 128):
        acc = np.zeros(T.shape[1], dtype=np.float32)
        for s in range(b0, min(b0 + 128, n)):
            acc = f32(acc + T[s])
        g = f32(g + acc)
    return g.astype(np.float64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forward_bound_contains_fp32_emulation(seed):
    X, _ = inp.mlp_samples(1500, seed=40 + seed)
    X = np.float32(X).astype(np.float64)
    P = _params(11 + seed)
    norm = _norm(X)
    ref, bound, flips = mb.forward_bound(P, norm, X)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        emu = emulate_tile(P, norm, X, rng)
        assert np.all(np.abs(emu - ref) <= bound)
    # the bound is a few tanh errors wide for a typical sample
    assert np.median(bound / np.abs(ref)) < 1e-2
    assert flips.sum() > 0  # near ties do occur and are covered


def test_forward_bound_catches_a_planted_mistake():
    X, _ = inp.mlp_samples(1500, seed=44)
    X = np.float32(X).astype(np.float64)
    P = _params(14)
    norm = _norm(X)
    emu = emulate_tile(P, norm, X, np.random.default_rng(9))
    for plant in ("swap_b1", "w2_transposed"):
        Pm = P.copy()
        if plant == "swap_b1":
            Pm[224 + 3], Pm[224 + 17] = P[224 + 17], P[224 + 3]
        else:
            Pm[256:1280] = P[256:1280].reshape(32, 32).T.ravel()
        ref, bound, _ = mb.forward_bound(Pm, norm, X)
        assert np.mean(np.abs(emu - ref) > bound) > 0.05, plant


@pytest.mark.parametrize("seed", [0, 1])
def test_grad_bound_contains_fp32_emulation(seed):
    X, t = inp.mlp_samples(1000, seed=50 + seed)
    X, t = (np.float32(a).astype(np.float64) for a in (X, t))
    P = _params(12 + seed)
    norm = _norm(X)
    keep = ~mb.near_ties_grad_kernel(P, norm, X)
    assert 0.6 < keep.mean() < 1.0
    X, t = X[keep], t[keep]
    _, g_ref = mlp.loss_and_grad(P, norm, X, t)
    bound = mb.grad_bound(P, norm, X, t)
    g = emulate_grad(P, norm, X, t, np.random.default_rng(seed))
    assert np.all(np.abs(g - g_ref) <= bound)
    # per block the bound is a small fraction of the gradient's size
    for lo, hi in ((0, 224), (224, 256), (256, 1280), (1280, 1312), (1312, 1344), (1344, 1345)):
        assert np.max(bound[lo:hi]) <= 1e-3 * np.max(np.abs(g_ref[lo:hi])) + 1e-30


def test_grad_bound_catches_a_planted_mistake():
    X, t = inp.mlp_samples(1000, seed=52)
    X, t = (np.float32(a).astype(np.float64) for a in (X, t))
    P = _params(15)
    norm = _norm(X)
    keep = ~mb.near_ties_grad_kernel(P, norm, X)
    X, t = X[keep], t[keep]
    g = emulate_grad(P, norm, X, t, np.random.default_rng(3))
    # the oracle's derivative of one b2 entry taken from its neighbour's row
    _, g_ref = mlp.loss_and_grad(P, norm, X, t)
    g_bad = g_ref.copy()
    g_bad[1280 + 4] = g_ref[1280 + 5]
    bound = mb.grad_bound(P, norm, X, t)
    assert np.abs(g - g_bad)[1280 + 4] > bound[1280 + 4]
    # a bias of the oracle's network off by 1e-3
    Pm = P.copy()
    Pm[224 + 9] += 1e-3
    _, g_ref2 = mlp.loss_and_grad(Pm, norm, X, t)
    assert np.any(np.abs(g - g_ref2) > mb.grad_bound(Pm, norm, X, t))
