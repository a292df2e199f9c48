"""FP64 numpy oracle of the learned relaxation-time closure and of its training
data (TEST INFRASTRUCTURE: imported only by tests, the smoke check and the
benchmark's CPU legs).

The paper has no learned closure; every definition here is the reading of the
closure stated for this library:

- network: x (7 features) -> normalise -> 32 -> SiLU -> 32 -> SiLU -> y ->
  dtau = out_scale * softplus(y); the relaxation time is tau0 + dtau;
- features: the six components of the non-equilibrium stress Pi^neq
  (xx, yy, zz, xy, xz, yz) and the density;
- precision of the GPU forward: normalised inputs, first-layer weights,
  first-layer activations and second-layer weights are rounded to BF16
  (nearest even); products accumulate in FP32, biases and the last layer are
  FP32.  ``bf16=True`` applies the same roundings here, in FP64 otherwise;
- gradients treat every rounding as the identity (straight-through), the loss
  is the mean squared error of dtau, and the optimiser is Adam (Kingma & Ba);
- training data: the fine velocity field box-filtered by a factor f, the
  subgrid stress tau_sgs = mean(u u) - mean(u) mean(u), the filtered strain
  S from second-order central differences on the coarse grid, the eddy
  viscosity that best explains the deviatoric stress,
  nu_t = max(0, -tau_sgs_dev : S / (2 S : S)), the target dtau* = 3 nu_t (in
  coarse lattice units), and features from the Chapman-Enskog relation
  Pi^neq = -2 rho c_s^2 tau0 S = -(2/3) rho tau0 S.

Parameter layout (1345 values): W1[32][7], b1[32], W2[32][32], b2[32],
w3[32], b3.  Normalisation vector (16 values): mean[7], std[7], out_scale,
unused.

Pins: tests/test_oracle_mlp.py (central finite differences of the FP64 loss,
Adam's first step in closed form, exact filters and strains on polynomial
fields, the eddy-viscosity fit on a stress built from a known viscosity).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 7, 32
NPARAM = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    o = 0
    W1 = P[o:o + N_H * N_IN].reshape(N_H, N_IN); o += N_H * N_IN
    b1 = P[o:o + N_H]; o += N_H
    W2 = P[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = P[o:o + N_H]; o += N_H
    w3 = P[o:o + N_H]; o += N_H
    b3 = P[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), via FP32, as float64."""
    x32 = np.asarray(x, dtype=np.float32).copy()
    b = x32.view(np.uint32)
    lsb = (b >> 16) & np.uint32(1)
    b += np.uint32(0x7FFF) + lsb
    b &= np.uint32(0xFFFF0000)
    return x32.astype(np.float64)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def softplus(z):
    return np.where(z > 30.0, z, np.log1p(np.exp(np.minimum(z, 30.0))))


def forward(P, norm, X, bf=True):
    """dtau for samples X (n, 7); returns (dtau, cache)."""
    W1, b1, W2, b2, w3, b3 = unpack(P)
    norm = np.asarray(norm, dtype=np.float64)
    mean, std, scale = norm[:7], norm[7:14], norm[14]
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    xn = r((np.asarray(X, dtype=np.float64) - mean) / std)
    W1r, W2r = r(W1), r(W2)
    z1 = xn @ W1r.T + b1
    h1 = r(silu(z1))
    z2 = h1 @ W2r.T + b2
    h2 = silu(z2)
    y = h2 @ w3 + b3
    dtau = scale * softplus(y)
    return dtau, dict(xn=xn, W1r=W1r, W2r=W2r, z1=z1, h1=h1, z2=z2, h2=h2, y=y, scale=scale, w3=w3)


def loss_and_grad(P, norm, X, target, bf=True):
    """Mean squared error of dtau and its gradient with respect to P."""
    dtau, c = forward(P, norm, X, bf)
    n = len(dtau)
    e = dtau - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(e * e))
    dy = (2.0 / n) * e * c["scale"] * sigmoid(c["y"])
    dw3 = c["h2"].T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, c["w3"]) * dsilu(c["z2"])
    dW2 = dz2.T @ c["h1"]
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ c["W2r"]) * dsilu(c["z1"])
    dW1 = dz1.T @ c["xn"]
    db1 = dz1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dw3, db3)


def adam(P, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1); returns (P, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return P - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# Training data from a fine field
# ---------------------------------------------------------------------------
def box_filter(q, f):
    """Mean over f^3 blocks of the last three axes (nz, ny, nx)."""
    q = np.asarray(q, dtype=np.float64)
    *lead, nz, ny, nx = q.shape
    r = q.reshape(*lead, nz // f, f, ny // f, f, nx // f, f)
    return r.mean(axis=(-5, -3, -1))


def strain(u):
    """S_ab = (d_a u_b + d_b u_a)/2 with second-order central differences on a
    periodic grid of unit spacing; u has shape (3, nz, ny, nx).  Returns the
    six components (xx, yy, zz, xy, xz, yz)."""
    axis = {0: -1, 1: -2, 2: -3}  # x, y, z -> array axis

    def d(a, comp):
        return 0.5 * (np.roll(u[comp], -1, axis=axis[a]) - np.roll(u[comp], 1, axis=axis[a]))

    g = [[d(a, b) for b in range(3)] for a in range(3)]  # g[a][b] = d_a u_b
    S = lambda a, b: 0.5 * (g[a][b] + g[b][a])
    return np.stack([S(0, 0), S(1, 1), S(2, 2), S(0, 1), S(0, 2), S(1, 2)])


def eddy_viscosity(tau6, S6):
    """nu_t = max(0, -tau_dev : S / (2 S : S)), components (xx, yy, zz, xy, xz, yz)."""
    tr = (tau6[0] + tau6[1] + tau6[2]) / 3.0
    dev = np.stack([tau6[0] - tr, tau6[1] - tr, tau6[2] - tr, tau6[3], tau6[4], tau6[5]])
    w = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0]).reshape((6,) + (1,) * (tau6.ndim - 1))
    num = -np.sum(w * dev * S6, axis=0)
    den = 2.0 * np.sum(w * S6 * S6, axis=0)
    nu = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return np.maximum(nu, 0.0)


def coarse_samples(rho, u, f, tau0):
    """Features (Nc, 7) and targets dtau* (Nc,) from fine rho (nz,ny,nx) and
    u (3,nz,ny,nx), filtered by f; tau0 is the coarse BGK relaxation time."""
    rb = box_filter(rho, f)
    ub = box_filter(u, f)
    uu = np.stack([box_filter(u[a] * u[b], f) for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))])
    tau6 = uu - np.stack([ub[a] * ub[b] for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))])
    S6 = strain(ub)
    target = 3.0 * eddy_viscosity(tau6, S6)
    pi6 = -(2.0 / 3.0) * rb[None] * tau0 * S6
    X = np.concatenate([pi6, rb[None]], axis=0).reshape(7, -1).T
    return X, target.ravel()
