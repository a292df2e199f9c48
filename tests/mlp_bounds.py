"""Error bounds for comparing the GPU closure network with the FP64 oracle
(oracle/mlp.py), sample by sample and parameter by parameter.  Test
infrastructure: used by tests/test_gpu_mlp.py, and checked on the CPU by
tests/test_mlp_bounds_cpu.py against an FP32 emulation of the GPU arithmetic.

Both sides apply the same BF16 roundings (normalised inputs, W1, first-layer
activations, W2).  The GPU computes the values that get rounded in FP32, so a
rounding decision can only differ where the exact value lies within the FP32
error band of a BF16 rounding midpoint (a "near tie"); anywhere else both
sides round to the same BF16 number and the difference that remains is FP32
arithmetic.  The bounds below follow that error through the network with
absolute values (first order in the errors, then doubled):

- FP32 sums: at most k * 2^-24 of the sum of the magnitudes of their k terms;
- SiLU of the inference tiles: (z/2)(1 + tanh(z/2)) with the hardware tanh,
  whose relative error is about 2^-11; 2^-10 is used;
- SiLU / sigmoid of the gradient kernel: __expf and __fdividef, a few FP32
  ulps for the arguments that occur (2^-19 relative is used);
- a near tie flips the rounded value by one BF16 ulp of it.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

U32 = 2.0 ** -24
TANH_REL = 2.0 ** -10


def bf16_ulp(v):
    """Spacing of BF16 numbers (8 significant bits) at |v|."""
    a = np.abs(np.asarray(v, dtype=np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 2.0 ** -133)


def midpoint_distance(v):
    """Distance of v from the nearest BF16 rounding midpoint."""
    a = np.abs(np.asarray(v, dtype=np.float64))
    ulp = bf16_ulp(a)
    r = a / ulp
    return np.abs(r - np.floor(r) - 0.5) * ulp


def _silu_tile_err(z):
    """Absolute error of the tiles' SiLU: (z/2) tanh(z/2) carries the tanh
    error; the final FMA adds one FP32 rounding."""
    hz = 0.5 * z
    return np.abs(hz * np.tanh(hz)) * TANH_REL + 2 * U32 * np.abs(mlp.silu(z)) + 1e-45


def forward_bound(P, norm, X):
    """Per-sample bound on |dtau_gpu - dtau_oracle| for the inference tiles
    (batch tcgen05 tile and the collide kernel's warp tile)."""
    dtau, c = mlp.forward(P, norm, X, bf=True)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(P)
    norm = np.asarray(norm, dtype=np.float64)
    mean, std, scale = norm[:7], norm[7:14], norm[14]
    W1r, W2r = c["W1r"], c["W2r"]
    xn_pre = (np.asarray(X, dtype=np.float64) - mean) / std
    # normalisation in FP32: difference, reciprocal, product
    e_xn = 4 * U32 * np.abs(xn_pre) + 4 * U32 * np.abs(mean / std)
    flip_xn = np.where(midpoint_distance(xn_pre) <= e_xn, bf16_ulp(xn_pre), 0.0)
    xn = c["xn"]
    # layer 1: accumulation error band plus the effect of flipped inputs
    e_z1 = np.abs(W1r) @ flip_xn.T
    e_z1 = e_z1.T + 10 * U32 * (np.abs(xn) @ np.abs(W1r).T + np.abs(b1))
    z1 = c["z1"]
    e_s1 = np.abs(mlp.dsilu(z1)) * e_z1 + _silu_tile_err(z1)
    s1 = mlp.silu(z1)
    flip_h1 = np.where(midpoint_distance(s1) <= e_s1, bf16_ulp(s1), 0.0)
    h1 = c["h1"]
    e_z2 = flip_h1 @ np.abs(W2r).T + 36 * U32 * (np.abs(h1) @ np.abs(W2r).T + np.abs(b2))
    z2 = c["z2"]
    e_h2 = np.abs(mlp.dsilu(z2)) * e_z2 + _silu_tile_err(z2)
    h2 = c["h2"]
    e_y = e_h2 @ np.abs(w3) + 36 * U32 * (np.abs(h2) @ np.abs(w3) + abs(b3))
    e_dtau = scale * mlp.sigmoid(c["y"]) * e_y + 16 * U32 * np.abs(dtau)
    flips = (flip_xn > 0).sum(axis=1) + (flip_h1 > 0).sum(axis=1)
    return dtau, 2.0 * e_dtau + 1e-30, flips


def near_ties_grad_kernel(P, norm, X):
    """Samples whose BF16 roundings in the gradient kernel could differ from
    the oracle's (a normalised input or first-layer activation within the
    FP32 error band of a midpoint).  That kernel computes SiLU as
    z * sigmoid(z) with __expf / __fdividef."""
    _, c = mlp.forward(P, norm, X, bf=True)
    W1, b1, *_ = mlp.unpack(P)
    norm = np.asarray(norm, dtype=np.float64)
    mean, std = norm[:7], norm[7:14]
    xn_pre = (np.asarray(X, dtype=np.float64) - mean) / std
    near = (midpoint_distance(xn_pre) <= 8 * U32 * (np.abs(xn_pre) + np.abs(mean / std))).any(axis=1)
    z1 = c["z1"]
    e_z1 = 10 * U32 * (np.abs(c["xn"]) @ np.abs(c["W1r"]).T + np.abs(b1))
    s1 = mlp.silu(z1)
    e_s1 = np.abs(mlp.dsilu(z1)) * e_z1 + 2.0 ** -19 * np.abs(s1) + 1e-45
    near |= (midpoint_distance(s1) <= 2 * e_s1).any(axis=1)
    return near


def grad_bound(P, norm, X, target, n_total=None):
    """Per-parameter bound on |grad_gpu - grad_oracle| for samples without near
    ties.  Every term of the gradient is followed with absolute values:
    |dy|, |dz2| = |dy| |w3| |silu'(z2)|, |dz1| = (|dz2| |W2r|) |silu'(z1)|,
    with the prediction error |dtau - target| widened by the FP32 error of
    dtau (where dtau ~ target the difference has no correct digits).  The
    FP32 error of a parameter's gradient is then at most
    (chain length + samples per block + blocks) * 2^-24 times its sum of
    term magnitudes."""
    dtau, c = mlp.forward(P, norm, X, bf=True)
    n = len(dtau) if n_total is None else n_total
    W1, b1, W2, b2, w3, b3 = mlp.unpack(P)
    scale = float(np.asarray(norm)[14])
    W1r, W2r = np.abs(c["W1r"]), np.abs(c["W2r"])
    h1, h2, xn = np.abs(c["h1"]), np.abs(c["h2"]), np.abs(c["xn"])
    ds1, ds2 = np.abs(mlp.dsilu(c["z1"])), np.abs(mlp.dsilu(c["z2"]))
    sy = mlp.sigmoid(c["y"])
    # FP32 error of dtau: accumulations of both layers and the output layer
    mag_z2 = h1 @ W2r.T + np.abs(b2)
    mag_y = h2 @ np.abs(w3) + abs(b3) + (ds2 * mag_z2) @ np.abs(w3)
    e_dt = scale * sy * 48 * U32 * mag_y + 16 * U32 * np.abs(dtau)
    err = np.abs(dtau - np.asarray(target, dtype=np.float64)) + e_dt
    dy = (2.0 / n) * err * scale * sy
    dz2 = dy[:, None] * np.abs(w3)[None, :] * ds2
    dz1 = (dz2 @ W2r) * ds1
    A = mlp.pack(dz1.T @ xn, dz1.sum(axis=0), dz2.T @ h1, dz2.sum(axis=0), h2.T @ dy, dy.sum())
    blocks = -(-len(dtau) // 128)
    k = 64 + 128 + blocks
    return 2.0 * k * U32 * A + 1e-30
