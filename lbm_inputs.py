"""Seeded synthetic inputs for the lattice Boltzmann workloads.

This module only generates inputs (initial fields, tag layouts, random sphere
lists, random populations).  It holds none of the method's arithmetic, and both
the FP64 oracle and the CUDA library consume what it produces.

Array conventions: scalar fields have shape (nz, ny, nx) (x fastest), vector
fields (3, nz, ny, nx), populations (Q, nz, ny, nx).
"""
from __future__ import annotations

import numpy as np

# Tag values of the library's tag scheme (integer per node, Sec. 2.3.2).
FLUID, FORCED, SOLID, WALL0 = 0, 1, 2, 3


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def tgv2d(nx: int, ny: int, nz: int, u0: float, rho0: float = 1.0):
    """z-extruded 2D Taylor-Green vortex with wavenumber k = 2*pi/nx.

    u = (-u0 cos kx sin ky, u0 sin kx cos ky, 0) and the matching pressure
    p - p0 = -(rho0 u0^2 / 4)(cos 2kx + cos 2ky), turned into a density with
    rho = rho0 + 3 (p - p0) (c_s^2 = 1/3).  Requires nx == ny.
    """
    if nx != ny:
        raise ValueError("the 2D Taylor-Green vortex needs nx == ny")
    x, y, _ = _grid(nx, ny, nz)
    k = 2.0 * np.pi / nx
    u = np.zeros((3, nz, ny, nx))
    u[0] = -u0 * np.cos(k * x) * np.sin(k * y)
    u[1] = u0 * np.sin(k * x) * np.cos(k * y)
    dp = -(rho0 * u0 * u0 / 4.0) * (np.cos(2 * k * x) + np.cos(2 * k * y))
    rho = rho0 + 3.0 * dp
    return rho, u


def tgv3d(n: int, u0: float, rho0: float = 1.0):
    """3D Taylor-Green vortex of Sec. 3.1 on an n^3 periodic box.

    Node i sits at the angle X = 2 pi i / n.  u_x = u0 sin X cos Y cos Z,
    u_y = -u0 cos X sin Y cos Z, u_z = 0, and the pressure deviation
    p - p0 = (rho0 u0^2 / 16)(cos 2Z + 2)(cos 2X + cos 2Y), read with u0
    squared for dimensional consistency, gives rho = rho0 + 3 (p - p0).
    """
    x, y, z = _grid(n, n, n)
    s = 2.0 * np.pi / n
    X, Y, Z = s * x, s * y, s * z
    u = np.zeros((3, n, n, n))
    u[0] = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    dp = (rho0 * u0 * u0 / 16.0) * (np.cos(2 * Z) + 2.0) * (np.cos(2 * X) + np.cos(2 * Y))
    rho = rho0 + 3.0 * dp
    return rho, u


def cavity_tags(n: int, ny: int | None = None, nz: int | None = None) -> np.ndarray:
    """Lid-driven cavity (Sec. 3.2): resting walls on the x, y faces and the
    bottom z face, the moving lid WALL0 over the whole top plane z = nz-1
    (edges included).  Interior fluid is (n-2) x (ny-2) x (nz-2)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    t = np.full((nz, ny, n), FLUID, dtype=np.uint8)
    t[:, :, 0] = SOLID
    t[:, :, -1] = SOLID
    t[:, 0, :] = SOLID
    t[:, -1, :] = SOLID
    t[0, :, :] = SOLID
    t[-1, :, :] = WALL0
    return t


def channel_tags(nx: int, ny: int, nz: int, *, moving_top: bool = False, fluid_tag: int = FORCED) -> np.ndarray:
    """Plane channel normal to y: solid rows at y = 0 and y = ny-1 (or a moving
    WALL0 top row for Couette flow); fluid rows carry ``fluid_tag``."""
    t = np.full((nz, ny, nx), fluid_tag, dtype=np.uint8)
    t[:, 0, :] = SOLID
    t[:, -1, :] = WALL0 if moving_top else SOLID
    return t


def sphere_list(shape, seed: int, rmin: float = 4.0, rmax: float = 10.0, count: int = 100000):
    """Seeded list of sphere centres (integer voxels) and radii U[rmin, rmax).

    Generated with numpy's PCG64 generator; centres and radii are drawn as two
    separate blocks so that a longer list extends a shorter one.
    """
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    cx = rng.integers(0, nx, size=count)
    cy = rng.integers(0, ny, size=count)
    cz = rng.integers(0, nz, size=count)
    r = rng.uniform(rmin, rmax, size=count)
    centres = np.stack([cx, cy, cz], axis=1).astype(np.int32)
    return centres, r.astype(np.float64)


def random_populations(weights, shape, seed: int, amplitude: float = 0.05) -> np.ndarray:
    """Positive random populations f_i = w_i (1 + amplitude * U(-1, 1))."""
    w = np.asarray(weights, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.uniform(-1.0, 1.0, size=(len(w),) + tuple(shape))
    return w.reshape((-1,) + (1,) * len(shape)) * (1.0 + amplitude * noise)


def random_tags(shape, seed: int, p_solid: float = 0.1, p_forced: float = 0.2, p_wall: float = 0.05,
                n_walls: int = 2) -> np.ndarray:
    """Random tag field mixing fluid, forced, solid and moving-wall nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(size=shape)
    t = np.full(shape, FLUID, dtype=np.uint8)
    t[r < p_forced + p_solid + p_wall] = FORCED
    t[r < p_solid + p_wall] = SOLID
    walls = r < p_wall
    t[walls] = (WALL0 + rng.integers(0, n_walls, size=int(walls.sum()))).astype(np.uint8)
    return t


def random_velocity_field(shape, seed: int, amplitude: float = 0.05):
    """Random rho ~ 1 + small, u ~ amplitude * U(-1, 1) fields."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = 1.0 + 0.01 * rng.uniform(-1.0, 1.0, size=shape)
    u = amplitude * rng.uniform(-1.0, 1.0, size=(3,) + tuple(shape))
    return rho, u


def mlp_init(seed: int, n_in: int = 7, n_h: int = 32) -> np.ndarray:
    """Initial closure weights (layout W1[32][7], b1, W2[32][32], b2, w3, b3):
    uniform Glorot-style weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def glorot(fan_out, fan_in):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=(fan_out, fan_in))

    W1 = glorot(n_h, n_in)
    W2 = glorot(n_h, n_h)
    w3 = glorot(1, n_h)[0]
    return np.concatenate([W1.ravel(), np.zeros(n_h), W2.ravel(), np.zeros(n_h), w3, [0.0]])


def mlp_samples(n: int, seed: int, scale: float = 1e-3):
    """Random closure features (n, 7): stress-like components ~ N(0, scale),
    density ~ 1 + N(0, 0.01); and positive targets ~ scale * U(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.empty((n, 7))
    X[:, :6] = rng.normal(0.0, scale, size=(n, 6))
    X[:, 6] = 1.0 + rng.normal(0.0, 0.01, size=n)
    y = scale * rng.uniform(0.0, 1.0, size=n)
    return X, y
