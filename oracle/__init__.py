"""FP64 CPU oracle of the lattice Boltzmann hot path.

TEST INFRASTRUCTURE.  This package is the plain, slow reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
does.  It shares no code with the CUDA library: the C half (``lbm_oracle.c``)
and the numpy half (``mlp.py``) restate the method from the paper's text.

Parity status of each function is stated where it is defined; the pins live
in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "lbm_oracle.c"
_LIB = _HERE / "_build" / "liblbm_oracle.so"
_LIB_OMP = _HERE / "_build" / "liblbm_oracle_omp.so"

# Tag values and closure ids of the oracle (its own statement of the tag
# scheme of Sec. 2.3.2; the CUDA library declares the same values itself).
FLUID, FORCED, SOLID, WALL0 = 0, 1, 2, 3
NWALLS = 8
BGK, SMAGORINSKY, MLP, STREAM_ONLY, TRT = 0, 1, 2, 3, 4
F64, F32, F16, BF16, F16_SCALED = 0, 1, 2, 3, 4
MLP_NPARAM = 32 * 7 + 32 + 32 * 32 + 32 + 32 + 1


def build(force: bool = False, openmp: bool = False) -> Path:
    """Compiles the C oracle into a shared library: plain gcc (the build the
    tests use), or with OpenMP over the z planes of a step (the build the
    CPU baseline times; same arithmetic per node, so the same results)."""
    lib_path = _LIB_OMP if openmp else _LIB
    lib_path.parent.mkdir(exist_ok=True)
    if force or not lib_path.exists() or lib_path.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = lib_path.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               *(["-fopenmp"] if openmp else []), str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib_path)
    return lib_path


class Params(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("closure", ctypes.c_int),
        ("cs_smag", ctypes.c_double),
        ("wall_u", (ctypes.c_double * 3) * NWALLS),
        ("rho_wall", ctypes.c_double),
        ("mlp_params", ctypes.POINTER(ctypes.c_double)),
        ("mlp_norm", ctypes.POINTER(ctypes.c_double)),
        ("mlp_bf16", ctypes.c_int),
        ("trt_magic", ctypes.c_double),
        ("wall_rho_local", ctypes.c_int),
    ]


class Reduction(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double),
        ("mom", ctypes.c_double * 3),
        ("vel", ctypes.c_double * 3),
        ("ke", ctypes.c_double),
        ("ke_rho", ctypes.c_double),
        ("umax", ctypes.c_double),
        ("n_fluid", ctypes.c_longlong),
        ("nonfinite", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        return {
            "mass": self.mass, "mom": list(self.mom), "vel": list(self.vel), "ke": self.ke,
            "ke_rho": self.ke_rho, "umax": self.umax, "n_fluid": self.n_fluid,
            "nonfinite": self.nonfinite,
        }


_libs = {}


def lib(openmp: bool = False):
    """The plain oracle library, or its OpenMP build (openmp=True)."""
    if openmp not in _libs:
        _lib = ctypes.CDLL(str(build(openmp=openmp)))
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.orc_set_threads.argtypes = [I]
        _lib.orc_lattice.argtypes = [I, P, P, P]
        _lib.orc_equilibrium.argtypes = [I, D, P, P]
        _lib.orc_equilibrium.restype = None
        _lib.orc_tau_smagorinsky.argtypes = [D, D, D, P]
        _lib.orc_tau_smagorinsky.restype = D
        _lib.orc_round_scalar.argtypes = [D, I]
        _lib.orc_round_scalar.restype = D
        _lib.orc_round_storage.argtypes = [I, ctypes.c_longlong, P, I]
        _lib.orc_mlp_dtau.argtypes = [P, P, I, P]
        _lib.orc_mlp_dtau.restype = D
        _lib.orc_step.argtypes = [I, I, I, I, P, ctypes.POINTER(Params), P, P]
        _lib.orc_closure_features.argtypes = [I, I, I, I, P, ctypes.POINTER(Params), P, P]
        _lib.orc_init_equilibrium.argtypes = [I, I, I, I, P, P, P]
        _lib.orc_moments.argtypes = [I, I, I, I, P, ctypes.POINTER(Params), P, P, P]
        _lib.orc_reduce.argtypes = [I, I, I, I, P, ctypes.POINTER(Params), P, ctypes.POINTER(Reduction)]
        _lib.orc_enstrophy.argtypes = [I, I, I, P, P]
        _lib.orc_enstrophy.restype = D
        _lib.orc_spheres.argtypes = [I, I, I, P, P, I, D, ctypes.c_ubyte, ctypes.c_ubyte, P, P]
        _libs[openmp] = _lib
    return _libs[openmp]


def set_threads(n: int) -> int:
    """Threads of the OpenMP build's steps (n <= 0 keeps the current count);
    returns the count in use."""
    return lib(openmp=True).orc_set_threads(int(n))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def lattice(Q: int):
    """Velocity set c[Q][3], weights w[Q] and opposite index opp[Q]."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    if lib().orc_lattice(Q, _ptr(c), _ptr(w), _ptr(opp)) != 0:
        raise ValueError(f"unknown lattice Q={Q}")
    return c, w, opp


def equilibrium(Q: int, rho: float, u) -> np.ndarray:
    feq = np.zeros(Q)
    uu = _f64(u)
    lib().orc_equilibrium(Q, float(rho), _ptr(uu), _ptr(feq))
    return feq


def tau_smagorinsky(tau0: float, cs: float, rho: float, pi6) -> float:
    p = _f64(pi6)
    return lib().orc_tau_smagorinsky(tau0, cs, rho, _ptr(p))


def round_scalar(h: float, dtype: int) -> float:
    return lib().orc_round_scalar(float(h), int(dtype))


def round_storage(f: np.ndarray, dtype: int) -> np.ndarray:
    """Returns w_i + round(f_i - w_i) in the emulated storage type."""
    out = np.ascontiguousarray(f, dtype=np.float64).copy()
    Q = out.shape[0]
    lib().orc_round_storage(Q, out[0].size, _ptr(out), int(dtype))
    return out


class Problem:
    """A lattice of shape (nz, ny, nx) with tags and parameters.

    ``f`` arrays have shape (Q, nz, ny, nx), unshifted, FP64.
    """

    def __init__(self, Q: int, nx: int, ny: int, nz: int, tags=None, *, tau: float,
                 force=(0.0, 0.0, 0.0), closure: int = BGK, cs_smag: float = 0.0,
                 wall_u=None, rho_wall: float = 1.0, mlp_params=None, mlp_norm=None,
                 mlp_bf16: bool = False, trt_magic: float = 3.0 / 16.0, wall_rho_local: bool = False,
                 openmp: bool = False):
        self.Q, self.nx, self.ny, self.nz = Q, nx, ny, nz
        self._lib = lib(openmp=openmp)
        self.tags = None if tags is None else np.ascontiguousarray(tags, dtype=np.uint8).reshape(nz, ny, nx)
        self.p = Params()
        self.p.tau = tau
        for a in range(3):
            self.p.force[a] = force[a]
        self.p.closure = closure
        self.p.cs_smag = cs_smag
        if wall_u is not None:
            for k, v in enumerate(wall_u):
                for a in range(3):
                    self.p.wall_u[k][a] = v[a]
        self.p.rho_wall = rho_wall
        self.p.wall_rho_local = 1 if wall_rho_local else 0
        self._mlp = None if mlp_params is None else _f64(mlp_params)
        self._norm = None if mlp_norm is None else _f64(mlp_norm)
        if self._mlp is not None:
            self.p.mlp_params = self._mlp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            self.p.mlp_norm = self._norm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.p.mlp_bf16 = int(mlp_bf16)
        self.p.trt_magic = trt_magic

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def init_equilibrium(self, rho=None, u=None) -> np.ndarray:
        f = np.zeros((self.Q,) + self.shape)
        r = _f64(rho)
        v = _f64(u)
        self._lib.orc_init_equilibrium(self.Q, self.nx, self.ny, self.nz, _ptr(r), _ptr(v), _ptr(f))
        return f

    def step(self, f: np.ndarray, n: int = 1) -> np.ndarray:
        a = _f64(f).copy()
        b = np.empty_like(a)
        for _ in range(n):
            rc = self._lib.orc_step(self.Q, self.nx, self.ny, self.nz, _ptr(self.tags), ctypes.byref(self.p),
                                    _ptr(a), _ptr(b))
            if rc != 0:
                raise ValueError("oracle step rejected its arguments")
            a, b = b, a
        return a

    def closure_features(self, f: np.ndarray) -> np.ndarray:
        """Inputs of the learned closure for the step that would follow f:
        (Pi^neq xx, yy, zz, xy, xz, yz, rho) of each node's pulled set, shape
        (nz, ny, nx, 7), zeros on solid and wall nodes."""
        x = np.zeros(self.shape + (7,))
        ff = _f64(f)
        rc = lib().orc_closure_features(self.Q, self.nx, self.ny, self.nz, _ptr(self.tags), ctypes.byref(self.p),
                                        _ptr(ff), _ptr(x))
        if rc != 0:
            raise ValueError("oracle closure features rejected their arguments")
        return x

    def moments(self, f: np.ndarray):
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        ff = _f64(f)
        lib().orc_moments(self.Q, self.nx, self.ny, self.nz, _ptr(self.tags), ctypes.byref(self.p), _ptr(ff),
                          _ptr(rho), _ptr(u))
        return rho, u

    def reduce(self, f: np.ndarray) -> dict:
        out = Reduction()
        ff = _f64(f)
        lib().orc_reduce(self.Q, self.nx, self.ny, self.nz, _ptr(self.tags), ctypes.byref(self.p), _ptr(ff),
                         ctypes.byref(out))
        return out.as_dict()


def init_equilibrium(Q, rho, u):
    """Equilibrium populations for fields rho (nz,ny,nx) and u (3,nz,ny,nx)."""
    nz, ny, nx = np.shape(rho)
    return Problem(Q, nx, ny, nz, tau=1.0).init_equilibrium(rho, u)


def mlp_dtau(params, norm, x, bf16: bool = False) -> float:
    P = _f64(params)
    nm = _f64(norm)
    xx = _f64(x)
    return lib().orc_mlp_dtau(_ptr(P), _ptr(nm), int(bf16), _ptr(xx))


def enstrophy(u: np.ndarray, return_omega: bool = False):
    """Enstrophy average (1/N) sum |curl u|^2/2 with the 8th-order centred curl."""
    uu = _f64(u)
    _, nz, ny, nx = uu.shape
    om = np.zeros_like(uu) if return_omega else None
    e = lib().orc_enstrophy(nx, ny, nz, _ptr(uu), _ptr(om))
    return (e, om) if return_omega else e


def spheres(shape, centres, radii, target: float, solid_tag: int = SOLID, pore_tag: int = FLUID):
    """Sequential random-sphere medium; returns (tags, n_used, porosity)."""
    nz, ny, nx = shape
    c = np.ascontiguousarray(centres, dtype=np.int32)
    r = _f64(radii)
    tags = np.zeros(shape, dtype=np.uint8)
    por = np.zeros(1)
    used = lib().orc_spheres(nx, ny, nz, _ptr(c), _ptr(r), len(r), float(target), solid_tag, pore_tag,
                             _ptr(tags), _ptr(por))
    return tags, used, float(por[0])


def kinetic_energy_fields(u: np.ndarray) -> float:
    """k = <|u|^2/2> over all cells (Sec. 3.1)."""
    return float(0.5 * np.mean(np.sum(np.asarray(u, dtype=np.float64) ** 2, axis=0)))


def permeability(u_mean_x: float, tau: float, g: float) -> float:
    """Body-force form of the Sec. 3.3 permeability: k = u_mean * nu / g, with
    nu = (tau - 1/2)/3 and u_mean averaged over all cells (solid = 0)."""
    return u_mean_x * ((tau - 0.5) / 3.0) / g


def glups_peak(bandwidth_bytes_per_s: float, Q: int, n_store: int, extra_bytes: int = 12) -> float:
    """Sec. 4.1 performance model: cells per second = B / n_t with
    n_t = 2 Q n_store + extra (the paper counts 8 + 4 bytes of flags)."""
    return bandwidth_bytes_per_s / (2 * Q * n_store + extra_bytes) / 1e9


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
