"""Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/liblbm.so``; this
module converts numpy arrays / torch tensors to pointers, passes torch's
caching allocator and current CUDA stream to the library, and turns status
codes into exceptions.  There is no CPU fallback: without the compiled
library, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "liblbm.so"

# Values of include/lbm.h.
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_UNSTABLE, ERR_TIMEOUT = range(7)
D3Q19, D3Q27 = 19, 27
F64, F32, F16_SHIFTED, BF16_SHIFTED, F16_SCALED = 0, 1, 2, 3, 4
DTYPES = {"f64": F64, "f32": F32, "f16": F16_SHIFTED, "bf16": BF16_SHIFTED, "f16s": F16_SCALED}
# torch element type of each storage type (scaled FP16 stores FP16 of h * 2^12)
STORAGE_TORCH_DTYPE = {F64: "float64", F32: "float32", F16_SHIFTED: "float16", BF16_SHIFTED: "bfloat16",
                       F16_SCALED: "float16"}
PATTERN_AB, PATTERN_AA = 0, 1
PATTERNS = {"ab": PATTERN_AB, "aa": PATTERN_AA}
TAG_FLUID, TAG_FORCED, TAG_SOLID, TAG_WALL0, NWALLS = 0, 1, 2, 3, 8
NTAGS = TAG_WALL0 + NWALLS
CLOSURE_BGK, CLOSURE_SMAGORINSKY, CLOSURE_MLP, CLOSURE_STREAM_ONLY, CLOSURE_TRT = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_STATE", 5: "ERR_UNSTABLE",
                6: "ERR_TIMEOUT"}


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class UnstableError(LBMError):
    """A reduction met a non-finite density or velocity."""

    def __init__(self, status, message, reduction):
        super().__init__(status, message)
        self.reduction = reduction


class Params(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("closure", ctypes.c_int),
        ("cs_smag", ctypes.c_double),
        ("wall_u", (ctypes.c_double * 3) * NWALLS),
        ("rho_wall", ctypes.c_double),
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
        return {"mass": self.mass, "mom": list(self.mom), "vel": list(self.vel), "ke": self.ke,
                "ke_rho": self.ke_rho, "umax": self.umax, "n_fluid": self.n_fluid, "nonfinite": self.nonfinite}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


# name -> (restype, argtypes) of every C ABI entry point.
_P, _I, _D, _LL, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t
SIGNATURES = {
    "lbm_create": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(Allocator), _P, ctypes.POINTER(_P)]),
    "lbm_create_ex": (_I, [_I, _I, _I, _I, _I, _I, ctypes.POINTER(Allocator), _P, ctypes.POINTER(_P)]),
    "lbm_closure_features": (_I, [_P, _P, _I]),
    "lbm_destroy": (_I, [_P]),
    "lbm_set_params": (_I, [_P, ctypes.POINTER(Params)]),
    "lbm_set_tags": (_I, [_P, _P, _I]),
    "lbm_get_tags": (_I, [_P, _P, _I]),
    "lbm_tag_census": (_I, [_P, _P]),
    "lbm_init_equilibrium": (_I, [_P, _P, _P, _I]),
    "lbm_step": (_I, [_P, _I]),
    "lbm_step_count": (_I, [_P, ctypes.POINTER(_LL)]),
    "lbm_use_graphs": (_I, [_P, _I]),
    "lbm_step_reduce": (_I, [_P, _I, ctypes.POINTER(Reduction)]),
    "lbm_moments": (_I, [_P, _P, _P, _I]),
    "lbm_reduce": (_I, [_P, ctypes.POINTER(Reduction)]),
    "lbm_sync": (_I, [_P, _I]),
    "lbm_get_populations": (_I, [_P, _P, _I]),
    "lbm_set_populations": (_I, [_P, _P, _I]),
    "lbm_get_state": (_I, [_P, _P, _SZ, ctypes.POINTER(_I), ctypes.POINTER(_LL), _I]),
    "lbm_set_state": (_I, [_P, _P, _SZ, _I, _LL, _I]),
    "lbm_info": (_I, [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lbm_fp64_fma_rate": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_geometry_spheres": (_I, [_P, _P, _P, _I, _D, ctypes.c_uint8, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "lbm_enstrophy": (_I, [_P, ctypes.POINTER(_D)]),
    "lbm_set_closure_weights": (_I, [_P, _P, _P, _I]),
    "lbm_mlp_forward": (_I, [_P, _P, _P, _I, _P, _P]),
    "lbm_mlp_workspace_bytes": (_SZ, [_I]),
    "lbm_mlp_loss_grad": (_I, [_P, _P, _P, _P, _I, _P, _P, _P, _SZ, _P]),
    "lbm_mlp_adam": (_I, [_P, _P, _P, _P, _I, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "lbm_coarse_samples": (_I, [_P, _P, _I, _I, _I, _I, _D, _P, _P, _P]),
    "lbm_box_filter": (_I, [_P, _I, _I, _I, _I, _I, _P, _P]),
    "lbm_reduce_noalloc": (_I, [_P, _I, _I, _I, _I, _I, _P, ctypes.POINTER(Params), _P, ctypes.POINTER(Reduction)]),
}

_lib = None


def library_path() -> Path:
    return _LIB_PATH


def load():
    """Loads the compiled library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise ImportError(f"CUDA library {_LIB_PATH} is missing: run __graft_entry__.build() first")
        lib = ctypes.CDLL(str(_LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, ctx=None):
    if status != OK:
        msg = load().lbm_last_error(ctx).decode(errors="replace")
        raise LBMError(status, msg)


def _buf(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, 0, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != dtype_torch(dtype):
                raise TypeError(f"expected a {dtype} tensor, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


def dtype_torch(np_dtype):
    import torch
    return {np.float64: torch.float64, np.uint8: torch.uint8, np.float32: torch.float32,
            np.int32: torch.int32}[np.dtype(np_dtype).type]


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching
    allocator on the given device."""

    def __init__(self, device: int):
        import torch
        self.device = device
        self._torch = torch

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0))
            except Exception:  # noqa: BLE001 - report as NULL (LBM_ERR_OOM)
                return None

        def _free(ptr, nbytes, stream, user):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self._alloc = ALLOC_FN(_alloc)
        self._free = FREE_FN(_free)
        self.struct = Allocator(self._alloc, self._free, None)


class Lattice:
    """One lattice (a library context) on one GPU.

    shape is (nx, ny, nz); fields use numpy order (nz, ny, nx) with x fastest.
    """

    def __init__(self, nx: int, ny: int, nz: int, lattice: int = D3Q19, dtype="f32", *, device: int = 0,
                 stream=None, torch_allocator: bool = True, pattern: str = "ab"):
        lib = load()
        self.pattern = PATTERNS[pattern] if isinstance(pattern, str) else int(pattern)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.Q = int(lattice)
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.device = device
        self._alloc = None
        stream_handle = None
        try:
            import torch
            if torch.cuda.is_available():
                torch.cuda.set_device(device)
                if stream is None:
                    stream = torch.cuda.current_stream(device)
                stream_handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
                if torch_allocator:
                    self._alloc = _TorchAllocator(device)
        except ImportError:  # pragma: no cover
            pass
        self._stream = stream
        ctx = ctypes.c_void_p()
        alloc_ptr = ctypes.byref(self._alloc.struct) if self._alloc else None
        _check(lib.lbm_create_ex(nx, ny, nz, self.Q, self.dtype, self.pattern, alloc_ptr, stream_handle,
                                 ctypes.byref(ctx)))
        self._ctx = ctx
        self._closure = None  # host copy of the closure weights, for checkpoints
        self.params = Params()
        self.params.tau = 1.0
        self.params.rho_wall = 1.0
        self.params.trt_magic = 3.0 / 16.0

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            load().lbm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def ctx(self):
        return self._ctx

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def _call(self, name, *args):
        st = getattr(load(), name)(self._ctx, *args)
        _check(st, self._ctx)
        return st

    # -- configuration -------------------------------------------------------
    def set_params(self, tau: float, *, force=(0.0, 0.0, 0.0), closure: int = CLOSURE_BGK, cs_smag: float = 0.0,
                   wall_u=None, rho_wall: float = 1.0, trt_magic: float = 3.0 / 16.0,
                   wall_rho_local: bool = False):
        p = Params()
        p.tau = tau
        for a in range(3):
            p.force[a] = force[a]
        p.closure = closure
        p.cs_smag = cs_smag
        if wall_u is not None:
            for k, v in enumerate(wall_u):
                for a in range(3):
                    p.wall_u[k][a] = v[a]
        p.rho_wall = rho_wall
        p.trt_magic = trt_magic
        p.wall_rho_local = 1 if wall_rho_local else 0
        self._call("lbm_set_params", ctypes.byref(p))
        self.params = p

    def set_tags(self, tags):
        ptr, dev, keep = _buf(tags, np.uint8)
        count = keep.numel() if hasattr(keep, "numel") else keep.size
        if count != self.N:
            raise ValueError("tags must have nx*ny*nz entries")
        self._call("lbm_set_tags", ptr, dev)

    def get_tags(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.uint8)
        self._call("lbm_get_tags", out.ctypes.data_as(ctypes.c_void_p), 0)
        return out

    def census(self) -> np.ndarray:
        out = np.zeros(NTAGS, dtype=np.int64)
        self._call("lbm_tag_census", out.ctypes.data_as(ctypes.c_void_p))
        return out

    # -- state -----------------------------------------------------------------
    def init_equilibrium(self, rho=None, u=None):
        r, dr, kr = _buf(rho, np.float64)
        v, dv, kv = _buf(u, np.float64)
        if rho is not None and u is not None and dr != dv:
            raise ValueError("rho and u must both be on the host or both on the device")
        self._call("lbm_init_equilibrium", r, v, dr if rho is not None else dv)

    def step(self, n: int = 1):
        self._call("lbm_step", int(n))

    def use_graphs(self, enable: bool = True):
        self._call("lbm_use_graphs", int(bool(enable)))

    def step_count(self) -> int:
        v = ctypes.c_longlong()
        self._call("lbm_step_count", ctypes.byref(v))
        return v.value

    def sync(self, timeout_ms: int = -1):
        self._call("lbm_sync", int(timeout_ms))

    def moments(self, rho=None, u=None):
        """Returns (rho, u) as numpy arrays, or fills the given device tensors."""
        if rho is None and u is None:
            rho = np.empty(self.shape)
            u = np.empty((3,) + self.shape)
        r, dr, _ = _buf(rho, np.float64)
        v, dv, _ = _buf(u, np.float64)
        self._call("lbm_moments", r, v, dr if rho is not None else dv)
        return rho, u

    def reduce(self) -> dict:
        out = Reduction()
        st = load().lbm_reduce(self._ctx, ctypes.byref(out))
        if st == ERR_UNSTABLE:
            raise UnstableError(st, load().lbm_last_error(self._ctx).decode(), out.as_dict())
        _check(st, self._ctx)
        return out.as_dict()

    def step_reduce(self, n: int) -> dict:
        """n steps and the reduction of the new state, fused into the last step."""
        out = Reduction()
        st = load().lbm_step_reduce(self._ctx, int(n), ctypes.byref(out))
        if st == ERR_UNSTABLE:
            raise UnstableError(st, load().lbm_last_error(self._ctx).decode(), out.as_dict())
        _check(st, self._ctx)
        return out.as_dict()

    def get_populations(self, out=None):
        if out is None:
            out = np.empty((self.Q,) + self.shape)
        p, d, _ = _buf(out, np.float64)
        self._call("lbm_get_populations", p, d)
        return out

    def set_populations(self, f):
        p, d, keep = _buf(f, np.float64)
        self._call("lbm_set_populations", p, d)
        self._keep = keep

    def get_state(self):
        """(raw, layout, steps): the stored populations byte for byte (storage
        type, padded layout), the layout word (1 after an odd number of AA
        steps, else 0) and the step counter; for bit-exact checkpoints."""
        raw = np.empty(self.info()["population_bytes"], dtype=np.uint8)
        layout, steps = ctypes.c_int(), ctypes.c_longlong()
        self._call("lbm_get_state", raw.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(raw.nbytes),
                   ctypes.byref(layout), ctypes.byref(steps), 0)
        return raw, layout.value, steps.value

    def set_state(self, raw, layout: int = 0, steps: int = 0):
        """Restores what get_state returned (set tags, parameters and closure
        weights first)."""
        raw = np.ascontiguousarray(raw, dtype=np.uint8).reshape(-1)
        self._call("lbm_set_state", raw.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(raw.nbytes), int(layout),
                   int(steps), 0)

    def save_checkpoint(self, path):
        """Writes everything a run needs to continue bit for bit to an .npz
        file: the raw state, layout word and step counter, the tags, the
        parameters, the closure weights if set, and the lattice's shape,
        velocity set, storage type and streaming pattern."""
        raw, layout, steps = self.get_state()
        extra = {}
        if self._closure is not None:
            extra = {"closure_params": self._closure[0], "closure_norm": self._closure[1]}
        np.savez(path, state=raw, layout=layout, steps=steps, tags=self.get_tags(),
                 params=np.frombuffer(bytes(self.params), dtype=np.uint8),
                 meta=np.array([self.nx, self.ny, self.nz, self.Q, self.dtype, self.pattern], dtype=np.int64),
                 **extra)

    @classmethod
    def from_checkpoint(cls, path, **kwargs):
        """A new lattice holding the state save_checkpoint wrote (kwargs go to
        the constructor: device, stream, torch_allocator)."""
        with np.load(path) as d:
            nx, ny, nz, Q, dtype, pattern = (int(v) for v in d["meta"])
            lat = cls(nx, ny, nz, Q, dtype, pattern=pattern, **kwargs)
            try:
                lat.set_tags(d["tags"])
                p = Params.from_buffer_copy(d["params"].tobytes())
                lat._call("lbm_set_params", ctypes.byref(p))
                lat.params = p
                if "closure_params" in d:
                    lat.set_closure_weights(d["closure_params"], d["closure_norm"])
                lat.set_state(d["state"], int(d["layout"]), int(d["steps"]))
            except Exception:
                lat.close()
                raise
        return lat

    def geometry_spheres(self, centres, radii, target_porosity: float, pore_tag: int = TAG_FLUID):
        """Random-sphere medium; returns (n_used, porosity)."""
        c = np.ascontiguousarray(centres, dtype=np.int32)
        r = np.ascontiguousarray(radii, dtype=np.float64)
        if c.shape != (len(r), 3):
            raise ValueError("centres must have shape (n, 3)")
        used, por = ctypes.c_int(), ctypes.c_double()
        self._call("lbm_geometry_spheres", c.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p),
                   len(r), float(target_porosity), int(pore_tag), ctypes.byref(used), ctypes.byref(por))
        return used.value, por.value

    def enstrophy(self) -> float:
        out = ctypes.c_double()
        self._call("lbm_enstrophy", ctypes.byref(out))
        return out.value

    def set_closure_weights(self, params, norm):
        """Installs the closure network (params[1345], norm[16]; numpy or CUDA tensors)."""
        p, dp, kp = _buf(params, np.float32)
        n, dn, kn = _buf(norm, np.float32)
        if dp != dn:
            raise ValueError("params and norm must both be on the host or both on the device")
        self._call("lbm_set_closure_weights", p, n, dp)
        host = [k.detach().cpu().numpy() if hasattr(k, "detach") else k for k in (kp, kn)]
        self._closure = (np.array(host[0], dtype=np.float32), np.array(host[1], dtype=np.float32))

    def closure_features(self, out=None):
        """The closure's inputs for the next step, (N, 7) FP32 with N in
        x-fastest node order: a numpy array, or written into the given CUDA
        tensor (which is returned)."""
        if out is None:
            out = np.empty((self.N, 7), dtype=np.float32)
        p, dev, _keep = _buf(out, np.float32)
        self._call("lbm_closure_features", p, dev)
        return out

    def info(self) -> dict:
        nbytes, px, q = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        self._call("lbm_info", ctypes.byref(nbytes), ctypes.byref(px), ctypes.byref(q))
        return {"population_bytes": nbytes.value, "pitch_x": px.value, "Q": q.value}


def reduce_noalloc(h, Q: int, dtype, nx: int, ny: int, nz: int, tags=None, force=(0.0, 0.0, 0.0), stream=None):
    """Domain reduction over caller-held device populations without any device
    allocation (``lbm_reduce_noalloc``).  ``h``: CUDA tensor of h = f - w in
    the storage type, shape (Q, nz, ny, nx); ``tags``: CUDA uint8 tensor of
    nx*ny*nz tags or None.  Both must sit on the current CUDA device, whose
    static scratch and current stream the library uses: any mismatch of
    shape, type, count or device raises ValueError before the call."""
    import torch
    lib = load()
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    if dt not in STORAGE_TORCH_DTYPE:
        raise ValueError(f"unknown storage type {dtype!r}")
    if not isinstance(h, torch.Tensor):
        raise TypeError("h must be a torch tensor")
    if tuple(h.shape) != (Q, nz, ny, nx):
        raise ValueError(f"h has shape {tuple(h.shape)}, expected (Q, nz, ny, nx) = {(Q, nz, ny, nx)}")
    if h.dtype != getattr(torch, STORAGE_TORCH_DTYPE[dt]):
        raise ValueError(f"h is {h.dtype}, the storage type needs torch.{STORAGE_TORCH_DTYPE[dt]}")
    if not h.is_contiguous():
        raise ValueError("h must be contiguous")
    if tags is not None:
        if not isinstance(tags, torch.Tensor) or tags.dtype != torch.uint8:
            raise ValueError("tags must be a uint8 tensor")
        if tags.numel() != nx * ny * nz or not tags.is_contiguous():
            raise ValueError(f"tags must be contiguous with nx*ny*nz = {nx * ny * nz} entries, got {tags.numel()}")
    for name, t in (("h", h), ("tags", tags)):
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {t.device}, not on the current device cuda:{torch.cuda.current_device()}")
    p = Params()
    for a in range(3):
        p.force[a] = force[a]
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    out = Reduction()
    st = lib.lbm_reduce_noalloc(ctypes.c_void_p(h.data_ptr()), Q, dt, nx, ny, nz,
                                ctypes.c_void_p(tags.data_ptr()) if tags is not None else None,
                                ctypes.byref(p), handle, ctypes.byref(out))
    if st == ERR_UNSTABLE:
        raise UnstableError(st, lib.lbm_last_error(None).decode(), out.as_dict())
    _check(st, None)
    return out.as_dict()


def fp64_fma_rate(stream=None) -> float:
    """FP64 operations per second of the current device (an FMA counts as
    two), measured by the library's FMA-chain kernel on torch's current
    stream: the arithmetic roof of the step on FP64 storage."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    out = ctypes.c_double()
    _check(load().lbm_fp64_fma_rate(handle, ctypes.byref(out)), None)
    return out.value


# -- closure training calls (device tensors, torch's current stream) ---------
MLP_NPARAM, MLP_NNORM = 1345, 16


def _dev(t, dtype_name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected torch.{dtype_name}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def mlp_forward(params, norm, x):
    """dtau for features x (n, 7) on the GPU's tensor-core tile."""
    import torch
    n = x.shape[0]
    out = torch.empty(n, dtype=torch.float32, device=x.device)
    _check(load().lbm_mlp_forward(_dev(params, "float32"), _dev(norm, "float32"), _dev(x, "float32"), n,
                                  _dev(out, "float32"), _stream()))
    return out


def mlp_loss_grad(params, norm, x, target, workspace=None):
    """(loss, grad) of the mean squared dtau error over (x, target)."""
    import torch
    n = x.shape[0]
    nbytes = load().lbm_mlp_workspace_bytes(n)
    if workspace is None or workspace.numel() * 4 < nbytes:
        workspace = torch.empty((nbytes + 3) // 4, dtype=torch.float32, device=x.device)
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(load().lbm_mlp_loss_grad(_dev(params, "float32"), _dev(norm, "float32"), _dev(x, "float32"),
                                    _dev(target, "float32"), n, _dev(grad, "float32"), _dev(loss, "float32"),
                                    _dev(workspace, "float32"), workspace.numel() * 4, _stream()))
    return loss, grad


def mlp_adam(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on device tensors."""
    _check(load().lbm_mlp_adam(_dev(params, "float32"), _dev(m, "float32"), _dev(v, "float32"),
                               _dev(grad, "float32"), params.numel(), int(t), float(lr), float(beta1), float(beta2),
                               float(eps), _stream()))


def coarse_samples(rho, u, factor, tau0):
    """Training features (Nc, 7) and targets (Nc,) from fine device fields
    rho (nz, ny, nx) and u (3, nz, ny, nx), FP64."""
    import torch
    nz, ny, nx = rho.shape
    nc = (nx // factor) * (ny // factor) * (nz // factor)
    X = torch.empty((nc, 7), dtype=torch.float32, device=rho.device)
    y = torch.empty(nc, dtype=torch.float32, device=rho.device)
    _check(load().lbm_coarse_samples(_dev(rho, "float64"), _dev(u, "float64"), nx, ny, nz, int(factor), float(tau0),
                                     _dev(X, "float32"), _dev(y, "float32"), _stream()))
    return X, y


def box_filter(field, factor):
    """Box-filtered copy of a device FP64 field of shape (c, nz, ny, nx) or
    (nz, ny, nx)."""
    import torch
    squeeze = field.dim() == 3
    f4 = field.unsqueeze(0) if squeeze else field
    c, nz, ny, nx = f4.shape
    out = torch.empty((c, nz // factor, ny // factor, nx // factor), dtype=torch.float64, device=field.device)
    _check(load().lbm_box_filter(_dev(f4.contiguous(), "float64"), c, nx, ny, nz, int(factor), _dev(out, "float64"),
                                 _stream()))
    return out[0] if squeeze else out
