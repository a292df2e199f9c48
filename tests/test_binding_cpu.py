"""The Python binding's host logic against a recording fake of the library
(no GPU, no CUDA): argument marshalling of the lattice calls and the
checkpoint file round trip (save_checkpoint, then from_checkpoint replays the
same tags, parameters, closure weights and raw state, in the order the
library requires)."""
import ctypes

import numpy as np
import pytest

from paper_2506_09242_gb300 import lbm


class FakeLib:
    """Stands in for liblbm.so: every entry point returns OK and is recorded;
    the few that write outputs write plausible ones."""

    def __init__(self, pop_bytes=4096):
        self.calls = []
        self.pop_bytes = pop_bytes
        self.state = np.arange(pop_bytes, dtype=np.uint64).astype(np.uint8)
        self.tags = None

    def __getattr__(self, name):
        if not name.startswith("lbm_"):
            raise AttributeError(name)

        def call(*args):
            self.calls.append((name, args))
            return getattr(self, "_" + name, lambda *a: lbm.OK)(*args)
        return call

    def _lbm_create_ex(self, nx, ny, nz, q, dtype, pattern, alloc, stream, out):
        out._obj.value = 0x1000
        self.shape = (nz, ny, nx)
        return lbm.OK

    def _lbm_info(self, ctx, nbytes, px, q):
        nbytes._obj.value = self.pop_bytes
        px._obj.value = 32
        q._obj.value = 19
        return lbm.OK

    def _lbm_get_state(self, ctx, buf, nbytes, layout, steps, on_device):
        assert nbytes.value == self.pop_bytes and on_device == 0
        ctypes.memmove(buf, self.state.ctypes.data, self.pop_bytes)
        layout._obj.value = 1
        steps._obj.value = 123
        return lbm.OK

    def _lbm_get_tags(self, ctx, buf, on_device):
        n = int(np.prod(self.shape))
        t = (np.arange(n) % 5).astype(np.uint8)
        ctypes.memmove(buf, t.ctypes.data, n)
        return lbm.OK

    def _lbm_set_state(self, ctx, buf, nbytes, layout, steps, on_device):
        got = np.empty(nbytes.value, np.uint8)
        ctypes.memmove(got.ctypes.data, buf, nbytes.value)
        self.restored = (got, layout, steps)
        return lbm.OK

    def _lbm_set_tags(self, ctx, buf, on_device):
        n = int(np.prod(self.shape))
        got = np.empty(n, np.uint8)
        ctypes.memmove(got.ctypes.data, buf.value, n)
        self.tags = got
        return lbm.OK

    def _lbm_set_params(self, ctx, p):
        self.params = bytes(p._obj)
        return lbm.OK

    def _lbm_set_closure_weights(self, ctx, params, norm, on_device):
        w = np.empty(lbm_nparam(), np.float32)
        ctypes.memmove(w.ctypes.data, params.value, w.nbytes)
        self.weights = w
        return lbm.OK


def lbm_nparam():
    return 32 * 7 + 32 + 32 * 32 + 32 + 32 + 1


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(lbm, "_lib", f)
    return f


def test_checkpoint_round_trip_through_the_file(fake, tmp_path):
    lat = lbm.Lattice(8, 4, 2, lbm.D3Q19, "f16", pattern="aa", torch_allocator=False)
    lat.set_params(0.7, force=(1e-5, 0.0, -2e-5), closure=lbm.CLOSURE_MLP, wall_u=[(0.1, 0.0, 0.0)])
    params_bytes = fake.params
    w = np.linspace(-1, 1, lbm_nparam()).astype(np.float32)
    lat.set_closure_weights(w, np.ones(16, np.float32))
    path = tmp_path / "ck.npz"
    lat.save_checkpoint(path)
    lat.close()  # through the fake: the context handle is not a real one

    fresh = FakeLib()
    lbm._lib = fresh
    back = lbm.Lattice.from_checkpoint(path, torch_allocator=False)
    names = [c[0] for c in fresh.calls]
    # order: create, tags, parameters, weights, then the state
    order = [names.index(n) for n in ("lbm_create_ex", "lbm_set_tags", "lbm_set_params",
                                      "lbm_set_closure_weights", "lbm_set_state")]
    assert order == sorted(order)
    create = fresh.calls[names.index("lbm_create_ex")][1]
    assert create[:6] == (8, 4, 2, 19, lbm.F16_SHIFTED, lbm.PATTERN_AA)
    assert np.array_equal(fresh.tags, (np.arange(64) % 5).astype(np.uint8))
    assert fresh.params == params_bytes
    assert np.array_equal(fresh.weights, w)
    raw, layout, steps = fresh.restored
    assert np.array_equal(raw, fake.state) and layout == 1 and steps == 123
    assert back.params.tau == 0.7 and back.params.closure == lbm.CLOSURE_MLP
    back.close()


def test_set_params_marshals_every_field(fake):
    lat = lbm.Lattice(8, 4, 2, torch_allocator=False)
    lat.set_params(0.9, force=(1.0, 2.0, 3.0), closure=lbm.CLOSURE_TRT, cs_smag=0.2,
                   wall_u=[(0.1, 0.2, 0.3), (0.4, 0.5, 0.6)], rho_wall=1.1, trt_magic=0.25, wall_rho_local=True)
    p = lbm.Params.from_buffer_copy(fake.params)
    assert p.tau == 0.9 and list(p.force) == [1.0, 2.0, 3.0] and p.closure == lbm.CLOSURE_TRT
    assert p.cs_smag == 0.2 and p.rho_wall == 1.1 and p.trt_magic == 0.25 and p.wall_rho_local == 1
    assert [list(p.wall_u[k]) for k in range(3)] == [[0.1, 0.2, 0.3], [0.4, 0.5, 0.6], [0.0, 0.0, 0.0]]
    lat.close()


def test_tags_must_cover_the_lattice(fake):
    lat = lbm.Lattice(8, 4, 2, torch_allocator=False)
    with pytest.raises(ValueError):
        lat.set_tags(np.zeros(10, np.uint8))
    lat.close()


def test_reduce_noalloc_checks_its_tensors_before_the_call(fake):
    """reduce_noalloc hands raw pointers to a library that reads Q*N elements
    and N tags on the current device: a wrong shape, element type, tag count
    or device is refused in Python, and the library is never called."""
    torch = pytest.importorskip("torch")
    nz, ny, nx = 3, 4, 5
    good = torch.zeros((19, nz, ny, nx), dtype=torch.float32)
    cases = [
        (torch.zeros((19, nz, ny, nx + 1)), None, "shape"),
        (torch.zeros((27, nz, ny, nx)), None, "shape"),
        (torch.zeros((19, nz, ny, nx), dtype=torch.float64), None, "float64"),
        (torch.zeros((19, nz, ny, nx), dtype=torch.float16), None, "float16"),
        (good, torch.zeros(nx * ny * nz, dtype=torch.int32), "uint8"),
        (good, torch.zeros(nx * ny * nz - 1, dtype=torch.uint8), "entries"),
        (good, None, "CUDA"),
        (torch.zeros((19, nz, nx, ny)).transpose(2, 3), None, "contiguous"),
    ]
    for h, tags, msg in cases:
        with pytest.raises(ValueError, match=msg):
            lbm.reduce_noalloc(h, 19, "f32", nx, ny, nz, tags=tags)
    with pytest.raises(ValueError, match="bfloat16"):
        lbm.reduce_noalloc(good, 19, "bf16", nx, ny, nz)
    with pytest.raises(ValueError, match="unknown storage"):
        lbm.reduce_noalloc(good, 19, 9, nx, ny, nz)
    assert not [c for c in fake.calls if c[0] == "lbm_reduce_noalloc"]
