"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function that include/*.h declares, the binding's signature table
covers them, and argument / allocation failures are reported as status codes
before any device work."""
import ctypes
import re
from pathlib import Path

import pytest

from paper_2506_09242_gb300 import _build, lbm

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = []
    for h in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_][a-z0-9_ ]*\**\s*\**(lbm_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lbm.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_set_tags", "lbm_init_equilibrium", "lbm_step", "lbm_moments",
                     "lbm_reduce"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
        assert name in lbm.SIGNATURES, f"binding lacks {name}"


def test_create_rejects_bad_arguments(lib):
    out = ctypes.c_void_p()
    for args in [(0, 4, 4, 19, 1), (4, -1, 4, 19, 1), (4, 4, 4, 15, 1), (4, 4, 4, 19, 9), (4, 4, 70000, 19, 1),
                 (1 << 20, 1 << 10, 4, 19, 1)]:
        st = lib.lbm_create(*args, None, None, ctypes.byref(out))
        assert st == lbm.ERR_ARG, args
        assert not out.value
        assert lib.lbm_last_error(None)
    assert lib.lbm_create(4, 4, 4, 19, 1, None, None, None) == lbm.ERR_ARG
    for pattern in (-1, 2, 7):  # streaming pattern: AB (0) or AA (1) only
        assert lib.lbm_create_ex(4, 4, 4, 19, 1, pattern, None, None, ctypes.byref(out)) == lbm.ERR_ARG
        assert not out.value
        assert b"pattern" in lib.lbm_last_error(None)


def test_allocator_failure_is_reported_as_oom(lib):
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, user):
        calls["alloc"] += 1
        return None

    def _free(ptr, nbytes, stream, user):
        calls["free"] += 1

    a = lbm.Allocator(lbm.ALLOC_FN(_alloc), lbm.FREE_FN(_free), None)
    out = ctypes.c_void_p()
    st = lib.lbm_create(8, 8, 8, 19, 1, ctypes.byref(a), None, ctypes.byref(out))
    assert st == lbm.ERR_OOM
    assert not out.value
    assert calls["alloc"] >= 2
    assert calls["free"] == 0  # nothing was handed out, nothing is freed
    assert b"allocation" in lib.lbm_last_error(None)


def test_null_context_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == lbm.ERR_ARG
    buf = ctypes.create_string_buffer(64)
    assert lib.lbm_get_state(None, buf, 64, None, None, 0) == lbm.ERR_ARG
    assert lib.lbm_set_state(None, buf, 64, 0, 0, 0) == lbm.ERR_ARG
    assert lib.lbm_destroy(None) == lbm.OK
    assert lib.lbm_sync(None, 0) == lbm.ERR_ARG


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises."""
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "_LIB_PATH", tmp_path / "missing.so")
    with pytest.raises(ImportError):
        lbm.load()
    with pytest.raises(ImportError):
        lbm.Lattice(8, 8, 8)


def test_params_struct_matches_the_header():
    """The binding's parameter struct has the header's fields in order."""
    text = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "lbm.h").read_text(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\} lbm_params;", text).group(1)
    names = re.findall(r"([a-z_]+)(?:\[[^\]]*\])*\s*;", body)
    assert names == [f[0] for f in lbm.Params._fields_]
    body = re.search(r"typedef struct \{([^}]*)\} lbm_reduction;", text).group(1)
    names = re.findall(r"([a-z_]+)(?:\[[^\]]*\])*\s*;", body)
    assert names == [f[0] for f in lbm.Reduction._fields_]


def test_noalloc_reduction_rejects_lattices_beyond_its_bound(lib):
    """lbm_reduce_noalloc walks node offsets in 32-bit integers: a lattice of
    LBM_NOALLOC_MAX_NODES + 1 = 2^31 - 256 nodes (the size lbm_create also
    refuses) is rejected before any device work, so the placeholder pointer
    is never used."""
    text = (ROOT / "include" / "lbm.h").read_text()
    bound = int(re.search(r"#define LBM_NOALLOC_MAX_NODES (\d+)LL", text).group(1))
    assert bound == (1 << 31) - 257
    nx, ny, nz = 178481, 47 * 256, 1  # 2^31 - 256 = 256 * 47 * 178481
    assert nx * ny * nz == bound + 1
    r = lbm.Reduction()
    for lattice, dtype in ((19, lbm.F32), (27, lbm.F16_SHIFTED), (19, lbm.F64)):
        st = lib.lbm_reduce_noalloc(ctypes.c_void_p(256), lattice, dtype, nx, ny, nz, None, None, None,
                                    ctypes.byref(r))
        assert st == lbm.ERR_ARG
        assert b"LBM_NOALLOC_MAX_NODES" in lib.lbm_last_error(None)
    # lbm_create refuses the same node count (x already a multiple of 32, so
    # no padding)
    out = ctypes.c_void_p()
    assert (32 * 178481) * (8 * 47) == bound + 1
    assert lib.lbm_create(32 * 178481, 8 * 47, 1, 19, 1, None, None, ctypes.byref(out)) == lbm.ERR_ARG
    assert not out.value
