"""The C ABI from plain C: tests/c/abi_host.c is compiled as C99 with
warnings as errors against include/lbm.h, linked against the library, and
run (it calls only what needs no GPU).  The header must also compile as
C++."""
import shutil
import subprocess

from pathlib import Path

import pytest

from paper_2506_09242_gb300 import _build

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def libdir():
    return _build.build().parent


def test_c_program_links_and_runs(tmp_path, libdir):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "abi_host"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", f"-I{ROOT / 'include'}",
                    str(ROOT / "tests" / "c" / "abi_host.c"), "-o", str(exe), f"-L{libdir}", "-llbm",
                    f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "abi_host: ok" in r.stdout


def test_header_compiles_as_cpp(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "h.cpp"
    src.write_text('#include "lbm.h"\nint main() { return lbm_destroy(nullptr) == LBM_OK ? 0 : 1; }\n')
    subprocess.run([cxx, "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", f"-I{ROOT / 'include'}", str(src)],
                   check=True)
