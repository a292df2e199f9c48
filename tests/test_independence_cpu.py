"""The oracle and the CUDA path share nothing: no module of the package
imports or loads the oracle, the oracle imports nothing of the package, no
CUDA source includes an oracle file, and the seeded input generators that
both sides use hold none of the method's arithmetic (they import neither)."""
import ast
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2506_09242_gb300"


def _imports(path: Path):
    tree = ast.parse(path.read_text())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def test_package_never_imports_the_oracle():
    for py in PKG.rglob("*.py"):
        assert "oracle" not in _imports(py), py
        assert "lbm_oracle" not in py.read_text(), py


def test_cuda_sources_include_no_oracle_file():
    for src in list((PKG / "csrc").glob("*.cu")) + list((PKG / "csrc").glob("*.cuh")):
        for inc in re.findall(r'#include\s+"([^"]+)"', src.read_text()):
            assert "oracle" not in inc, (src, inc)


def test_oracle_imports_nothing_of_the_package():
    for py in (ROOT / "oracle").glob("*.py"):
        assert "paper_2506_09242_gb300" not in _imports(py), py
    assert "#include \"" not in (ROOT / "oracle" / "lbm_oracle.c").read_text()


def test_input_generators_are_independent_of_both():
    assert not {"oracle", "paper_2506_09242_gb300"} & _imports(ROOT / "lbm_inputs.py")


def test_bench_uses_the_oracle_only_in_its_baseline_legs():
    """bench.py may run the oracle only for the CPU baseline and the
    reference arm; the timed GPU path never imports it."""
    tree = ast.parse((ROOT / "bench.py").read_text())
    users = set()
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        for node in ast.walk(fn):
            if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                users.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any(isinstance(n, ast.Import) and any(a.name == "oracle" for a in n.names) for n in top)
    assert users == {"oracle_timing", "run_reference"}
