"""The CUDA path and the oracle stay apart, and the product path has no CPU
fallback.

* Nothing in the package (Python, CUDA sources) or its header imports,
  includes or loads anything from oracle/, and the oracle's sources include
  nothing from the package or its header.
* bench.py touches the oracle only in its CPU-baseline leg and its
  reference arm.
* Without a CUDA device the binding raises instead of computing anything.
"""
import ast
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2003_03508_gb300"
ORACLE = ROOT / "oracle"

ORACLE_REF = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s*[<\"].*oracle)|liboracle", re.M)
PKG_REF = re.compile(r"#\s*include\s*[<\"].*(hmm_gb300|hmm_internal|hmm_tc_common)|paper_2003_03508_gb300")


def _strip_comments(text, suffix):
    if suffix in (".c", ".h", ".cu", ".cuh"):
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
    return text


def test_package_does_not_reach_the_oracle():
    files = [p for p in PKG.rglob("*") if p.suffix in (".py", ".cu", ".cuh") and "_build" not in p.parts]
    files += list((ROOT / "include").glob("*.h"))
    assert files
    for p in files:
        text = _strip_comments(p.read_text(), p.suffix)
        assert not ORACLE_REF.search(text), p


def test_oracle_does_not_reach_the_package():
    files = [p for p in ORACLE.glob("*") if p.suffix in (".c", ".h", ".py")]
    assert files
    for p in files:
        text = _strip_comments(p.read_text(), p.suffix)
        assert not PKG_REF.search(text), p


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse((ROOT / "bench.py").read_text())
    allowed = {"cpu_baseline", "run_reference"}
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, (ast.Import, ast.ImportFrom)):
                    names = [a.name for a in node.names] + [getattr(node, "module", None) or ""]
                    if any(n == "oracle" or n.startswith("oracle.") for n in names):
                        users.add(fn.name)
    # module-level imports of the oracle are not allowed either
    for node in tree.body:
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            names = [a.name for a in node.names] + [getattr(node, "module", None) or ""]
            assert not any(n == "oracle" for n in names)
    assert users <= allowed, users
    assert "cpu_baseline" in users


def test_binding_raises_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2003_03508_gb300 import api
    with pytest.raises(RuntimeError):
        api.Context(0)
