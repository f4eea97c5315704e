"""The oracle and the CUDA path stay apart: the product package never imports the
oracle, the two share no source file or header, bench.py reaches the oracle only in
its CPU-baseline and reference legs, and the binding raises instead of falling back
when the library is missing."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1801_10277_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name, node
        elif isinstance(node, ast.ImportFrom) and node.module:
            yield node.module, node


def test_package_never_imports_the_oracle():
    for f in _files(PKG, (".py",)):
        for mod, _ in _imported_modules(f):
            assert not mod.split(".")[0] == "oracle", f
        assert "oracle/" not in open(f).read(), f


def test_no_shared_sources_or_headers():
    inc = re.compile(r'#\s*include\s*[<"]([^>"]+)[>"]')
    for f in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h", ".cpp")):
        for h in inc.findall(open(f).read()):
            assert "oracle" not in h, (f, h)
    for f in _files(os.path.join(ROOT, "oracle"), (".cpp", ".h", ".c", ".py")):
        text = open(f).read()
        for h in inc.findall(text):
            assert "celeste.h" not in h and "csrc" not in h and ".cuh" not in h, (f, h)
        if f.endswith(".py"):
            for mod, _ in _imported_modules(f):
                assert not mod.startswith("paper_1801_10277_gb300"), (f, mod)


def test_bench_reaches_the_oracle_only_in_its_baseline_legs():
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path).read(), path)
    allowed = {"oracle_rate", "reference_sample", "reference_arm"}
    for fn in ast.walk(tree):
        if not isinstance(fn, ast.FunctionDef):
            continue
        for node in ast.walk(fn):
            mods = []
            if isinstance(node, ast.ImportFrom) and node.module:
                mods = [node.module]
            elif isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            if any(m.split(".")[0] == "oracle" for m in mods):
                assert fn.name in allowed, fn.name
    for node in tree.body:   # nothing at module level
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            mods = [node.module] if isinstance(node, ast.ImportFrom) else [a.name for a in node.names]
            assert not any((m or "").split(".")[0] == "oracle" for m in mods)


def test_binding_raises_when_the_library_is_missing(monkeypatch, tmp_path):
    from paper_1801_10277_gb300 import celeste
    monkeypatch.setattr(celeste, "_lib", None)
    monkeypatch.setattr(celeste, "lib_path", lambda: str(tmp_path / "libceleste.so"))
    with pytest.raises(RuntimeError, match="not built"):
        celeste.load()
