"""The product path and the oracle share no code: no module of the package
imports the oracle, the oracle imports nothing of the package, and the CUDA
sources include nothing from the oracle (CPU only)."""

import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1108_4181_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""


def _py_files(top):
    for dirpath, _, files in os.walk(top):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        bad = [m for m in _imports(path) if m == "oracle" or m.startswith("oracle.")]
        assert not bad, (path, bad)


def test_oracle_never_imports_the_package():
    for path in _py_files(os.path.join(ROOT, "oracle")):
        bad = [m for m in _imports(path) if m.startswith("paper_1108_4181_gb300")]
        assert not bad, (path, bad)


def test_cuda_sources_include_nothing_from_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        src = open(os.path.join(csrc, f)).read()
        assert "oracle" not in src, f
