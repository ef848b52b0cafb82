"""The product path stands alone: no module of the package imports the
oracle (test infrastructure), and the binding fails loudly when the CUDA
library is missing instead of falling back to anything else."""
import ast
import glob
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1304_3771_b300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            yield from (a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""


def test_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(PKG, "*.py"))
    assert files
    for f in files:
        for name in _imports(f):
            assert name.split(".")[0] != "oracle", f"{os.path.basename(f)} imports {name}"


def test_cuda_sources_never_include_oracle_code():
    for f in glob.glob(os.path.join(PKG, "csrc", "*")):
        text = open(f, errors="replace").read()
        assert "cvd_oracle" not in text and "oracle/" not in text, os.path.basename(f)


def test_binding_raises_without_the_library(monkeypatch):
    from paper_1304_3771_b300 import cvd
    monkeypatch.setattr(cvd, "_lib", None)
    monkeypatch.setattr(cvd, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libcvd.so"))
    with pytest.raises(ImportError):
        cvd.lib()
