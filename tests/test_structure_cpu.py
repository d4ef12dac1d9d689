"""Structural guards of the product path (CPU): the package and the CUDA
sources never reach the oracle (no import, no include, no load of its shared
object), and the binding fails loudly when the CUDA library is missing instead
of falling back to anything."""
import ast
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1112_5239_gb300")


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), path
        assert "libci_oracle" not in open(path).read(), path


def test_cuda_sources_never_reach_the_oracle():
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        text = open(path).read()
        assert not re.search(r'#include\s+[<"][^>"]*oracle', text), path
        assert "libci_oracle" not in text and "ci_oracle.c" not in text, path


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_1112_5239_gb300 import _lib

    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libci_prng.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.lib()
