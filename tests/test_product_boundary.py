"""Separation of the product, the oracle and the input generators (CPU):

* nothing in the product package (CUDA sources, binding, build) imports or
  names the oracle, and the seeded input generators import neither;
* the oracle imports nothing of the product;
* the binding fails loudly, naming the missing library, when libnk.so is
  absent: there is no CPU fallback to drop into.
"""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2303_05420_gb300")


def _sources(top, exts):
    for dirpath, _, files in os.walk(top):
        if "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_product_does_not_use_the_oracle():
    bad = []
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        if re.search(r"\boracle\b", open(path, encoding="utf-8").read()):
            bad.append(os.path.relpath(path, ROOT))
    assert not bad, bad


def test_inputs_module_imports_neither_side():
    for path in _sources(os.path.join(ROOT, "nkdata"), (".py",)):
        src = open(path, encoding="utf-8").read()
        assert not re.search(r"^\s*(import|from)\s+(oracle|paper_2303_05420_gb300)\b", src, re.M), path


def test_oracle_does_not_import_the_product():
    for path in _sources(os.path.join(ROOT, "oracle"), (".py",)):
        src = open(path, encoding="utf-8").read()
        assert not re.search(r"^\s*(import|from)\s+paper_2303_05420_gb300\b", src, re.M), path


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2303_05420_gb300 import _lib

    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libnk.so"))
    with pytest.raises(Exception) as ei:
        _lib.lib()
    assert "libnk.so" in str(ei.value)
