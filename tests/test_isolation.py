"""The oracle and the CUDA path share no code, and the library has no
fallback: a missing shared library is an error, not a slower path."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2107_04074_gb300")


def _sources(top, exts):
    for dirpath, _, files in os.walk(top):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_library_never_touches_the_oracle():
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".h")):
        text = open(path).read()
        assert not re.search(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|skm_oracle|oracle/", text), path


def test_oracle_never_touches_the_library():
    for path in _sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(path).read()
        assert not re.search(r"\bimport\s+paper_2107_04074_gb300|\bfrom\s+paper_2107_04074_gb300|"
                             r"#include\s*[<\"][^>\"]*(csrc|skm\.h|skm_internal)", text), path


def test_missing_library_is_an_error(monkeypatch, tmp_path):
    from paper_2107_04074_gb300 import skm
    monkeypatch.setattr(skm, "_LIB", None)
    monkeypatch.setattr(skm._build, "LIB", str(tmp_path / "libskm.so"))
    with pytest.raises(RuntimeError, match="missing"):
        skm.load(build_if_missing=False)
