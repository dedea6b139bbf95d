"""The C ABI library loads and exports every declared symbol; host-side logic
that needs no GPU."""
import ctypes
import os
import re

import pytest

from paper_2107_04074_gb300 import skm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "skm.h")).read()
    return sorted(set(re.findall(r"\b(skm_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(skm.EXPORTS)


def test_library_exports_every_symbol():
    lib = skm.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_and_bound_accounting():
    lib = skm.load()
    assert lib.skm_strerror(0) == b"ok"
    assert b"invalid" in lib.skm_strerror(-1)
    n, k = 1842986, 100
    # two FP32 bounds per point (the paper's Hamerly keeps three FP64 values: 24 B)
    assert skm.bound_bytes("hamerly", n, k) == 8 * n
    assert skm.bound_bytes("elkan", n, k) == 4 * n * (k + 1)
    assert skm.bound_bytes("standard", n, k) == 0


def test_init_rejects_bad_arguments_without_touching_the_gpu():
    lib = skm.load()
    h = ctypes.c_void_p()
    assert lib.skm_init(ctypes.byref(h), None, 3, 0, None, 0, None, None) == skm.EINVAL
    d = skm.skm_data(n=10, d=5, layout=0, dtype=0, memspace=1, reserved=0, row_ptr=None, col_idx=None, values=None)
    assert lib.skm_init(ctypes.byref(h), ctypes.byref(d), 3, 0, None, 0, None, None) == skm.EINVAL
    assert lib.skm_init(ctypes.byref(h), ctypes.byref(d), 30, 0, None, 0, None, None) == skm.EINVAL  # k > n
    assert lib.skm_init(ctypes.byref(h), ctypes.byref(d), 3, 9, None, 0, None, None) == skm.EINVAL  # variant
    assert h.value is None
