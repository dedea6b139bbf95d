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


def test_unsupported_combinations_rejected_without_the_gpu():
    """Combinations the library does not offer are refused before any CUDA
    call: dense rows with Elkan or Yin-Yang or non-FP32 values, the BF16
    precision form with d not a multiple of 8 (FP8: 16) or an unknown
    precision, Elkan with k > 4096, Yin-Yang with k > 1024, a CSR center table of 16 GB or more, a
    tile of centers that is not 128, 256, 512 or 1024 (or any tile for
    Yin-Yang, dense rows or a batch), and the batched form with Yin-Yang
    bounds or with a malformed run table."""
    import numpy as np
    lib = skm.load()
    h = ctypes.c_void_p()
    buf = np.zeros(64, np.float32)
    rp = np.zeros(11, np.int64)
    ci = np.zeros(4, np.int32)

    def data(layout, dtype=0, n=10, d=16):  # dtype 0: FP32, 1: FP16
        return skm.skm_data(n=n, d=d, layout=layout, dtype=dtype, memspace=skm.HOST, reserved=0,
                            row_ptr=rp.ctypes.data if layout == skm.CSR else None,
                            col_idx=ci.ctypes.data if layout == skm.CSR else None, values=buf.ctypes.data)

    def init(x, k, variant, opt=None):
        rc = lib.skm_init(ctypes.byref(h), ctypes.byref(x), k, variant, None, 0,
                          ctypes.byref(opt) if opt is not None else None, None)
        assert h.value is None
        return rc

    V = skm.VARIANTS
    assert init(data(skm.DENSE), 3, V["elkan"]) == skm.EUNSUPPORTED
    assert init(data(skm.DENSE), 3, V["simp_elkan"]) == skm.EUNSUPPORTED
    assert init(data(skm.DENSE), 3, V["yinyang"]) == skm.EUNSUPPORTED
    assert init(data(skm.DENSE, dtype=1), 3, V["standard"]) == skm.EUNSUPPORTED  # FP16 dense
    opt = skm.skm_options()
    lib.skm_default_options(ctypes.byref(opt))
    opt.precision = skm.PREC_BF16
    assert init(data(skm.DENSE, d=12), 3, V["standard"], opt) == skm.EUNSUPPORTED  # d % 8 != 0
    opt.precision = skm.PREC_FP8
    assert init(data(skm.DENSE, d=24), 3, V["standard"], opt) == skm.EUNSUPPORTED  # d % 16 != 0
    opt.precision = 7
    assert init(data(skm.DENSE, d=32), 3, V["standard"], opt) == skm.EINVAL  # no such precision
    assert init(data(skm.CSR, n=5000), 4097, V["elkan"]) == skm.EUNSUPPORTED
    assert init(data(skm.CSR, n=5000), 1025, V["yinyang"]) == skm.EUNSUPPORTED  # one pass over a row
    assert init(data(skm.CSR, n=5000, d=2 ** 22), 1024, V["standard"]) == skm.EUNSUPPORTED  # Ct of 16 GB
    topt = skm.skm_options()
    lib.skm_default_options(ctypes.byref(topt))
    topt.k_tile = 100  # not a tile size
    assert init(data(skm.CSR), 3, V["elkan"], topt) == skm.EINVAL
    topt.k_tile = 256
    assert init(data(skm.CSR), 3, V["yinyang"], topt) == skm.EUNSUPPORTED  # Yin-Yang walks a row once
    assert init(data(skm.DENSE), 3, V["standard"], topt) == skm.EUNSUPPORTED  # the tile is the CSR kernel's

    x = data(skm.CSR)
    ks = np.array([2, 3], np.int32)

    def batch(run_rows, ks, variant, xb=x):
        run_rows = np.asarray(run_rows, np.int64)
        rc = lib.skm_batch_init(ctypes.byref(h), ctypes.byref(xb), run_rows.ctypes.data, ks.ctypes.data, len(ks),
                                variant, None, 0, None, None)
        assert h.value is None
        return rc

    # Yin-Yang in a batch: runs of at most 512 centers (one pass over a row)
    assert batch([0, 10, 600], np.array([3, 513], np.int32), V["yinyang"], data(skm.CSR, n=600)) == \
        skm.EUNSUPPORTED
    rr = np.asarray([0, 4, 10], np.int64)
    assert lib.skm_batch_init(ctypes.byref(h), ctypes.byref(x), rr.ctypes.data, ks.ctypes.data, 2, V["standard"],
                              None, 0, ctypes.byref(topt), None) == skm.EUNSUPPORTED  # no tile choice in a batch
    assert h.value is None
    assert batch([0, 4, 9], ks, V["standard"]) == skm.EINVAL      # does not end at n
    assert batch([1, 4, 10], ks, V["standard"]) == skm.EINVAL     # does not start at 0
    assert batch([0, 2, 10], np.array([3, 3], np.int32), V["standard"]) == skm.EINVAL  # k > rows of the run
    assert batch([0, 4, 10], np.array([0, 3], np.int32), V["standard"]) == skm.EINVAL  # k < 1
