"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package draws data only; it contains none of the clustering method's
arithmetic.  The C generator (``gen.c``) is built on first use with gcc.

Workloads (stand-ins for the paper's data sets, Section 6 / Table 1, which are
not available here):

* ``tfidf(cfg)`` -- sparse TF-IDF document vectors (CSR, unit rows).
* ``vmf(...)``   -- dense embedding-like unit vectors from a vMF mixture.
* ``init_rows``  -- k distinct seeded row ids (the paper's uniform random
  initialisation, Section 6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def _lib_path() -> str:
    return os.path.join(_HERE, "_build", "libsynth.so")


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (idempotent)."""
    out = _lib_path()
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            i64, u64, dbl, ip = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.synth_row_nnz.argtypes = [i64, i64, u64, ctypes.c_int, dbl, dbl, i64, i64, ip]
            lib.synth_row_nnz.restype = None
            lib.synth_tfidf_fill.argtypes = [i64, i64, u64, dbl, ip, ip, ip, ctypes.c_int]
            lib.synth_tfidf_fill.restype = ctypes.c_int
            lib.synth_vmf.argtypes = [i64, i64, i64, dbl, u64, ip, ip, ip, ctypes.c_int]
            lib.synth_vmf.restype = ctypes.c_int
            lib.synth_init_rows.argtypes = [i64, i64, u64, ip]
            lib.synth_init_rows.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _threads(t):
    return int(t) if t else max(1, min(16, os.cpu_count() or 1))


@dataclass(frozen=True)
class SparseCfg:
    """Recipe of a sparse TF-IDF workload."""
    n: int
    d: int
    seed: int
    nnz_kind: int  # 0 = Poisson(a) (0 redrawn), 1 = lognormal(mean a, sigma b)
    a: float
    b: float
    lo: int
    hi: int
    zipf: float
    dtype: str = "f32"  # stored value type: f32 | f16


# The sparse workloads: TF-IDF-shaped rows whose lengths follow nnz_kind (a, b, lo, hi) and whose
# terms follow a Zipf law over the vocabulary.
CSR_TINY = SparseCfg(n=2000, d=5000, seed=1, nnz_kind=0, a=50.0, b=0.0, lo=1, hi=5000, zipf=1.1)
CSR_RCV1_LIKE = SparseCfg(n=100_000, d=50_000, seed=2, nnz_kind=1, a=120.0, b=0.8, lo=5, hi=2000, zipf=1.1)
CSR_LARGE = SparseCfg(n=4_000_000, d=200_000, seed=5, nnz_kind=1, a=200.0, b=0.9, lo=10, hi=5000, zipf=1.05,
                      dtype="f16")


def scaled(cfg: SparseCfg, n: int | None = None, d: int | None = None, seed: int | None = None) -> SparseCfg:
    """Same recipe with a different row count / vocabulary / seed."""
    return SparseCfg(n=n or cfg.n, d=d or cfg.d, seed=cfg.seed if seed is None else seed, nnz_kind=cfg.nnz_kind,
                     a=cfg.a, b=cfg.b, lo=cfg.lo, hi=cfg.hi, zipf=cfg.zipf, dtype=cfg.dtype)


@dataclass
class CSR:
    n: int
    d: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz], sorted within each row
    val: np.ndarray      # float32 or float16 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self, idx) -> "CSR":
        """Sub-matrix of the given rows (in the given order)."""
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.row_ptr[idx + 1] - self.row_ptr[idx]
        rp = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        take = np.concatenate([np.arange(self.row_ptr[i], self.row_ptr[i + 1]) for i in idx]) if len(idx) else \
            np.zeros(0, dtype=np.int64)
        return CSR(len(idx), self.d, rp, self.col[take], self.val[take])

    def dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.d), dtype=np.float64)
        r = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        out[r, self.col] = self.val.astype(np.float64)
        return out


def tfidf(cfg: SparseCfg, threads: int | None = None) -> CSR:
    """Sparse TF-IDF rows drawn per the recipe ``cfg`` (unit L2 rows)."""
    lib = _lib()
    nnz = np.empty(cfg.n, dtype=np.int64)
    lib.synth_row_nnz(cfg.n, cfg.d, cfg.seed, cfg.nnz_kind, cfg.a, cfg.b, cfg.lo, cfg.hi, _ptr(nnz))
    rp = np.zeros(cfg.n + 1, dtype=np.int64)
    np.cumsum(nnz, out=rp[1:])
    col = np.empty(int(rp[-1]), dtype=np.int32)
    val = np.empty(int(rp[-1]), dtype=np.float32)
    rc = lib.synth_tfidf_fill(cfg.n, cfg.d, cfg.seed, cfg.zipf, _ptr(rp), _ptr(col), _ptr(val), _threads(threads))
    if rc != 0:
        raise MemoryError("synth_tfidf_fill failed")
    if cfg.dtype == "f16":
        val = val.astype(np.float16)
    return CSR(cfg.n, cfg.d, rp, col, val)


def csr_from_dense(X: np.ndarray) -> CSR:
    """CSR view of a small dense matrix (zeros dropped); used for hand-made cases."""
    X = np.asarray(X)
    n, d = X.shape
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(X[i])[0]
        cols.append(nz.astype(np.int32))
        vals.append(X[i, nz])
        rp[i + 1] = rp[i] + len(nz)
    col = np.concatenate(cols) if cols else np.zeros(0, np.int32)
    val = np.concatenate(vals).astype(np.float32) if vals else np.zeros(0, np.float32)
    return CSR(n, d, rp, col.astype(np.int32), val)


def vmf(n: int, d: int, ncomp: int, kappa: float, seed: int, threads: int | None = None,
        return_comp: bool = False):
    """Dense unit rows (float32, n x d) from a uniform mixture of vMF(kappa)."""
    lib = _lib()
    X = np.empty((n, d), dtype=np.float32)
    comp = np.empty(n, dtype=np.int32)
    means = np.empty((ncomp, d), dtype=np.float64)
    rc = lib.synth_vmf(n, d, ncomp, kappa, seed, _ptr(X), _ptr(comp), _ptr(means), _threads(threads))
    if rc != 0:
        raise MemoryError("synth_vmf failed")
    if return_comp:
        return X, comp, means
    return X


def init_rows(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct seeded row ids in [0, n)."""
    if k > n:
        raise ValueError("k > n")
    out = np.empty(k, dtype=np.int64)
    _lib().synth_init_rows(n, k, seed, _ptr(out))
    return out


# The batched workload: many independent runs of uneven size and k.
BATCH_K_CHOICES = (10, 50, 100, 250, 500)


def batch_runs(nruns: int = 64, d: int = 20_000, seed: int = 4, n_lo: int = 5_000, n_hi: int = 200_000,
               k_choices=BATCH_K_CHOICES, row_cfg: SparseCfg = CSR_RCV1_LIKE):
    """Recipes of `nruns` independent runs: run r has n_r rows with
    ln n_r ~ Normal(ln sqrt(n_lo n_hi), (ln(n_hi / n_lo) / 4)^2) clipped to
    [n_lo, n_hi], rows drawn like ``row_cfg`` over a vocabulary of d terms
    with seed 1000 + r, and k_r uniform over k_choices.  Returns (list of
    SparseCfg, numpy int32 array of k_r)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = 0.5 * (np.log(n_lo) + np.log(n_hi))
    sigma = np.log(n_hi / n_lo) / 4.0
    ns = np.clip(np.exp(rng.normal(mu, sigma, nruns)), n_lo, n_hi).astype(np.int64)
    ks = np.asarray(k_choices, dtype=np.int32)[rng.integers(0, len(k_choices), nruns)]
    cfgs = [SparseCfg(n=int(ns[r]), d=d, seed=1000 + r, nnz_kind=row_cfg.nnz_kind, a=row_cfg.a, b=row_cfg.b,
                      lo=row_cfg.lo, hi=row_cfg.hi, zipf=row_cfg.zipf, dtype=row_cfg.dtype) for r in range(nruns)]
    return cfgs, ks


def concat(parts) -> tuple:
    """Stack CSR blocks (same d) into one CSR; returns (CSR, run_rows)."""
    d = parts[0].d
    run_rows = np.zeros(len(parts) + 1, dtype=np.int64)
    np.cumsum([p.n for p in parts], out=run_rows[1:])
    nnz = np.zeros(len(parts) + 1, dtype=np.int64)
    np.cumsum([p.nnz for p in parts], out=nnz[1:])
    rp = np.concatenate([parts[0].row_ptr[:1]] + [p.row_ptr[1:] + nnz[r] for r, p in enumerate(parts)])
    col = np.concatenate([p.col for p in parts])
    val = np.concatenate([p.val for p in parts])
    return CSR(int(run_rows[-1]), d, rp.astype(np.int64), col, val), run_rows
