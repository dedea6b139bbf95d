"""FP64 spherical k-means oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU implementation of what the GPU path computes, written from
the paper ("Accelerating Spherical k-Means", Schubert, Lang, Feher; arXiv
2107.04074).  The arithmetic lives in ``skm_oracle.c`` (plain C, FP64,
single-threaded); this module only builds it with gcc and marshals numpy
arrays.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import it; the library under ``paper_2107_04074_gb300`` never
does, and this package never imports that library.

Functions and the passages they follow:

* ``rinv``            row normalisation (Section 5, first paragraph)
* ``sim``             cosine = dot product of unit vectors (Section 2)
* ``assign``          a(i) = argmax_j <x(i), c(j)> (Section 5), tie rule T
* ``update``          c(j) = normalised member sum (Section 5), rule E
* ``drift``           p(j) = <c(j), c'(j)> (Section 4) and its sine
* ``center_bounds``   cc(i,j), s(i) (Section 5.2)
* ``l_update``        Eq. (eqn:l-bound), clamped (rule CL)
* ``u_update``        Eq. (eqn:u-elkan), clamped (rule CL)
* ``u_hamerly``       Eq. (eqn:u-hamerly-2) under rule HG (Section 5.3)
* ``run``             full runs of the five variants (Sections 5, 5.1-5.4) and of
                      Yin-Yang group bounds (Section 5.5)
* ``kmeanspp``        spherical k-means++ seeding (Section 5.6)
* ``kmeanspp_bounds`` the same, with the first assignment and the bounds
                      pre-initialised from the seeding's similarities
                      (Section 5.6's remark, Section 7's outlook)

The rule letters (T, E, CL, HG, V, D, M) are defined in the header of
``skm_oracle.c``.
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

STANDARD, HAMERLY, ELKAN, SIMP_HAMERLY, SIMP_ELKAN, YINYANG = 0, 1, 2, 3, 4, 5
VARIANTS = {"standard": STANDARD, "hamerly": HAMERLY, "elkan": ELKAN, "simp_hamerly": SIMP_HAMERLY,
            "simp_elkan": SIMP_ELKAN, "yinyang": YINYANG}


def _lib_path() -> str:
    return os.path.join(_HERE, "_build", "libskm_oracle.so")


def build(force: bool = False) -> str:
    """Compile skm_oracle.c with gcc (idempotent)."""
    out = _lib_path()
    src = os.path.join(_HERE, "skm_oracle.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, ip = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            ci = ctypes.c_int
            data = [i64, i64, ci, ip, ip, ip]
            lib.sko_rinv.argtypes = data + [ip]
            lib.sko_rinv.restype = None
            lib.sko_sim.argtypes = data + [ip, i64, ip]
            lib.sko_sim.restype = dbl
            lib.sko_assign.argtypes = data + [ip, i64, ip, ip, ip, ip, ip]
            lib.sko_assign.restype = i64
            lib.sko_update.argtypes = data + [ip, i64, ip, ip, ip, ip]
            lib.sko_update.restype = dbl
            lib.sko_drift.argtypes = [i64, i64, ip, ip, ip, ip]
            lib.sko_drift.restype = None
            lib.sko_center_bounds.argtypes = [i64, i64, ip, ip, ip]
            lib.sko_center_bounds.restype = None
            lib.sko_l_update.argtypes = [dbl, dbl, dbl]
            lib.sko_l_update.restype = dbl
            lib.sko_u_update.argtypes = [dbl, dbl, dbl]
            lib.sko_u_update.restype = dbl
            lib.sko_u_hamerly.argtypes = [dbl, dbl, dbl, ci]
            lib.sko_u_hamerly.restype = dbl
            lib.sko_run.argtypes = data + [ip, i64, ci, ip, i32, ci, ci, ip, ip, ip, ip, ip, ip]
            lib.sko_run.restype = ci
            lib.sko_kmeanspp.argtypes = data + [ip, i64, ip, ip]
            lib.sko_kmeanspp.restype = ci
            lib.sko_kmeanspp_bounds.argtypes = data + [ip, i64, ip, ip, ip, ip, ip, ip]
            lib.sko_kmeanspp_bounds.restype = ci
            _LIB = lib
    return _LIB


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


@dataclass
class Data:
    """Stored vectors promoted to float64 (CSR or dense)."""
    n: int
    d: int
    dense: bool
    row_ptr: np.ndarray | None
    col: np.ndarray | None
    val: np.ndarray

    @staticmethod
    def from_csr(csr) -> "Data":
        return Data(csr.n, csr.d, False, np.ascontiguousarray(csr.row_ptr, dtype=np.int64),
                    np.ascontiguousarray(csr.col, dtype=np.int32),
                    np.ascontiguousarray(np.asarray(csr.val).astype(np.float64)))

    @staticmethod
    def from_dense(X) -> "Data":
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
        return Data(X.shape[0], X.shape[1], True, None, None, X.reshape(-1))

    def args(self):
        return (self.n, self.d, 1 if self.dense else 0, _p(self.row_ptr), _p(self.col), _p(self.val))

    def row_len(self) -> np.ndarray:
        if self.dense:
            return np.full(self.n, self.d, dtype=np.int64)
        return np.diff(self.row_ptr)


def rinv(X: Data) -> np.ndarray:
    out = np.empty(X.n, dtype=np.float64)
    _lib().sko_rinv(*X.args(), _p(out))
    return out


def unit_rows(X: Data, rows) -> np.ndarray:
    """x_i = stored_i / |stored_i| as dense float64 rows (for initial centers)."""
    ri = rinv(X)
    out = np.zeros((len(rows), X.d), dtype=np.float64)
    for q, i in enumerate(np.asarray(rows)):
        if X.dense:
            out[q] = X.val[i * X.d:(i + 1) * X.d] * ri[i]
        else:
            b, e = X.row_ptr[i], X.row_ptr[i + 1]
            out[q, X.col[b:e]] = X.val[b:e] * ri[i]
    return out


def sim(X: Data, ri: np.ndarray, i: int, c: np.ndarray) -> float:
    c = np.ascontiguousarray(c, dtype=np.float64)
    return _lib().sko_sim(*X.args(), _p(ri), int(i), _p(c))


def kmeanspp(X: Data, ri: np.ndarray, u) -> np.ndarray:
    """Spherical k-means++ seeding (Section 5.6) from the uniform draws u (k of
    them, in [0, 1)); returns the chosen rows."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    rows = np.empty(len(u), dtype=np.int64)
    _lib().sko_kmeanspp(*X.args(), _p(ri), len(u), _p(u), _p(rows))
    return rows


def kmeanspp_bounds(X: Data, ri: np.ndarray, u, with_sims: bool = False):
    """Spherical k-means++ seeding (Section 5.6) with the bound
    pre-initialisation of Section 5.6's remark and Section 7's outlook: the
    seeding's own similarities give the first assignment from the seeded
    centers.  Returns (rows, labels, s_best, s_second, S) -- S the n x k
    similarities (Elkan's initial upper bounds) when with_sims, else None."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    k = len(u)
    rows = np.empty(k, dtype=np.int64)
    lab = np.empty(X.n, dtype=np.int32)
    s1 = np.empty(X.n)
    s2 = np.empty(X.n)
    S = np.empty((X.n, k)) if with_sims else None
    _lib().sko_kmeanspp_bounds(*X.args(), _p(ri), k, _p(u), _p(rows), _p(lab), _p(s1), _p(s2), _p(S))
    return rows, lab, s1, s2, S


def assign(X: Data, ri: np.ndarray, C: np.ndarray, a: np.ndarray | None = None):
    """Standard assignment.  Returns (labels, changed, s_best, s_second, top_gap)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    k = C.shape[0]
    lab = np.full(X.n, -1, dtype=np.int32) if a is None else np.array(a, dtype=np.int32, copy=True)
    sb = np.empty(X.n)
    ss = np.empty(X.n)
    gap = np.empty(X.n)
    ch = _lib().sko_assign(*X.args(), _p(ri), k, _p(C), _p(lab), _p(sb), _p(ss), _p(gap))
    return lab, int(ch), sb, ss, gap


def update(X: Data, ri: np.ndarray, a: np.ndarray, C_old: np.ndarray):
    """Center update.  Returns (C_new, norms, J)."""
    C_old = np.ascontiguousarray(C_old, dtype=np.float64)
    k = C_old.shape[0]
    a = np.ascontiguousarray(a, dtype=np.int32)
    Cn = np.empty_like(C_old)
    nr = np.empty(k)
    J = _lib().sko_update(*X.args(), _p(ri), k, _p(a), _p(C_old), _p(Cn), _p(nr))
    return Cn, nr, float(J)


def drift(C_old: np.ndarray, C_new: np.ndarray):
    C_old = np.ascontiguousarray(C_old, dtype=np.float64)
    C_new = np.ascontiguousarray(C_new, dtype=np.float64)
    k, d = C_old.shape
    p = np.empty(k)
    sp = np.empty(k)
    _lib().sko_drift(k, d, _p(C_old), _p(C_new), _p(p), _p(sp))
    return p, sp


def center_bounds(C: np.ndarray):
    C = np.ascontiguousarray(C, dtype=np.float64)
    k, d = C.shape
    cc = np.empty((k, k))
    s = np.empty(k)
    _lib().sko_center_bounds(k, d, _p(C), _p(cc), _p(s))
    return cc, s


def l_update(l: float, p: float, sp: float | None = None) -> float:
    if sp is None:
        sp = float(np.sqrt(max(0.0, (1 - p) * (1 + p))))
    return _lib().sko_l_update(l, p, sp)


def u_update(u: float, p: float, sp: float | None = None) -> float:
    if sp is None:
        sp = float(np.sqrt(max(0.0, (1 - p) * (1 + p))))
    return _lib().sko_u_update(u, p, sp)


def u_hamerly(u: float, pp: float, spp: float | None = None, tight: bool = False) -> float:
    if spp is None:
        spp = float(np.sqrt(max(0.0, (1 - pp) * (1 + pp))))
    return _lib().sko_u_hamerly(u, pp, spp, 1 if tight else 0)


@dataclass
class Trace:
    labels: np.ndarray    # iters x n int32, labels after each assignment
    changed: np.ndarray   # iters int64
    sims: np.ndarray      # iters int64, exact similarities computed
    J: np.ndarray         # iters float64, objective after each iteration
    iters: int
    C: np.ndarray         # final centers k x d
    violations: int


def run(X: Data, C0: np.ndarray, variant: str | int = "standard", max_iters: int = 100,
        hamerly_tight: bool = False, check_bounds: bool = False, ri: np.ndarray | None = None) -> Trace:
    """One full run from the initial centers C0 (k x d unit rows)."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    C = np.array(C0, dtype=np.float64, copy=True, order="C")
    k = C.shape[0]
    ri = rinv(X) if ri is None else ri
    lt = np.empty((max_iters, X.n), dtype=np.int32)
    ch = np.zeros(max_iters, dtype=np.int64)
    sm = np.zeros(max_iters, dtype=np.int64)
    J = np.zeros(max_iters)
    it = ctypes.c_int32(0)
    viol = ctypes.c_int64(0)
    rc = _lib().sko_run(*X.args(), _p(ri), k, v, _p(C), int(max_iters), 1 if hamerly_tight else 0,
                        1 if check_bounds else 0, _p(lt), _p(ch), _p(sm), _p(J), ctypes.byref(it),
                        ctypes.byref(viol))
    if rc != 0:
        raise MemoryError("oracle run failed")
    n_it = it.value
    return Trace(lt[:n_it].copy(), ch[:n_it].copy(), sm[:n_it].copy(), J[:n_it].copy(), n_it, C, int(viol.value))
