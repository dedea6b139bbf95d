"""Thin ctypes binding of libskm (include/skm.h).

Argument marshalling only: every step of the clustering runs in the CUDA
library.  Device buffers are torch CUDA tensors (torch is used for device
memory and streams); host buffers are numpy arrays.  If the library cannot be
loaded this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ESTATE, ETOOBIG = 0, -1, -2, -3, -4, -5, -6, -7
STANDARD, HAMERLY, ELKAN, SIMP_HAMERLY, SIMP_ELKAN, YINYANG = 0, 1, 2, 3, 4, 5
VARIANTS = {"standard": STANDARD, "hamerly": HAMERLY, "elkan": ELKAN, "simp_hamerly": SIMP_HAMERLY,
            "simp_elkan": SIMP_ELKAN, "yinyang": YINYANG}
F32, F16, BF16 = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
CSR, DENSE = 0, 1
DEVICE, HOST = 0, 1

# every exported symbol of include/skm.h
EXPORTS = ["skm_default_options", "skm_init", "skm_reset", "skm_assign", "skm_update_centers", "skm_run",
           "skm_get_labels", "skm_get_centers", "skm_set_centers", "skm_set_labels", "skm_get_bounds",
           "skm_get_stats", "skm_bound_bytes", "skm_kernel_launches", "skm_profile", "skm_profile_read",
           "skm_destroy", "skm_strerror", "skm_assign_noalloc", "skm_get_bf16_topk", "skm_batch_init",
           "skm_autotune", "skm_selftest_wait", "skm_seed_kmeanspp", "skm_seed_kmeanspp_assign", "skm_measure_peak"]


class SkmError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_strerror(code)} ({code})")
        self.code = code


class skm_data(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("layout", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("memspace", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class skm_options(ctypes.Structure):
    _fields_ = [("hamerly_tight", ctypes.c_int32), ("validate", ctypes.c_int32), ("row_threshold", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("graph", ctypes.c_int32), ("graph_check", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("fused_update", ctypes.c_int32),
                ("screen", ctypes.c_int32), ("k_tile", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class skm_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("last_changed", ctypes.c_int64), ("last_sims", ctypes.c_int64),
                ("total_sims", ctypes.c_int64), ("last_survivors", ctypes.c_int64),
                ("last_rechecks", ctypes.c_int64), ("objective", ctypes.c_double),
                ("last_cand_rechecks", ctypes.c_int64), ("last_skipped", ctypes.c_int64)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libskm.so (building it first if needed); raises if impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libskm.so is missing at {path}; run paper_2107_04074_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "skm_default_options": (None, [P]),
        "skm_init": (ctypes.c_int, [P, P, i32, i32, P, u64, P, P]),
        "skm_reset": (ctypes.c_int, [P, P, u64]),
        "skm_assign": (ctypes.c_int, [P, P]),
        "skm_update_centers": (ctypes.c_int, [P, P]),
        "skm_run": (ctypes.c_int, [P, i32, P, P]),
        "skm_get_labels": (ctypes.c_int, [P, P, i32]),
        "skm_get_centers": (ctypes.c_int, [P, P, i32]),
        "skm_set_centers": (ctypes.c_int, [P, P, i32]),
        "skm_set_labels": (ctypes.c_int, [P, P, i32]),
        "skm_get_bounds": (ctypes.c_int, [P, P, P, i32]),
        "skm_get_stats": (ctypes.c_int, [P, P]),
        "skm_bound_bytes": (ctypes.c_int, [i32, i64, i32, P]),
        "skm_kernel_launches": (i64, []),
        "skm_profile": (ctypes.c_int, [P, i32]),
        "skm_profile_read": (ctypes.c_int, [P, i32, P, i32, P, P]),
        "skm_destroy": (None, [P]),
        "skm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "skm_assign_noalloc": (ctypes.c_int, [P, i32, P, P, P, P]),
        "skm_get_bf16_topk": (ctypes.c_int, [P, P, P, P, i32]),
        "skm_batch_init": (ctypes.c_int, [P, P, P, P, i32, i32, P, u64, P, P]),
        "skm_autotune": (ctypes.c_int, [P, ctypes.c_char_p, i32, P]),
        "skm_selftest_wait": (ctypes.c_int, [i64, P]),
        "skm_seed_kmeanspp": (ctypes.c_int, [P, P, P]),
        "skm_seed_kmeanspp_assign": (ctypes.c_int, [P, P, P, P]),
        "skm_measure_peak": (ctypes.c_int, [i32, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _strerror(code: int) -> str:
    try:
        return load(build_if_missing=False).skm_strerror(code).decode()
    except Exception:  # pragma: no cover
        return "unknown"


def _check(code: int, what: str):
    if code != OK:
        raise SkmError(code, what)


def selftest_wait(timeout_ns: int, stream=None) -> int:
    """Status of a device wait on a barrier nothing completes (SKM_ETIMEOUT expected)."""
    return int(load().skm_selftest_wait(int(timeout_ns), ctypes.c_void_p(stream or 0)))


PEAK_FP32_FMA, PEAK_FP64_FMA, PEAK_FP32_FMA2, PEAK_L2_GATHER = 0, 1, 2, 3


def measure_peak(kind: str, stream=None) -> float:
    """Measured FMA rate of the current GPU in TFLOP/s (skm_measure_peak):
    kind "fp32", "fp64" or "fp32x2" (FP32 FMAs issued as packed pairs); kind
    "l2_gather": TB/s of 416-byte rows gathered from an L2-resident table."""
    out = ctypes.c_double(0)
    code = {"fp32": PEAK_FP32_FMA, "fp64": PEAK_FP64_FMA, "fp32x2": PEAK_FP32_FMA2,
            "l2_gather": PEAK_L2_GATHER}[kind]
    _check(load().skm_measure_peak(code, ctypes.byref(out), ctypes.c_void_p(stream or 0)), "skm_measure_peak")
    return out.value


def kernel_launches() -> int:
    return int(load().skm_kernel_launches())


def bound_bytes(variant, n: int, k: int) -> int:
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    out = ctypes.c_int64(0)
    _check(load().skm_bound_bytes(v, n, k, ctypes.byref(out)), "skm_bound_bytes")
    return out.value


def assign_noalloc(n: int, d: int, row_ptr, col_idx, values, k: int, centers, labels, stream=None,
                   count: bool = True):
    """Standard assignment without device allocation (skm_assign_noalloc).

    All arrays are torch CUDA tensors; labels (int32[n]) is updated in place.
    count=True: returns the number of changed labels (synchronises; a malformed
    row raises SkmError EINVAL).  count=False: passes no host output, so the
    call only enqueues its kernels and returns None."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    data = skm_data(n=n, d=d, layout=CSR, dtype=_dtype_code(values.dtype), memspace=DEVICE, reserved=0,
                    row_ptr=_ptr(row_ptr), col_idx=_ptr(col_idx), values=_ptr(values))
    out = ctypes.c_int64(0)
    _check(load().skm_assign_noalloc(ctypes.byref(data), int(k), _ptr(centers), _ptr(labels),
                                     ctypes.byref(out) if count else None, ctypes.c_void_p(stream)),
           "skm_assign_noalloc")
    return out.value if count else None


def _ptr(x):
    """Address of a torch tensor (device) or numpy array (host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def _dtype_code(dt) -> int:
    s = str(dt)
    if s.endswith("bfloat16"):
        return BF16
    if s.endswith("float32"):
        return F32
    if s.endswith("float16"):
        return F16
    raise ValueError(f"unsupported value dtype {dt}")


@dataclass
class Stats:
    iterations: int
    last_changed: int
    last_sims: int
    total_sims: int
    last_survivors: int
    last_rechecks: int
    objective: float
    last_cand_rechecks: int = 0
    last_skipped: int = 0


class KMeans:
    """One clustering context (skm_ctx) over CSR data.

    row_ptr / col_idx / values: torch CUDA tensors (borrowed: keep them alive)
    or numpy arrays (copied to the device by the library).
    """

    def __init__(self, n: int, d: int, row_ptr, col_idx, values, k: int, variant="standard", init_rows=None,
                 seed: int = 0, hamerly_tight: bool = False, row_threshold: int = 0, stream=None,
                 precision: str = "fp32", graph: bool = False, graph_check: int = 0, blocks_per_sm: int = 0,
                 fused_update: bool = False, screen: bool | None = None, k_tile: int = 0):
        lib = load()
        host = isinstance(values, np.ndarray)
        self._keep = (row_ptr, col_idx, values)
        dense = row_ptr is None
        data = skm_data(n=n, d=d, layout=DENSE if dense else CSR, dtype=_dtype_code(values.dtype),
                        memspace=HOST if host else DEVICE, reserved=0, row_ptr=_ptr(row_ptr),
                        col_idx=_ptr(col_idx), values=_ptr(values))
        opt = skm_options()
        lib.skm_default_options(ctypes.byref(opt))
        opt.hamerly_tight = 1 if hamerly_tight else 0
        opt.precision = {"fp32": PREC_FP32, "bf16": PREC_BF16, "fp8": PREC_FP8}[precision]
        opt.row_threshold = int(row_threshold)
        opt.graph = 1 if graph else 0
        opt.graph_check = int(graph_check)
        opt.blocks_per_sm = int(blocks_per_sm)
        opt.fused_update = 1 if fused_update else 0
        # screen: None = the library's choice (on for Elkan with k > 128), True / False = on / off
        opt.screen = 0 if screen is None else (1 if screen else 2)
        # centers per pass of the whole-row kernel: 0 = the smallest tile that holds k
        opt.k_tile = int(k_tile)
        self.n, self.d, self.k = int(n), int(d), int(k)
        self.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        rows = None
        if init_rows is not None:
            rows = np.ascontiguousarray(np.asarray(init_rows, dtype=np.int64))
            if rows.shape != (k,):
                raise ValueError("init_rows must have k entries")
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if not host else 0
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.skm_init(ctypes.byref(h), ctypes.byref(data), int(k), self.variant, _ptr(rows), int(seed),
                            ctypes.byref(opt), ctypes.c_void_p(stream)), "skm_init")
        self._h = h

    @classmethod
    def dense(cls, X, k: int, **kw) -> "KMeans":
        """Dense rows X (n x d FP32; torch CUDA tensor, borrowed, or numpy array, copied)."""
        n, d = X.shape
        return cls(n, d, None, None, X, k, **kw)

    def close(self):
        if getattr(self, "_h", None):
            load().skm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, init_rows=None, seed: int = 0):
        rows = None if init_rows is None else np.ascontiguousarray(np.asarray(init_rows, dtype=np.int64))
        _check(load().skm_reset(self._h, _ptr(rows), int(seed)), "skm_reset")

    def assign(self, sync: bool = True):
        out = ctypes.c_int64(0)
        _check(load().skm_assign(self._h, ctypes.byref(out) if sync else None), "skm_assign")
        return out.value if sync else None

    def update_centers(self, sync: bool = True):
        out = ctypes.c_double(0)
        _check(load().skm_update_centers(self._h, ctypes.byref(out) if sync else None), "skm_update_centers")
        return out.value if sync else None

    def run(self, max_iters: int):
        it = ctypes.c_int32(0)
        J = ctypes.c_double(0)
        _check(load().skm_run(self._h, int(max_iters), ctypes.byref(it), ctypes.byref(J)), "skm_run")
        return it.value, J.value

    def labels(self, out=None):
        if out is None:
            out = np.empty(self.n, dtype=np.int32)
        _check(load().skm_get_labels(self._h, _ptr(out), HOST if isinstance(out, np.ndarray) else DEVICE),
               "skm_get_labels")
        return out

    def centers(self, out=None):
        if out is None:
            out = np.empty((self.k, self.d), dtype=np.float32)
        _check(load().skm_get_centers(self._h, _ptr(out), HOST if isinstance(out, np.ndarray) else DEVICE),
               "skm_get_centers")
        return out

    def set_centers(self, C):
        if isinstance(C, np.ndarray):
            C = np.ascontiguousarray(C, dtype=np.float32)
        _check(load().skm_set_centers(self._h, _ptr(C), HOST if isinstance(C, np.ndarray) else DEVICE),
               "skm_set_centers")

    def set_labels(self, a):
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.int32)
        _check(load().skm_set_labels(self._h, _ptr(a), HOST if isinstance(a, np.ndarray) else DEVICE),
               "skm_set_labels")

    def bounds(self):
        l = np.empty(self.n, dtype=np.float32)
        elk = self.variant in (ELKAN, SIMP_ELKAN)
        if self.variant == YINYANG:
            u = np.empty(((self.k + 7) // 8, self.n), dtype=np.float32)
        else:
            u = np.empty((self.n, self.k) if elk else self.n, dtype=np.float32)
        _check(load().skm_get_bounds(self._h, _ptr(l), _ptr(u), HOST), "skm_get_bounds")
        return l, u

    def profile(self, enable: bool = True):
        _check(load().skm_profile(self._h, 1 if enable else 0), "skm_profile")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} recorded since profiling started."""
        out = {}
        buf = ctypes.create_string_buffer(64)
        idx = 0
        while True:
            ms = ctypes.c_double(0)
            cnt = ctypes.c_int64(0)
            rc = load().skm_profile_read(self._h, idx, buf, 64, ctypes.byref(ms), ctypes.byref(cnt))
            if rc != OK:
                break
            out[buf.value.decode()] = (ms.value, cnt.value)
            idx += 1
        return out

    def bf16_topk(self):
        """(n x 8 best BF16 similarities in descending order, n x 8 their centers) of the last
        assignment, and each row's error bound eps (n floats) against the exact similarities."""
        vals = np.empty((self.n, 8), dtype=np.float32)
        idx = np.empty((self.n, 8), dtype=np.int32)
        eps = np.empty(self.n, dtype=np.float32)
        _check(load().skm_get_bf16_topk(self._h, _ptr(vals), _ptr(idx), _ptr(eps), HOST),
               "skm_get_bf16_topk")
        return vals, idx, eps

    def seed_kmeanspp(self, u) -> np.ndarray:
        """Spherical k-means++ seeding from the k uniform draws u (Section 5.6);
        returns the chosen rows, which become the centers."""
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
        if u.shape != (self.k,):
            raise ValueError("u must have k entries")
        rows = np.empty(self.k, dtype=np.int64)
        _check(load().skm_seed_kmeanspp(self._h, _ptr(u), _ptr(rows)), "skm_seed_kmeanspp")
        return rows

    def seed_kmeanspp_assign(self, u, sync: bool = True):
        """Seeding plus the first assignment from the seeding's similarities
        (skm_seed_kmeanspp_assign): returns (rows, labels changed or None)."""
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
        if u.shape != (self.k,):
            raise ValueError("u must have k entries")
        rows = np.empty(self.k, dtype=np.int64)
        out = ctypes.c_int64(0)
        _check(load().skm_seed_kmeanspp_assign(self._h, _ptr(u), _ptr(rows), ctypes.byref(out) if sync else None),
               "skm_seed_kmeanspp_assign")
        return rows, (out.value if sync else None)

    def autotune(self, cache_path=None, iters: int = 3) -> bool:
        """Pick, by timing, the persistent kernels' launch shape and the Elkan
        whole-row threshold, then the whole-row kernel's tile of centers and
        whether the screened pass is used (see skm_autotune); True when the
        choice came from cache_path."""
        fc = ctypes.c_int32(0)
        path = None if cache_path is None else str(cache_path).encode()
        _check(load().skm_autotune(self._h, path, int(iters), ctypes.byref(fc)), "skm_autotune")
        return bool(fc.value)

    def stats(self) -> Stats:
        s = skm_stats()
        _check(load().skm_get_stats(self._h, ctypes.byref(s)), "skm_get_stats")
        return Stats(s.iterations, s.last_changed, s.last_sims, s.total_sims, s.last_survivors, s.last_rechecks,
                     s.objective, s.last_cand_rechecks, s.last_skipped)


class Batch(KMeans):
    """Batched form: independent runs over row blocks of one CSR matrix.

    run_rows: nruns + 1 row offsets; ks: centers per run; init_rows: for each
    run in order ks[r] row indices local to the run (or None: seeded).
    labels() are local to each run; centers() stacks the runs' centers.
    """

    def __init__(self, n: int, d: int, row_ptr, col_idx, values, run_rows, ks, variant="simp_elkan",
                 init_rows=None, seed: int = 0, row_threshold: int = 0, stream=None, graph: bool = False,
                 graph_check: int = 0, blocks_per_sm: int = 0):
        lib = load()
        host = isinstance(values, np.ndarray)
        self._keep = (row_ptr, col_idx, values)
        data = skm_data(n=n, d=d, layout=CSR, dtype=_dtype_code(values.dtype), memspace=HOST if host else DEVICE,
                        reserved=0, row_ptr=_ptr(row_ptr), col_idx=_ptr(col_idx), values=_ptr(values))
        opt = skm_options()
        lib.skm_default_options(ctypes.byref(opt))
        opt.row_threshold = int(row_threshold)
        opt.graph = 1 if graph else 0
        opt.graph_check = int(graph_check)
        opt.blocks_per_sm = int(blocks_per_sm)
        self.run_rows = np.ascontiguousarray(np.asarray(run_rows, dtype=np.int64))
        self.ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int32))
        self.nruns = len(self.ks)
        if self.run_rows.shape != (self.nruns + 1,):
            raise ValueError("run_rows must have nruns + 1 entries")
        self.n, self.d, self.k = int(n), int(d), int(self.ks.sum())
        self.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        rows = None
        if init_rows is not None:
            rows = np.ascontiguousarray(np.asarray(init_rows, dtype=np.int64))
            if rows.shape != (self.k,):
                raise ValueError("init_rows must have sum(ks) entries")
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if not host else 0
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.skm_batch_init(ctypes.byref(h), ctypes.byref(data), _ptr(self.run_rows), _ptr(self.ks),
                                  self.nruns, self.variant, _ptr(rows), int(seed), ctypes.byref(opt),
                                  ctypes.c_void_p(stream)), "skm_batch_init")
        self._h = h

    def run_centers(self, C=None):
        """List of per-run center arrays (k_r x d) from centers()."""
        C = self.centers() if C is None else C
        off = np.concatenate([[0], np.cumsum(self.ks)])
        return [C[off[r]:off[r + 1]] for r in range(self.nruns)]

    def run_labels(self, lab=None):
        lab = self.labels() if lab is None else lab
        return [lab[self.run_rows[r]:self.run_rows[r + 1]] for r in range(self.nruns)]
