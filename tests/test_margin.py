"""The exactness margin (reading M): the canonical FP32 similarity of a row
with m stored entries -- a sequential FP32 FMA chain over the entries in
order, times the FP32 1/|x| -- is within delta = g / (1 - g), g = (m + 10) 2^-24,
of the exact cosine for every unit FP32 center.  The chain is emulated on the
CPU step by step (each FMA as the FP64 sum of an exact product, rounded to
FP32; the rare double rounding this allows is far inside the 10-unit slack);
the exact cosine is an exactly rounded FP64 sum."""
import math

import numpy as np

import synth

U = 2.0 ** -24


def delta(m):
    g = (m + 10.0) * U
    return g / (1.0 - g)


def canonical(vals, cols, C32, ri):
    """fl32(chain(sum_p v_p C[:, t_p]) * ri) for one row against all centers."""
    acc = np.zeros(C32.shape[0], dtype=np.float32)
    for v, t in zip(vals, cols):
        acc = (np.float64(v) * C32[:, t].astype(np.float64) + acc.astype(np.float64)).astype(np.float32)
    return (acc.astype(np.float64) * np.float64(ri)).astype(np.float32).astype(np.float64)


def unit_centers(k, d, seed):
    rng = np.random.default_rng(seed)
    C = np.abs(rng.standard_normal((k, d))) ** 3  # skewed, like TF-IDF means
    return (C / np.linalg.norm(C, axis=1, keepdims=True)).astype(np.float32)


def check_rows(csr, C32, rows):
    worst = 0.0
    for i in rows:
        b, e = csr.row_ptr[i], csr.row_ptr[i + 1]
        vals, cols = csr.val[b:e].astype(np.float32), csr.col[b:e]
        v64 = vals.astype(np.float64)
        nrm = math.sqrt(math.fsum(v64 * v64))
        ri = np.float32(1.0 / nrm)
        f = canonical(vals, cols, C32, ri)
        s = np.array([math.fsum(v64 * C32[j, cols].astype(np.float64)) / nrm for j in range(len(C32))])
        err = np.abs(f - s).max()
        assert err <= delta(e - b), (i, e - b, err, delta(e - b))
        worst = max(worst, err / delta(e - b))
    return worst


def test_margin_bounds_the_canonical_similarity_tfidf_rows():
    csr = synth.tfidf(synth.CSR_TINY)
    C32 = unit_centers(16, csr.d, 1)
    longest = np.argsort(np.diff(csr.row_ptr))[-20:]
    worst = check_rows(csr, C32, list(range(60)) + list(longest))
    assert worst < 1.0


def _one_row(vals, cols, d):
    return synth.CSR(1, d, np.array([0, len(vals)], np.int64), np.asarray(cols, np.int32),
                     np.asarray(vals, np.float32))


def test_margin_bounds_long_same_sign_rows():
    """A long row of equal-sign terms and centers aligned with it (no
    cancellation, the running sum grows with every entry): within delta, and
    above a margin without the m term, 10u -- so that term is needed."""
    rng = np.random.default_rng(7)
    m, d = 20000, 24000
    cols = np.sort(rng.choice(d, m, replace=False))
    vals = (1.0 + rng.random(m)).astype(np.float32)
    row = np.zeros(d, np.float64)
    row[cols] = vals
    C = np.stack([row + 0.01 * rng.random(d) for _ in range(4)])
    C32 = (C / np.linalg.norm(C, axis=1, keepdims=True)).astype(np.float32)
    csr = _one_row(vals, cols, d)
    assert check_rows(csr, C32, [0]) < 1.0
    f = canonical(vals, cols, C32, np.float32(1.0 / np.linalg.norm(vals.astype(np.float64))))
    s = C32.astype(np.float64)[:, cols] @ vals.astype(np.float64) / np.linalg.norm(vals.astype(np.float64))
    assert np.abs(f - s).max() > delta(0)


def test_margin_is_absolute_not_relative_to_the_similarity():
    """Terms that cancel (a row orthogonal to the center up to rounding):
    the similarity is ~0 while the chain's error follows sum |v c| ~ 1, so a
    margin of (m + 10) u |s| would fail; delta holds."""
    rng = np.random.default_rng(9)
    m = 4000
    c = rng.standard_normal(m)
    c /= np.linalg.norm(c)
    v = rng.standard_normal(m)
    v -= (v @ c) * c  # orthogonal in FP64; FP32 storage leaves a tiny similarity
    vals = v.astype(np.float32)
    C32 = c[None, :].astype(np.float32)
    cols = np.arange(m)
    csr = _one_row(vals, cols, m)
    assert check_rows(csr, C32, [0]) < 1.0
    v64 = vals.astype(np.float64)
    nrm = np.linalg.norm(v64)
    s = math.fsum(v64 * C32[0].astype(np.float64)) / nrm
    f = canonical(vals, cols, C32, np.float32(1.0 / nrm))[0]
    assert abs(f - s) > (m + 10) * U * abs(s)
