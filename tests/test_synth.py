"""The seeded input generators follow their stated recipes."""
import numpy as np
import pytest
from scipy import special

import synth


def test_tfidf_shape_and_recipe():
    cfg = synth.scaled(synth.CSR_RCV1_LIKE, n=20000)
    c = synth.tfidf(cfg)
    lens = np.diff(c.row_ptr)
    assert lens.min() >= cfg.lo and lens.max() <= cfg.hi
    assert abs(lens.mean() - cfg.a) / cfg.a < 0.03          # lognormal with arithmetic mean a
    for i in range(0, c.n, 997):
        row = c.col[c.row_ptr[i]:c.row_ptr[i + 1]]
        assert np.all(np.diff(row) > 0) and row.min() >= 0 and row.max() < c.d
    nrm = np.sqrt(np.add.reduceat(c.val.astype(np.float64) ** 2, c.row_ptr[:-1]))
    np.testing.assert_allclose(nrm, 1.0, atol=1e-6)
    assert np.all(c.val > 0)
    # Zipf head: the most frequent term appears in far more rows than the median one
    df = np.bincount(c.col, minlength=c.d)
    assert df.max() > 50 * max(1, np.median(df))


def test_tfidf_deterministic_and_thread_independent():
    cfg = synth.scaled(synth.CSR_TINY, n=500)
    a = synth.tfidf(cfg, threads=1)
    b = synth.tfidf(cfg, threads=7)
    np.testing.assert_array_equal(a.row_ptr, b.row_ptr)
    np.testing.assert_array_equal(a.col, b.col)
    np.testing.assert_array_equal(a.val, b.val)
    lens = np.diff(synth.tfidf(synth.CSR_TINY).row_ptr)
    assert abs(lens.mean() - 50) < 1.0                         # Poisson(50)


def test_vmf_mean_resultant_length():
    """The cosine to the component mean has expectation A_d(kappa) = I_{d/2}/I_{d/2-1}."""
    d, kappa = 64, 40.0
    X, comp, means = synth.vmf(20000, d, 5, kappa, seed=3, return_comp=True)
    w = np.sum(X.astype(np.float64) * means[comp], axis=1)
    want = special.ive(d / 2, kappa) / special.ive(d / 2 - 1, kappa)
    assert abs(w.mean() - want) < 5e-3
    np.testing.assert_allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-6)


def test_init_rows_distinct():
    r = synth.init_rows(1000, 200, 9)
    assert len(set(r.tolist())) == 200 and r.min() >= 0 and r.max() < 1000
    with pytest.raises(ValueError):
        synth.init_rows(5, 6, 1)
