"""Bound pre-initialisation from the spherical k-means++ seeding (the remark
of Section 5.6 and the outlook of Section 7), in the FP64 oracle: the
seeding's own similarities give the first assignment from the seeded centers
and its Hamerly and Elkan bounds.  Pinned against brute force (all n k
cosines by numpy), against the oracle's separate assignment step, and on an
exact tie that checks the tie rule follows center order, not row order."""
import numpy as np
import pytest

import oracle
import synth


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


@pytest.mark.parametrize("seed", range(6))
def test_seeding_bounds_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, d, k = int(rng.integers(6, 64)), int(rng.integers(2, 16)), int(rng.integers(1, 6))
    k = min(k, n)
    Xs = np.abs(rng.standard_normal((n, d))) * rng.uniform(0.5, 3.0, size=(n, 1))
    Xs[rng.random((n, d)) < 0.3] = 0.0
    Xs[:, 0] += 1e-3
    u = rng.random(k)
    for dense in (True, False):
        csr = synth.csr_from_dense(Xs)
        X = oracle.Data.from_dense(Xs) if dense else oracle.Data.from_csr(csr)
        ri = oracle.rinv(X)
        rows, lab, s1, s2, S = oracle.kmeanspp_bounds(X, ri, u, with_sims=True)
        np.testing.assert_array_equal(rows, oracle.kmeanspp(X, ri, u))  # the same seeding
        Xn = _unit(Xs) if dense else csr.dense() * ri[:, None]
        Sb = Xn @ Xn[rows].T                                             # every cosine, brute force
        np.testing.assert_allclose(S, Sb, rtol=0, atol=1e-13)
        np.testing.assert_array_equal(lab, np.argmax(Sb, axis=1))      # first maximum: lowest index
        np.testing.assert_allclose(s1, Sb.max(axis=1), rtol=0, atol=1e-13)
        if k > 1:
            np.testing.assert_allclose(s2, np.sort(Sb, axis=1)[:, -2], rtol=0, atol=1e-13)
        else:
            assert np.all(np.isneginf(s2))


def test_seeding_bounds_equal_the_first_assignment():
    """The same FP64 similarities as the oracle's assignment step from the
    seeded centers, bit for bit: labels, best and second best."""
    csr = synth.tfidf(synth.scaled(synth.CSR_TINY, n=600, seed=5))
    X = oracle.Data.from_csr(csr)
    ri = oracle.rinv(X)
    u = np.random.default_rng(5).random(15)
    rows, lab, s1, s2, _ = oracle.kmeanspp_bounds(X, ri, u)
    want, ch, sb, ss, _ = oracle.assign(X, ri, oracle.unit_rows(X, rows))
    np.testing.assert_array_equal(lab, want)
    np.testing.assert_array_equal(s1, sb)
    np.testing.assert_array_equal(s2, ss)
    assert ch == X.n
    # and an Elkan run from the seeded centers makes that first assignment
    tr = oracle.run(X, oracle.unit_rows(X, rows), "elkan", max_iters=1)
    np.testing.assert_array_equal(tr.labels[0], lab)


def test_seeding_bounds_tie_rule_follows_center_order():
    """Rows e1, e0, e0 + e1 (normalised), seeded e1 first then e0: the third
    row is equally close to both centers and takes center 0 (the first chosen,
    row 0 = e1), although e0 is the lower row index."""
    Xs = np.array([[0, 1, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]], dtype=np.float64)
    X = oracle.Data.from_dense(Xs)
    ri = oracle.rinv(X)
    # u0 = 0.1 picks row 0 (e1); the second draw follows 1 - cos: rows 1 and 3
    # weigh most, u1 = 0 picks the first row with positive weight, row 1 (e0)
    rows, lab, s1, s2, _ = oracle.kmeanspp_bounds(X, ri, [0.1, 0.0])
    assert rows.tolist() == [0, 1]
    assert lab.tolist() == [0, 1, 0, 0]
    assert s1[2] == s2[2]  # the tie: best and second best are equal
