"""Spherical k-means++ seeding on the GPU (Section 5.6) against the FP64
oracle: the same draws give the same rows (the weights differ only in their
last bits, far below the spacing of the prefix sums), the centers become the
normalised chosen rows, and a run continues from them."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402


def _ctx_csr(X, k, variant="simp_elkan"):
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    return skm.KMeans(X.n, X.d, *dev, k, variant=variant, seed=1), dev


@pytest.mark.parametrize("cfg,k,seed", [(synth.CSR_TINY, 20, 1), (synth.CSR_TINY, 60, 2),
                                        (synth.scaled(synth.CSR_RCV1_LIKE, n=20000, d=20000, seed=9), 100, 3)])
def test_seed_csr_matches_oracle(cfg, k, seed):
    X = synth.tfidf(cfg)
    u = np.random.default_rng(seed).random(k)
    km, keep = _ctx_csr(X, k)
    rows = km.seed_kmeanspp(u)
    d = oracle.Data.from_csr(X)
    want = oracle.kmeanspp(d, oracle.rinv(d), u)
    np.testing.assert_array_equal(rows, want)
    assert len(set(rows.tolist())) == k
    np.testing.assert_allclose(km.centers(), oracle.unit_rows(d, rows), atol=2e-7)
    # a run continues from the seeded centers and agrees with the oracle
    C = km.centers()
    km.assign()
    lab, _, _, _, gap = oracle.assign(d, oracle.rinv(d), C.astype(np.float64))
    assert np.all((lab == km.labels()) | (gap < 1e-6))
    it, _ = km.run(50)
    assert it >= 1
    km.close()


def test_seed_dense_matches_oracle():
    Xs = synth.vmf(3000, 64, 12, 20.0, seed=4)
    u = np.random.default_rng(7).random(40)
    km = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 40, variant="hamerly")
    rows = km.seed_kmeanspp(u)
    d = oracle.Data.from_dense(Xs)
    np.testing.assert_array_equal(rows, oracle.kmeanspp(d, oracle.rinv(d), u))
    km.close()


def test_seed_rejections():
    X = synth.tfidf(synth.scaled(synth.CSR_TINY, n=300))
    km, keep = _ctx_csr(X, 5)
    with pytest.raises(skm.SkmError):
        km.seed_kmeanspp(np.array([0.1, 0.2, 1.0, 0.3, 0.4]))
    with pytest.raises(skm.SkmError):
        km.seed_kmeanspp(np.array([0.1, -0.2, 0.5, 0.3, 0.4]))
    km.close()
    runs = np.array([0, 150, 300])
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    b = skm.Batch(X.n, X.d, *dev, runs, [3, 4])
    with pytest.raises(skm.SkmError):
        b.seed_kmeanspp(np.full(7, 0.5))
    b.close()
