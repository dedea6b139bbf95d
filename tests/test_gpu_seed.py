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


# ------------------------------------------ bound pre-initialisation

PRE_VARIANTS = ["standard", "hamerly", "simp_hamerly", "elkan", "simp_elkan"]


def _state(km, variant):
    out = [km.labels(), km.centers()]
    if variant != "standard":
        out += list(km.bounds())
    return out


@pytest.mark.parametrize("variant", PRE_VARIANTS)
def test_seed_assign_equals_seed_then_assign(variant):
    """skm_seed_kmeanspp_assign leaves exactly the state of skm_seed_kmeanspp
    followed by skm_assign (labels, centers, l and every u, bit for bit), and
    the runs that continue from both states are identical."""
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=8000, d=6000, seed=13))
    k = 37
    u = np.random.default_rng(13).random(k)
    a, ka = _ctx_csr(X, k, variant)
    b, kb = _ctx_csr(X, k, variant)
    rows_a = a.seed_kmeanspp(u)
    ch_a = a.assign()
    rows_b, ch_b = b.seed_kmeanspp_assign(u)
    np.testing.assert_array_equal(rows_a, rows_b)
    assert ch_a == ch_b == X.n
    assert b.stats().last_sims == X.n * k and b.stats().iterations == 1
    for x, y in zip(_state(a, variant), _state(b, variant)):
        np.testing.assert_array_equal(x, y)
    for _ in range(25):
        a.update_centers()
        b.update_centers()
        ca, cb = a.assign(), b.assign()
        assert ca == cb
        np.testing.assert_array_equal(a.labels(), b.labels())
        if ca == 0:
            break
    np.testing.assert_array_equal(a.centers(), b.centers())
    a.close()
    b.close()


def test_seed_assign_matches_oracle_and_bounds_hold():
    """Against the FP64 oracle's pre-initialisation (the seeding's own
    similarities): the same rows, the same labels up to near-ties, and bounds
    that hold for the exact similarities -- l(i) <= s(i, a(i)), Elkan's
    u(i, j) >= s(i, j) for every center."""
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=3000, d=5000, seed=17))
    k = 24
    u = np.random.default_rng(17).random(k)
    d = oracle.Data.from_csr(X)
    ri = oracle.rinv(d)
    rows_o, lab_o, s1, s2, S = oracle.kmeanspp_bounds(d, ri, u, with_sims=True)
    km, keep = _ctx_csr(X, k, "elkan")
    rows, ch = km.seed_kmeanspp_assign(u)
    np.testing.assert_array_equal(rows, rows_o)
    lab = km.labels()
    bad = (lab != lab_o) & (s1 - s2 >= 1e-6)
    assert not bad.any()
    l, U = km.bounds()
    assert np.all(l.astype(np.float64) <= S[np.arange(X.n), lab])
    assert np.all(U.astype(np.float64) >= S)
    km.close()


@pytest.mark.parametrize("variant,precision", [("standard", "fp32"), ("hamerly", "fp32"), ("standard", "bf16"),
                                               ("hamerly", "bf16")])
def test_seed_assign_dense(variant, precision):
    """Dense rows, FP32 path and the BF16 precision form: the runs continued
    from the pre-initialised state and from seeding + first assignment give
    the same labels, iteration by iteration."""
    Xs = synth.vmf(4000, 96, 20, 30.0, seed=19)
    k = 33
    u = np.random.default_rng(19).random(k)
    Xd = torch.from_numpy(Xs).cuda()
    a = skm.KMeans.dense(Xd, k, variant=variant, precision=precision, seed=1)
    b = skm.KMeans.dense(Xd, k, variant=variant, precision=precision, seed=1)
    a.seed_kmeanspp(u)
    a.assign()
    b.seed_kmeanspp_assign(u)
    np.testing.assert_array_equal(a.labels(), b.labels())
    for _ in range(15):
        a.update_centers()
        b.update_centers()
        ca, cb = a.assign(), b.assign()
        assert ca == cb
        np.testing.assert_array_equal(a.labels(), b.labels())
        if ca == 0:
            break
    a.close()
    b.close()


def test_seed_assign_rejections():
    X = synth.tfidf(synth.scaled(synth.CSR_TINY, n=300))
    km, keep = _ctx_csr(X, 5, "yinyang")
    with pytest.raises(skm.SkmError) as e:
        km.seed_kmeanspp_assign(np.full(5, 0.5))
    assert e.value.code == skm.EUNSUPPORTED
    km.close()
