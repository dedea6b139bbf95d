"""The batched form through the C ABI: many independent runs in one context.

Each run of a batch must follow exactly the trajectory of the same run alone
(the per-row arithmetic is the same canonical FP32 chain, and the center sums
are exact), so labels and centers are compared bit for bit with single-run
contexts, and each run is pinned to the FP64 oracle through teacher-forced
assignments.  Also covered: CUDA-graph replay of the iteration, the
autotuner and its cache, the getters' layout and the unsupported calls."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402

GAP = 1e-6


@pytest.fixture(scope="module")
def small_batch():
    # uneven runs, k not a multiple of 8, one run with k = 1
    cfgs, ks = synth.batch_runs(nruns=7, d=3000, seed=11, n_lo=200, n_hi=2500, k_choices=(3, 10, 25, 60))
    ks = ks.copy()
    ks[3] = 1
    parts = [synth.tfidf(c) for c in cfgs]
    X, run_rows = synth.concat(parts)
    inits = [synth.init_rows(p.n, int(k), 100 + r) for r, (p, k) in enumerate(zip(parts, ks))]
    return parts, X, run_rows, ks, inits


def _batch(X, run_rows, ks, inits, variant, **kw):
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    return skm.Batch(X.n, X.d, dev[0], dev[1], dev[2], run_rows, ks, variant=variant,
                     init_rows=np.concatenate(inits), **kw), dev


def _single(part, k, init, variant, **kw):
    dev = [torch.from_numpy(a).cuda() for a in (part.row_ptr, part.col, part.val)]
    return skm.KMeans(part.n, part.d, dev[0], dev[1], dev[2], int(k), variant=variant, init_rows=init, **kw), dev


BATCH_VARIANTS = ["standard", "hamerly", "simp_hamerly", "elkan", "simp_elkan", "yinyang"]


@pytest.mark.parametrize("variant", BATCH_VARIANTS)
def test_batch_equals_single_runs(small_batch, variant):
    parts, X, run_rows, ks, inits = small_batch
    b, keep = _batch(X, run_rows, ks, inits, variant)
    singles = [_single(p, k, ini, variant) for p, k, ini in zip(parts, ks, inits)]
    for it in range(12):
        ch = b.assign()
        chs = [s.assign() for s, _ in singles]
        assert ch == sum(chs)
        labs = b.run_labels()
        for r, (s, _) in enumerate(singles):
            np.testing.assert_array_equal(labs[r], s.labels(), err_msg=f"run {r} iteration {it}")
            assert labs[r].min() >= 0 and labs[r].max() < ks[r]
        if ch == 0:
            break
        J = b.update_centers()
        Js = [s.update_centers() for s, _ in singles]
        assert abs(J - sum(Js)) <= 1e-9 * abs(J)
        C = b.run_centers()
        for r, (s, _) in enumerate(singles):
            np.testing.assert_array_equal(C[r], s.centers(), err_msg=f"run {r} iteration {it}")
    for s, _ in singles:
        s.close()
    b.close()


@pytest.mark.parametrize("variant", ["simp_elkan", "elkan", "hamerly", "yinyang"])
def test_batch_runs_match_oracle(small_batch, variant):
    """Teacher-forced: every run's assignment from the batch's centers equals
    the FP64 oracle's (up to near-ties), and its center update matches."""
    parts, X, run_rows, ks, inits = small_batch
    b, keep = _batch(X, run_rows, ks, inits, variant)
    data = [oracle.Data.from_csr(p) for p in parts]
    ris = [oracle.rinv(dd) for dd in data]
    prev = [np.full(p.n, -1, np.int32) for p in parts]
    for it in range(6):
        Cs = b.run_centers()
        b.assign()
        labs = b.run_labels()
        for r in range(len(parts)):
            want, _, _, _, gap = oracle.assign(data[r], ris[r], Cs[r].astype(np.float64), prev[r])
            bad = np.flatnonzero((want != labs[r]) & (gap >= GAP))
            assert bad.size == 0, f"run {r}: {bad.size} label mismatches"
        b.update_centers()
        C2 = b.run_centers()
        for r in range(len(parts)):
            Co, _, _ = oracle.update(data[r], ris[r], labs[r], Cs[r].astype(np.float64))
            assert np.max(np.abs(C2[r] - Co)) < 1e-5
            prev[r] = labs[r].copy()
    b.close()


def test_yinyang_batch_large_runs():
    """Yin-Yang in a batch with runs of up to 512 centers (all four 128-center
    slices of the row kernel, a ragged last group of 8): every run follows its
    single-run trajectory bit for bit, labels and centers."""
    cfgs, _ = synth.batch_runs(nruns=4, d=4000, seed=23, n_lo=1500, n_hi=4000, k_choices=(3,))
    ks = np.array([512, 129, 300, 77], np.int32)
    parts = [synth.tfidf(c) for c in cfgs]
    X, run_rows = synth.concat(parts)
    inits = [synth.init_rows(p.n, int(k), 200 + r) for r, (p, k) in enumerate(zip(parts, ks))]
    b, keep = _batch(X, run_rows, ks, inits, "yinyang")
    singles = [_single(p, k, ini, "yinyang") for p, k, ini in zip(parts, ks, inits)]
    for it in range(15):
        ch = b.assign()
        assert ch == sum(s.assign() for s, _ in singles)
        labs = b.run_labels()
        for r, (s, _) in enumerate(singles):
            np.testing.assert_array_equal(labs[r], s.labels(), err_msg=f"run {r} iteration {it}")
        if ch == 0:
            break
        b.update_centers()
        for s, _ in singles:
            s.update_centers()
        C = b.run_centers()
        for r, (s, _) in enumerate(singles):
            np.testing.assert_array_equal(C[r], s.centers(), err_msg=f"run {r} iteration {it}")
    # and the same run as the standard algorithm's
    st, k2 = _batch(X, run_rows, ks, inits, "standard")
    yy, k3 = _batch(X, run_rows, ks, inits, "yinyang")
    assert yy.run(25) == st.run(25)
    np.testing.assert_array_equal(yy.labels(), st.labels())
    for h in [b, st, yy] + [s for s, _ in singles]:
        h.close()


@pytest.mark.parametrize("variant", BATCH_VARIANTS)
def test_graph_replay_equals_eager(small_batch, variant):
    parts, X, run_rows, ks, inits = small_batch
    eager, k1 = _batch(X, run_rows, ks, inits, variant)
    it_e, J_e = eager.run(40)
    for check in (1, 3, 8):
        g, k2 = _batch(X, run_rows, ks, inits, variant, graph=True, graph_check=check)
        n0 = skm.kernel_launches()
        it_g, J_g = g.run(40)
        assert skm.kernel_launches() > n0
        assert it_g == it_e and J_g == J_e
        np.testing.assert_array_equal(g.labels(), eager.labels())
        np.testing.assert_array_equal(g.centers(), eager.centers())
        assert g.stats().iterations == it_e
        g.close()
    eager.close()


def test_graph_replay_single_run():
    X = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=6000, d=4000, seed=21))
    init = synth.init_rows(X.n, 40, 21)
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    out = {}
    for variant in ("standard", "elkan", "simp_elkan", "hamerly", "yinyang"):
        for graph in (False, True):
            km = skm.KMeans(X.n, X.d, *dev, 40, variant=variant, init_rows=init, graph=graph)
            out[(variant, graph)] = (km.run(60), km.labels())
            km.close()
    ref = out[("standard", False)]
    for key, (res, lab) in out.items():
        assert res == ref[0], key
        np.testing.assert_array_equal(lab, ref[1])


def test_autotune_and_cache(small_batch, tmp_path):
    """The tuner's choice changes speed only: runs after tuning (by timing,
    then from the cache file) give the untuned run's result."""
    parts, X, run_rows, ks, inits = small_batch
    ref, k0 = _batch(X, run_rows, ks, inits, "simp_elkan")
    want = ref.run(30)
    cache = tmp_path / "tune.txt"
    b, k1 = _batch(X, run_rows, ks, inits, "simp_elkan")
    assert b.autotune(cache, iters=2) is False
    assert cache.exists() and len(cache.read_text().splitlines()) == 1
    assert b.run(30) == want
    np.testing.assert_array_equal(b.labels(), ref.labels())
    c2, k2 = _batch(X, run_rows, ks, inits, "simp_elkan")
    assert c2.autotune(cache, iters=2) is True
    assert c2.run(30) == want
    np.testing.assert_array_equal(c2.labels(), ref.labels())
    for h in (ref, b, c2):
        h.close()


def test_batch_rejections(small_batch):
    parts, X, run_rows, ks, inits = small_batch
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    big = ks.copy()
    r = int(np.argmax([p.n for p in parts]))
    big[r] = 513  # Yin-Yang's group bounds come from one pass over at most 512 centers
    assert parts[r].n >= 513
    with pytest.raises(skm.SkmError):
        skm.Batch(X.n, X.d, *dev, run_rows, big, variant="yinyang")
    bad = ks.copy()
    bad[0] = parts[0].n + 1
    with pytest.raises(skm.SkmError):
        skm.Batch(X.n, X.d, *dev, run_rows, bad)
    rr = run_rows.copy()
    rr[-1] -= 1
    with pytest.raises(skm.SkmError):
        skm.Batch(X.n, X.d, *dev, rr, ks)
    b = skm.Batch(X.n, X.d, *dev, run_rows, ks, variant="simp_elkan", seed=3)
    b.assign()
    with pytest.raises(skm.SkmError):
        b.set_centers(np.zeros((int(ks.sum()), X.d), np.float32))
    with pytest.raises(skm.SkmError):
        b.bounds()
    lab = b.run_labels()
    assert all(l.min() >= 0 and l.max() < k for l, k in zip(lab, ks))
    b.close()


@pytest.mark.parametrize("variant", ["elkan", "hamerly"])
def test_batch_full_variants_prune_with_center_bounds(small_batch, variant):
    """The full variants' per-run center-center bounds do prune: over a whole
    run the batch computes no more exact similarities than its simplified
    variant (same labels), and about as many as the runs alone (their Gram
    sums the same products in other chunks, so the bounds may differ in the
    last bits and prune a few pairs differently)."""
    parts, X, run_rows, ks, inits = small_batch
    simp = "simp_" + variant
    sims = {}
    for v in (variant, simp):
        b, keep = _batch(X, run_rows, ks, inits, v)
        it, _ = b.run(40)
        sims[v] = (it, b.stats().total_sims, b.labels())
        b.close()
    assert sims[variant][0] == sims[simp][0]
    np.testing.assert_array_equal(sims[variant][2], sims[simp][2])
    assert sims[variant][1] <= sims[simp][1]
    single = 0
    for p, k, ini in zip(parts, ks, inits):
        s, keep = _single(p, k, ini, variant)
        s.run(40)
        single += s.stats().total_sims
        s.close()
    assert abs(sims[variant][1] - single) <= 0.02 * single
