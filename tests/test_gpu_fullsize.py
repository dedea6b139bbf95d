"""Parity at the workloads' full sizes, in the configurations bench.py times,
on sampled rows the FP64 oracle can afford: teacher-forced assignments (the
oracle assigns the sampled rows from the GPU's centers and previous labels)
must give the GPU's labels except below the 1e-6 similarity gap.  Every
workload runs at its full size, the 8e8-nonzero one included."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402

GAP = 1e-6
NSAMPLE = 2000


def _sample(n, seed=55):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(NSAMPLE, n), replace=False))


def _check_sparse(km, csr, sample, prev, C):
    sub = oracle.Data.from_csr(csr.rows(sample))
    want, _, _, _, gap = oracle.assign(sub, oracle.rinv(sub), C.astype(np.float64), prev[sample])
    lab = km.labels()[sample]
    bad = np.flatnonzero((want != lab) & (gap >= GAP))
    assert bad.size == 0, f"{bad.size} of {len(sample)} sampled labels differ from the oracle"


def _teacher_forced_sparse(km, csr, iters, check_at):
    sample = _sample(csr.n)
    prev = np.full(csr.n, -1, np.int32)
    for t in range(iters):
        C = km.centers() if t in check_at else None
        ch = km.assign()
        if C is not None:
            _check_sparse(km, csr, sample, prev, C)
        prev = km.labels()
        if ch == 0:
            return t + 1
        km.update_centers()
    return iters


def test_rcv1_like_full_size():
    """n = 1e5, d = 5e4, k = 100, simplified Elkan (the bench variant) to
    convergence: the same labels as the standard variant, and sampled parity
    at the first, fifth and last assignment."""
    csr = synth.tfidf(synth.CSR_RCV1_LIKE)
    init = synth.init_rows(csr.n, 100, 7)
    dev = [torch.from_numpy(a).cuda() for a in (csr.row_ptr, csr.col, csr.val)]
    std = skm.KMeans(csr.n, csr.d, *dev, 100, variant="standard", init_rows=init)
    it_s, _ = std.run(100)
    km = skm.KMeans(csr.n, csr.d, *dev, 100, variant="simp_elkan", init_rows=init)
    it = _teacher_forced_sparse(km, csr, 100, {0, 4, it_s - 1})
    assert it == it_s
    np.testing.assert_array_equal(km.labels(), std.labels())
    km.close()
    std.close()


def test_embedding_full_size_bf16():
    """n = 1e6, d = 384, k = 1000 dense, the precision form (BF16 tensor-core
    bulk, FP32 candidate recheck): sampled parity over three assignments."""
    Xs = synth.vmf(1_000_000, 384, 1000, 40.0, seed=3)
    init = synth.init_rows(len(Xs), 1000, 3)
    km = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 1000, variant="standard", init_rows=init, precision="bf16")
    sample = _sample(len(Xs))
    sub = oracle.Data.from_dense(Xs[sample])
    ri = oracle.rinv(sub)
    prev = np.full(NSAMPLE, -1, np.int32)
    for t in range(3):
        C = km.centers()
        km.assign()
        lab = km.labels()[sample]
        want, _, _, _, gap = oracle.assign(sub, ri, C.astype(np.float64), prev)
        bad = np.flatnonzero((want != lab) & (gap >= GAP))
        assert bad.size == 0, f"iteration {t}: {bad.size} sampled labels differ"
        prev = lab
        km.update_centers()
    km.close()


def test_batch_full_size():
    """64 runs (sum n ~ 2.9e6, d = 2e4), simplified Elkan with graph replay
    and autotuned launches, 50 iterations: three runs checked against the
    oracle (teacher-forced at the first assignment, then the final labels
    against a fresh single-run context)."""
    cfgs, ks = synth.batch_runs(64)
    parts = [synth.tfidf(c) for c in cfgs]
    X, run_rows = synth.concat(parts)
    inits = [synth.init_rows(p.n, int(k), 1000 + r) for r, (p, k) in enumerate(zip(parts, ks))]
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    b = skm.Batch(X.n, X.d, *dev, run_rows, ks, variant="simp_elkan", init_rows=np.concatenate(inits))
    C0 = b.run_centers()
    b.assign()
    labs = b.run_labels()
    for r in (0, 31, 63):
        sample = _sample(parts[r].n, seed=r)
        sub = oracle.Data.from_csr(parts[r].rows(sample))
        want, _, _, _, gap = oracle.assign(sub, oracle.rinv(sub), C0[r].astype(np.float64))
        bad = np.flatnonzero((want != labs[r][sample]) & (gap >= GAP))
        assert bad.size == 0, f"run {r}: {bad.size} sampled labels differ"
    g = skm.Batch(X.n, X.d, *dev, run_rows, ks, variant="simp_elkan", init_rows=np.concatenate(inits),
                  graph=True)
    g.autotune(None, iters=2)
    g.run(50)
    final = g.run_labels()
    for r in (0, 31, 63):
        pd = [torch.from_numpy(a).cuda() for a in (parts[r].row_ptr, parts[r].col, parts[r].val)]
        s = skm.KMeans(parts[r].n, parts[r].d, *pd, int(ks[r]), variant="standard", init_rows=inits[r])
        s.run(50)
        np.testing.assert_array_equal(final[r], s.labels())
        s.close()
    b.close()
    g.close()


def test_large_sparse_full_size():
    """n = 4e6 rows, d = 2e5, ~200 nnz/row (8e8 non-zeros), FP16 values,
    k = 1000, 30 iterations: Elkan keeps n * 1000 FP32 bounds (16 GB, 4e9
    elements, past signed 32-bit indexing).  Sampled parity at the first and the last
    assignment; Hamerly and the standard variant reach the same labels after
    the same 30 iterations."""
    csr = synth.tfidf(synth.CSR_LARGE)
    assert csr.nnz > 7.5e8 and csr.n * 1000 > 2 ** 31
    init = synth.init_rows(csr.n, 1000, synth.CSR_LARGE.seed)
    dev = [torch.from_numpy(a).cuda() for a in (csr.row_ptr, csr.col, csr.val)]
    iters = 30
    km = skm.KMeans(csr.n, csr.d, *dev, 1000, variant="elkan", init_rows=init)
    it = _teacher_forced_sparse(km, csr, iters, {0, iters - 1})
    ref = km.labels()
    sims_elkan = km.stats().total_sims
    km.close()
    assert sims_elkan < it * csr.n * 1000
    for variant in ("hamerly", "standard"):
        o = skm.KMeans(csr.n, csr.d, *dev, 1000, variant=variant, init_rows=init)
        it_o, _ = o.run(iters)
        assert it_o == it
        np.testing.assert_array_equal(o.labels(), ref)
        o.close()
