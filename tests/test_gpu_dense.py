"""Dense rows through the C ABI: the plain FP32 GEMM path and the precision
form (BF16 tensor-core bulk + FP32 recheck) against the FP64 oracle, and the
precision form's labels against the FP32 path's (they must be identical)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402

GAP = 1e-6
CTOL = 1e-5


def _teacher_forced_dense(Xs, k, variant, precision, init, iters):
    X = oracle.Data.from_dense(Xs)
    ri = oracle.rinv(X)
    km = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), k, variant=variant, init_rows=init, precision=precision)
    prev = np.full(len(Xs), -1, np.int32)
    seq = []
    for _ in range(iters):
        C = km.centers()
        ch = km.assign()
        lab = km.labels()
        assert ch == int(np.sum(lab != prev))
        want, _, _, _, gap = oracle.assign(X, ri, C.astype(np.float64), prev)
        bad = np.flatnonzero((want != lab) & (gap >= GAP))
        assert bad.size == 0, f"{bad.size} label mismatches"
        seq.append(lab.copy())
        if ch == 0:
            break
        J = km.update_centers()
        Co, _, Jo = oracle.update(X, ri, lab, C.astype(np.float64))
        assert np.max(np.linalg.norm(km.centers() - Co, axis=1)) < CTOL
        assert abs(J - Jo) <= CTOL * abs(Jo)
        prev = lab
    st = km.stats()
    km.close()
    return seq, st


@pytest.fixture(scope="module")
def emb():
    # vMF mixture, ragged sizes: n not a multiple of 128, k not a multiple of 256
    return synth.vmf(3001, 96, 40, 30.0, seed=41)


@pytest.mark.parametrize("variant", ["standard", "hamerly", "simp_hamerly"])
@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_dense_teacher_forced(emb, variant, precision):
    init = synth.init_rows(len(emb), 37, 5)
    _teacher_forced_dense(emb, 37, variant, precision, init, 15)


def test_precision_form_labels_equal_fp32_path():
    """Section 5's labels with the BF16 bulk equal those of the plain FP32 path
    bit for bit, over a whole run, for the standard and Hamerly variants."""
    Xs = synth.vmf(20000, 384, 200, 40.0, seed=3)
    init = synth.init_rows(len(Xs), 300, 3)
    Xd = torch.from_numpy(Xs).cuda()
    seqs = {}
    for v in ("standard", "hamerly"):
        for p in ("fp32", "bf16", "fp8"):
            km = skm.KMeans.dense(Xd, 300, variant=v, init_rows=init, precision=p)
            labs = []
            for _ in range(12):
                ch = km.assign()
                labs.append(km.labels())
                if ch == 0:
                    break
                km.update_centers()
            seqs[(v, p)] = labs
            km.close()
    ref = seqs[("standard", "fp32")]
    for key, labs in seqs.items():
        assert len(labs) == len(ref), key
        for a, b in zip(labs, ref):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("d", [768, 1024])
def test_precision_form_wide_embeddings(d):
    """Embedding widths 768 and 1024 (12 and 16 K blocks of the tensor-core
    loop): the BF16 bulk is teacher-forced against the FP64 oracle step by
    step, and its label sequence equals the FP32 path's."""
    Xs = synth.vmf(3001, d, 40, 80.0, seed=43)
    init = synth.init_rows(len(Xs), 37, 43)
    seq_b, st = _teacher_forced_dense(Xs, 37, "standard", "bf16", init, 8)
    seq_f, _ = _teacher_forced_dense(Xs, 37, "standard", "fp32", init, 8)
    assert len(seq_b) == len(seq_f)
    for a, b in zip(seq_b, seq_f):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("d", [384, 1024])
def test_bf16_error_bound_holds(d):
    """Every BF16 similarity of the candidate list is within its row's bound
    eps_i of the exact FP64 one, the list is descending with distinct centers,
    and every center outside it is at most v8 + eps_i exactly (the facts the
    precision form relies on).  eps_i never exceeds the worst-case constant
    2^-7 + 2^-15 + (d + 16) 2^-23 and, from the actual rounding errors, is
    well below it.  Lists may end in entries with center -1 that carry a
    bound instead of a center; a row whose candidate buffer overflowed is all
    -1 / +inf (it gets a whole-row recheck) and must be rare."""
    Xs = synth.vmf(4000, d, 100, 40.0 * d / 384, seed=9)
    init = synth.init_rows(len(Xs), 256, 9)
    km = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 256, variant="standard", init_rows=init, precision="bf16")
    Xn = Xs.astype(np.float64) / np.linalg.norm(Xs.astype(np.float64), axis=1, keepdims=True)
    for it in range(4):
        C = km.centers().astype(np.float64)
        km.assign()
        tv, ti, eps = km.bf16_topk()
        km.update_centers()
        eps = eps.astype(np.float64)
        worst = 2.0 ** -7 + 2.0 ** -15 + (Xs.shape[1] + 16) * 2.0 ** -23
        assert np.all(eps > 0) and np.all(eps <= worst), (eps.min(), eps.max(), worst)
        assert eps.mean() < 0.75 * worst, (eps.mean(), worst)
        Cn = C / np.linalg.norm(C, axis=1, keepdims=True)
        S = Xn @ Cn.T
        over = ti[:, 0] < 0
        assert np.all(np.isposinf(tv[over])) and np.all(ti[over] == -1)
        assert over.mean() < 0.02, over.mean()
        tv, ti, S, eps = tv[~over], ti[~over], S[~over], eps[~over]
        real = ti >= 0
        # real entries first, then bound entries
        assert np.all(np.diff(real.astype(np.int8), axis=1) <= 0)
        assert np.all(np.diff(tv, axis=1) <= 0)
        for r in range(len(tv)):
            js = ti[r][real[r]]
            assert len(set(js.tolist())) == len(js)
        exact = np.take_along_axis(S, np.where(real, ti, 0).astype(np.int64), axis=1)
        err = np.where(real, np.abs(tv.astype(np.float64) - exact), 0.0)
        assert np.all(err <= eps[:, None]), (err.max(), eps.min())
        outside = S.copy()
        for r in range(len(tv)):
            outside[r, ti[r][real[r]]] = -np.inf
        assert np.all(outside.max(axis=1) <= tv[:, 7].astype(np.float64) + eps)
    km.close()


def _label_runs(Xs, k, init, iters, keys):
    Xd = torch.from_numpy(Xs).cuda()
    seqs, stats = {}, {}
    for v, p in keys:
        km = skm.KMeans.dense(Xd, k, variant=v, init_rows=init, precision=p)
        labs, sts = [], []
        for _ in range(iters):
            ch = km.assign()
            labs.append(km.labels())
            sts.append(km.stats())
            if ch == 0:
                break
            km.update_centers()
        if p != "fp32":
            stats[(v, p)] = (sts, km.bf16_topk())
        seqs[(v, p)] = labs
        km.close()
    return seqs, stats


KEYS = [("standard", "fp32"), ("standard", "bf16"), ("hamerly", "bf16"), ("simp_hamerly", "bf16"),
        ("standard", "fp8"), ("hamerly", "fp8")]


@pytest.mark.parametrize("k", [5, 8, 9])
def test_bf16_candidate_recheck_small_k(k):
    """k < 8 (the list ends in center -1), k = 8 and k = 9: the candidate
    recheck gives the FP32 path's labels over a whole run."""
    Xs = synth.vmf(3000, 64, 6, 8.0, seed=4)
    init = synth.init_rows(len(Xs), k, 4)
    seqs, stats = _label_runs(Xs, k, init, 10, KEYS)
    ref = seqs[("standard", "fp32")]
    for key, labs in seqs.items():
        assert len(labs) == len(ref), key
        for a, b in zip(labs, ref):
            np.testing.assert_array_equal(a, b)
    _, (tv, ti, _) = stats[("standard", "bf16")]
    if k < 8:
        assert np.all(ti[:, k:] == -1)


def test_bf16_candidate_window_overflow():
    """One tight cluster and 32 centers inside it: the similarities of a row
    to many centers lie within the error window, all eight BF16 candidates
    qualify and the row falls back to a whole-row FP32 recheck; labels still
    equal the FP32 path's."""
    Xs = synth.vmf(2000, 64, 1, 3000.0, seed=6)
    init = synth.init_rows(len(Xs), 32, 6)
    seqs, stats = _label_runs(Xs, 32, init, 6, KEYS)
    ref = seqs[("standard", "fp32")]
    for key, labs in seqs.items():
        assert len(labs) == len(ref), key
        for a, b in zip(labs, ref):
            np.testing.assert_array_equal(a, b)
    sts, _ = stats[("standard", "bf16")]
    assert sts[0].last_cand_rechecks > 0
    assert max(s.last_rechecks for s in sts) > 0


def test_dense_host_input_and_rejections():
    Xs = synth.vmf(500, 40, 5, 20.0, seed=2)
    init = synth.init_rows(500, 7, 2)
    a = skm.KMeans.dense(Xs, 7, variant="hamerly", init_rows=init)            # host copy
    b = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 7, variant="hamerly", init_rows=init)
    assert a.run(30) == b.run(30)
    np.testing.assert_array_equal(a.labels(), b.labels())
    with pytest.raises(skm.SkmError):
        skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 7, variant="elkan", init_rows=init)
    odd = synth.vmf(100, 500, 3, 20.0, seed=3)  # d = 500 is not a multiple of 8: no BF16 bulk
    with pytest.raises(skm.SkmError):
        skm.KMeans.dense(torch.from_numpy(odd).cuda(), 3, precision="bf16")


def _e4m3(y):
    """Nearest E4M3 value (ties to even), as FP64 (the emulation pinned
    against PyTorch in test_fp8_bound.py)."""
    y = np.asarray(y, dtype=np.float64)
    ay = np.abs(y)
    e = np.maximum(np.floor(np.log2(np.where(ay > 0, ay, 1.0))), -6.0)
    q = 2.0 ** (e - 3)
    return np.clip(np.round(y / q) * q, -448.0, 448.0)


def _unit32(M):
    M = np.asarray(M, dtype=np.float32)
    ss = np.einsum("ij,ij->i", M.astype(np.float64), M.astype(np.float64))
    return (M * (1.0 / np.sqrt(ss)).astype(np.float32)[:, None]).astype(np.float32)


def test_fp8_error_bound_holds():
    """FP8 form: every listed E4M3 similarity is within its row's bound eps_i
    of the exact FP64 one, every center left out is at most v8 + eps_i, and
    eps_i lies near the E4M3 rounding scale (about 16x the BF16 bound)."""
    Xs = synth.vmf(4000, 384, 100, 40.0, seed=9)
    init = synth.init_rows(len(Xs), 256, 9)
    km = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 256, variant="standard", init_rows=init, precision="fp8")
    Xn = Xs.astype(np.float64) / np.linalg.norm(Xs.astype(np.float64), axis=1, keepdims=True)
    for it in range(3):
        C = km.centers().astype(np.float64)
        km.assign()
        tv, ti, eps = km.bf16_topk()
        km.update_centers()
        eps = eps.astype(np.float64)
        assert np.all(eps > 0.005) and np.all(eps < 0.15), (eps.min(), eps.max())
        S = Xn @ (C / np.linalg.norm(C, axis=1, keepdims=True)).T
        over = ti[:, 0] < 0
        tv, ti, S, eps = tv[~over], ti[~over], S[~over], eps[~over]
        real = ti >= 0
        exact = np.take_along_axis(S, np.where(real, ti, 0).astype(np.int64), axis=1)
        err = np.where(real, np.abs(tv.astype(np.float64) - exact), 0.0)
        assert np.all(err <= eps[:, None]), (err.max(), eps.min())
        outside = S.copy()
        for r in range(len(tv)):
            outside[r, ti[r][real[r]]] = -np.inf
        assert np.all(outside.max(axis=1) <= tv[:, 7].astype(np.float64) + eps)
    km.close()


def test_fp8_tensor_core_sums_the_exact_products():
    """The FP8 similarities the tensor cores return are the FP32-accumulated
    sums of the exact E4M3 products, unscaled exactly: against the sums of the
    same quantised operands in FP64 they differ by at most (d + 16) 2^-23
    times the sum of |products| (reading TC of the bound).  The rows are built
    so that large partial sums cancel: rows 2.. are (+a..., -a..., small
    entries) and the two centers (rows 0 and 1) are (a..., a..., small
    entries), so each of those similarities is a small sum left after
    products of 64 x 64 entries cancel; an accumulator that kept fewer bits
    than FP32 would lose the small products and fail here."""
    d, n = 256, 64
    rng = np.random.default_rng(17)
    M = np.zeros((n, d), np.float64)
    M[:, :64] = 1.0
    M[:, 64:128] = -1.0
    M[:2, 64:128] = 1.0
    M[:, 128:] = rng.uniform(-2.0 ** -5, 2.0 ** -5, size=(n, 128))
    Y = _unit32(M)
    km = skm.KMeans.dense(torch.from_numpy(Y).cuda(), 2, variant="standard", init_rows=np.array([0, 1]),
                          precision="fp8")
    C = km.centers()  # unit rows 0 and 1 (FP32)
    km.assign()
    tv, ti, _ = km.bf16_topk()
    km.close()
    e = 7 - np.floor(np.log2(np.abs(Y.astype(np.float64)).max(axis=1))).astype(np.int64)
    s = np.ldexp(1.0, e)[:, None]
    Xq = _e4m3(Y.astype(np.float64) * s)                   # scaled row operands
    Cq = _e4m3(C.astype(np.float64) * 256.0)              # scaled center operands
    P = Xq @ Cq.T                                           # exact sums of the products
    A = np.abs(Xq) @ np.abs(Cq).T
    got = np.full((n, 2), np.nan)
    for r in range(n):
        for q in range(8):
            if ti[r, q] >= 0:
                got[r, ti[r, q]] = tv[r, q] * s[r, 0] * 256.0  # back to the accumulator's units
    have = ~np.isnan(got)
    assert have[2:].all()  # both centers are candidates of every test row
    assert np.all(np.abs(P[2:]) < 0.01 * A[2:])  # the large products do cancel
    tol = (d + 16) * 2.0 ** -23 * A
    assert np.all(np.abs(got[have] - P[have]) <= tol[have]), np.max(np.abs(got - P)[have] / A[have])
