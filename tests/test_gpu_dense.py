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
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
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
        for p in ("fp32", "bf16"):
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


def test_bf16_error_bound_holds():
    """|BF16 similarity - exact FP64 similarity| <= eps_b for the reported
    best center of every row (the bound the precision form relies on)."""
    Xs = synth.vmf(4000, 384, 100, 40.0, seed=9)
    init = synth.init_rows(len(Xs), 256, 9)
    km = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 256, variant="standard", init_rows=init, precision="bf16")
    for _ in range(3):
        C = km.centers().astype(np.float64)
        km.assign()
        t2, eps = km.bf16_top2()
        km.update_centers()
    Xn = Xs.astype(np.float64) / np.linalg.norm(Xs.astype(np.float64), axis=1, keepdims=True)
    Cn = C / np.linalg.norm(C, axis=1, keepdims=True)
    j1 = t2[:, 1].view(np.int32) if t2.dtype == np.float32 else t2[:, 1]
    j1 = np.frombuffer(t2[:, 1].tobytes(), dtype=np.int32)
    exact = np.sum(Xn * Cn[j1], axis=1)
    err = np.abs(t2[:, 0].astype(np.float64) - exact)
    assert err.max() <= eps, (err.max(), eps)
    # the top-1 of the BF16 bulk is a true near-maximum
    S = Xn @ Cn.T
    assert np.all(S.max(axis=1) - exact <= 2 * eps)
    km.close()


def test_dense_host_input_and_rejections():
    Xs = synth.vmf(500, 40, 5, 20.0, seed=2)
    init = synth.init_rows(500, 7, 2)
    a = skm.KMeans.dense(Xs, 7, variant="hamerly", init_rows=init)            # host copy
    b = skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 7, variant="hamerly", init_rows=init)
    assert a.run(30) == b.run(30)
    np.testing.assert_array_equal(a.labels(), b.labels())
    with pytest.raises(skm.SkmError):
        skm.KMeans.dense(torch.from_numpy(Xs).cuda(), 7, variant="elkan", init_rows=init)
    odd = synth.vmf(100, 500, 3, 20.0, seed=3)  # d = 500 > 448: no BF16 bulk
    with pytest.raises(skm.SkmError):
        skm.KMeans.dense(torch.from_numpy(odd).cuda(), 3, precision="bf16")
