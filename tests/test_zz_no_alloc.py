"""skm_assign_noalloc: the standard assignment step for callers that cannot
allocate device memory (code inside another framework's memory pool, under a
fixed memory budget, or a service that must not allocate after start-up).

Its scratch is a static device array owned by the library, so the test checks
that two calls in a row -- the second one reusing the array the first one
filled -- give exactly the labels of the regular entry point (skm_assign of a
standard context holding the same centers and current labels)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402


def test_noalloc_assign_matches_regular_entry_point_twice():
    csr = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=6000, d=8000, seed=31))
    k = 40
    init = synth.init_rows(csr.n, k, 31)
    rp, col, val = (torch.from_numpy(a).cuda() for a in (csr.row_ptr, csr.col, csr.val))
    ref = skm.KMeans(csr.n, csr.d, rp, col, val, k, variant="standard", init_rows=init)
    # call 1: the initial centers, no current labels
    C1 = ref.centers()
    want1_changed = ref.assign()
    want1 = ref.labels()
    # call 2: the centers after one update, with call 1's labels as current
    ref.update_centers()
    C2 = ref.centers()
    ref.set_centers(C2)
    ref.set_labels(want1)
    want2_changed = ref.assign()
    want2 = ref.labels()
    ref.close()

    labels = torch.full((csr.n,), -1, dtype=torch.int32, device="cuda")
    got1_changed = skm.assign_noalloc(csr.n, csr.d, rp, col, val, k, torch.from_numpy(C1).cuda(), labels)
    np.testing.assert_array_equal(labels.cpu().numpy(), want1)
    assert got1_changed == want1_changed == csr.n
    got2_changed = skm.assign_noalloc(csr.n, csr.d, rp, col, val, k, torch.from_numpy(C2).cuda(), labels)
    np.testing.assert_array_equal(labels.cpu().numpy(), want2)
    assert got2_changed == want2_changed
    assert 0 < got2_changed < csr.n


def test_noalloc_rejects_oversized_problem():
    csr = synth.csr_from_dense(np.eye(8, dtype=np.float32))
    rp, col, val = (torch.from_numpy(a).cuda() for a in (csr.row_ptr, csr.col, csr.val))
    labels = torch.full((8,), -1, dtype=torch.int32, device="cuda")
    big_d = (1 << 22) // 8 + 1   # d * round_up(k, 8) just above the static limit
    centers = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(skm.SkmError) as e:
        skm.assign_noalloc(8, big_d, rp, col, val, 8, centers, labels)
    assert e.value.code == skm.ETOOBIG


def _with_bad_rows(csr, bad_at):
    """The rows of csr with three malformed rows inserted before the rows
    bad_at[0..2]: an empty row (zero norm), a row with a column index past d,
    and a row holding +inf.  Returns (row_ptr, col, val, positions of the good
    rows, positions of the bad rows)."""
    rows_c, rows_v = [], []
    good_pos, bad_pos = [], []
    kinds = dict(zip(bad_at, ("empty", "column", "inf")))
    for i in range(csr.n):
        if i in kinds:
            bad_pos.append(len(rows_c))
            if kinds[i] == "empty":
                rows_c.append(np.zeros(0, np.int32))
                rows_v.append(np.zeros(0, np.float32))
            elif kinds[i] == "column":
                rows_c.append(np.array([1, 7, csr.d + 5], np.int32))
                rows_v.append(np.array([0.6, 0.6, 0.52915026], np.float32))
            else:
                rows_c.append(np.array([2, 9], np.int32))
                rows_v.append(np.array([np.inf, 0.5], np.float32))
        b, e = csr.row_ptr[i], csr.row_ptr[i + 1]
        good_pos.append(len(rows_c))
        rows_c.append(csr.col[b:e])
        rows_v.append(csr.val[b:e])
    rp = np.zeros(len(rows_c) + 1, np.int64)
    rp[1:] = np.cumsum([len(c) for c in rows_c])
    return rp, np.concatenate(rows_c), np.concatenate(rows_v), np.array(good_pos), np.array(bad_pos)


def test_noalloc_malformed_rows_get_no_label():
    """Rows with a zero norm, an out-of-range column or an infinite value get
    label -1 and make a counting call fail with EINVAL; the other rows keep the
    labels of the regular entry point.  Without a host count the call returns
    OK and the labels are the same.  (The kernel checks a row before it reads
    any center value through the row's column indices.)"""
    csr = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=600, d=3000, seed=37))
    k = 24
    init = synth.init_rows(csr.n, k, 37)
    rp, col, val = (torch.from_numpy(a).cuda() for a in (csr.row_ptr, csr.col, csr.val))
    ref = skm.KMeans(csr.n, csr.d, rp, col, val, k, variant="standard", init_rows=init)
    C = ref.centers()
    ref.assign()
    want = ref.labels()
    ref.close()

    brp, bcol, bval, good, bad = _with_bad_rows(csr, (5, 300, 599))
    nb = len(brp) - 1
    drp, dcol, dval = (torch.from_numpy(a).cuda() for a in (brp, bcol, bval))
    Cd = torch.from_numpy(C).cuda()
    for count in (True, False):
        labels = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
        if count:
            with pytest.raises(skm.SkmError) as e:
                skm.assign_noalloc(nb, csr.d, drp, dcol, dval, k, Cd, labels, count=True)
            assert e.value.code == skm.EINVAL
        else:
            assert skm.assign_noalloc(nb, csr.d, drp, dcol, dval, k, Cd, labels, count=False) is None
            torch.cuda.synchronize()
        got = labels.cpu().numpy()
        np.testing.assert_array_equal(got[bad], -1)
        np.testing.assert_array_equal(got[good], want)


def test_noalloc_nan_centers_give_no_label():
    """Centers holding NaN leave every similarity NaN: no row gets a label
    (all -1, EINVAL), never an out-of-range one."""
    csr = synth.tfidf(synth.scaled(synth.CSR_RCV1_LIKE, n=200, d=2000, seed=41))
    k = 9
    rp, col, val = (torch.from_numpy(a).cuda() for a in (csr.row_ptr, csr.col, csr.val))
    C = torch.full((k, csr.d), float("nan"), dtype=torch.float32, device="cuda")
    labels = torch.full((csr.n,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(skm.SkmError) as e:
        skm.assign_noalloc(csr.n, csr.d, rp, col, val, k, C, labels)
    assert e.value.code == skm.EINVAL
    np.testing.assert_array_equal(labels.cpu().numpy(), -1)
