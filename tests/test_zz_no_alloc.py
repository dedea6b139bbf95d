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
