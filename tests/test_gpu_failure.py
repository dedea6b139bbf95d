"""Failure detection without a GPU fault: a device wait that nothing
completes gives up after its limit and reports SKM_ETIMEOUT through the
status the host reads, and the GPU context stays usable afterwards (a
clustering run on the same process gives the oracle's labels)."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402


@pytest.mark.parametrize("limit_ms", [1, 20])
def test_wait_times_out_and_context_survives(limit_ms):
    t0 = time.perf_counter()
    rc = skm.selftest_wait(limit_ms * 1_000_000)
    dt = time.perf_counter() - t0
    assert rc == skm.ETIMEOUT
    assert dt >= limit_ms / 1e3 * 0.5  # it did wait, then gave up
    assert dt < 5.0
    # the context is still usable: a small run matches the oracle
    X = synth.tfidf(synth.scaled(synth.CSR_TINY, n=500))
    init = synth.init_rows(X.n, 7, 3)
    dev = [torch.from_numpy(a).cuda() for a in (X.row_ptr, X.col, X.val)]
    km = skm.KMeans(X.n, X.d, *dev, 7, variant="elkan", init_rows=init)
    C = km.centers()
    km.assign()
    d = oracle.Data.from_csr(X)
    want, _, _, _, gap = oracle.assign(d, oracle.rinv(d), C.astype(np.float64))
    assert np.all((want == km.labels()) | (gap < 1e-6))
    km.close()


def test_wait_selftest_rejects_bad_limits():
    assert skm.selftest_wait(0) == skm.EINVAL
    assert skm.selftest_wait(3_000_000_000) == skm.EINVAL

