"""Host-side arithmetic of bench.py's roofline (no GPU): the algorithmic
bytes per launch, the gathered bytes, and the guard that a recorded ncu
traffic figure is only used while its kernel's source is unchanged."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes():
    n, d, k, nnz = 1000, 500, 100, 50_000
    row = 8 + 8 * (nnz / n) + 16
    # the Elkan bound pass reads and writes u(i, j) and touches four per-row words
    assert bench.kernel_bytes("k_elk_bounds", n, n, d, k, nnz, "simp_elkan") == 8 * n * k + 16 * n
    # a whole-row pass reads each row once and the centers once; the bounded
    # variants also write their bounds
    assert bench.kernel_bytes("k_rows_top2", n, n, d, k, nnz, "standard") == int(n * row + 4 * d * k)
    assert bench.kernel_bytes("k_rows_top2(list)", 10, n, d, k, nnz, "simp_elkan") == \
        int(10 * (row + 4 * k + 8 + 4) + 4 * d * k)
    # an incremental center update moves nothing through the full-sum kernel
    assert bench.kernel_bytes("k_center_sum", n, n, d, k, nnz, "standard", full_sum=False) == 0
    assert bench.kernel_bytes("k_unknown", n, n, d, k, nnz, "standard") is None


def test_gathered_bytes_use_the_padded_center_slice():
    n, k, nnz = 1000, 100, 50_000
    assert bench.gather_bytes("k_rows_top2", n, n, k, nnz) == int(n * (nnz / n) * 4 * 104)
    assert bench.gather_bytes("k_elk_bounds", n, n, k, nnz) is None


def test_recorded_traffic_lines_are_well_formed():
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    lines = [ln.split() for ln in open(path).read().splitlines() if ln and not ln.startswith("#")]
    assert lines
    for f in lines:
        assert len(f) == 4 and len(f[2]) == 12 and int(f[3]) > 0
        got = bench.recorded_traffic(f[0], f[1])
        assert got is None or got == int(f[3])


def test_recorded_traffic_is_dropped_when_the_source_changes(monkeypatch):
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    f = next(ln.split() for ln in open(path).read().splitlines() if ln and not ln.startswith("#"))
    monkeypatch.setattr(bench, "source_hash", lambda kernel=None: f[2])
    assert bench.recorded_traffic(f[0], f[1]) == int(f[3])
    assert bench.recorded_traffic(f[0], "another-workload") is None
    monkeypatch.setattr(bench, "source_hash", lambda kernel=None: "0" * 12)
    assert bench.recorded_traffic(f[0], f[1]) is None


@pytest.mark.parametrize("kernel", ["k_rows_top2(list)", "k_bf16_topk"])
def test_hash_covers_the_kernel_file_and_the_shared_header(kernel):
    h = bench.source_hash(kernel)
    assert len(h) == 12 and h != bench.source_hash(None)


def test_launch_traffic_scales_a_per_row_record(monkeypatch):
    """Whole-row launches treat a different number of rows every iteration: a
    per-row DRAM record is scaled by the launch's average rows, a per-launch
    record is used as it is."""
    recs = {("k_rows_top2(list)", "rcv1-like-k100-per-row"): 1468, ("k_elk_bounds", "rcv1-like-k100"): 43620000}
    monkeypatch.setattr(bench, "recorded_traffic", lambda name, wl: recs.get((name, wl)))
    assert bench.launch_traffic("k_rows_top2(list)", 37000.0) == 1468 * 37000
    assert bench.launch_traffic("k_elk_bounds", 1.0) == 43620000
    assert bench.launch_traffic("k_unknown", 10.0) is None
