"""Why the precision form has no FP8-E4M3 bulk: on the embedding recipe the
proven error bound of an E4M3 similarity (per-row scale, the same per-row
Cauchy-Schwarz bound as the BF16 form) leaves almost every row ambiguous,
so the FP32 recheck would redo most of the work the FP8 rate saves.  FP64
on the CPU, with E4M3 and BF16 rounding emulated (the E4M3 rounding pinned
against PyTorch's conversion)."""
import numpy as np
import pytest

import synth


def round_to(y, mbits, emin, vmax):
    """Nearest (ties to even) value with mbits fraction bits, exponents down
    to emin (subnormal spacing below), saturated at vmax."""
    y = np.asarray(y, dtype=np.float64)
    ay = np.abs(y)
    e = np.maximum(np.floor(np.log2(np.where(ay > 0, ay, 1.0))), emin)
    q = 2.0 ** (e - mbits)
    return np.clip(np.round(y / q) * q, -vmax, vmax)


def e4m3(y):
    return round_to(y, 3, -6, 448.0)


def bf16(y):
    return round_to(y, 7, -126, 3.38e38)


def e4m3_rows(M):
    """Per-row scale to the E4M3 range, round, scale back."""
    s = 448.0 / np.abs(M).max(axis=1, keepdims=True)
    return e4m3(M * s) / s


def test_rounding_emulation_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this PyTorch")
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.uniform(-448, 448, 2000), rng.standard_normal(2000) * 2.0 ** -7,
                        (1.0 + (np.arange(8) + 0.5) / 8.0) * 2.0 ** 3,  # midpoints
                        (np.arange(1, 8) + 0.5) * 2.0 ** -9]).astype(np.float32)  # subnormal midpoints
    want = torch.from_numpy(a).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(e4m3(a.astype(np.float64)), want)
    b = (rng.standard_normal(4000) * 10.0 ** rng.integers(-8, 8, 4000)).astype(np.float32)
    want = torch.from_numpy(b).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(bf16(b.astype(np.float64)), want)


def _certain_fraction(X, C, F, quant):
    Xq, Cq = quant(X), quant(C)
    ex = np.linalg.norm(Xq - X, axis=1)
    Ec = np.linalg.norm(Cq - C, axis=1).max()
    eps = ex * (1.0 + Ec) + Ec  # |c| = 1 in FP64; products summed exactly enough in FP64
    S = Xq @ Cq.T
    assert np.all(np.abs(S - F) <= eps[:, None] + 1e-12)  # the bound holds
    v1 = S.max(axis=1)
    cands = (S + eps[:, None] >= (v1 - eps)[:, None]).sum(axis=1)
    return np.mean(cands == 1), cands.mean(), eps.mean()


def test_fp8_bound_leaves_most_rows_ambiguous():
    """vMF(kappa = 40) rows in d = 384, ~200 rows per cluster after five
    Lloyd iterations (the regime of the embedding workload)."""
    n, d, k = 20000, 384, 100
    X = synth.vmf(n, d, 100, 40.0, seed=3).astype(np.float64)
    C = X[synth.init_rows(n, k, 3)].copy()
    for _ in range(5):
        a = np.argmax(X @ C.T, axis=1)
        S = np.zeros((k, d))
        np.add.at(S, a, X)
        nrm = np.linalg.norm(S, axis=1)
        C[nrm > 0] = S[nrm > 0] / nrm[nrm > 0, None]
    F = X @ C.T
    bf_certain, bf_cands, bf_eps = _certain_fraction(X, C, F, bf16)
    f8_certain, f8_cands, f8_eps = _certain_fraction(X, C, F, e4m3_rows)
    assert bf_certain > 0.85 and bf_cands < 1.5, (bf_certain, bf_cands)
    assert f8_certain < 0.1 and f8_cands > 10, (f8_certain, f8_cands)
    assert 10 < f8_eps / bf_eps < 30  # 4 fewer significant bits: ~16x the error
