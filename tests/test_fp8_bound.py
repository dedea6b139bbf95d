"""The FP8-E4M3 precision form's per-row error bound, checked on the CPU with
E4M3 rounding emulated bit for bit (pinned against PyTorch's conversion).

The library scales each unit row y_i (FP32) by the power of two 2^e_i with
e_i = 7 - floor(log2 max|y_i|), so the largest scaled entry lies in
[128, 256) and none saturates, and every center by 2^8.  With
xq_i = e4m3(2^e_i y_i) 2^-e_i and cq_j = e4m3(2^8 c_j) 2^-8, the same
Cauchy-Schwarz split as the BF16 form gives

    |<xq, cq> - <x, c>| <= |xq - x| (|c| + |cq - c|) + |cq - c|,

and the FP32 accumulation term uses the factor 1.25 >= (1 + ex)(1 + 6u + E_c).
The tests below pin each of those facts, and constructed pairs reach each
term of the bound."""
import numpy as np
import pytest

import synth

U = 2.0 ** -24


def e4m3(y):
    """Nearest E4M3 value (ties to even; 3 fraction bits, exponents down to -6
    with subnormal spacing 2^-9 below, saturating at 448), as FP64."""
    y = np.asarray(y, dtype=np.float64)
    ay = np.abs(y)
    e = np.maximum(np.floor(np.log2(np.where(ay > 0, ay, 1.0))), -6.0)
    q = 2.0 ** (e - 3)
    return np.clip(np.round(y / q) * q, -448.0, 448.0)


def unit32(M):
    """Rows scaled to unit norm the way the library does it: FP64 norm,
    reciprocal rounded to FP32, product rounded to FP32."""
    M = np.asarray(M, dtype=np.float32)
    ss = np.einsum("ij,ij->i", M.astype(np.float64), M.astype(np.float64))
    rinv = (1.0 / np.sqrt(ss)).astype(np.float32)
    return (M * rinv[:, None]).astype(np.float32)


def row_exponents(Y32):
    m = np.abs(Y32.astype(np.float64)).max(axis=1)
    return 7 - np.floor(np.log2(m)).astype(np.int64)


def quant_rows(Y32):
    e = row_exponents(Y32)
    s = np.ldexp(1.0, e)[:, None]
    return e4m3(Y32.astype(np.float64) * s) / s, e


def quant_centers(C32):
    return e4m3(C32.astype(np.float64) * 256.0) / 256.0


def bound_terms(Y32, C32):
    Xh = Y32.astype(np.float64)
    Xh /= np.linalg.norm(Xh, axis=1, keepdims=True)  # the exact unit rows (FP64)
    Xq, _ = quant_rows(Y32)
    Cq = quant_centers(C32)
    C = C32.astype(np.float64)
    ex = np.linalg.norm(Xq - Xh, axis=1)
    ec = np.linalg.norm(Cq - C, axis=1)
    err = np.abs(Xq @ Cq.T - Xh @ C.T)
    return ex, ec, err


def eps_rows(ex, ec):
    Ec = ec.max()
    return ex * (1.0 + 6.0 * U + Ec) + Ec


def test_e4m3_emulation_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this PyTorch")
    rng = np.random.default_rng(21)
    a = np.concatenate([rng.uniform(-256, 256, 4000), rng.standard_normal(4000) * 2.0 ** -8,
                        (1.0 + (np.arange(8) + 0.5) / 8.0) * 2.0 ** 5,      # normal midpoints
                        (np.arange(1, 8) + 0.5) * 2.0 ** -9]).astype(np.float32)  # subnormal midpoints
    want = torch.from_numpy(a).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(e4m3(a), want)


def test_scales_keep_every_entry_in_range():
    """The largest scaled entry of each row lies in [128, 256) and centers
    scaled by 2^8 stay at or below 256 (1 + 6u rounds to 256 exactly in E4M3's
    grid), so neither saturates at 448."""
    Y = unit32(synth.vmf(2000, 384, 30, 40.0, seed=4))
    e = row_exponents(Y)
    top = np.abs(Y.astype(np.float64)).max(axis=1) * np.ldexp(1.0, e)
    assert np.all((top >= 128.0) & (top < 256.0))
    assert e4m3(256.0 * (1.0 + 6.0 * U)) == 256.0


def test_rounding_error_is_exact_in_fp32():
    """y - e4m3(2^e y) 2^-e, computed in FP32, equals the FP64 difference: the
    library sums the squares of exact FP32 differences."""
    Y = unit32(synth.vmf(500, 384, 10, 40.0, seed=6))
    Xq, _ = quant_rows(Y)
    d32 = (Y - Xq.astype(np.float32)).astype(np.float32)
    np.testing.assert_array_equal(d32.astype(np.float64), Y.astype(np.float64) - Xq)


def test_accumulation_factor_covers_the_operand_norms():
    """(1 + ex_i)(1 + 6u + E_c) <= 1.25: an E4M3 rounding of a normal value errs
    by at most 2^-4 of it, so ex_i, E_c stay near 2^-4 at most."""
    Y = unit32(synth.vmf(3000, 384, 50, 40.0, seed=1))
    C = unit32(Y[synth.init_rows(len(Y), 200, 1)] + 0.01)
    ex, ec, _ = bound_terms(Y, C)
    assert ex.max() <= 2.0 ** -4 + 1e-6 and ec.max() <= 2.0 ** -4 + 1e-6
    assert np.all((1 + ex) * (1 + 6 * U + ec.max()) <= 1.25)


@pytest.mark.parametrize("seed", [1, 2])
def test_bound_holds_on_embedding_rows(seed):
    Y = unit32(synth.vmf(3000, 384, 50, 40.0, seed=seed))
    C = unit32(Y[synth.init_rows(len(Y), 200, seed)] + 0.01)
    ex, ec, err = bound_terms(Y, C)
    eps = eps_rows(ex, ec)
    assert np.all(err <= eps[:, None])
    # the bound is about 16x the BF16 one on the same rows (4 vs 8 significant bits)
    assert 0.01 < eps.mean() < 0.08


def test_bound_holds_at_rounding_midpoints():
    """Entries halfway between E4M3 neighbours after scaling (the largest
    relative rounding error) in both the rows and the centers."""
    rng = np.random.default_rng(9)
    d = 128
    mant = rng.integers(0, 8, size=(64, d))
    sign = rng.choice([-1.0, 1.0], size=(64, d))
    expo = rng.integers(-6, 0, size=(64, d))
    M = sign * (1.0 + (mant + 0.5) / 8.0) * 2.0 ** expo
    Y = unit32(M[:32])
    C = unit32(M[32:])
    ex, ec, err = bound_terms(Y, C)
    assert np.all(err <= eps_rows(ex, ec)[:, None])


def test_row_term_is_reached():
    """Centers exactly representable (entries +-1/8 in d = 64, scaled by 2^8
    they are 32) along the signs of each row's rounding error: the center term
    is 0 and the error is a large part of |xq - x|."""
    Y = unit32(synth.vmf(40, 64, 5, 20.0, seed=7))
    Xh = Y.astype(np.float64) / np.linalg.norm(Y.astype(np.float64), axis=1, keepdims=True)
    Xq, _ = quant_rows(Y)
    C = (np.where(Xq - Xh >= 0, 1.0, -1.0) / 8.0).astype(np.float32)
    ex, ec, err = bound_terms(Y, C)
    assert np.all(ec == 0)
    assert np.all(err <= eps_rows(ex, ec)[:, None])
    assert np.all(np.diag(err) >= 0.5 * ex)  # a bound without the row term would fail here


def test_center_term_is_reached():
    """Rows exactly representable (entries +-1/8 in d = 64: max 1/8 scales by
    2^10 to 128) along the signs of each center's rounding error: the row term
    is 0 and the error is a large part of |cq - c|."""
    C = unit32(synth.vmf(40, 64, 5, 20.0, seed=8))
    Y = (np.where(quant_centers(C) - C.astype(np.float64) >= 0, 1.0, -1.0) / 8.0).astype(np.float32)
    ex, ec, err = bound_terms(Y, C)
    assert np.all(ex == 0)
    assert np.all(err <= eps_rows(ex, ec)[:, None])
    assert np.all(np.diag(err) >= 0.5 * ec)  # a bound without the center term would fail here
