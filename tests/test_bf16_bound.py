"""The precision form's per-row error bound, checked on the CPU with BF16
rounding emulated bit for bit: for a unit row x and a center c rounded to xb
and cb, <xb, cb> - <x, c> = <xb - x, cb> + <x, cb - c>, so by Cauchy-Schwarz

    |<xb, cb> - <x, c>| <= |xb - x| (|c| + |cb - c|) + |cb - c|

(the GPU adds the FP32 accumulation term and rounds up).  Both terms are
needed: constructed pairs reach each of them."""
import numpy as np
import pytest

import synth

U = 2.0 ** -24


def bf16(a):
    """Round float32 values to BF16 (nearest, ties to even), returned as FP64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unit32(M):
    """Rows scaled to unit norm the way the library does it: FP64 norm,
    reciprocal rounded to FP32, product rounded to FP32."""
    M = np.asarray(M, dtype=np.float32)
    ss = np.einsum("ij,ij->i", M.astype(np.float64), M.astype(np.float64))
    rinv = (1.0 / np.sqrt(ss)).astype(np.float32)
    return (M * rinv[:, None]).astype(np.float32)


def bound_terms(X32, C32):
    Xh = X32.astype(np.float64)
    Xh /= np.linalg.norm(Xh, axis=1, keepdims=True)  # the exact unit rows (FP64)
    Xb, Cb = bf16(X32), bf16(C32)
    C = C32.astype(np.float64)
    ex = np.linalg.norm(Xb - Xh, axis=1)
    ec = np.linalg.norm(Cb - C, axis=1)
    err = np.abs(Xb @ Cb.T - Xh @ C.T)
    return ex, ec, err


def eps_rows(ex, ec):
    Ec = ec.max()
    return ex * (1.0 + 6.0 * U + Ec) + Ec


@pytest.mark.parametrize("seed", [1, 2])
def test_bound_holds_on_embedding_rows(seed):
    X = synth.vmf(3000, 384, 50, 40.0, seed=seed)
    C = unit32(X[synth.init_rows(len(X), 200, seed)] + 0.01)
    ex, ec, err = bound_terms(X, C)
    eps = eps_rows(ex, ec)
    assert np.all(err <= eps[:, None])
    worst = 2.0 ** -7 + 2.0 ** -15
    assert np.all(eps <= worst)
    # with real data the rounding errors are far from their worst case
    assert eps.mean() < 0.6 * worst


def test_bound_holds_at_rounding_midpoints():
    """Entries halfway between BF16 neighbours (the largest relative
    rounding error) in both the rows and the centers."""
    rng = np.random.default_rng(5)
    d = 128
    mant = rng.integers(0, 128, size=(64, d))
    sign = rng.choice([-1.0, 1.0], size=(64, d))
    expo = rng.integers(-8, 0, size=(64, d))
    M = sign * (1.0 + (mant + 0.5) / 128.0) * 2.0 ** expo  # exact midpoints in FP32
    X = unit32(M[:32])
    C = unit32(M[32:])
    ex, ec, err = bound_terms(X, C)
    assert np.all(err <= eps_rows(ex, ec)[:, None])


def test_row_term_is_reached():
    """Centers exactly representable (entries +-1/8 in d = 64, norm 1) along
    the signs of each row's rounding error: the center term is 0 and the
    error is |xb - x|_1 / 8, a large part of |xb - x|."""
    X = synth.vmf(40, 64, 5, 20.0, seed=7)
    Xh = X.astype(np.float64) / np.linalg.norm(X.astype(np.float64), axis=1, keepdims=True)
    C = (np.where(bf16(X) - Xh >= 0, 1.0, -1.0) / 8.0).astype(np.float32)
    ex, ec, err = bound_terms(X, C)
    assert np.all(ec == 0)
    assert np.all(err <= eps_rows(ex, ec)[:, None])
    diag = np.diag(err)
    assert np.all(diag >= 0.5 * ex)  # a bound without the row term would fail here


def test_center_term_is_reached():
    """Rows exactly representable (entries +-1/8 in d = 64) along the signs
    of each center's rounding error: the row term is 0 and the error is
    |cb - c|_1 / 8."""
    C = unit32(synth.vmf(40, 64, 5, 20.0, seed=8))
    X = (np.where(bf16(C) - C.astype(np.float64) >= 0, 1.0, -1.0) / 8.0).astype(np.float32)
    ex, ec, err = bound_terms(X, C)
    assert np.all(ex == 0)
    assert np.all(err <= eps_rows(ex, ec)[:, None])
    diag = np.diag(err)
    assert np.all(diag >= 0.5 * ec)  # a bound without the center term would fail here


def test_bf16_emulation_matches_torch():
    """The bit-level rounding above is the BF16 conversion PyTorch's CPU
    kernels perform (nearest, ties to even), on random values and midpoints."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.standard_normal(4096) * 10.0 ** rng.integers(-6, 6, 4096),
                        (1.0 + (np.arange(256) + 0.5) / 128.0) * 2.0 ** -3]).astype(np.float32)
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(bf16(a), want)


@pytest.mark.parametrize("scale", [1.0, 3.7e-3, 2.9e4])
def test_row_error_split(scale):
    """The row term the library computes: with y = fl32(x * fl32(1/|x|)) (the
    values it rounds to BF16), |bf16(y) - x/|x|| <= |bf16(y) - y| +
    2^-23 (1 + (d + 8) 2^-30), on unit and on scaled rows."""
    d = 384
    X = (synth.vmf(500, d, 20, 40.0, seed=11) * np.float32(scale)).astype(np.float32)
    X64 = X.astype(np.float64)
    nrm = np.sqrt(np.einsum("ij,ij->i", X64, X64))
    ri = (1.0 / nrm).astype(np.float32)
    y = (X * ri[:, None]).astype(np.float32)
    yb = bf16(y)
    lhs = np.linalg.norm(yb - X64 / nrm[:, None], axis=1)
    rhs = np.linalg.norm(yb - y.astype(np.float64), axis=1) + 2.0 ** -23 * (1 + (d + 8) * 2.0 ** -30)
    assert np.all(lhs <= rhs)
    assert np.all(rhs - lhs <= 2.0 ** -22)  # the added term is small against the BF16 error
