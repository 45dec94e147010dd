"""Gram products G = A^T B through lrfsi_gram on both paths: the FP64 FMA
kernels and the BF16 tensor cores by error-free splitting (Ozaki, Ogita,
Oishi, Rump 2012).

* integer-valued factors: every path must return the exact integer Gram (the
  splitting is then exact and the level sums are integers);
* factors whose 8 digits sit at their largest magnitudes in every row of a
  256-row window: the level sums come within 2^23.3 of the FP32 limit, the
  result must still agree with the exactly rounded Gram to 1e-15 relative;
* random, column-graded factors against an extended-precision reference,
  within the error of an FP64 Gram (ragged M, ragged column tiles, the
  symmetric product and a product of two different factors).
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_10275_gb300 import lrfsi  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lrfsi.load()
    prev = lrfsi.gram_path()
    yield
    lrfsi.gram_path(prev)


def _gram(A, B, path, sym):
    lrfsi.gram_path(path)
    M, p = A.shape
    Ad = torch.tensor(A, dtype=torch.float64, device=DEV)
    if sym:
        Bd, q, ldb = Ad, p, p
    else:
        Bd = torch.tensor(B, dtype=torch.float64, device=DEV)
        q, ldb = B.shape[1], B.shape[1]
    G = torch.full((p, q), np.nan, dtype=torch.float64, device=DEV)
    lrfsi.lrfsi_gram(Ad, p, p, Bd, ldb, q, M, G, q)
    torch.cuda.synchronize()
    return G.cpu().numpy()


@pytest.mark.parametrize("path", [1, 0])
@pytest.mark.parametrize("M,p,q", [(1000, 37, 37), (3 * 256 + 17, 130, 70), (40, 5, 200)])
def test_gram_integer_factors_exact(path, M, p, q):
    rng = np.random.default_rng(M + p + q)
    A = rng.integers(-1024, 1025, (M, p)).astype(np.float64) * 2.0 ** -5
    B = rng.integers(-1024, 1025, (M, q)).astype(np.float64) * 2.0 ** 3
    exact = (A * 2 ** 5).astype(np.int64).T @ (B * 2 ** -3).astype(np.int64)
    G = _gram(A, B, path, sym=False)
    assert np.array_equal(G, exact.astype(np.float64) * 2.0 ** -2)
    if p == q:
        S = _gram(A, None, path, sym=True)
        assert np.array_equal(S, ((A * 2 ** 5).astype(np.int64).T @ (A * 2 ** 5).astype(np.int64)) * 2.0 ** -10)


def test_gram_largest_digits_window():
    """Every row holds x = (127 * 2^49 + 63 (2^42 + ... + 1)) 2^(e - 56): digit 0
    is 127 and the other 7 digits are 63 (the largest magnitudes), so each
    256-row window drives the level sums to ~10.2e6 of the 16.8e6 that FP32
    holds exactly."""
    v = 127 * 2 ** 49 + sum(63 * 2 ** (7 * k) for k in range(7))
    M, p = 2 * 256 + 100, 3
    x = float(Fraction(v, 2 ** 56))   # |x| < 1; rounded to FP64, which changes only the last digit
    A = np.full((M, p), x)
    A[:, 1] *= -2.0 ** 10
    A[:, 2] *= 2.0 ** -20
    G = _gram(A, None, 1, sym=True)
    for i in range(p):
        for j in range(p):
            ref = float(M * Fraction(A[0, i]) * Fraction(A[0, j]))
            assert abs(G[i, j] - ref) <= 1e-15 * abs(ref), (i, j, G[i, j], ref)


@pytest.mark.parametrize("path", [1, 0])
@pytest.mark.parametrize("M,p,q,sym", [(5000, 67, 67, True), (2 * 256 + 3, 200, 45, False), (777, 129, 129, True)])
def test_gram_fp64_accuracy(path, M, p, q, sym):
    rng = np.random.default_rng(7 * M + p)
    A = rng.standard_normal((M, p)) * 10.0 ** rng.uniform(-6, 3, p)        # graded columns
    A[rng.random((M, p)) < 0.1] *= 1e-9                                     # and graded rows
    B = A if sym else rng.standard_normal((M, q)) * 10.0 ** rng.uniform(-3, 3, q)
    G = _gram(A, None if sym else B, path, sym)
    ref = A.astype(np.longdouble).T @ B.astype(np.longdouble)
    absAB = np.abs(A).T @ np.abs(B)
    # FP64-level bound: 2^-48 |A|^T |B| (an FP64 Gram's error is ~2^-53 log2(M) |A|^T |B|)
    err = np.abs(G.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= 2.0 ** -48 * absAB), (err / absAB).max()
    if sym:
        assert np.array_equal(G, G.T)
