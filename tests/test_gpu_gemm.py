"""Tall FP64 GEMMs C = alpha A B + beta C through lrfsi_gemm on both paths
(tensor cores by error-free splitting with an equilibrated contraction index;
FP64 FMA kernels).

* integer-valued factors: the exact product on both paths;
* random factors with columns of A graded over 12 orders of magnitude and the
  rows of B graded inversely (the structure of X R^-1 in the truncation) and
* an orthonormal-by-graded product (U V^T with V carrying singular values
  1 .. 1e-10, the dense residual columns):
  within the error bound of each path against extended precision (_bound);
* alpha, beta and ragged sizes (m not a multiple of 128, n of 32, k of 16).
"""
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


def _gemm(A, B, C0, alpha, beta, path):
    lrfsi.gram_path(path)
    m, k = A.shape
    n = B.shape[1]
    # row-major device copies (torch.tensor keeps the order of a transposed array)
    Ad = torch.tensor(np.ascontiguousarray(A), dtype=torch.float64, device=DEV)
    Bd = torch.tensor(np.ascontiguousarray(B), dtype=torch.float64, device=DEV)
    Cd = torch.tensor(np.ascontiguousarray(C0), dtype=torch.float64, device=DEV)
    lrfsi.lrfsi_gemm(m, n, k, Ad, k, Bd, n, Cd, n, alpha, beta, tensor=True)
    torch.cuda.synchronize()
    return Cd.cpu().numpy()


@pytest.mark.parametrize("path", [1, 0])
@pytest.mark.parametrize("m,n,k", [(3000, 100, 40), (2 * 128 * 9 + 5, 37, 163), (4096, 70, 400)])
def test_gemm_integer_factors_exact(path, m, n, k):
    rng = np.random.default_rng(m + n + k)
    A = rng.integers(-512, 513, (m, k)).astype(np.float64) * 2.0 ** -3
    B = rng.integers(-512, 513, (k, n)).astype(np.float64) * 2.0 ** 4
    exact = ((A * 8).astype(np.int64) @ (B / 16).astype(np.int64)).astype(np.float64) * 2.0
    C = _gemm(A, B, np.zeros((m, n)), 1.0, 0.0, path)
    assert np.array_equal(C, exact)


def _ref(A, B, C0, alpha, beta):
    L = np.longdouble
    return (L(alpha) * (A.astype(L) @ B.astype(L)) + L(beta) * C0.astype(L))


def _bound(A, B, C0, alpha, beta, path):
    """FP64 path: 2^-48 |alpha| (|A| |B|) + 2^-52 |beta C0|.  Tensor path, the
    error bound of the splitting: with the contraction index equilibrated
    (column l of A over 2^e_l, row l of B times 2^e_l, e_l the exponent above
    the column's largest entry), each entry rounded to 56 bits of its row or
    column maximum and the digit levels t + u >= 8 dropped, a term is off by
    at most 2^-50.7 rmax_i cmax_j: 2^-50 k rmax_i cmax_j |alpha| in total."""
    if path == 0:
        return 2.0 ** -48 * abs(alpha) * (np.abs(A) @ np.abs(B)) + 2.0 ** -52 * np.abs(beta * C0)
    e = np.frexp(np.abs(A).max(axis=0))[1].astype(np.float64)
    Ap, Bp = A * 2.0 ** -e, B * 2.0 ** e[:, None]
    rmax, cmax = np.abs(Ap).max(axis=1), np.abs(Bp).max(axis=0)
    return 2.0 ** -50 * A.shape[1] * abs(alpha) * np.outer(rmax, cmax) + 2.0 ** -52 * np.abs(beta * C0)


@pytest.mark.parametrize("path", [1, 0])
def test_gemm_graded_contraction(path):
    """Columns of A from 1 to 1e-12, rows of B the inverse (X R^-1)."""
    rng = np.random.default_rng(5)
    m, n, k = 5000, 90, 120
    g = 10.0 ** -np.linspace(0, 12, k)
    A = rng.standard_normal((m, k)) * g
    B = np.triu(rng.standard_normal((k, n)) + 3 * np.eye(k, n)) / g[:, None]
    C0 = rng.standard_normal((m, n))
    C = _gemm(A, B, C0, -1.0, 1.0, path)
    err = np.abs(C.astype(np.longdouble) - _ref(A, B, C0, -1.0, 1.0)).astype(np.float64)
    bound = _bound(A, B, C0, -1.0, 1.0, path)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("path", [1, 0])
def test_gemm_orthonormal_times_graded(path):
    """U (orthonormal columns) times V^T with V carrying singular values 1 .. 1e-10."""
    rng = np.random.default_rng(6)
    m, n, k = 4000, 100, 40
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    Vt = np.linalg.qr(rng.standard_normal((n, k)))[0].T * np.logspace(0, -10, k)[:, None]
    C = _gemm(U, Vt, np.zeros((m, n)), 2.0, 0.0, path)
    err = np.abs(C.astype(np.longdouble) - _ref(U, Vt, np.zeros((m, n)), 2.0, 0.0)).astype(np.float64)
    bound = _bound(U, Vt, np.zeros((m, n)), 2.0, 0.0, path)
    assert np.all(err <= bound), (err / bound).max()
