"""Pins of the oracle's subset matrix equation, truncation and Chebyshev
iteration (CPU only).

* Chebyshev closed form: for F(S) = A S with A = diag(lambda), lambda in
  [d - c, d + c], and P = I, k steps from S0 = 0 leave the error
  T_k((d - A) / c) / T_k(d / c) applied to the initial error (the defining
  property of Chebyshev acceleration); a restart squares the factor.  A wrong
  rho recurrence, coefficient or sign breaks it.
* Truncation closed form: X = A diag(s) B^T with orthonormal A, B built from
  QR of random matrices; T keeps exactly the leading r terms.
* Vector notation (Eq. (newtonstep_vectornot1)) == matrix equation (Eq.
  (newton_matrix1)): the column-by-column solution with directly assembled
  J(x~; mu_i, nu_i), R(x~; mu_i, nu_i) solves the affine F(S) = B; rank(B) <= 3
  (Sec. 4.2, "Multiple Newton Steps").
* The untruncated iteration converges to the brute-force solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import algorithm1, fsi, lowrank, newton, params


class _Identity:
    def solve(self, X):
        return np.array(X, copy=True)


@pytest.mark.parametrize("c,d,k,cycles", [(0.1, 1.0, 6, 1), (0.6, 1.0, 5, 2), (0.3, 0.8, 7, 1)])
def test_chebyshev_closed_form(c, d, k, cycles):
    rng = np.random.default_rng(0)
    n, m = 40, 5
    lam = np.linspace(d - c, d + c, n)
    A = sp.diags(lam).tocsr()
    Z = sp.csr_matrix((n, n))
    B = rng.standard_normal((n, m))
    S = lowrank.chebyshev_T(A, Z, Z, _Identity(), B, np.ones(m), np.ones(m), c, d,
                            iters=k, cycles=cycles, truncated=False)
    Sstar = B / lam[:, None]
    p = np.polynomial.chebyshev.chebval((d - lam) / c, [0] * k + [1]) / np.cosh(k * np.arccosh(d / c))
    expect_err = (p ** cycles)[:, None] * Sstar            # e_0 = S* - 0
    assert np.allclose(Sstar - S, expect_err, rtol=1e-9, atol=1e-13 * abs(Sstar).max())


def test_truncation_closed_form():
    rng = np.random.default_rng(1)
    M, m, n = 60, 12, 10
    A, _ = np.linalg.qr(rng.standard_normal((M, n)))
    Bm, _ = np.linalg.qr(rng.standard_normal((m, n)))
    s = 10.0 ** -np.arange(n)                                # 1, 1e-1, ..., 1e-9
    X = (A * s) @ Bm.T
    for tol, cap, r in ((3e-8, 20, 8), (3e-3, 20, 3), (0.0, 20, 10), (3e-8, 5, 5)):
        Xr = lowrank.truncate(X, tol, cap)
        assert np.allclose(Xr, (A[:, :r] * s[:r]) @ Bm[:, :r].T, atol=1e-14)
        assert np.linalg.matrix_rank(Xr, tol=1e-12) == r
    # the rule: smallest r with ||s[r:]|| <= tol ||s||
    assert lowrank.truncation_rank(np.array([3.0, 4.0]), 0.81, 10) == 1
    assert lowrank.truncation_rank(np.array([3.0, 4.0]), 0.79, 10) == 2
    assert lowrank.truncation_rank(np.zeros(3), 0.1, 10) == 0


@pytest.fixture(scope="module")
def small_subset():
    m = fsi.Mesh(fsi.Problem(20, 4))   # the flap is 1 x 2 cells: mu_s acts (the 10 x 2 mesh has no solid cell)
    assert m.cell_solid.any()
    mu_k = np.repeat(np.linspace(6e5, 9e5, 3), 2)
    nu_k = np.tile(np.array([3.0e-3, 3.4e-3]), 3)
    med = params.upper_median_position(len(mu_k))
    xt, it, r = newton.newton(m, mu_k[med], nu_k[med], eps=1e-11)
    return m, xt, mu_k, nu_k


def test_vector_notation_equals_matrix_equation(small_subset):
    m, xt, mu_k, nu_k = small_subset
    S = lowrank.brute_force(m, xt, mu_k, nu_k)
    J0, Jmu, Jnu = fsi.affine_jacobian(m, xt)
    R0, Rmu, Rnu = fsi.affine_residual(m, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu_k, nu_k)
    F = lowrank.apply_F(J0, Jmu, Jnu, S, mu_k, nu_k)
    assert np.linalg.norm(F - B) <= 1e-9 * np.linalg.norm(B)
    sv = np.linalg.svd(B, compute_uv=False)
    assert sv[3] <= 1e-13 * sv[0]                           # rank(B) <= 3
    # one subset step is a Newton step for every column: the median column's update is ~0
    med = params.upper_median_position(len(mu_k))
    assert np.linalg.norm(S[:, med]) <= 1e-8 * np.linalg.norm(S)


def test_untruncated_chebyshev_converges_to_brute_force(small_subset):
    m, xt, mu_k, nu_k = small_subset
    S_bf = lowrank.brute_force(m, xt, mu_k, nu_k)
    J0, Jmu, Jnu = fsi.affine_jacobian(m, xt)
    R0, Rmu, Rnu = fsi.affine_residual(m, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu_k, nu_k)
    mb, nb = params.midpoint_parameters(mu_k, nu_k)
    P = lowrank.preconditioner(J0, Jmu, Jnu, mb, nb)
    cor = params.corner_parameters(mu_k, nu_k)
    lo, hi = lowrank.spectrum_interval(J0, Jmu, Jnu, P, mu_k[cor], nu_k[cor])
    c, d = lowrank.chebyshev_cd(lo, hi)
    errs = []
    for cycles in (1, 2, 4):
        S = lowrank.chebyshev_T(J0, Jmu, Jnu, P, B, mu_k, nu_k, c, d, iters=6, cycles=cycles,
                                truncated=False)
        errs.append(np.linalg.norm(S - S_bf) / np.linalg.norm(S_bf))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9, errs
    # truncated with a generous cap behaves the same to the truncation level
    S_t = lowrank.chebyshev_T(J0, Jmu, Jnu, P, B, mu_k, nu_k, c, d, iters=6, cycles=4,
                              tol=1e-12, rank_cap=len(mu_k))
    assert np.linalg.norm(S_t - S_bf) <= 1e-9 * np.linalg.norm(S_bf)


def test_relative_residual_definition_and_subset_step(small_subset):
    m, xt, mu_k, nu_k = small_subset
    rr0 = algorithm1.relative_residuals(m, np.repeat(m.bD[:, None], len(mu_k), 1), mu_k, nu_k)
    assert np.allclose(rr0, 1.0)
    # the chord corrections contract ~15-30x each here (5.8e-7 after 3, 6.5e-11 after 6)
    opt = algorithm1.Options(c=0.5, d=1.0, iters=6, cycles=3, truncated=False, chord_steps=6)
    X = algorithm1.subset_step(m, xt, mu_k, nu_k, opt)
    rr = algorithm1.relative_residuals(m, X, mu_k, nu_k)
    assert rr.max() < 1e-8


def test_equilibration_unit_max_norms_and_scaling_invariance(small_subset):
    m, xt, mu_k, nu_k = small_subset
    J0, Jmu, Jnu = fsi.affine_jacobian(m, xt)
    mb, nb = params.midpoint_parameters(mu_k, nu_k)
    r, c = lowrank.equilibration(J0, Jmu, Jnu, mb, nb)
    P = (J0 + mb * Jmu + nb * Jnu).toarray()
    Ps = np.abs(r[:, None] * P * c[None, :])
    assert np.allclose(Ps.max(axis=0), 1.0, rtol=1e-14)          # every column max is 1
    assert np.all(Ps.max(axis=1) <= 1.0 + 1e-14)
    # untruncated Chebyshev is invariant under the two-sided scaling (similarity)
    R0, Rmu, Rnu = fsi.affine_residual(m, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu_k, nu_k)
    Pl = lowrank.preconditioner(J0, Jmu, Jnu, mb, nb)
    S1 = lowrank.chebyshev_T(J0, Jmu, Jnu, Pl, B, mu_k, nu_k, 0.5, 1.0, iters=5, cycles=2, truncated=False)
    S2 = lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mu_k, nu_k, mb, nb, 0.5, 1.0, iters=5, cycles=2,
                                    truncated=False)
    assert np.linalg.norm(S1 - S2) <= 1e-10 * np.linalg.norm(S1)


def test_subset_step_to_target_stops_at_the_first_correction_that_meets_it(small_subset):
    m, xt, mu_k, nu_k = small_subset
    opt = algorithm1.Options(c=0.5, d=1.0, iters=6, cycles=1, truncated=False)
    X, k, rr = algorithm1.subset_step_to_target(m, xt, mu_k, nu_k, opt, 1e-9)
    assert rr.max() <= 1e-9 and k >= 1
    # the same iterate as the fixed-count subset step with k corrections, and
    # k - 1 corrections were not enough
    opt.chord_steps = k
    Xk = algorithm1.subset_step(m, xt, mu_k, nu_k, opt)
    assert np.abs(Xk - X).max() <= 1e-12 * np.abs(X).max()
    opt.chord_steps = k - 1
    rr_prev = algorithm1.relative_residuals(m, algorithm1.subset_step(m, xt, mu_k, nu_k, opt), mu_k, nu_k)
    assert rr_prev.max() > 1e-9
    assert np.allclose(rr, algorithm1.relative_residuals(m, X, mu_k, nu_k))
