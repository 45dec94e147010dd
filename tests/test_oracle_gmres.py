"""Pins of the oracle's truncated GMRES (``oracle.lowrank.gmres_T``), CPU only.

* Minimal residual over the Krylov space: untruncated, one cycle of k steps
  equals the minimiser of ||b - A P^{-1} z||_2 over z in K_k(A P^{-1}, b),
  computed independently on the Kronecker (vec) form of the matrix equation
  (vec(J S D) = (D kron J) vec(S) for diagonal D) with an explicit Krylov
  matrix, numpy QR and least squares.  A dropped term in F, a wrong
  Hessenberg entry, a transposed inner product or left instead of right
  preconditioning all break it.
* A restart continues from the current iterate: two cycles equal two
  brute-force minimisations in sequence.
* Finite termination: F(S) = (I + u v^T) S has two distinct eigenvalues, so
  two steps solve it exactly for any B.
* Untruncated, the true residual does not increase from cycle to cycle.
* T with tolerance 0 and a full cap changes nothing; a cap of 1 returns a
  rank-1 iterate.
* On the FSI subset the untruncated iteration converges to the brute-force
  Newton step (Eq. (newtonstep_vectornot1)).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fsi, lowrank, newton, params


def _problem(M=7, m=3, seed=0):
    rng = np.random.default_rng(seed)
    J0 = 2.0 * np.eye(M) + 0.3 * rng.standard_normal((M, M))
    Jmu = 0.2 * rng.standard_normal((M, M))
    Jnu = 0.1 * rng.standard_normal((M, M))
    mu = rng.uniform(0.5, 1.5, m)
    nu = rng.uniform(0.5, 1.5, m)
    B = rng.standard_normal((M, m))
    P = J0 + 1.0 * Jmu + 1.0 * Jnu + 0.05 * rng.standard_normal((M, M))
    return J0, Jmu, Jnu, mu, nu, B, P


def _vec_operator(J0, Jmu, Jnu, mu, nu):
    m = len(mu)
    return np.kron(np.eye(m), J0) + np.kron(np.diag(mu), Jmu) + np.kron(np.diag(nu), Jnu)


def _krylov_minimiser(A, Pinv, b, s0, k):
    """argmin ||b - A s|| over s in s0 + P^{-1} K_k(A P^{-1}, r0)."""
    r0 = b - A @ s0
    AP = A @ Pinv
    K = np.zeros((len(b), k))
    v = r0.copy()
    for i in range(k):
        K[:, i] = v
        v = AP @ v
    Q = np.linalg.qr(K)[0]
    y = np.linalg.lstsq(AP @ Q, r0, rcond=None)[0]
    return s0 + Pinv @ (Q @ y)


def _vec(S):
    return S.flatten(order="F")


def _unvec(s, M):
    return s.reshape((M, -1), order="F")


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_one_cycle_is_the_krylov_minimiser(k):
    J0, Jmu, Jnu, mu, nu, B, P = _problem()
    M = J0.shape[0]
    P_lu = spla.splu(sp.csc_matrix(P))
    S = lowrank.gmres_T(J0, Jmu, Jnu, P_lu, B, mu, nu, iters=k, cycles=1, truncated=False)
    A = _vec_operator(J0, Jmu, Jnu, mu, nu)
    Pinv = np.kron(np.eye(len(mu)), np.linalg.inv(P))
    s = _krylov_minimiser(A, Pinv, _vec(B), np.zeros(B.size), k)
    assert np.linalg.norm(_vec(S) - s) <= 1e-10 * np.linalg.norm(s), k


def test_restart_continues_from_the_iterate():
    J0, Jmu, Jnu, mu, nu, B, P = _problem(seed=1)
    P_lu = spla.splu(sp.csc_matrix(P))
    S = lowrank.gmres_T(J0, Jmu, Jnu, P_lu, B, mu, nu, iters=2, cycles=2, truncated=False)
    A = _vec_operator(J0, Jmu, Jnu, mu, nu)
    Pinv = np.kron(np.eye(len(mu)), np.linalg.inv(P))
    s1 = _krylov_minimiser(A, Pinv, _vec(B), np.zeros(B.size), 2)
    s2 = _krylov_minimiser(A, Pinv, _vec(B), s1, 2)
    assert np.linalg.norm(_vec(S) - s2) <= 1e-10 * np.linalg.norm(s2)
    # and it is not the one-cycle result
    assert np.linalg.norm(s2 - s1) > 1e-6 * np.linalg.norm(s2)


def test_two_distinct_eigenvalues_solve_in_two_steps():
    rng = np.random.default_rng(2)
    M, m = 9, 4
    u, v = rng.standard_normal(M), rng.standard_normal(M)
    J0 = np.eye(M) + np.outer(u, v) / M
    Z = np.zeros((M, M))
    B = rng.standard_normal((M, m))
    S = lowrank.gmres_T(J0, Z, Z, spla.splu(sp.identity(M, format="csc")), B, np.ones(m), np.ones(m),
                        iters=2, cycles=1, truncated=False)
    X = np.linalg.solve(J0, B)
    assert np.linalg.norm(S - X) <= 1e-12 * np.linalg.norm(X)
    # one step is not enough
    S1 = lowrank.gmres_T(J0, Z, Z, spla.splu(sp.identity(M, format="csc")), B, np.ones(m), np.ones(m),
                         iters=1, cycles=1, truncated=False)
    assert np.linalg.norm(S1 - X) > 1e-3 * np.linalg.norm(X)


def test_residual_does_not_increase_across_cycles():
    J0, Jmu, Jnu, mu, nu, B, P = _problem(M=12, m=4, seed=3)
    P_lu = spla.splu(sp.csc_matrix(P))
    hist = []
    lowrank.gmres_T(J0, Jmu, Jnu, P_lu, B, mu, nu, iters=3, cycles=5, truncated=False, history=hist)
    assert len(hist) == 6
    assert all(b <= a * (1 + 1e-12) for a, b in zip(hist, hist[1:])), hist
    assert hist[-1] < 1e-3


def test_truncation_limits():
    J0, Jmu, Jnu, mu, nu, B, P = _problem(M=10, m=4, seed=4)
    P_lu = spla.splu(sp.csc_matrix(P))
    S0 = lowrank.gmres_T(J0, Jmu, Jnu, P_lu, B, mu, nu, iters=4, cycles=2, truncated=False)
    S1 = lowrank.gmres_T(J0, Jmu, Jnu, P_lu, B, mu, nu, iters=4, cycles=2, tol=0.0, rank_cap=4)
    assert np.linalg.norm(S1 - S0) <= 1e-10 * np.linalg.norm(S0)
    S2 = lowrank.gmres_T(J0, Jmu, Jnu, P_lu, B, mu, nu, iters=4, cycles=2, tol=0.0, rank_cap=1)
    sv = np.linalg.svd(S2, compute_uv=False)
    assert sv[1] <= 1e-12 * sv[0]


def test_eta_stops_at_the_first_cycle_that_meets_it():
    J0, Jmu, Jnu, mu, nu, B, P = _problem(M=12, m=4, seed=5)
    P_lu = spla.splu(sp.csc_matrix(P))
    hist = []
    S = lowrank.gmres_T(J0, Jmu, Jnu, P_lu, B, mu, nu, iters=3, cycles=8, truncated=False, eta=1e-2,
                        history=hist)
    res = np.linalg.norm(B - lowrank.apply_F(J0, Jmu, Jnu, S, mu, nu)) / np.linalg.norm(B)
    assert res <= 1e-2
    assert hist[-1] == pytest.approx(res, rel=1e-12) and all(h > 1e-2 for h in hist[:-1])


@pytest.fixture(scope="module")
def small_subset():
    m = fsi.Mesh(fsi.Problem(20, 4))   # the flap is 1 x 2 cells: mu_s acts
    mu_k = np.repeat(np.linspace(6e5, 9e5, 3), 2)
    nu_k = np.tile(np.array([3.0e-3, 3.4e-3]), 3)
    med = params.upper_median_position(len(mu_k))
    xt, it, r = newton.newton(m, mu_k[med], nu_k[med], eps=1e-11)
    return m, xt, mu_k, nu_k


def test_untruncated_gmres_converges_to_brute_force(small_subset):
    m, xt, mu_k, nu_k = small_subset
    S_bf = lowrank.brute_force(m, xt, mu_k, nu_k)
    J0, Jmu, Jnu = fsi.affine_jacobian(m, xt)
    R0, Rmu, Rnu = fsi.affine_residual(m, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu_k, nu_k)
    mb, nb = params.midpoint_parameters(mu_k, nu_k)
    errs = []
    for cycles in (1, 2, 3):
        S = lowrank.gmres_T_scaled(J0, Jmu, Jnu, B, mu_k, nu_k, mb, nb, iters=6, cycles=cycles, truncated=False)
        errs.append(np.linalg.norm(S - S_bf) / np.linalg.norm(S_bf))
    # the second cycle gains orders of magnitude; the third sits at the
    # rounding floor of the comparison (~1e-11)
    assert errs[0] > 10 * errs[1] and max(errs[1:]) < 1e-9, errs
    S_t = lowrank.gmres_T_scaled(J0, Jmu, Jnu, B, mu_k, nu_k, mb, nb, iters=6, cycles=3, tol=1e-12,
                                 rank_cap=len(mu_k))
    assert np.linalg.norm(S_t - S_bf) <= 1e-9 * np.linalg.norm(S_bf)
