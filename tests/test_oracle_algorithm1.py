"""Pins of the oracle's Algorithm 1 driver, its spectrum estimate and the
equilibration reading (CPU only).

* ``algorithm1.algorithm1`` (Sec. 4, Algorithm 1): on hand-counted layouts the
  subsets are the contiguous blocks of Eq. (clustering1) and the medians the
  upper medians of Sec. 3.3 (written out by hand here, not taken from
  ``params``); every median solution solves its own problem; every column is
  the subset step at its subset's median solution; the warm start x~^{k-1}
  (Sec. 5.1) changes the Newton counts, not the result.
* ``lowrank.spectrum_interval`` (Sec. 5.1.1): on operators built as
  A(mu, nu) = P (T0 + mu T1 + nu T2) with upper-triangular T_i, the
  eigenvalues of P^{-1} A are the diagonal of T0 + mu T1 + nu T2 (closed form),
  including negative and complex-free cases where |lambda| matters.
* ``params.corner_parameters``: on a 3 x 3 grid the four corners, in order.
* Equilibration (a reading, not in the paper): on the 20 x 4 mesh with a
  20-parameter subset, the unscaled truncated ChebyshevT stalls at a linear
  relative residual above 1e-2 while the max-norm equilibrated one at the same
  rank cap and tolerance goes below 1e-4, and the untruncated iteration to
  1e-8 (the measurement that motivated the reading).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import algorithm1, fsi, lowrank, newton, params


@pytest.fixture(scope="module")
def mesh():
    m = fsi.Mesh(fsi.Problem(20, 4))
    assert m.cell_solid.any()
    return m


@pytest.mark.parametrize("m_params,K,bounds,medians", [
    (6, 2, [(0, 3), (3, 6)], [1, 4]),          # sizes 3, 3: upper median at 1-based position 2
    (7, 3, [(0, 2), (2, 4), (4, 7)], [1, 3, 5]),  # sizes 2, 2, 3 (remainder last)
])
def test_algorithm1_subsets_medians_and_columns(mesh, m_params, K, bounds, medians):
    mus = np.linspace(6e5, 1.2e6, m_params)
    nus = np.linspace(2e-3, 4e-3, m_params)
    opt = algorithm1.Options(K=K, eps_N=1e-9, c=0.65, d=1.0, iters=6, cycles=2, truncated=False)
    X, info = algorithm1.algorithm1(mesh, mus, nus, opt)
    assert info["medians"] == medians
    for k, ((a, b), med) in enumerate(zip(bounds, medians)):
        xt = info["xt"][k]
        # the median solution solves the median's problem
        assert np.linalg.norm(fsi.residual(mesh, xt, mus[med], nus[med])) <= 1e-9
        # the subset's columns are the subset step at that median solution
        Xk = algorithm1.subset_step(mesh, xt, mus[a:b], nus[a:b], opt)
        assert np.abs(X[:, a:b] - Xk).max() <= 1e-12 * np.abs(Xk).max()
        # the median column's update is (nearly) zero: x~ already solves it
        assert np.linalg.norm(X[:, med] - xt) <= 1e-6 * np.linalg.norm(xt)
    # warm start: same result, different Newton counts
    opt_cold = algorithm1.Options(**{**opt.__dict__, "warm_start": False})
    Xc, info_c = algorithm1.algorithm1(mesh, mus, nus, opt_cold)
    assert info_c["medians"] == medians
    assert np.abs(Xc - X).max() <= 1e-7 * np.abs(X).max()
    assert info_c["newton_steps"][0] == info["newton_steps"][0]
    assert sum(info_c["newton_steps"][1:]) > sum(info["newton_steps"][1:])


class _Lu:
    def __init__(self, P):
        self.lu = spla.splu(sp.csc_matrix(P))

    def solve(self, X):
        return self.lu.solve(np.asarray(X))


def test_spectrum_interval_closed_form():
    rng = np.random.default_rng(5)
    n = 6
    P = rng.standard_normal((n, n)) + 4 * np.eye(n)
    t0 = np.array([1.0, -2.0, 0.5, 3.0, -0.25, 1.5])
    t1 = np.array([0.1, 0.0, -0.2, 0.05, 0.3, 0.0])
    t2 = np.array([0.0, 1.0, 0.5, -1.0, 0.0, 2.0])
    T = [np.diag(t) + np.triu(rng.standard_normal((n, n)), 1) for t in (t0, t1, t2)]
    J0, Jmu, Jnu = (sp.csr_matrix(P @ Ti) for Ti in T)
    mu_pts = np.array([-1.0, 2.0, 2.0, -1.0])
    nu_pts = np.array([0.5, 0.5, -1.5, -1.5])
    lo, hi = lowrank.spectrum_interval(J0, Jmu, Jnu, _Lu(P), mu_pts, nu_pts)
    lam = np.abs(np.array([t0 + a * t1 + b * t2 for a, b in zip(mu_pts, nu_pts)]))
    assert lo == pytest.approx(lam.min(), rel=1e-10, abs=1e-12)
    assert hi == pytest.approx(lam.max(), rel=1e-10)
    # a single point gives that point's extremes
    lo1, hi1 = lowrank.spectrum_interval(J0, Jmu, Jnu, _Lu(P), mu_pts[:1], nu_pts[:1])
    assert (lo1, hi1) == (pytest.approx(lam[0].min(), abs=1e-12), pytest.approx(lam[0].max(), rel=1e-10))
    # c, d of the interval
    c, d = lowrank.chebyshev_cd(0.9, 1.1)
    assert (c, d) == (pytest.approx(0.1), pytest.approx(1.0))


def test_corner_parameters_of_a_grid():
    mu = np.tile([1.0, 2.0, 3.0], 3)
    nu = np.repeat([10.0, 20.0, 30.0], 3)
    assert params.corner_parameters(mu, nu).tolist() == [0, 2, 6, 8]


@pytest.mark.slow
def test_equilibration_reading_unscaled_truncation_stalls(mesh):
    mus = np.linspace(5e5, 2e6, 10)
    nus = np.linspace(1e-3, 5e-3, 10)
    mu_k = np.tile(mus[:5], 4)
    nu_k = np.repeat(nus[:4], 5)
    med = params.upper_median_position(len(mu_k))
    xt, _, _ = newton.newton(mesh, mu_k[med], nu_k[med], eps=1e-10)
    J0, Jmu, Jnu = fsi.affine_jacobian(mesh, xt)
    B = lowrank.rhs(*fsi.affine_residual(mesh, xt), mu_k, nu_k)
    mb, nb = params.midpoint_parameters(mu_k, nu_k)
    P = lowrank.preconditioner(J0, Jmu, Jnu, mb, nb)
    kw = dict(iters=6, cycles=4, tol=1e-8, rank_cap=12)

    def lin(S):
        return np.linalg.norm(B - lowrank.apply_F(J0, Jmu, Jnu, S, mu_k, nu_k)) / np.linalg.norm(B)

    unscaled = lin(lowrank.chebyshev_T(J0, Jmu, Jnu, P, B, mu_k, nu_k, 0.65, 1.0, **kw))
    scaled = lin(lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mu_k, nu_k, mb, nb, 0.65, 1.0, **kw))
    full = lin(lowrank.chebyshev_T(J0, Jmu, Jnu, P, B, mu_k, nu_k, 0.65, 1.0, iters=6, cycles=4,
                                   truncated=False))
    assert unscaled > 1e-2 and scaled < 1e-4 and full < 1e-8, (unscaled, scaled, full)
