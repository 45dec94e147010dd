"""Pins of the oracle's four-parameter extension (Sec. 4.4: mu_s, nu_f,
lambda_s, rho_f all vary), CPU only.

* At the problem's own lambda_s and rho_f the four-parameter residual and
  Jacobian are the two-parameter ones (which are pinned by manufactured
  solutions and central differences in test_oracle_fe.py).
* The direct assembly is affine in lambda_s and in rho_f separately (a
  midpoint identity that uses no affine pieces), and the five affine pieces
  reproduce it: R0 + mu Rmu + (nu rho) Rnurho + lam Rlam + rho Rrho = R and
  likewise for J, at parameters far from the problem's constants.
* The Jacobian is the derivative of the residual (central differences) at
  non-default lambda_s, rho_f.
* The little-endian order of four indices, written out for 2 x 2 x 1 x 2,
  2 x 1 x 3 x 1 and 1 x 1 x 2 x 3 sets from the key's definition.
* The matrix equation (Eq. (matrix_fourpars1)) equals the vector notation: the
  column-by-column Newton steps with directly assembled J and R solve
  F(S) = B with the affine pieces; rank(B) <= 5; and the untruncated
  ChebyshevT and GMREST with the two further terms converge to them.
"""
import numpy as np
import pytest

from oracle import fsi, lowrank, newton, params
from paper_2008_10275_gb300 import inputs


@pytest.fixture(scope="module")
def mesh():
    m = fsi.Mesh(fsi.Problem(20, 4))   # the flap is 1 x 2 cells (the 10 x 2 mesh has no solid cell)
    assert m.cell_solid.any() and not m.cell_solid.all()
    return m


def _state(mesh, seed):
    return mesh.bD + inputs.random_state(mesh.M, seed, nq2=mesh.NQ2)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_reduces_to_two_parameters_at_the_problem_constants(mesh):
    x = _state(mesh, 1)
    lam, rho = mesh.prob.lam_s, mesh.prob.rho_f
    R4 = fsi.residual4(mesh, x, 7e5, 3e-3, lam, rho)
    R2 = fsi.residual(mesh, x, 7e5, 3e-3)
    assert _rel(R4, R2) <= 1e-15
    J4 = fsi.jacobian4(mesh, x, 7e5, 3e-3, lam, rho).toarray()
    J2 = fsi.jacobian(mesh, x, 7e5, 3e-3).toarray()
    assert _rel(J4, J2) <= 1e-15


def test_direct_assembly_is_affine_in_lambda_and_rho(mesh):
    x = _state(mesh, 2)
    mu, nu = 9e5, 2e-3
    for name, args in (("lam", lambda v: (v, 1.1e3)), ("rho", lambda v: (1.5e6, v))):
        a, b = (3e5, 4e6) if name == "lam" else (400.0, 3000.0)
        Ra = fsi.residual4(mesh, x, mu, nu, *args(a))
        Rb = fsi.residual4(mesh, x, mu, nu, *args(b))
        Rm = fsi.residual4(mesh, x, mu, nu, *args(0.5 * (a + b)))
        assert _rel(0.5 * (Ra + Rb), Rm) <= 1e-13, name
        Ja = fsi.jacobian4(mesh, x, mu, nu, *args(a)).toarray()
        Jb = fsi.jacobian4(mesh, x, mu, nu, *args(b)).toarray()
        Jm = fsi.jacobian4(mesh, x, mu, nu, *args(0.5 * (a + b))).toarray()
        assert _rel(0.5 * (Ja + Jb), Jm) <= 1e-13, name
        assert _rel(Ra, Rb) > 1e-6, name  # the parameter does act


@pytest.mark.parametrize("seed", [3, 4])
def test_affine_pieces_reproduce_direct_assembly(mesh, seed):
    x = _state(mesh, seed)
    rng = np.random.default_rng(seed)
    mu, nu, lam, rho = rng.uniform(4e5, 2e6), rng.uniform(1e-3, 5e-3), rng.uniform(5e5, 5e6), rng.uniform(500, 2000)
    R0, Rmu, Rnr, Rlam, Rrho = fsi.affine_residual4(mesh, x)
    R = R0 + mu * Rmu + nu * rho * Rnr + lam * Rlam + rho * Rrho
    assert _rel(R, fsi.residual4(mesh, x, mu, nu, lam, rho)) <= 1e-13
    J0, Jmu, Jnr, Jlam, Jrho = fsi.affine_jacobian4(mesh, x)
    J = (J0 + mu * Jmu + nu * rho * Jnr + lam * Jlam + rho * Jrho).toarray()
    assert _rel(J, fsi.jacobian4(mesh, x, mu, nu, lam, rho).toarray()) <= 1e-13


def test_jacobian_is_the_derivative_of_the_residual(mesh):
    x = _state(mesh, 5)
    mu, nu, lam, rho = 8e5, 4e-3, 3.5e6, 1.6e3
    J = fsi.jacobian4(mesh, x, mu, nu, lam, rho)
    d = np.random.default_rng(6).standard_normal(mesh.M) * 1e-3
    errs = []
    for eps in (1e-2, 5e-3):
        fd = (fsi.residual4(mesh, x + eps * d, mu, nu, lam, rho) - fsi.residual4(mesh, x - eps * d, mu, nu, lam, rho))
        fd /= 2 * eps
        errs.append(np.linalg.norm(fd - J @ d) / np.linalg.norm(J @ d))
    # second order: halving eps quarters the error (or it is already at rounding level)
    assert errs[1] <= 0.3 * errs[0] or errs[1] < 1e-9, errs


def test_little_endian_order_of_four_indices():
    order = params.little_endian_order4(2, 2, 1, 2)
    assert order == [(1, 1, 1, 1), (2, 1, 1, 1), (1, 2, 1, 1), (2, 2, 1, 1),
                     (1, 1, 1, 2), (2, 1, 1, 2), (1, 2, 1, 2), (2, 2, 1, 2)]
    order = params.little_endian_order4(2, 1, 3, 1)
    assert order == [(1, 1, 1, 1), (2, 1, 1, 1), (1, 1, 2, 1), (2, 1, 2, 1), (1, 1, 3, 1), (2, 1, 3, 1)]
    # lambda before rho: key (i3 - 1) m1 m2 + (i4 - 1) m1 m2 m3 with m1 = m2 = 1, m3 = 2
    order = params.little_endian_order4(1, 1, 2, 3)
    assert order == [(1, 1, 1, 1), (1, 1, 2, 1), (1, 1, 1, 2), (1, 1, 2, 2), (1, 1, 1, 3), (1, 1, 2, 3)]
    # the two-parameter order is its m3 = m4 = 1 special case
    assert [t[:2] for t in params.little_endian_order4(3, 4, 1, 1)] == params.little_endian_order(3, 4)
    assert params.affine_midpoints([1.0, 3.0], [2.0, 8.0, 5.0]) == (2.0, 5.0)


@pytest.fixture(scope="module")
def subset(mesh):
    rng = np.random.default_rng(7)
    m = 6
    mu = rng.uniform(6e5, 9e5, m)
    nu = rng.uniform(3.0e-3, 3.4e-3, m)
    lam = rng.uniform(1.8e6, 2.2e6, m)
    rho = rng.uniform(0.9e3, 1.1e3, m)
    med = params.upper_median_position(m)
    x, it, r = newton.newton4(mesh, mu[med], nu[med], lam[med], rho[med], eps=1e-11)
    assert r <= 1e-11
    return x, mu, nu, lam, rho


def test_matrix_equation_equals_vector_notation(mesh, subset):
    xt, mu, nu, lam, rho = subset
    S = lowrank.brute_force4(mesh, xt, mu, nu, lam, rho)
    J0, Jmu, Jnr, Jlam, Jrho = fsi.affine_jacobian4(mesh, xt)
    B = lowrank.rhs_terms(fsi.affine_residual4(mesh, xt), [mu, nu * rho, lam, rho])
    F = lowrank.apply_F(J0, Jmu, Jnr, S, mu, nu * rho) + lowrank.apply_terms([(Jlam, lam), (Jrho, rho)], S)
    assert np.linalg.norm(F - B) <= 1e-9 * np.linalg.norm(B)
    sv = np.linalg.svd(B, compute_uv=False)
    assert sv[5] <= 1e-13 * sv[0]                           # rank(B) <= 5
    med = params.upper_median_position(len(mu))
    assert np.linalg.norm(S[:, med]) <= 1e-8 * np.linalg.norm(S)


@pytest.mark.parametrize("solver", ["chebyshev", "gmres"])
def test_untruncated_solvers_with_further_terms_converge(mesh, subset, solver):
    xt, mu, nu, lam, rho = subset
    S_bf = lowrank.brute_force4(mesh, xt, mu, nu, lam, rho)
    J0, Jmu, Jnr, Jlam, Jrho = fsi.affine_jacobian4(mesh, xt)
    B = lowrank.rhs_terms(fsi.affine_residual4(mesh, xt), [mu, nu * rho, lam, rho])
    mb, nrb, lb, rb = params.affine_midpoints(mu, nu * rho, lam, rho)
    extra = [(Jlam, lam, lb), (Jrho, rho, rb)]
    if solver == "gmres":
        S = lowrank.gmres_T_scaled(J0, Jmu, Jnr, B, mu, nu * rho, mb, nrb, extra=extra, iters=6, cycles=3,
                                   truncated=False)
    else:
        S = lowrank.chebyshev_T_scaled(J0, Jmu, Jnr, B, mu, nu * rho, mb, nrb, 0.5, 1.0, extra=extra, iters=6,
                                       cycles=6, truncated=False)
    assert np.linalg.norm(S - S_bf) <= 1e-8 * np.linalg.norm(S_bf)


@pytest.mark.parametrize("solver", ["chebyshev", "gmres"])
def test_algorithm1_four_parameters_reaches_the_target(mesh, solver):
    """Algorithm 1 with Eq. (matrix_fourpars1) on a 2 x 2 x 2 x 2 set in
    little-endian order, K = 2: untruncated subset steps plus chord
    corrections bring every column below 1e-8; the column order is the
    four-index order."""
    from oracle import algorithm1
    grid = (np.array([6e5, 9e5]), np.array([2.8e-3, 3.4e-3]), np.array([1.8e6, 2.3e6]), np.array([0.9e3, 1.1e3]))
    order = params.little_endian_order4(2, 2, 2, 2)
    mus, nus, lams, rhos = (np.array([g[t[q] - 1] for t in order]) for q, g in enumerate(grid))
    assert list(mus[:2]) == [6e5, 9e5] and nus[1] == 2.8e-3 and nus[2] == 3.4e-3 and lams[4] == 2.3e6
    # the chord corrections contract ~10x each (4e-2 after the subset step, 9e-11 after 7)
    opt = algorithm1.Options(K=2, c=0.5, d=1.0, iters=6, cycles=3, truncated=False, chord_steps=7, solver=solver,
                             eps_N=1e-10)
    X, info = algorithm1.algorithm1_4(mesh, mus, nus, lams, rhos, opt)
    rr = algorithm1.relative_residuals4(mesh, X, mus, nus, lams, rhos)
    assert rr.max() < 1e-8, rr.max()
    assert info["medians"] == [4, 12]


def test_five_operators_from_three_two_parameter_assemblies(mesh):
    """The two-parameter affine assembly at (rho_f, lambda_s) = (0, 0), (1, 0),
    (0, 1) yields the five four-parameter operators: the rho and lambda parts
    live in element blocks of their own (fluid momentum x velocity, solid
    momentum x deformation), so the differences below cancel nothing.  Here
    they agree to the rounding of the sparse assembly's summation order (the
    explicit zero entries of the rho = 0 pass reorder it)."""
    import dataclasses
    x = _state(mesh, 8)

    def aff(rho, lam):
        m = fsi.Mesh(dataclasses.replace(mesh.prob, rho_f=rho, lam_s=lam))
        return [A.toarray() for A in fsi.affine_jacobian(m, x)]

    a00, a10, a01 = aff(0.0, 0.0), aff(1.0, 0.0), aff(0.0, 1.0)
    J0, Jmu, Jnr, Jlam, Jrho = (A.toarray() for A in fsi.affine_jacobian4(mesh, x))
    close = lambda a, b: np.abs(a - b).max() <= 1e-15 * np.abs(b).max()
    assert close(a00[0], J0) and close(a00[1], Jmu)
    assert close(a10[2], Jnr)                               # Jnu' = rho_f A2
    assert close(a10[0] - a00[0], Jrho)
    assert close(a01[0] - a00[0], Jlam)
