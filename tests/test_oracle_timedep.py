"""Pins of the oracle's theta-scheme (Sec. 4.3; CPU only).

* The fluid mass matrix against closed forms of the Q2 mass on a uniform
  cell: a cell-midpoint node's diagonal entry is (8 hx / 15)(8 hy / 15), a
  vertex node shared by four fluid cells (4 hx / 15)(4 hy / 15); the matrix is
  symmetric on the rows and columns of interior fluid velocity DOFs.
* theta = 1 and dt -> infinity reduce a time step to the stationary
  problem: the time-step Newton solution is the stationary Newton solution.
* Consistency: the change over one step shrinks linearly with dt.
* The matrix equation of a subset time step equals the column-by-column
  Newton steps (Eq. (timedep_matrix1) is Eq. (time_indiv1) for every column).
* A subset time step with chord corrections reaches the target.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import algorithm1, fsi, lowrank, newton, params, timedep


@pytest.fixture(scope="module")
def mesh():
    return fsi.Mesh(fsi.Problem(20, 4))


def test_mass_closed_forms(mesh):
    Mf = timedep.mass_fluid(mesh)
    hx, hy = mesh.hx, mesh.hy
    NQ2 = mesh.NQ2
    nnx = 2 * mesh.nx + 1
    # node (ix, iy) = (3, 3): a cell midpoint in the fluid near the inflow; (4, 4): a vertex
    for (ix, iy), val in (((3, 3), (8 * hx / 15) * (8 * hy / 15)), ((4, 4), (4 * hx / 15) * (4 * hy / 15))):
        node = ix + nnx * iy
        row = mesh.node_mom_row[node, 0]
        assert row >= 0
        assert Mf[row, node] == pytest.approx(val, rel=1e-13)
        assert Mf[mesh.node_mom_row[node, 1], node + NQ2] == pytest.approx(val, rel=1e-13)
    # symmetric on interior fluid velocity DOFs (rows and columns in the same node order)
    nodes = [ix + nnx * iy for ix in range(2, 8) for iy in range(2, 6)]
    rows = [mesh.node_mom_row[n, 0] for n in nodes]
    sub = Mf[rows][:, nodes].toarray()
    assert np.abs(sub - sub.T).max() <= 1e-15 * np.abs(sub).max()


def test_stationary_limit(mesh):
    mu, nu = 8e5, 3e-3
    x_st, _, _ = newton.newton(mesh, mu, nu, eps=1e-10)
    x_t, it, r = timedep.newton_theta(mesh, mesh.bD, mu, nu, theta=1.0, dt=1e30, eps=1e-10)
    assert r <= 1e-10
    assert np.abs(x_t - x_st).max() <= 1e-8 * np.abs(x_st).max()


def test_consistency_first_order_in_dt(mesh):
    """From the stationary state at nu, one step at 2 nu: the fluid velocities
    (the unknowns with a time derivative) move by O(dt); pressure, extension
    and the quasi-static solid are algebraic and adjust at once."""
    mu, nu = 8e5, 3e-3
    x0, _, _ = newton.newton(mesh, mu, nu, eps=1e-10)
    Mf = timedep.mass_fluid(mesh)
    vel = np.unique(Mf.indices)                     # velocity DOFs with a mass term
    d = []
    for dt in (1e-3, 5e-4):
        x1, _, _ = timedep.newton_theta(mesh, x0, mu, 2 * nu, theta=0.5, dt=dt, eps=1e-11, Mf=Mf)
        d.append(np.linalg.norm((x1 - x0)[vel]))
    assert d[1] == pytest.approx(d[0] / 2, rel=0.05), d


@pytest.fixture(scope="module")
def step_case(mesh):
    mu_k = np.repeat(np.linspace(7e5, 9e5, 3), 2)
    nu_k = np.tile(np.array([3.0e-3, 3.4e-3]), 3)
    theta, dt = 0.6, 0.02
    X_prev = np.repeat(mesh.bD[:, None], len(mu_k), 1)
    med = params.upper_median_position(len(mu_k))
    xt, _, _ = timedep.newton_theta(mesh, X_prev[:, med], mu_k[med], nu_k[med], theta, dt, eps=1e-11)
    return mu_k, nu_k, theta, dt, X_prev, xt


def test_matrix_equation_equals_columnwise_newton_steps(mesh, step_case):
    mu_k, nu_k, theta, dt, X_prev, xt = step_case
    Mf = timedep.mass_fluid(mesh)
    J0, Jmu, Jnu = timedep.theta_operators(mesh, xt, theta, dt, Mf)
    Xt = np.repeat(xt[:, None], len(mu_k), 1)
    B = timedep.theta_rhs(mesh, Xt, X_prev, mu_k, nu_k, theta, dt, Mf)
    S = np.zeros_like(B)
    for j in range(len(mu_k)):
        A = timedep.theta_jacobian(mesh, xt, mu_k[j], nu_k[j], theta, dt, Mf)
        S[:, j] = spla.spsolve(A.tocsc(), B[:, j])
    F = lowrank.apply_F(J0, Jmu, Jnu, S, mu_k, nu_k)
    assert np.linalg.norm(F - B) <= 1e-9 * np.linalg.norm(B)


def test_subset_time_step_reaches_target(mesh, step_case):
    mu_k, nu_k, theta, dt, X_prev, xt = step_case
    opt = algorithm1.Options(c=0.5, d=1.0, iters=6, cycles=3, truncated=False)
    X, k, rr = timedep.subset_step_theta(mesh, xt, X_prev, mu_k, nu_k, theta, dt, opt, target=1e-9)
    assert rr.max() <= 1e-9
    # the median column solves its own time step already (its update is ~0)
    med = params.upper_median_position(len(mu_k))
    assert np.linalg.norm(X[:, med] - xt) <= 1e-6 * np.linalg.norm(xt - X_prev[:, med])
