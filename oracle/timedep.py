"""The time-dependent problem with the theta-scheme (Sec. 4.3; oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (fsi_problem_time_weak1) adds rho_s <d_t v, phi>_S and rho_f <d_t v,
phi>_F to the stationary weak form; the theta-scheme of Sec. 4.3 gives, per
time step t_{i-1} -> t_i and parameter (mu, nu), the nonlinear system

    R_theta(x) = (rho_f A_t^f / dt) (x - x_prev) + theta R(x; mu, nu)
                 + (1 - theta) R(x_prev; mu, nu) = 0,

solved by Newton with the matrix (rho_f A_t^f / dt) + theta J(x; mu, nu)
(Eq. (time_indiv1)); on a subset the Newton step at the median's time-step
solution x~ is one matrix equation (Eq. (timedep_matrix1)):

    (rho_f A_t^f / dt) S + theta F(S) = -[R_theta(x~; X_prev_j, mu_j, nu_j)]_j,

i.e. the stationary matrix equation with the affine operators
J0' = theta J0 + rho_f A_t^f / dt, Jmu'' = theta Jmu', Jnu'' = theta Jnu'.

Readings (the paper does not fix them):
* A_t^f discretises <v, phi>_F in the fluid momentum rows (the rows the
  stationary residual gives the fluid momentum equation; Dirichlet rows keep
  x - b_D).  A_t^s: the weak form states no kinematic equation d_t u = v in S,
  and in the stationary row ownership v = 0 on the closed solid (its v-rows
  are identity rows), so rho_s <d_t v, phi>_S vanishes: the solid is
  quasi-static.
* b_D does not depend on time (B^i = B^{i-1}).
* The (***) term of Eq. (timedep_matrix1) is evaluated exactly, column by
  column (the paper's remark offers a rank-3 approximation to save CPU time).
* Relative residual of a column: ||R_theta(x)||_2 / ||R(b_D; mu, nu)||_2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import algorithm1, fsi, lowrank, params


def mass_fluid(mesh):
    """A_t^f: <v, phi>_F on the fluid momentum rows and velocity columns
    (3 x 3 Gauss, exact for Q2 x Q2 products on the affine cells)."""
    F = np.flatnonzero(~mesh.cell_solid)
    w, N = mesh.w, mesh.N
    Ne = np.einsum("q,aq,bq->ab", w, N, N)                     # element mass of one component
    eye = np.eye(2)
    E = np.einsum("ab,ik->aibk", Ne, eye)                       # [a, i, b, k]
    coo = fsi._COO(mesh.M)
    if len(F):
        fsi._add_block(coo, mesh.momrow[F], mesh.vdof[F], np.broadcast_to(E, (len(F),) + E.shape))
    return coo.csr()


def theta_residual(mesh, x, x_prev, mu, nu, theta, dt, Mf=None):
    """R_theta(x) of one time step (see the module docstring)."""
    Mf = mass_fluid(mesh) if Mf is None else Mf
    rho = mesh.prob.rho_f
    return (rho / dt) * (Mf @ (x - x_prev)) + theta * fsi.residual(mesh, x, mu, nu) \
        + (1.0 - theta) * fsi.residual(mesh, x_prev, mu, nu)


def theta_jacobian(mesh, x, mu, nu, theta, dt, Mf=None):
    """d R_theta / dx = (rho_f A_t^f / dt) + theta J(x; mu, nu) (Eq. (time_indiv1))."""
    Mf = mass_fluid(mesh) if Mf is None else Mf
    return ((mesh.prob.rho_f / dt) * Mf + theta * fsi.jacobian(mesh, x, mu, nu)).tocsr()


def newton_theta(mesh, x_prev, mu, nu, theta, dt, x0=None, eps=1e-8, max_it=30, Mf=None):
    """Newton iteration of one time step from x0 (default x_prev); stops at
    ||R_theta||_2 <= eps.  Returns (x, iterations, final residual norm)."""
    Mf = mass_fluid(mesh) if Mf is None else Mf
    x = np.array(x_prev if x0 is None else x0, dtype=np.float64)
    r = theta_residual(mesh, x, x_prev, mu, nu, theta, dt, Mf)
    it = 0
    while np.linalg.norm(r) > eps and it < max_it:
        J = theta_jacobian(mesh, x, mu, nu, theta, dt, Mf)
        x = x + spla.spsolve(J.tocsc(), -r)
        r = theta_residual(mesh, x, x_prev, mu, nu, theta, dt, Mf)
        it += 1
    return x, it, np.linalg.norm(r)


def theta_operators(mesh, xt, theta, dt, Mf=None):
    """(J0', Jmu'', Jnu'') of the time-step matrix equation at x~."""
    Mf = mass_fluid(mesh) if Mf is None else Mf
    J0, Jmu, Jnu = fsi.affine_jacobian(mesh, xt)
    return ((theta * J0 + (mesh.prob.rho_f / dt) * Mf).tocsr(), (theta * Jmu).tocsr(), (theta * Jnu).tocsr())


def theta_rhs(mesh, X, X_prev, mu_k, nu_k, theta, dt, Mf=None):
    """-R_theta of every column of X (M x m) against its previous state."""
    Mf = mass_fluid(mesh) if Mf is None else Mf
    return -np.stack([theta_residual(mesh, X[:, j], X_prev[:, j], mu_k[j], nu_k[j], theta, dt, Mf)
                      for j in range(len(mu_k))], axis=1)


def relative_residuals_theta(mesh, X, X_prev, mu_k, nu_k, theta, dt, Mf=None):
    """||R_theta(X_j)||_2 / ||R(b_D; mu_j, nu_j)||_2 per column."""
    Mf = mass_fluid(mesh) if Mf is None else Mf
    out = np.zeros(len(mu_k))
    for j in range(len(mu_k)):
        num = np.linalg.norm(theta_residual(mesh, X[:, j], X_prev[:, j], mu_k[j], nu_k[j], theta, dt, Mf))
        out[j] = num / np.linalg.norm(fsi.residual(mesh, mesh.bD, mu_k[j], nu_k[j]))
    return out


def subset_step_theta(mesh, xt, X_prev, mu_k, nu_k, theta, dt, opt: algorithm1.Options, target=None,
                      max_chord=40, Mf=None):
    """One time step on a subset (Eq. (timedep_matrix1)): the Newton step at
    the median's time-step solution x~ as one matrix equation, solved by the
    truncated ChebyshevT with the mean-based preconditioner of the time-step
    operators, then chord corrections (right-hand side -R_theta of the
    current columns, operators kept at x~) until every column's relative
    residual is <= target (``opt.chord_steps`` corrections if target is None).
    Returns (X, corrections, relative residuals)."""
    Mf = mass_fluid(mesh) if Mf is None else Mf
    J0, Jmu, Jnu = theta_operators(mesh, xt, theta, dt, Mf)
    mb, nb = params.midpoint_parameters(mu_k, nu_k)
    kw = dict(iters=opt.iters, cycles=opt.cycles, tol=opt.tol, rank_cap=opt.rank_cap, truncated=opt.truncated,
              eta=opt.eta)
    run = lambda B: lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mu_k, nu_k, mb, nb, opt.c, opt.d, **kw)
    Xt = np.repeat(xt[:, None], len(mu_k), 1)
    X = Xt + run(theta_rhs(mesh, Xt, X_prev, mu_k, nu_k, theta, dt, Mf))
    k = 0
    rr = relative_residuals_theta(mesh, X, X_prev, mu_k, nu_k, theta, dt, Mf)
    while (rr.max() > target if target is not None else k < opt.chord_steps) and k < max_chord:
        X = X + run(theta_rhs(mesh, X, X_prev, mu_k, nu_k, theta, dt, Mf))
        k += 1
        rr = relative_residuals_theta(mesh, X, X_prev, mu_k, nu_k, theta, dt, Mf)
    return X, k, rr
