"""Per-parameter Newton iteration (oracle).  TEST INFRASTRUCTURE ONLY.

Sec. 3.2, Eq. (newton_step_indiv1): A(x_{j-1}; mu, nu) dx_j = b_D - g(x_{j-1}),
x_j = x_{j-1} + dx_j, started at x_0 = b_D (or a given start), stopped when
the Euclidean residual norm is <= eps_N (Algorithm 1, Sec. 5.1); ``newton4``
is the same iteration for the four parameters of Sec. 4.4.  The linear
solve is a sparse direct LU (SuperLU via scipy, a library primitive).

Safeguard that the paper does not state: if the full
step increases the residual norm, the step is halved up to 20 times.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fsi


def newton(mesh, mu, nu, x0=None, eps=1e-8, max_it=30, source=None, history=None):
    """Returns (x, iterations, final residual norm).  ``history`` (a list)
    receives the residual norm of every iterate."""
    return _iterate(mesh, lambda x: fsi.residual(mesh, x, mu, nu, source), lambda x: fsi.jacobian(mesh, x, mu, nu),
                    x0, eps, max_it, history)


def newton4(mesh, mu, nu, lam, rho, x0=None, eps=1e-8, max_it=30, history=None):
    """The same iteration for the four-parameter problem of Sec. 4.4 (the
    Jacobian A(x; mu_s, nu_f, lambda_s, rho_f) given there)."""
    return _iterate(mesh, lambda x: fsi.residual4(mesh, x, mu, nu, lam, rho),
                    lambda x: fsi.jacobian4(mesh, x, mu, nu, lam, rho), x0, eps, max_it, history)


def _iterate(mesh, residual, jacobian, x0, eps, max_it, history):
    x = mesh.bD.copy() if x0 is None else np.array(x0, dtype=np.float64)
    R = residual(x)
    r = np.linalg.norm(R)
    if history is not None:
        history.append(r)
    it = 0
    while r > eps and it < max_it:
        J = jacobian(x)
        dx = spla.splu(J.tocsc()).solve(-R)
        t = 1.0
        for _ in range(20):
            xn = x + t * dx
            Rn = residual(xn)
            rn = np.linalg.norm(Rn)
            if rn < r or t < 1e-5:
                break
            t *= 0.5
        x, R, r = xn, Rn, rn
        it += 1
        if history is not None:
            history.append(r)
    return x, it, r


def standard_newton(mesh, mus, nus, eps=1e-6, max_it=30, x0=None):
    """The paper's reference method (Sec. 5.1.2): the m problems solved one
    after another, each started from the previous solution (the first from
    b_D).  Returns the solutions (M x m), total Newton steps and final norms."""
    X = np.zeros((mesh.M, len(mus)))
    steps, norms = 0, []
    x = x0
    for i, (mu, nu) in enumerate(zip(mus, nus)):
        x, it, r = newton(mesh, mu, nu, x0=x, eps=eps, max_it=max_it)
        X[:, i] = x
        steps += it
        norms.append(r)
    return X, steps, np.array(norms)


def standard_newton_problem(nx, ny, mus, nus, eps=1e-6, max_it=30):
    """standard_newton on a freshly built nx x ny channel mesh; returns the
    Newton steps taken (a self-contained unit of work for a process pool)."""
    mesh = fsi.Mesh(fsi.Problem(nx, ny))
    X, steps, norms = standard_newton(mesh, mus, nus, eps=eps, max_it=max_it)
    return int(steps)
