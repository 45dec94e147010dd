"""Algorithm 1 of the paper and its accuracy metric (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Algorithm 1 (Sec. 4): split the ordered parameter set into K subsets; for each
subset compute the Newton solution x~ of the upper-median problem (stop at
||residual||_2 <= eps_N); take one Newton step on the whole subset as the
matrix equation F(S_k) = B_k solved by the truncated Chebyshev iteration (or
the truncated GMRES) with the mean-based preconditioner; X^k = x~ 1^T + S_k.

Reading for accuracy targets the paper does not reach in one step:
``chord_steps`` further subset corrections in the same matrix
form, the right-hand side being minus the per-column residuals
R(X_i; mu_i, nu_i) and the operators and preconditioner kept at x~.

Relative residual of a column (Sec. 5.1.2):
||R(x_i; mu_i, nu_i)||_2 / ||R(b_D; mu_i, nu_i)||_2.

Four parameters (Sec. 4.4): the same algorithm over the little-endian order of
(mu_s, nu_f, lambda_s, rho_f) with the matrix equation replaced by Eq.
(matrix_fourpars1) (``*4`` functions).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fsi, lowrank, newton, params


@dataclasses.dataclass
class Options:
    K: int = 2
    eps_N: float = 1e-8
    rank_cap: int = 20
    tol: float = 1e-8
    c: float = 0.5
    d: float = 1.0
    iters: int = 6
    cycles: int = 2
    truncated: bool = True
    eta: float | None = None
    chord_steps: int = 0
    warm_start: bool = True        # x~^{k-1} starts the median Newton of subset k (Sec. 5.1)
    solver: str = "chebyshev"      # "chebyshev" (ChebyshevT) or "gmres" (GMREST), Algorithm 1 step 3


def relative_residuals(mesh, X, mus, nus):
    out = np.zeros(X.shape[1])
    for i in range(X.shape[1]):
        num = np.linalg.norm(fsi.residual(mesh, X[:, i], mus[i], nus[i]))
        den = np.linalg.norm(fsi.residual(mesh, mesh.bD, mus[i], nus[i]))
        out[i] = num / den
    return out


def _subset_solver(mesh, xt, mu_k, nu_k, opt: Options, history=None):
    """The subset's right-hand side B_k and the low-rank solve F_k(S) = B'
    (operators and preconditioner at x~)."""
    J0, Jmu, Jnu = fsi.affine_jacobian(mesh, xt)
    R0, Rmu, Rnu = fsi.affine_residual(mesh, xt)
    mu_bar, nu_bar = params.midpoint_parameters(mu_k, nu_k)
    B = lowrank.rhs(R0, Rmu, Rnu, mu_k, nu_k)
    kw = dict(iters=opt.iters, cycles=opt.cycles, tol=opt.tol, rank_cap=opt.rank_cap,
              truncated=opt.truncated, eta=opt.eta, history=history)
    if opt.solver == "gmres":
        run = lambda B_: lowrank.gmres_T_scaled(J0, Jmu, Jnu, B_, mu_k, nu_k, mu_bar, nu_bar, **kw)
    else:
        run = lambda B_: lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B_, mu_k, nu_k, mu_bar, nu_bar, opt.c, opt.d,
                                                    **kw)
    return B, run


def _chord_rhs(mesh, X, mu_k, nu_k):
    return -np.stack([fsi.residual(mesh, X[:, i], mu_k[i], nu_k[i]) for i in range(len(mu_k))], axis=1)


def subset_step(mesh, xt, mu_k, nu_k, opt: Options, X0=None, history=None):
    """One Newton step on a subset (Sec. 3.4) plus ``opt.chord_steps`` chord
    corrections.  Returns X^k (M x m_k)."""
    B, run = _subset_solver(mesh, xt, mu_k, nu_k, opt, history)
    X = xt[:, None] + run(B)
    for _ in range(opt.chord_steps):
        X = X + run(_chord_rhs(mesh, X, mu_k, nu_k))
    return X


def subset_step_to_target(mesh, xt, mu_k, nu_k, opt: Options, target, max_chord=40):
    """The subset step followed by chord corrections until every column's
    relative residual (Sec. 5.1.2) is <= target or max_chord corrections were
    made (reading for targets beyond one step).  Returns (X, corrections,
    relative residuals)."""
    B, run = _subset_solver(mesh, xt, mu_k, nu_k, opt)
    X = xt[:, None] + run(B)
    k = 0
    rr = relative_residuals(mesh, X, mu_k, nu_k)
    while rr.max() > target and k < max_chord:
        X = X + run(_chord_rhs(mesh, X, mu_k, nu_k))
        k += 1
        rr = relative_residuals(mesh, X, mu_k, nu_k)
    return X, k, rr


def algorithm1(mesh, mus, nus, opt: Options):
    """Algorithm 1 over an already ordered parameter list.  Returns (X, info)."""
    mus, nus = np.asarray(mus, float), np.asarray(nus, float)
    m = len(mus)
    X = np.zeros((mesh.M, m))
    info = dict(newton_steps=[], medians=[], xt=[])
    start = 0
    x_prev = None
    for size in params.cluster_sizes(m, opt.K):
        idx = np.arange(start, start + size)
        med = idx[params.upper_median_position(size)]
        xt, it, r = newton.newton(mesh, mus[med], nus[med], x0=x_prev, eps=opt.eps_N)
        info["newton_steps"].append(it)
        info["medians"].append(int(med))
        info["xt"].append(xt)
        X[:, idx] = subset_step(mesh, xt, mus[idx], nus[idx], opt)
        if opt.warm_start:
            x_prev = xt
        start += size
    return X, info


def relative_residuals4(mesh, X, mus, nus, lams, rhos):
    """Sec. 5.1.2's relative residual for the four-parameter problem."""
    out = np.zeros(X.shape[1])
    for i in range(X.shape[1]):
        num = np.linalg.norm(fsi.residual4(mesh, X[:, i], mus[i], nus[i], lams[i], rhos[i]))
        den = np.linalg.norm(fsi.residual4(mesh, mesh.bD, mus[i], nus[i], lams[i], rhos[i]))
        out[i] = num / den
    return out


def subset_step4(mesh, xt, mu_k, nu_k, lam_k, rho_k, opt: Options, history=None):
    """One Newton step on a four-parameter subset (Eq. (matrix_fourpars1):
    affine coefficients mu, nu rho, lambda, rho; the mean-based
    preconditioner at the midpoints of their ranges) plus ``opt.chord_steps``
    chord corrections.  Returns X^k (M x m_k)."""
    mu_k, nu_k, lam_k, rho_k = (np.asarray(a, float) for a in (mu_k, nu_k, lam_k, rho_k))
    nr_k = nu_k * rho_k
    J0, Jmu, Jnr, Jlam, Jrho = fsi.affine_jacobian4(mesh, xt)
    B = lowrank.rhs_terms(fsi.affine_residual4(mesh, xt), [mu_k, nr_k, lam_k, rho_k])
    mb, nrb, lb, rb = params.affine_midpoints(mu_k, nr_k, lam_k, rho_k)
    extra = [(Jlam, lam_k, lb), (Jrho, rho_k, rb)]
    kw = dict(iters=opt.iters, cycles=opt.cycles, tol=opt.tol, rank_cap=opt.rank_cap,
              truncated=opt.truncated, eta=opt.eta, history=history, extra=extra)
    if opt.solver == "gmres":
        run = lambda B_: lowrank.gmres_T_scaled(J0, Jmu, Jnr, B_, mu_k, nr_k, mb, nrb, **kw)
    else:
        run = lambda B_: lowrank.chebyshev_T_scaled(J0, Jmu, Jnr, B_, mu_k, nr_k, mb, nrb, opt.c, opt.d, **kw)
    X = xt[:, None] + run(B)
    for _ in range(opt.chord_steps):
        Bc = -np.stack([fsi.residual4(mesh, X[:, i], mu_k[i], nu_k[i], lam_k[i], rho_k[i])
                        for i in range(len(mu_k))], axis=1)
        X = X + run(Bc)
    return X


def algorithm1_4(mesh, mus, nus, lams, rhos, opt: Options):
    """Algorithm 1 for four parameters over an already ordered parameter list
    (Sec. 4.4).  Returns (X, info)."""
    mus, nus, lams, rhos = (np.asarray(a, float) for a in (mus, nus, lams, rhos))
    m = len(mus)
    X = np.zeros((mesh.M, m))
    info = dict(newton_steps=[], medians=[], xt=[])
    start = 0
    x_prev = None
    for size in params.cluster_sizes(m, opt.K):
        idx = np.arange(start, start + size)
        med = idx[params.upper_median_position(size)]
        xt, it, r = newton.newton4(mesh, mus[med], nus[med], lams[med], rhos[med], x0=x_prev, eps=opt.eps_N)
        info["newton_steps"].append(it)
        info["medians"].append(int(med))
        info["xt"].append(xt)
        X[:, idx] = subset_step4(mesh, xt, mus[idx], nus[idx], lams[idx], rhos[idx], opt)
        if opt.warm_start:
            x_prev = xt
        start += size
    return X, info


def split_subset(start, size):
    """The two halves of the contiguous subset [start, start + size): the
    clustering rule of Eq. (clustering1) with K = 2 applied to the subset
    (floor(size / 2), then the remainder)."""
    a = size // 2
    return [(start, a), (start + a, size - a)]


def algorithm1_adaptive(mesh, mus, nus, opt: Options, target, min_size=1, max_levels=3):
    """Algorithm 1 with adaptively refined subsets (reading of Sec. 5,
    "Alternative ways to cluster the parameter set": more, smaller subsets
    lower the largest relative residual, and the paper leaves adaptive
    refinement open).  Start from the K subsets of ``opt``; after the subset
    step, every subset whose largest relative residual (Sec. 5.1.2) is above
    ``target`` and that has at least 2 * min_size parameters is split into its
    two halves, each solved again from its own upper median (Newton from b_D);
    at most ``max_levels`` refinements.  No chord corrections here.
    Returns (X, subsets) with subsets = [(start, size, median position)]."""
    mus, nus = np.asarray(mus, float), np.asarray(nus, float)
    m = len(mus)
    X = np.zeros((mesh.M, m))
    subsets, start = [], 0
    for size in params.cluster_sizes(m, opt.K):
        subsets.append((start, size))
        start += size

    def solve(start, size):
        idx = np.arange(start, start + size)
        med = start + params.upper_median_position(size)
        xt, _, _ = newton.newton(mesh, mus[med], nus[med], eps=opt.eps_N)
        X[:, idx] = subset_step(mesh, xt, mus[idx], nus[idx], opt)
        return relative_residuals(mesh, X[:, idx], mus[idx], nus[idx]).max()

    worst = {s: solve(*s) for s in subsets}
    for _ in range(max_levels):
        refine = [s for s in subsets if worst[s] > target and s[1] >= 2 * min_size]
        if not refine:
            break
        nxt = []
        for s in subsets:
            if s in refine:
                for h in split_subset(*s):
                    worst[h] = solve(*h)
                    nxt.append(h)
            else:
                nxt.append(s)
        subsets = nxt
    return X, [(a, n, a + params.upper_median_position(n)) for a, n in subsets]
