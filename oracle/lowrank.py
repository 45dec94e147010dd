"""The subset Newton step as a matrix equation, solved densely (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``rhs``          -- B_k of Sec. 3.4, Eq. (rhs_matrix1), written with the
                      affine pieces: B_k = -(R0 1^T + Rmu mu^T + Rnu nu^T).
* ``apply_F``      -- F(S_k) of Eq. (newton_matrix1) in the affine notation
                      J0 S + Jmu' S D_mu + Jnu' S D_nu (the reference values
                      mu_s, nu_f of Eq. (pardep_matrix1) cancel).
* ``brute_force``  -- the vector notation, Eq. (newtonstep_vectornot1): one
                      sparse solve J(x~; mu_i, nu_i) s_i = -R(x~; mu_i, nu_i)
                      per column, with J and R assembled directly (not through
                      the affine pieces).
* ``truncate``     -- the truncation operator T onto rank <= R (Sec. 5,
                      htucker's truncation; for an order-2 tensor this is the
                      truncated SVD, Eckart-Young): keep the smallest rank r
                      with sqrt(sum_{i>r} s_i^2) <= tol ||s||_2, r <= rank_cap.
* ``chebyshev_T``  -- the truncated, preconditioned Chebyshev iteration.  The
                      paper cites it ([WeiBR20, Alg. 3]) without restating it;
                      this is the textbook Chebyshev acceleration (centre d,
                      half-width c of the spectrum of P^{-1} A, Sec. 5.1.1)
                      with left preconditioning by the mean-based P_T^k
                      (Sec. 4.2) and T applied after every update of the
                      iterate, the residual (before preconditioning) and the
                      search direction; the true residual B - F(S) is formed
                      every step; a cycle of ``iters`` steps is restarted
                      ``cycles - 1`` times from the current iterate (Sec. 5.1:
                      "restarted once after 6 iterations" = 2 cycles of 6).
* ``gmres_T``      -- the truncated GMRES (GMREST), the paper's other low-rank
                      solver (Sec. 4, Algorithm 1 step 3; Sec. 5.1, Table 1),
                      also cited ([WeiBR20, Alg. 1]) without being restated.
                      Reading: the textbook restarted GMRES (Arnoldi with the
                      Frobenius inner product <X, Y> = trace(X^T Y), least
                      squares on the Hessenberg matrix) with right
                      preconditioning by the mean-based P_T^k (Sec. 4.2), so
                      that it minimises the true residual ||B - F(S)||_F, and T
                      applied to the starting residual, to every operator
                      application, to every Gram-Schmidt result and to every
                      update of the iterate; classical Gram-Schmidt against
                      the basis; the same restart rule as ChebyshevT.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fsi


def rhs(R0, Rmu, Rnu, mu_k, nu_k):
    """B_k (M x m_k), Eq. (rhs_matrix1)."""
    mu_k, nu_k = np.asarray(mu_k, float), np.asarray(nu_k, float)
    return -(np.outer(R0, np.ones_like(mu_k)) + np.outer(Rmu, mu_k) + np.outer(Rnu, nu_k))


def apply_F(J0, Jmu, Jnu, S, mu_k, nu_k):
    """F(S) = J0 S + Jmu' S D_mu + Jnu' S D_nu (Eq. (newton_matrix1))."""
    return J0 @ S + (Jmu @ S) * np.asarray(mu_k)[None, :] + (Jnu @ S) * np.asarray(nu_k)[None, :]


def apply_terms(terms, S):
    """sum_t J_t S D_t for further affine terms [(J_t, diag(D_t))] (Sec. 4.4,
    Eq. (matrix_fourpars1): the lambda and rho terms); 0 for none."""
    return sum((J @ S) * np.asarray(c)[None, :] for J, c in terms)


def rhs_terms(R_terms, coeffs):
    """B_k = -(R0 1^T + sum_t R_t c_t^T) for the affine pieces [R0, R_1, ...]
    and coefficient vectors [c_1, ...] (Sec. 4.4, B_k^{mu,nu,lambda,rho})."""
    B = -np.outer(R_terms[0], np.ones(len(coeffs[0])))
    for R, c in zip(R_terms[1:], coeffs):
        B -= np.outer(R, np.asarray(c, float))
    return B


def brute_force4(mesh, xt, mu_k, nu_k, lam_k, rho_k):
    """Exact four-parameter S_k column by column (the vector form of Eq.
    (matrix_fourpars1)): J(x~; mu_i, nu_i, lam_i, rho_i) s_i = -R(x~; ...)."""
    S = np.zeros((mesh.M, len(mu_k)))
    for i in range(len(mu_k)):
        J = fsi.jacobian4(mesh, xt, mu_k[i], nu_k[i], lam_k[i], rho_k[i])
        S[:, i] = spla.splu(J.tocsc()).solve(-fsi.residual4(mesh, xt, mu_k[i], nu_k[i], lam_k[i], rho_k[i]))
    return S


def brute_force(mesh, xt, mu_k, nu_k):
    """Exact S_k column by column (Eq. (newtonstep_vectornot1))."""
    S = np.zeros((mesh.M, len(mu_k)))
    for i, (mu, nu) in enumerate(zip(mu_k, nu_k)):
        J = fsi.jacobian(mesh, xt, mu, nu)
        S[:, i] = spla.splu(J.tocsc()).solve(-fsi.residual(mesh, xt, mu, nu))
    return S


def truncation_rank(s, tol, rank_cap):
    """Smallest r with sqrt(sum_{i >= r} s_i^2) <= tol * ||s||_2, capped."""
    s = np.asarray(s, float)
    if s.size == 0 or s[0] == 0.0:
        return 0
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])          # tail[r] = ||s[r:]||
    tail = np.append(tail, 0.0)
    total = tail[0]
    r = int(np.argmax(tail <= tol * total))
    return min(r, rank_cap)


def truncate(X, tol, rank_cap):
    """Best approximation of rank <= r (truncated SVD)."""
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    r = truncation_rank(s, tol, rank_cap)
    return (U[:, :r] * s[:r]) @ Vt[:r]


def preconditioner(J0, Jmu, Jnu, mu_bar, nu_bar, extra=()):
    """LU of P_T^k = J(x~; mu_bar, nu_bar) = J0 + mu_bar Jmu' + nu_bar Jnu' (Sec. 4.2)
    (+ sum_t bar_t J_t for further affine terms extra = [(J_t, bar_t)], Sec. 4.4)."""
    P = J0 + mu_bar * Jmu + nu_bar * Jnu
    for J, b in extra:
        P = P + b * J
    return spla.splu(P.tocsc())


def chebyshev_T(J0, Jmu, Jnu, P_lu, B, mu_k, nu_k, c, d, iters=6, cycles=2,
                tol=1e-8, rank_cap=None, truncated=True, eta=None, history=None, extra_terms=()):
    """Truncated preconditioned Chebyshev iteration for F(S) = B, S0 = 0.

    One step j (centre d, half-width c, sigma = d / c, rho_0 = 1 / sigma):
        S_{j+1}   = T(S_j + Delta_j)
        Res_{j+1} = T(B - F(S_{j+1}))
        Z_{j+1}   = P^{-1} Res_{j+1}
        rho_{j+1} = 1 / (2 sigma - rho_j)
        Delta_{j+1} = T(rho_{j+1} rho_j Delta_j + (2 rho_{j+1} / c) Z_{j+1})
    and each cycle starts with Res = T(B - F(S)), Delta = P^{-1} Res / d.
    The last step of a cycle stops after the update of S.  With ``eta`` the
    iteration also stops once ||B - F(S)||_F <= eta ||B||_F (checked whenever
    the true residual is formed).  ``history`` receives ||B - F(S)||_F / ||B||_F.
    ``extra_terms`` [(J_t, diag(D_t))] adds further affine terms to F (Sec. 4.4).
    """
    m = B.shape[1]
    rank_cap = m if rank_cap is None else rank_cap
    T = (lambda X: truncate(X, tol, rank_cap)) if truncated else (lambda X: X)
    F = lambda S: apply_F(J0, Jmu, Jnu, S, mu_k, nu_k) + apply_terms(extra_terms, S)
    sigma = d / c
    nB = np.linalg.norm(B)
    S = np.zeros_like(B)
    for _ in range(cycles):
        Res = B - F(S)
        if history is not None:
            history.append(np.linalg.norm(Res) / nB)
        if eta is not None and np.linalg.norm(Res) <= eta * nB:
            return S
        Delta = P_lu.solve(T(Res)) / d
        rho = 1.0 / sigma
        for j in range(iters):
            S = T(S + Delta)
            if j == iters - 1:
                break
            Res = B - F(S)
            if history is not None:
                history.append(np.linalg.norm(Res) / nB)
            if eta is not None and np.linalg.norm(Res) <= eta * nB:
                return S
            Z = P_lu.solve(T(Res))
            rho_new = 1.0 / (2.0 * sigma - rho)
            Delta = T(rho_new * rho * Delta + (2.0 * rho_new / c) * Z)
            rho = rho_new
    if history is not None:
        history.append(np.linalg.norm(B - F(S)) / nB)
    return S


def frobenius_inner(X, Y):
    """<X, Y>_F = trace(X^T Y)."""
    return float(np.sum(X * Y))


def gmres_T(J0, Jmu, Jnu, P_lu, B, mu_k, nu_k, iters=6, cycles=2, tol=1e-8, rank_cap=None,
            truncated=True, eta=None, history=None, extra_terms=()):
    """Truncated right-preconditioned restarted GMRES for F(S) = B, S0 = 0.

    One cycle from the current S:
        Res = B - F(S);  V_0 = T(Res) / beta,  beta = ||T(Res)||_F
        for j = 0 .. iters-1:
            Z_j = P^{-1} V_j
            W   = T(F(Z_j))
            h_ij = <W, V_i>_F  (i <= j);  W = T(W - sum_i h_ij V_i)
            h_{j+1,j} = ||W||_F;  V_{j+1} = W / h_{j+1,j}
            stop early when h_{j+1,j} = 0 or the least-squares residual
            min_y ||beta e_1 - H y|| is <= eta ||B||_F
        y = argmin ||beta e_1 - H y||_2  (H: (n+1) x n upper Hessenberg)
        S = T(S + sum_j y_j Z_j)
    The true residual is checked against eta at the start of every cycle;
    ``history`` receives ||B - F(S)||_F / ||B||_F there and at the end.
    ``extra_terms`` [(J_t, diag(D_t))] adds further affine terms to F (Sec. 4.4).
    """
    m = B.shape[1]
    rank_cap = m if rank_cap is None else rank_cap
    T = (lambda X: truncate(X, tol, rank_cap)) if truncated else (lambda X: X)
    F = lambda S: apply_F(J0, Jmu, Jnu, S, mu_k, nu_k) + apply_terms(extra_terms, S)
    nB = np.linalg.norm(B)
    S = np.zeros_like(B)
    for _ in range(cycles):
        Res = B - F(S)
        if history is not None:
            history.append(np.linalg.norm(Res) / nB)
        if eta is not None and np.linalg.norm(Res) <= eta * nB:
            return S
        R = T(Res)
        beta = np.linalg.norm(R)
        if beta == 0.0:
            return S
        V = [R / beta]
        Z = []
        H = np.zeros((iters + 1, iters))
        n = 0
        for j in range(iters):
            Z.append(P_lu.solve(V[j]))
            W = T(F(Z[j]))
            h = np.array([frobenius_inner(W, Vi) for Vi in V])
            W = T(W - sum(hi * Vi for hi, Vi in zip(h, V)))
            H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(W)
            n = j + 1
            g = np.zeros(j + 2)
            g[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], g, rcond=None)[0]
            est = np.linalg.norm(g - H[:j + 2, :j + 1] @ y)
            if H[j + 1, j] == 0.0 or (eta is not None and est <= eta * nB):
                break
            V.append(W / H[j + 1, j])
        g = np.zeros(n + 1)
        g[0] = beta
        y = np.linalg.lstsq(H[:n + 1, :n], g, rcond=None)[0]
        S = T(S + sum(y[i] * Z[i] for i in range(n)))
    if history is not None:
        history.append(np.linalg.norm(B - F(S)) / nB)
    return S


def equilibration(J0, Jmu, Jnu, mu_bar, nu_bar, extra=()):
    """Row and column scales (r, c) of the max-norm equilibration of the
    preconditioner matrix P = J0 + mu_bar Jmu' + nu_bar Jnu':
        r_i = 1 / max_j |P_ij|,   c_j = 1 / max_i r_i |P_ij|
    so that diag(r) P diag(c) has unit max-norm in every row and column.
    Reading (not in the paper): the truncation operator is applied to the
    equilibrated quantities -- the unknowns mix m/s, m and Pa and the
    equations mix fluid and solid (mu ~ 1e6) scales, so an unscaled Euclidean
    truncation discards the deformation components that dominate F(S)."""
    P = J0 + mu_bar * Jmu + nu_bar * Jnu
    for J, b in extra:
        P = P + b * J
    A = abs(P.tocsr())
    rmax = A.max(axis=1).toarray().ravel()
    r = np.where(rmax > 0, 1.0 / np.where(rmax > 0, rmax, 1.0), 1.0)
    cmax = (sp.diags(r) @ A).max(axis=0).toarray().ravel()
    c = np.where(cmax > 0, 1.0 / np.where(cmax > 0, cmax, 1.0), 1.0)
    return r, c


def _scaled_system(J0, Jmu, Jnu, mu_bar, nu_bar, extra):
    """The equilibrated operators, extra terms and preconditioner, and the
    row and column scales (see ``equilibration``).  extra = [(J_t, diag(D_t),
    bar_t)] for further affine terms (Sec. 4.4)."""
    r, cc = equilibration(J0, Jmu, Jnu, mu_bar, nu_bar, [(J, b) for J, _, b in extra])
    Dr, Dc = sp.diags(r), sp.diags(cc)
    sc = lambda J: (Dr @ J @ Dc).tocsr()
    J0s, Jmus, Jnus = sc(J0), sc(Jmu), sc(Jnu)
    ext = [(sc(J), c, b) for J, c, b in extra]
    P = preconditioner(J0s, Jmus, Jnus, mu_bar, nu_bar, [(J, b) for J, _, b in ext])
    return J0s, Jmus, Jnus, [(J, c) for J, c, _ in ext], P, r, cc


def chebyshev_T_scaled(J0, Jmu, Jnu, B, mu_k, nu_k, mu_bar, nu_bar, c, d, extra=(), **kw):
    """ChebyshevT on the equilibrated equation diag(r) F(diag(c) S~) = diag(r) B
    with the equilibrated preconditioner; returns S = diag(c) S~.  The
    spectrum of P^{-1} A is unchanged (similarity), so c and d are too.
    extra = [(J_t, diag(D_t), bar_t)]: further affine terms (Sec. 4.4)."""
    J0s, Jmus, Jnus, ext, P, r, cc = _scaled_system(J0, Jmu, Jnu, mu_bar, nu_bar, extra)
    Ss = chebyshev_T(J0s, Jmus, Jnus, P, r[:, None] * B, mu_k, nu_k, c, d, extra_terms=ext, **kw)
    return cc[:, None] * Ss


def gmres_T_scaled(J0, Jmu, Jnu, B, mu_k, nu_k, mu_bar, nu_bar, extra=(), **kw):
    """GMREST on the equilibrated equation diag(r) F(diag(c) S~) = diag(r) B
    with the equilibrated preconditioner; returns S = diag(c) S~.  GMRES
    minimises the residual in the row-scaled norm ||diag(r) (B - F(S))||_F.
    extra = [(J_t, diag(D_t), bar_t)]: further affine terms (Sec. 4.4)."""
    J0s, Jmus, Jnus, ext, P, r, cc = _scaled_system(J0, Jmu, Jnu, mu_bar, nu_bar, extra)
    Ss = gmres_T(J0s, Jmus, Jnus, P, r[:, None] * B, mu_k, nu_k, extra_terms=ext, **kw)
    return cc[:, None] * Ss


def spectrum_interval(J0, Jmu, Jnu, P_lu, mu_pts, nu_pts):
    """Smallest and largest |lambda| of P^{-1} A(mu, nu) over the given
    parameters (Sec. 5.1.1), by dense eigenvalues (small M only)."""
    M = J0.shape[0]
    Pinv = P_lu.solve(np.eye(M))
    lo, hi = np.inf, 0.0
    for mu, nu in zip(mu_pts, nu_pts):
        A = (J0 + mu * Jmu + nu * Jnu).toarray()
        lam = np.abs(np.linalg.eigvals(Pinv @ A))
        lo, hi = min(lo, lam.min()), max(hi, lam.max())
    return lo, hi


def chebyshev_cd(lam_min, lam_max):
    """Centre d and half-width c of the interval [lam_min, lam_max]
    (reading of Sec. 5.1.1: c = 0.1, d = 1 for the spectrum in [0.9, 1.1])."""
    return 0.5 * (lam_max - lam_min), 0.5 * (lam_max + lam_min)
