"""Stationary 2D FSI finite element residual and Jacobian (oracle, FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Weak form: Sec. 2, Eq. (fsi_problem_weak1) -- divergence equation tested with
xi on F, momentum equation tested with a global phi, harmonic deformation
extension tested with psi on F.  Unknown x = (v, u, p): velocity and
deformation in Q2 (biquadratic), pressure in Q1 (bilinear) on a structured
quadrilateral mesh of the channel [0, Lx] x [0, Ly] with the elastic flap S
attached to the bottom wall.

Readings of the paper that this file fixes:

* Gradient convention (grad u)_ij = d u_i / d x_j; the solid terms are taken
  literally from Eq. (fsi_problem_weak1): mu_s <G + G^T + G^T G, grad phi>_S and
  lambda_s <tr(G + G^T G / 2) I, grad phi>_S with G = grad u (the typo
  tr(grad u^T grad u^T) of Sec. 3 is read as tr(grad u^T grad u)).
* Row ownership of the monolithic system (the coupling conditions are
  "implicitly included", Sec. 2): at nodes of the closed solid S-bar the
  momentum test function lives in the u-rows and v = 0 (kinematic condition);
  at fluid nodes the momentum equation lives in the v-rows and the extension
  equation in the u-rows; u = 0 on the outer boundary; v = v_in on the inflow,
  v = 0 on the walls; the outflow x = Lx is natural (do-nothing for the
  symmetric-gradient form); p-rows carry the divergence equation at Q1
  vertices of F-bar and the identity elsewhere.
* The residual is R(x; mu, nu) = g(x; mu, nu) - b_D, where g has the
  variational residual in equation rows and x itself in Dirichlet/identity
  rows; Newton solves J dx = -R (Sec. 3.2, Eq. (newton_step_indiv1) with
  b_D - g = -R).
* Affine split (Sec. 3, Eq. (pardep_matrix1) with the reference values
  mu_s = nu_f = 0): R = R0 + mu Rmu + nu Rnu with
  Rmu = <G + G^T + G^T G, grad phi>_S, Rnu = rho_f <grad v + grad v^T,
  grad phi>_F, and R0 the rest; likewise J = J0 + mu Jmu' + nu Jnu'.
* 3 x 3 Gauss-Legendre quadrature on every cell.

Oracle DOF ordering (an interface fact, not shared code): field-blocked
[v_x | v_y | u_x | u_y] over the Q2 nodes, node id = i + (2 nx + 1) j, then p
over the Q1 vertices, vertex id = a + (nx + 1) b.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# Reference elements on [0, 1]^2
# ----------------------------------------------------------------------------

_G3_T = np.array([0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)])
_G3_W = np.array([5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0])


def _lagrange2(t):
    """1D quadratic Lagrange basis at nodes 0, 1/2, 1 and its derivative."""
    t = np.asarray(t, dtype=np.float64)
    val = np.stack([(2 * t - 1) * (t - 1), 4 * t * (1 - t), t * (2 * t - 1)])
    der = np.stack([4 * t - 3, 4 - 8 * t, 4 * t - 1])
    return val, der


def _lagrange1(t):
    t = np.asarray(t, dtype=np.float64)
    return np.stack([1 - t, t]), np.stack([-np.ones_like(t), np.ones_like(t)])


def reference_basis(tx, ty):
    """Q2 basis N[a, q], gradients dN[a, q, 2] (reference coordinates) and Q1
    basis P[b, q] at the points (tx[q], ty[q]).  Local Q2 node a = ax + 3 ay,
    local Q1 vertex b = bx + 2 by."""
    lx, dlx = _lagrange2(tx)
    ly, dly = _lagrange2(ty)
    mx, _ = _lagrange1(tx)
    my, _ = _lagrange1(ty)
    nq = len(tx)
    N = np.zeros((9, nq))
    dN = np.zeros((9, nq, 2))
    for ay in range(3):
        for ax in range(3):
            a = ax + 3 * ay
            N[a] = lx[ax] * ly[ay]
            dN[a, :, 0] = dlx[ax] * ly[ay]
            dN[a, :, 1] = lx[ax] * dly[ay]
    P = np.zeros((4, nq))
    for by in range(2):
        for bx in range(2):
            P[bx + 2 * by] = mx[bx] * my[by]
    return N, dN, P


def gauss_2d(npts=3):
    t, w = np.polynomial.legendre.leggauss(npts)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    if npts == 3:
        t, w = _G3_T, _G3_W
    tx = np.tile(t, npts)
    ty = np.repeat(t, npts)
    return tx, ty, np.tile(w, npts) * np.repeat(w, npts)


# ----------------------------------------------------------------------------
# Mesh, DOF layout, row ownership
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Problem:
    """Geometry and constants of the 2D channel-with-flap FSI problem."""
    nx: int
    ny: int
    Lx: float = 2.0
    Ly: float = 0.4
    flap: tuple | None = (0.6, 0.7, 0.0, 0.2)  # (x0, x1, y0, y1); None = no solid
    all_solid: bool = False                     # every cell solid (MMS only)
    rho_f: float = 1.0e3
    lam_s: float = 2.0e6
    v_mean: float = 0.2                         # mean inflow velocity


class Mesh:
    """Structured Q2/Q1 mesh with DOF numbering, Dirichlet data and row ownership."""

    def __init__(self, prob: Problem, bD: np.ndarray | None = None):
        self.prob = prob
        nx, ny = prob.nx, prob.ny
        self.nx, self.ny = nx, ny
        self.hx, self.hy = prob.Lx / nx, prob.Ly / ny
        self.nnx, self.nny = 2 * nx + 1, 2 * ny + 1           # Q2 node grid
        self.NQ2 = self.nnx * self.nny
        self.NQ1 = (nx + 1) * (ny + 1)
        self.M = 4 * self.NQ2 + self.NQ1
        self.ncell = nx * ny

        ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
        ci, cj = ci.ravel(), cj.ravel()                        # cell id = ci + nx cj
        self.cell_ij = np.stack([ci, cj], axis=1)
        self.cell_nodes = np.zeros((self.ncell, 9), dtype=np.int64)
        for ay in range(3):
            for ax in range(3):
                self.cell_nodes[:, ax + 3 * ay] = (2 * ci + ax) + self.nnx * (2 * cj + ay)
        self.cell_verts = np.zeros((self.ncell, 4), dtype=np.int64)
        for by in range(2):
            for bx in range(2):
                self.cell_verts[:, bx + 2 * by] = (ci + bx) + (nx + 1) * (cj + by)
        xc = (ci + 0.5) * self.hx
        yc = (cj + 0.5) * self.hy
        if prob.all_solid:
            solid = np.ones(self.ncell, dtype=bool)
        elif prob.flap is None:
            solid = np.zeros(self.ncell, dtype=bool)
        else:
            x0, x1, y0, y1 = prob.flap
            solid = (xc > x0) & (xc < x1) & (yc > y0) & (yc < y1)
        self.cell_solid = solid

        ni, nj = np.meshgrid(np.arange(self.nnx), np.arange(self.nny), indexing="xy")
        ni, nj = ni.ravel(), nj.ravel()
        self.node_ij = np.stack([ni, nj], axis=1)
        self.node_xy = np.stack([ni * 0.5 * self.hx, nj * 0.5 * self.hy], axis=1)
        in_sbar = np.zeros(self.NQ2, dtype=bool)
        in_sbar[self.cell_nodes[solid].ravel()] = True
        inflow = ni == 0
        outflow = ni == self.nnx - 1
        wall = (nj == 0) | (nj == self.nny - 1)
        on_bnd = inflow | outflow | wall
        v_dir = inflow | wall | in_sbar
        self.in_sbar, self.on_bnd, self.v_dir = in_sbar, on_bnd, v_dir
        self.inflow, self.outflow, self.wall = inflow, outflow, wall
        vert_in_fbar = np.zeros(self.NQ1, dtype=bool)
        vert_in_fbar[self.cell_verts[~solid].ravel()] = True
        self.vert_in_fbar = vert_in_fbar

        NQ2 = self.NQ2
        nodes = np.arange(NQ2)
        # Row of the momentum test function phi_n e_i (Sec. 2: v-rows in F, u-rows on S-bar).
        self.node_mom_row = np.full((NQ2, 2), -1, dtype=np.int64)
        self.node_ext_row = np.full((NQ2, 2), -1, dtype=np.int64)
        for i in range(2):
            fluid_mom = ~v_dir
            solid_mom = in_sbar & ~on_bnd
            self.node_mom_row[fluid_mom, i] = i * NQ2 + nodes[fluid_mom]
            self.node_mom_row[solid_mom, i] = (2 + i) * NQ2 + nodes[solid_mom]
            ext = ~on_bnd & ~in_sbar
            self.node_ext_row[ext, i] = (2 + i) * NQ2 + nodes[ext]
        self.vert_div_row = np.where(vert_in_fbar, 4 * NQ2 + np.arange(self.NQ1), -1)

        kind = np.zeros(self.M, dtype=np.int64)                # 0 = identity row
        for arr, k in ((self.node_mom_row, 1), (self.node_ext_row, 2), (self.vert_div_row, 3)):
            r = arr[arr >= 0]
            assert np.all(kind[r] == 0), "a row owned twice"
            kind[r] = k
        self.row_kind = kind
        self.ident_rows = np.flatnonzero(kind == 0)

        if bD is None:
            bD = np.zeros(self.M)
            y = self.node_xy[:, 1]
            H = prob.Ly
            vin = prob.v_mean * 6.0 / H ** 2 * y * (H - y)    # parabolic, mean v_mean
            bD[np.flatnonzero(inflow)] = vin[inflow]
        self.bD = np.where(kind == 0, bD, 0.0)

        # per-cell DOF maps
        self.vdof = np.stack([self.cell_nodes, self.cell_nodes + NQ2], axis=2)          # (c, a, i)
        self.udof = np.stack([self.cell_nodes + 2 * NQ2, self.cell_nodes + 3 * NQ2], axis=2)
        self.pdof = self.cell_verts + 4 * NQ2
        self.momrow = self.node_mom_row[self.cell_nodes]                               # (c, a, i)
        self.extrow = self.node_ext_row[self.cell_nodes]
        self.divrow = self.vert_div_row[self.cell_verts]

        tx, ty, w = gauss_2d(3)
        N, dNr, P = reference_basis(tx, ty)
        self.N, self.P = N, P
        self.dN = dNr / np.array([self.hx, self.hy])
        self.w = w * self.hx * self.hy
        self.cell_origin = np.stack([ci * self.hx, cj * self.hy], axis=1)
        self.qxy = self.cell_origin[:, None, :] + np.stack([tx * self.hx, ty * self.hy], axis=1)[None]

    # -- field extraction -------------------------------------------------
    def split(self, x):
        x = np.asarray(x, dtype=np.float64)
        V = x[self.vdof]          # (c, 9, 2)
        U = x[self.udof]
        Pv = x[self.pdof]         # (c, 4)
        return V, U, Pv

    def field_names(self):
        return ("vx", "vy", "ux", "uy", "p")


# ----------------------------------------------------------------------------
# Quadrature-point fields and element terms
# ----------------------------------------------------------------------------


def _qp_fields(mesh, x):
    V, U, Pv = mesh.split(x)
    v = np.einsum("cai,aq->cqi", V, mesh.N)
    Gv = np.einsum("cai,aqj->cqij", V, mesh.dN)         # Gv[c,q,i,j] = d v_i / d x_j
    Gu = np.einsum("cai,aqj->cqij", U, mesh.dN)
    p = np.einsum("cb,bq->cq", Pv, mesh.P)
    return v, Gv, Gu, p


def element_residual_terms(mesh, x, rho=None, lam=None):
    """Element vectors of every term of Eq. (fsi_problem_weak1) on every cell
    (rho, lam: override the problem's rho_f, lambda_s; Sec. 4.4 varies them).

    Returns a dict of arrays over all cells (callers mask fluid / solid cells):
      conv[c,a,i]  = rho_f <(v . grad) v, phi_a e_i>
      pres[c,a,i]  = -<p, div(phi_a e_i)>
      visc[c,a,i]  = rho_f <grad v + grad v^T, grad(phi_a e_i)>      (times nu)
      div[c,b]     = <div v, xi_b>
      ext[c,a,i]   = <grad u_i, grad phi_a>
      smu[c,a,i]   = <G + G^T + G^T G, grad(phi_a e_i)>              (times mu)
      slam[c,a,i]  = lambda_s <tr(G + G^T G / 2), div(phi_a e_i)>
    """
    rho = mesh.prob.rho_f if rho is None else rho
    lam = mesh.prob.lam_s if lam is None else lam
    v, Gv, Gu, p = _qp_fields(mesh, x)
    w, N, dN, P = mesh.w, mesh.N, mesh.dN, mesh.P
    adv = np.einsum("cqj,cqij->cqi", v, Gv)                             # (v . grad) v
    conv = rho * np.einsum("q,cqi,aq->cai", w, adv, N)
    pres = -np.einsum("q,cq,aqi->cai", w, p, dN)
    symv = Gv + np.swapaxes(Gv, 2, 3)
    visc = rho * np.einsum("q,cqij,aqj->cai", w, symv, dN)
    divv = Gv[:, :, 0, 0] + Gv[:, :, 1, 1]
    div = np.einsum("q,cq,bq->cb", w, divv, P)
    ext = np.einsum("q,cqij,aqj->cai", w, Gu, dN)
    GtG = np.einsum("cqki,cqkj->cqij", Gu, Gu)                         # (G^T G)_ij
    E2 = Gu + np.swapaxes(Gu, 2, 3) + GtG
    smu = np.einsum("q,cqij,aqj->cai", w, E2, dN)
    tr = Gu[:, :, 0, 0] + Gu[:, :, 1, 1] + 0.5 * np.einsum("cqkj,cqkj->cq", Gu, Gu)
    slam = lam * np.einsum("q,cq,aqi->cai", w, tr, dN)
    return dict(conv=conv, pres=pres, visc=visc, div=div, ext=ext, smu=smu, slam=slam)


def _scatter(M, rows, vals):
    out = np.zeros(M)
    rows = rows.ravel()
    vals = vals.ravel()
    keep = rows >= 0
    np.add.at(out, rows[keep], vals[keep])
    return out


def residual(mesh, x, mu, nu, source=None):
    """R(x; mu, nu) assembled directly with the given parameters (Sec. 2, Eq.
    (fsi_problem_weak1); Dirichlet/identity rows x - b_D).  ``source`` (tests
    only) is subtracted from the equation rows."""
    t = element_residual_terms(mesh, x)
    F, S = ~mesh.cell_solid, mesh.cell_solid
    mom = np.zeros_like(t["conv"])
    mom[F] = t["conv"][F] + t["pres"][F] + nu * t["visc"][F]
    mom[S] = mu * t["smu"][S] + t["slam"][S]
    R = _scatter(mesh.M, mesh.momrow, mom)
    R += _scatter(mesh.M, mesh.extrow[F], t["ext"][F])
    R += _scatter(mesh.M, mesh.divrow[F], t["div"][F])
    x = np.asarray(x, dtype=np.float64)
    R[mesh.ident_rows] = x[mesh.ident_rows] - mesh.bD[mesh.ident_rows]
    if source is not None:
        eq = mesh.row_kind != 0
        R[eq] -= source[eq]
    return R


def affine_residual(mesh, x):
    """The affine pieces (R0, Rmu, Rnu) with R = R0 + mu Rmu + nu Rnu
    (Sec. 3.4, Eq. (rhs_matrix1): -B_k = R0 (x) 1 + Rmu (x) diag(D_mu) +
    Rnu (x) diag(D_nu), Rmu = A1 x + g_mu(x), Rnu = rho_f A2 x)."""
    t = element_residual_terms(mesh, x)
    F, S = ~mesh.cell_solid, mesh.cell_solid
    M = mesh.M
    R0 = _scatter(M, mesh.momrow[F], t["conv"][F] + t["pres"][F])
    R0 += _scatter(M, mesh.momrow[S], t["slam"][S])
    R0 += _scatter(M, mesh.extrow[F], t["ext"][F])
    R0 += _scatter(M, mesh.divrow[F], t["div"][F])
    x = np.asarray(x, dtype=np.float64)
    R0[mesh.ident_rows] = x[mesh.ident_rows] - mesh.bD[mesh.ident_rows]
    Rmu = _scatter(M, mesh.momrow[S], t["smu"][S])
    Rnu = _scatter(M, mesh.momrow[F], t["visc"][F])
    return R0, Rmu, Rnu


# ----------------------------------------------------------------------------
# Element Jacobians (Sec. 3.1 "The Jacobian matrices")
# ----------------------------------------------------------------------------


def element_jacobian_terms(mesh, x, rho=None, lam=None):
    """Element matrices of the derivatives of every term (rho, lam: override
    the problem's rho_f, lambda_s), indexed
    [c, a, i, b, k] = d(term for test (a, i)) / d(trial dof (b, k)).

      conv_vv : rho_f * (phi_b d_k v_i + delta_ik v . grad phi_b) phi_a      (J_rho)
      visc_vv : rho_f * (delta_ik grad phi_b . grad phi_a + d_i phi_b d_k phi_a)
      pres_vp : -xi_b d_i phi_a                       [c, a, i, b]
      div_pv  : d_k phi_b xi_a                        [c, a, b, k] (a = Q1 test)
      ext_uu  : delta_ik grad phi_b . grad phi_a
      smu_uu  : delta_ik gb.ga + d_i phi_b d_k phi_a + d_i phi_b (G_k . ga) + G_ki gb.ga
      slam_uu : lambda_s (d_k phi_b + G_k . grad phi_b) d_i phi_a            (J_lambda)
    with G = grad u, G_k the k-th row of G, ga = grad phi_a, gb = grad phi_b.
    """
    rho = mesh.prob.rho_f if rho is None else rho
    lam = mesh.prob.lam_s if lam is None else lam
    v, Gv, Gu, p = _qp_fields(mesh, x)
    w, N, dN, P = mesh.w, mesh.N, mesh.dN, mesh.P
    eye = np.eye(2)
    gg = np.einsum("aqj,bqj->qab", dN, dN)                              # grad phi_a . grad phi_b
    # convection: phi_b (d_k v_i) phi_a + delta_ik (v . grad phi_b) phi_a
    t1 = np.einsum("q,aq,bq,cqik->caibk", w, N, N, Gv)
    vgb = np.einsum("cqj,bqj->cqb", v, dN)
    t2 = np.einsum("q,aq,cqb,ik->caibk", w, N, vgb, eye)
    conv = rho * (t1 + t2)
    visc = rho * (np.einsum("q,qab,ik->aibk", w, gg, eye)
                  + np.einsum("q,bqi,aqk->aibk", w, dN, dN))
    pres = -np.einsum("q,bq,aqi->aib", w, P, dN)
    div = np.einsum("q,bqk,aq->abk", w, dN, P)
    ext = np.einsum("q,qab,ik->aibk", w, gg, eye)
    # solid mu-part: derivative of <G + G^T + G^T G, grad(phi_a e_i)>
    Gka = np.einsum("cqkj,aqj->cqka", Gu, dN)                           # G_k . grad phi_a
    smu = (np.einsum("q,qab,ik->aibk", w, gg, eye)[None]
           + np.einsum("q,bqi,aqk->aibk", w, dN, dN)[None]
           + np.einsum("q,bqi,cqka->caibk", w, dN, Gka)
           + np.einsum("q,cqki,qab->caibk", w, Gu, gg))
    Gkb = np.einsum("cqkj,bqj->cqkb", Gu, dN)                           # G_k . grad phi_b
    dtr = np.einsum("bqk,c->cqbk", dN, np.ones(mesh.ncell)) + np.swapaxes(Gkb, 2, 3)
    slam = lam * np.einsum("q,cqbk,aqi->caibk", w, dtr, dN)
    return dict(conv=conv, visc=visc, pres=pres, div=div, ext=ext, smu=smu, slam=slam)


class _COO:
    def __init__(self, M):
        self.M = M
        self.r, self.c, self.v = [], [], []

    def add(self, rows, cols, vals):
        rows, cols, vals = np.broadcast_arrays(rows, cols, vals)
        rows, cols, vals = rows.ravel(), cols.ravel(), vals.ravel()
        keep = rows >= 0
        self.r.append(rows[keep])
        self.c.append(cols[keep])
        self.v.append(vals[keep])

    def csr(self):
        if not self.r:
            return sp.csr_matrix((self.M, self.M))
        A = sp.coo_matrix((np.concatenate(self.v), (np.concatenate(self.r), np.concatenate(self.c))),
                          shape=(self.M, self.M)).tocsr()
        A.sum_duplicates()
        return A


def _add_block(coo, rows, cols, E):
    """Scatter element matrices E[c, ...rowshape, ...colshape] into COO."""
    nc = rows.shape[0]
    r = rows.reshape(nc, -1)
    c = cols.reshape(nc, -1)
    E = E.reshape(nc, r.shape[1], c.shape[1])
    coo.add(r[:, :, None], c[:, None, :], E)


def _bcast(E, nc):
    return E if E.shape[0] == nc and E.ndim == 5 else np.broadcast_to(E, (nc,) + E.shape)


def jacobian(mesh, x, mu, nu):
    """J(x; mu, nu) = dR/dx assembled directly (Sec. 3.2, Eq. (pardep_matrix1))."""
    t = element_jacobian_terms(mesh, x)
    F = np.flatnonzero(~mesh.cell_solid)
    S = np.flatnonzero(mesh.cell_solid)
    coo = _COO(mesh.M)
    nf = len(F)
    if nf:
        Jvv = t["conv"][F] + nu * _bcast(t["visc"], nf)
        _add_block(coo, mesh.momrow[F], mesh.vdof[F], Jvv)
        _add_block(coo, mesh.momrow[F], mesh.pdof[F], np.broadcast_to(t["pres"], (nf,) + t["pres"].shape))
        _add_block(coo, mesh.divrow[F], mesh.vdof[F], np.broadcast_to(t["div"], (nf,) + t["div"].shape))
        _add_block(coo, mesh.extrow[F], mesh.udof[F], np.broadcast_to(t["ext"], (nf,) + t["ext"].shape))
    if len(S):
        Juu = mu * t["smu"][S] + t["slam"][S]
        _add_block(coo, mesh.momrow[S], mesh.udof[S], Juu)
    d = mesh.ident_rows
    coo.add(d, d, np.ones(len(d)))
    return coo.csr()


def affine_jacobian(mesh, x):
    """(J0, Jmu', Jnu') with J(x; mu, nu) = J0 + mu Jmu' + nu Jnu'
    (Sec. 3, Eq. (pardep_matrix1) with mu_s = nu_f = 0: Jmu' = A1 + J_mu(x),
    Jnu' = rho_f A2, J0 = A0 + lambda_s J_lambda(x) + rho_f J_rho(x))."""
    t = element_jacobian_terms(mesh, x)
    F = np.flatnonzero(~mesh.cell_solid)
    S = np.flatnonzero(mesh.cell_solid)
    nf = len(F)
    J0, Jmu, Jnu = _COO(mesh.M), _COO(mesh.M), _COO(mesh.M)
    if nf:
        _add_block(J0, mesh.momrow[F], mesh.vdof[F], t["conv"][F])
        _add_block(J0, mesh.momrow[F], mesh.pdof[F], np.broadcast_to(t["pres"], (nf,) + t["pres"].shape))
        _add_block(J0, mesh.divrow[F], mesh.vdof[F], np.broadcast_to(t["div"], (nf,) + t["div"].shape))
        _add_block(J0, mesh.extrow[F], mesh.udof[F], np.broadcast_to(t["ext"], (nf,) + t["ext"].shape))
        _add_block(Jnu, mesh.momrow[F], mesh.vdof[F], np.broadcast_to(t["visc"], (nf,) + t["visc"].shape))
    if len(S):
        _add_block(J0, mesh.momrow[S], mesh.udof[S], t["slam"][S])
        _add_block(Jmu, mesh.momrow[S], mesh.udof[S], t["smu"][S])
    d = mesh.ident_rows
    J0.add(d, d, np.ones(len(d)))
    return J0.csr(), Jmu.csr(), Jnu.csr()


# ----------------------------------------------------------------------------
# Four parameters (Sec. 4.4, "Extension to further parameters"): mu_s, nu_f,
# lambda_s and rho_f all vary; nu_f enters as the product nu_f rho_f.
# ----------------------------------------------------------------------------


def residual4(mesh, x, mu, nu, lam, rho):
    """R(x; mu_s, nu_f, lambda_s, rho_f) assembled directly (Eq.
    (fsi_problem_weak1) with all four constants given)."""
    t = element_residual_terms(mesh, x, rho=rho, lam=lam)
    F, S = ~mesh.cell_solid, mesh.cell_solid
    mom = np.zeros_like(t["conv"])
    mom[F] = t["conv"][F] + t["pres"][F] + nu * t["visc"][F]
    mom[S] = mu * t["smu"][S] + t["slam"][S]
    R = _scatter(mesh.M, mesh.momrow, mom)
    R += _scatter(mesh.M, mesh.extrow[F], t["ext"][F])
    R += _scatter(mesh.M, mesh.divrow[F], t["div"][F])
    x = np.asarray(x, dtype=np.float64)
    R[mesh.ident_rows] = x[mesh.ident_rows] - mesh.bD[mesh.ident_rows]
    return R


def jacobian4(mesh, x, mu, nu, lam, rho):
    """J(x; mu_s, nu_f, lambda_s, rho_f) = dR/dx assembled directly (the
    Jacobian of Sec. 4.4 with its reference values cancelled)."""
    t = element_jacobian_terms(mesh, x, rho=rho, lam=lam)
    F = np.flatnonzero(~mesh.cell_solid)
    S = np.flatnonzero(mesh.cell_solid)
    coo = _COO(mesh.M)
    nf = len(F)
    if nf:
        _add_block(coo, mesh.momrow[F], mesh.vdof[F], t["conv"][F] + nu * _bcast(t["visc"], nf))
        _add_block(coo, mesh.momrow[F], mesh.pdof[F], np.broadcast_to(t["pres"], (nf,) + t["pres"].shape))
        _add_block(coo, mesh.divrow[F], mesh.vdof[F], np.broadcast_to(t["div"], (nf,) + t["div"].shape))
        _add_block(coo, mesh.extrow[F], mesh.udof[F], np.broadcast_to(t["ext"], (nf,) + t["ext"].shape))
    if len(S):
        _add_block(coo, mesh.momrow[S], mesh.udof[S], mu * t["smu"][S] + t["slam"][S])
    d = mesh.ident_rows
    coo.add(d, d, np.ones(len(d)))
    return coo.csr()


def affine_residual4(mesh, x):
    """(R0, Rmu, Rnurho, Rlam, Rrho) with R = R0 + mu Rmu + (nu rho) Rnurho +
    lam Rlam + rho Rrho (Sec. 4.4, the right-hand side B_k^{mu,nu,lambda,rho}
    with the reference values set to 0): Rmu = A1 x + g_mu(x), Rnurho = A2 x,
    Rlam = A3 x + g_lambda(x), Rrho = g_rho(x) (convection), R0 the rest
    (pressure, divergence, extension, Dirichlet rows x - b_D)."""
    t1 = element_residual_terms(mesh, x, rho=1.0, lam=1.0)
    F, S = ~mesh.cell_solid, mesh.cell_solid
    M = mesh.M
    R0 = _scatter(M, mesh.momrow[F], t1["pres"][F])
    R0 += _scatter(M, mesh.extrow[F], t1["ext"][F])
    R0 += _scatter(M, mesh.divrow[F], t1["div"][F])
    x = np.asarray(x, dtype=np.float64)
    R0[mesh.ident_rows] = x[mesh.ident_rows] - mesh.bD[mesh.ident_rows]
    Rmu = _scatter(M, mesh.momrow[S], t1["smu"][S])
    Rnurho = _scatter(M, mesh.momrow[F], t1["visc"][F])
    Rlam = _scatter(M, mesh.momrow[S], t1["slam"][S])
    Rrho = _scatter(M, mesh.momrow[F], t1["conv"][F])
    return R0, Rmu, Rnurho, Rlam, Rrho


def affine_jacobian4(mesh, x):
    """(J0, Jmu', Jnurho', Jlam', Jrho') with J = J0 + mu Jmu' + (nu rho)
    Jnurho' + lam Jlam' + rho Jrho' (Sec. 4.4, Eq. (matrix_fourpars1) with
    the reference values set to 0): Jmu' = A1 + J_mu(x), Jnurho' = A2,
    Jlam' = A3 + J_lambda(x), Jrho' = J_rho(x), J0 = A0."""
    t1 = element_jacobian_terms(mesh, x, rho=1.0, lam=1.0)
    F = np.flatnonzero(~mesh.cell_solid)
    S = np.flatnonzero(mesh.cell_solid)
    nf = len(F)
    J0, Jmu, Jnr, Jlam, Jrho = (_COO(mesh.M) for _ in range(5))
    if nf:
        _add_block(J0, mesh.momrow[F], mesh.pdof[F], np.broadcast_to(t1["pres"], (nf,) + t1["pres"].shape))
        _add_block(J0, mesh.divrow[F], mesh.vdof[F], np.broadcast_to(t1["div"], (nf,) + t1["div"].shape))
        _add_block(J0, mesh.extrow[F], mesh.udof[F], np.broadcast_to(t1["ext"], (nf,) + t1["ext"].shape))
        _add_block(Jnr, mesh.momrow[F], mesh.vdof[F], np.broadcast_to(t1["visc"], (nf,) + t1["visc"].shape))
        _add_block(Jrho, mesh.momrow[F], mesh.vdof[F], t1["conv"][F])
    if len(S):
        _add_block(Jmu, mesh.momrow[S], mesh.udof[S], t1["smu"][S])
        _add_block(Jlam, mesh.momrow[S], mesh.udof[S], t1["slam"][S])
    d = mesh.ident_rows
    J0.add(d, d, np.ones(len(d)))
    return J0.csr(), Jmu.csr(), Jnr.csr(), Jlam.csr(), Jrho.csr()


# ----------------------------------------------------------------------------
# Load vectors and error norms (manufactured-solution tests)
# ----------------------------------------------------------------------------


def load_vector(mesh, f_fluid_mom=None, f_solid_mom=None, f_ext=None, f_div=None,
                t_outflow=None):
    """Right-hand side of the weak form for manufactured solutions:
    int f . phi over the cells of each equation's domain, and the boundary
    traction int_{x = Lx} t . phi of the natural outflow condition.  Each f_*
    maps (X, Y) arrays to an array with trailing component axis (2) or a
    scalar array (f_div)."""
    M = mesh.M
    b = np.zeros(M)
    X, Y = mesh.qxy[..., 0], mesh.qxy[..., 1]
    w, N, P = mesh.w, mesh.N, mesh.P
    F, S = ~mesh.cell_solid, mesh.cell_solid
    if f_fluid_mom is not None:
        f = f_fluid_mom(X, Y)
        b += _scatter(M, mesh.momrow[F], np.einsum("q,cqi,aq->cai", w, f, N)[F])
    if f_solid_mom is not None:
        f = f_solid_mom(X, Y)
        b += _scatter(M, mesh.momrow[S], np.einsum("q,cqi,aq->cai", w, f, N)[S])
    if f_ext is not None:
        f = f_ext(X, Y)
        b += _scatter(M, mesh.extrow[F], np.einsum("q,cqi,aq->cai", w, f, N)[F])
    if f_div is not None:
        f = f_div(X, Y)
        b += _scatter(M, mesh.divrow[F], np.einsum("q,cq,bq->cb", w, f, P)[F])
    if t_outflow is not None:
        # cells of the last column, edge xi = 1; only nodes with ax = 2 are nonzero there
        t1, w1 = np.polynomial.legendre.leggauss(5)
        t1, w1 = 0.5 * (t1 + 1), 0.5 * w1 * mesh.hy
        ly, _ = _lagrange2(t1)
        cells = np.flatnonzero((mesh.cell_ij[:, 0] == mesh.nx - 1) & F)
        for c in cells:
            y = mesh.cell_origin[c, 1] + t1 * mesh.hy
            tr = t_outflow(np.full_like(y, mesh.prob.Lx), y)                # (q, 2)
            for ay in range(3):
                a = 2 + 3 * ay
                for i in range(2):
                    r = mesh.momrow[c, a, i]
                    if r >= 0:
                        b[r] += np.sum(w1 * tr[:, i] * ly[ay])
    return b


def interpolate(mesh, fields):
    """Nodal interpolant: ``fields`` maps name in {vx, vy, ux, uy, p} to a
    function of (X, Y)."""
    x = np.zeros(mesh.M)
    X, Y = mesh.node_xy[:, 0], mesh.node_xy[:, 1]
    for f, name in enumerate(("vx", "vy", "ux", "uy")):
        if name in fields:
            x[f * mesh.NQ2:(f + 1) * mesh.NQ2] = fields[name](X, Y)
    if "p" in fields:
        vx = np.arange(mesh.NQ1) % (mesh.nx + 1) * mesh.hx
        vy = np.arange(mesh.NQ1) // (mesh.nx + 1) * mesh.hy
        x[4 * mesh.NQ2:] = fields["p"](vx, vy)
    return x


def l2_error(mesh, x, field, exact, cells=None, npts=5):
    """|| field_h - exact ||_L2 over the given cells with an npts x npts Gauss rule."""
    tx, ty, wq = gauss_2d(npts)
    N, _, P = reference_basis(tx, ty)
    cells = np.arange(mesh.ncell) if cells is None else np.asarray(cells)
    qx = mesh.cell_origin[cells, 0:1] + tx[None] * mesh.hx
    qy = mesh.cell_origin[cells, 1:2] + ty[None] * mesh.hy
    x = np.asarray(x)
    if field == "p":
        vals = np.einsum("cb,bq->cq", x[mesh.pdof[cells]], P)
    else:
        f = ("vx", "vy", "ux", "uy").index(field)
        vals = np.einsum("ca,aq->cq", x[f * mesh.NQ2 + mesh.cell_nodes[cells]], N)
    err = vals - exact(qx, qy)
    return float(np.sqrt(np.sum(err ** 2 * wq[None] * mesh.hx * mesh.hy)))
