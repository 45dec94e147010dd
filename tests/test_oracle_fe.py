"""Pins of the oracle's finite element residual and Jacobian (CPU only).

What pins what:
* manufactured solutions (sympy derives the strong-form sources from the
  weak form of Sec. 2, Eq. (fsi_problem_weak1)) on three meshes: Q2 fields
  converge like h^3 and the Q1 pressure like h^2 in L2 -- a dropped term, a
  wrong sign, index or coefficient breaks the rates;
* central finite differences reproduce J dx to rounding (the residual is a
  quadratic polynomial in x, so the central difference is exact);
* the affine split J0 + mu Jmu' + nu Jnu' = J(x; mu, nu) and R0 + mu Rmu +
  nu Rnu = R(x; mu, nu) to 1e-13 (Eq. (pardep_matrix1));
* A1 (<grad u + grad u^T, grad phi>_S), A2 and the extension block are
  symmetric on their row/column sets, J_rho vanishes for v = 0, J_mu and
  J_lambda vanish for u = 0 (Sec. 3.1);
* DOF counts of the channel meshes and the Dirichlet profile's mean.
"""
import numpy as np
import pytest
import sympy as sy

from oracle import fsi, newton


def _rate(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def _sym_fluid(nu, rho):
    X, Y = sy.symbols("X Y")
    psi = sy.Rational(1, 10) * sy.sin(2 * X) * sy.cos(3 * Y) + sy.Rational(1, 5) * Y ** 2 * (1 + X / 4)
    vx, vy = sy.diff(psi, Y), -sy.diff(psi, X)
    p = sy.cos(X) * sy.sin(2 * Y) + X / 3
    ux = sy.Rational(1, 100) * sy.sin(X + 1) * sy.cos(5 * Y)
    uy = sy.Rational(1, 100) * sy.exp(X / 2) * sy.sin(3 * Y + 1)
    v = [vx, vy]
    G = [[sy.diff(v[i], [X, Y][j]) for j in range(2)] for i in range(2)]
    sig = [[nu * rho * (G[i][j] + G[j][i]) - (p if i == j else 0) for j in range(2)] for i in range(2)]
    f = [rho * sum(v[j] * G[i][j] for j in range(2)) - sum(sy.diff(sig[i][j], [X, Y][j]) for j in range(2))
         for i in range(2)]
    fext = [-(sy.diff(ux, X, 2) + sy.diff(ux, Y, 2)), -(sy.diff(uy, X, 2) + sy.diff(uy, Y, 2))]
    trac = [sig[0][0], sig[1][0]]                       # sigma n with n = e_x at the outflow
    lam = lambda e: sy.lambdify((X, Y), e, "numpy")
    vec = lambda es: (lambda x, y: np.stack([np.broadcast_to(lam(e)(x, y), np.shape(x)) for e in es], axis=-1))
    return dict(vx=lam(vx), vy=lam(vy), p=lam(p), ux=lam(ux), uy=lam(uy),
                f=vec(f), fext=vec(fext), trac=vec(trac))


def _sym_solid(mu, lam_s):
    X, Y = sy.symbols("X Y")
    ux = sy.Rational(3, 100) * sy.sin(2 * X + 1) * sy.cos(3 * Y)
    uy = sy.Rational(2, 100) * sy.cos(X) * sy.sin(4 * Y + 1)
    u = [ux, uy]
    G = [[sy.diff(u[i], [X, Y][j]) for j in range(2)] for i in range(2)]
    GtG = [[sum(G[k][i] * G[k][j] for k in range(2)) for j in range(2)] for i in range(2)]
    tr = G[0][0] + G[1][1] + sy.Rational(1, 2) * (GtG[0][0] + GtG[1][1])
    sig = [[mu * (G[i][j] + G[j][i] + GtG[i][j]) + (lam_s * tr if i == j else 0) for j in range(2)]
           for i in range(2)]
    f = [-sum(sy.diff(sig[i][j], [X, Y][j]) for j in range(2)) for i in range(2)]
    lam = lambda e: sy.lambdify((X, Y), e, "numpy")
    vec = lambda es: (lambda x, y: np.stack([np.broadcast_to(lam(e)(x, y), np.shape(x)) for e in es], axis=-1))
    return dict(ux=lam(ux), uy=lam(uy), f=vec(f))


def test_mms_navier_stokes_and_extension_rates():
    nu, rho = 0.1, 1.0
    s = _sym_fluid(nu, rho)
    errs = {k: [] for k in ("vx", "vy", "p", "ux", "uy")}
    for k in (2, 4, 8):
        prob = fsi.Problem(5 * k, k, flap=None, rho_f=rho, lam_s=0.0)
        m0 = fsi.Mesh(prob)
        bD = fsi.interpolate(m0, dict(vx=s["vx"], vy=s["vy"], ux=s["ux"], uy=s["uy"]))
        m = fsi.Mesh(prob, bD=bD)
        src = fsi.load_vector(m, f_fluid_mom=s["f"], f_ext=s["fext"], t_outflow=s["trac"])
        x, it, r = newton.newton(m, 1.0, nu, x0=bD, eps=1e-11, source=src)
        assert r < 1e-10
        for f in errs:
            errs[f].append(fsi.l2_error(m, x, f, s[f]))
    for f in ("vx", "vy", "ux", "uy"):
        assert min(_rate(errs[f])) > 2.7, (f, errs[f])
    assert min(_rate(errs["p"])) > 1.8, errs["p"]


def test_mms_nonlinear_solid_rates():
    mu, lam_s = 1.0, 2.0
    s = _sym_solid(mu, lam_s)
    errs = {"ux": [], "uy": []}
    for k in (2, 4, 8):
        prob = fsi.Problem(5 * k, k, all_solid=True, lam_s=lam_s)
        m0 = fsi.Mesh(prob)
        bD = fsi.interpolate(m0, dict(ux=s["ux"], uy=s["uy"]))
        m = fsi.Mesh(prob, bD=bD)
        src = fsi.load_vector(m, f_solid_mom=s["f"])
        x, it, r = newton.newton(m, mu, 0.0, x0=bD, eps=1e-12, source=src)
        assert r < 1e-11
        for f in errs:
            errs[f].append(fsi.l2_error(m, x, f, s[f]))
    for f in errs:
        assert min(_rate(errs[f])) > 2.7, (f, errs[f])


def _scaled_random(m, rng, amp=1.0):
    sc = np.r_[np.full(2 * m.NQ2, 0.3), np.full(2 * m.NQ2, 1e-3), np.full(m.NQ1, 50.0)]
    return amp * sc * rng.standard_normal(m.M)


@pytest.mark.parametrize("nx,ny", [(20, 4), (10, 2)])
def test_central_difference_reproduces_jacobian(nx, ny):
    m = fsi.Mesh(fsi.Problem(nx, ny))
    rng = np.random.default_rng(1)
    x = m.bD + _scaled_random(m, rng)
    dx = _scaled_random(m, rng)
    for mu, nu in ((5e5, 1e-3), (2e6, 5e-3)):
        J = fsi.jacobian(m, x, mu, nu)
        Jd = J @ dx
        fd = (fsi.residual(m, x + dx, mu, nu) - fsi.residual(m, x - dx, mu, nu)) / 2.0
        assert np.linalg.norm(fd - Jd) <= 1e-12 * np.linalg.norm(Jd)
        # the residual is genuinely nonlinear: the second difference is not zero
        sd = fsi.residual(m, x + dx, mu, nu) + fsi.residual(m, x - dx, mu, nu) - 2 * fsi.residual(m, x, mu, nu)
        assert np.linalg.norm(sd) > 1e-6 * np.linalg.norm(Jd)


def test_affine_split_reproduces_direct_assembly():
    m = fsi.Mesh(fsi.Problem(20, 4))
    rng = np.random.default_rng(2)
    x = m.bD + _scaled_random(m, rng)
    J0, Jmu, Jnu = fsi.affine_jacobian(m, x)
    R0, Rmu, Rnu = fsi.affine_residual(m, x)
    for mu, nu in ((5e5, 1e-3), (1.3e6, 2.2e-3), (2e6, 5e-3)):
        J = fsi.jacobian(m, x, mu, nu)
        D = (J0 + mu * Jmu + nu * Jnu - J)
        assert abs(D).max() <= 1e-13 * abs(J).max()
        R = fsi.residual(m, x, mu, nu)
        assert np.linalg.norm(R0 + mu * Rmu + nu * Rnu - R) <= 1e-13 * np.linalg.norm(R)
    # Jnu' does not depend on x; Rmu, Rnu vanish in Dirichlet rows
    J0b, Jmub, Jnub = fsi.affine_jacobian(m, m.bD)
    assert abs(Jnub - Jnu).max() == 0.0
    assert np.all(Rmu[m.ident_rows] == 0) and np.all(Rnu[m.ident_rows] == 0)


def test_operator_symmetries_and_vanishing_nonlinear_parts():
    m = fsi.Mesh(fsi.Problem(20, 4))
    # At u = 0 the solid Jacobian J_mu' equals A1 (symmetric on the solid u-rows/cols),
    # and with v = 0 the convection Jacobian vanishes; Jnu' = rho_f A2 is symmetric on fluid v-dofs.
    x0 = np.zeros(m.M)
    J0, Jmu, Jnu = fsi.affine_jacobian(m, x0)
    r = np.unique(m.momrow[m.cell_solid].ravel())
    r = r[r >= 0]
    A1 = Jmu[r][:, r].toarray()
    assert np.allclose(A1, A1.T, atol=1e-12 * abs(A1).max())
    v_rows = np.unique(m.momrow[~m.cell_solid].ravel())
    v_rows = v_rows[(v_rows >= 0) & (v_rows < 2 * m.NQ2)]
    A2 = Jnu[v_rows][:, v_rows].toarray()
    assert np.allclose(A2, A2.T, atol=1e-12 * abs(A2).max())
    e = np.unique(m.extrow.ravel())
    e = e[e >= 0]
    E = J0[e][:, e].toarray()
    assert np.allclose(E, E.T, atol=1e-12 * abs(E).max())
    # convection Jacobian vanishes at v = 0: J0 at x = 0 equals J0 at x with only u/p set
    rng = np.random.default_rng(3)
    xu = np.zeros(m.M)
    xu[2 * m.NQ2:] = _scaled_random(m, rng)[2 * m.NQ2:]
    J0u, Jmuu, _ = fsi.affine_jacobian(m, xu)
    xv = np.zeros(m.M)
    xv[:2 * m.NQ2] = _scaled_random(m, rng)[:2 * m.NQ2]
    J0v, Jmuv, _ = fsi.affine_jacobian(m, xv)
    assert abs(Jmuv - Jmu).max() == 0.0                    # J_mu depends on u only
    fl = np.setdiff1d(np.unique(m.momrow[~m.cell_solid].ravel()), m.momrow[m.cell_solid].ravel())
    fl = fl[fl >= 0]                                       # rows reached by fluid cells only
    assert abs((J0u - J0)[fl]).max() == 0.0               # J_rho depends on v only
    assert abs((J0v - J0)[fl]).max() > 0.0


def test_dof_counts_and_inflow_profile():
    for (nx, ny), M in (((20, 4), 1581), ((80, 16), 22629), ((320, 64), 351621)):
        prob = fsi.Problem(nx, ny)
        NQ2 = (2 * nx + 1) * (2 * ny + 1)
        NQ1 = (nx + 1) * (ny + 1)
        assert 4 * NQ2 + NQ1 == M
    m = fsi.Mesh(fsi.Problem(80, 16))
    assert m.M == 22629
    assert m.cell_solid.sum() == 4 * 8                     # flap [0.6,0.7]x[0,0.2] is 4 x 8 cells
    y = m.node_xy[m.inflow, 1]
    vin = m.bD[np.flatnonzero(m.inflow)]
    # Simpson on the Q2 node column integrates the parabola exactly: mean = 0.2
    h = y[1] - y[0]
    w = np.ones(len(y)); w[1:-1:2] = 4; w[2:-1:2] = 2
    assert abs(np.sum(w * vin) * h / 3 / 0.4 - 0.2) < 1e-14
