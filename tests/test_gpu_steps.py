"""The exported single steps against the oracle, through the C ABI, and the
truncated solvers at the benchmark's truncation settings.

* lrfsi_precond_apply: P_k^{-1} X for the mean-based preconditioner
  (Sec. 4.2) vs a sparse direct solve of the oracle's P_k (scipy splu), on
  the 20 x 4 and 80 x 16 meshes, two uneven subsets.  Two backward-stable
  solvers agree only to about cond(P_k) eps (P_k mixes unit Dirichlet rows
  with solid rows of size mu ~ 1e6), so the test checks the backward error of
  the GPU solution, ||P y - x||_inf / (||P||_inf ||y||_inf + ||x||_inf) <=
  1e-12, and the forward agreement with splu to max(1e-10, 20 cond_1(P) eps)
  per column, cond_1 estimated with onenormest on the splu factors.
* lrfsi_truncate: T (Sec. 5, the best rank-<= R approximation) vs the oracle's
  SVD truncation on factors with a known, well-separated spectrum; the kept
  product to 1e-12 of the largest singular value, the same rank, U
  orthonormal.
* lrfsi_residual: relative residuals of x~ 1^T + U V^T (Sec. 5.1.2) vs the
  oracle's column-by-column definition; 1e-10 relative.
* ChebyshevT and GMREST with truncation that decides the result (tol 1e-8,
  rank cap below m_k, as in the benchmark) vs the oracle's truncated solvers,
  element by element.  Truncation is only well-defined where the kept and
  dropped singular values are separated; the oracle records every
  truncation's relative gap (s_r - s_{r+1}) / s_r and the test requires it to
  be >= 1e-6 (the cases are chosen so that it is).  With such gaps a
  perturbation of one ulp moves a truncated subspace by at most ~1e-10, so
  the bar is 1e-8 per column relative to the largest column.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import algorithm1, fsi, lowrank, newton, params  # noqa: E402
from paper_2008_10275_gb300 import build, lrfsi  # noqa: E402
from tests.gpu_common import perm_lib_to_oracle  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _two_subsets(nx, ny, sizes=(7, 12), seed=4):
    lm = lrfsi.Mesh(nx, ny)
    om = fsi.Mesh(fsi.Problem(nx, ny))
    perm = perm_lib_to_oracle(lm, om)
    rng = np.random.default_rng(seed)
    subs = []
    for k, m in enumerate(sizes):
        mu = np.sort(rng.uniform(6e5 + 3e5 * k, 9e5 + 3e5 * k, m))
        nu = rng.uniform(2.5e-3, 3.5e-3, m)
        med = params.upper_median_position(m)
        xt, _, _ = newton.newton(om, mu[med], nu[med], eps=1e-10)
        subs.append((mu, nu, xt))
    return lm, om, perm, subs


@pytest.mark.parametrize("lu_mode", [1, 0])
@pytest.mark.parametrize("nx,ny", [(20, 4), (80, 16)])
def test_precond_apply_matches_sparse_direct_solve(nx, ny, lu_mode):
    prev = lrfsi.lu_mode(lu_mode)
    try:
        _precond_case(nx, ny)
    finally:
        lrfsi.lu_mode(prev)


@pytest.mark.parametrize("lu_mode", [1, 0])
def test_newton_median_both_lu_modes(lu_mode):
    """The batched median Newton with either sparse LU reaches the oracle's
    Newton solution (1e-9) in the same number of steps."""
    prev = lrfsi.lu_mode(lu_mode)
    try:
        lm = lrfsi.Mesh(20, 4)
        om = fsi.Mesh(fsi.Problem(20, 4))
        perm = perm_lib_to_oracle(lm, om)
        mus, nus = np.array([5e5, 1.3e6, 2e6]), np.array([1e-3, 3e-3, 5e-3])
        X = _dev(np.tile(om.bD[perm], (3, 1)))
        it, res, st = lrfsi.lrfsi_newton_median(lm, X, mus, nus, 1e-10, 30)
        Xh = X.cpu().numpy()
        for k in range(3):
            xo, ito, _ = newton.newton(om, mus[k], nus[k], eps=1e-10)
            assert res[k] <= 1e-10
            assert np.abs(Xh[k] - xo[perm]).max() <= 1e-9 * np.abs(xo).max()
            assert abs(int(it[k]) - ito) <= 1
    finally:
        lrfsi.lu_mode(prev)


@pytest.mark.parametrize("nx,ny", [(20, 4), (80, 16)])
def test_precond_apply_tensor_core_sweeps(nx, ny):
    """With >= 8 right-hand sides the sweeps of the nested-dissection solve run
    their large GEMMs on the tensor cores (fixed factor blocks sliced once per
    factorisation); the same handle with the FP64 sweeps (path 0) and with the
    tensor sweeps meets the same bars against splu, and the two agree to the
    forward bar."""
    prev_lu, prev_path = lrfsi.lu_mode(1), lrfsi.gram_path(1)
    try:
        Y1 = _precond_case(nx, ny, r=(20, 13), ld=24, paths=(1, 0))
        assert np.all(np.isfinite(Y1))
    finally:
        lrfsi.lu_mode(prev_lu)
        lrfsi.gram_path(prev_path)


def _precond_case(nx, ny, r=(5, 3), ld=6, paths=(None,)):
    lm, om, perm, subs = _two_subsets(nx, ny)
    K = len(subs)
    mu = np.concatenate([s[0] for s in subs])
    nu = np.concatenate([s[1] for s in subs])
    xt = _dev(np.stack([s[2][perm] for s in subs]))
    sizes = [len(s[0]) for s in subs]
    sub = lrfsi.Subsets(lm, xt, mu, nu, sizes, [8, 8])
    r = list(r)
    rng = np.random.default_rng(9)
    Xh = rng.standard_normal((K, lm.M, ld))
    outs = []
    for path in paths:
        if path is not None:
            lrfsi.gram_path(path)
        Y = torch.zeros(K * lm.M * ld, dtype=torch.float64, device=DEV)
        lrfsi.lrfsi_precond_apply(sub, _dev(Xh.reshape(-1)), ld, r, Y, ld)
        outs.append(Y.cpu().numpy().reshape(K, lm.M, ld))
    Yh = outs[0]
    inv = np.argsort(perm)
    for k, (mu_k, nu_k, xt_k) in enumerate(subs):
        J0, Jmu, Jnu = fsi.affine_jacobian(om, xt_k)
        mb, nb = params.midpoint_parameters(mu_k, nu_k)
        P = lowrank.preconditioner(J0, Jmu, Jnu, mb, nb)
        xk = np.ascontiguousarray(Xh[k][:, :r[k]][inv])
        ref = P.solve(xk)
        A = (J0 + mb * Jmu + nb * Jnu).tocsr()
        Pinv = spla.LinearOperator(A.shape, matvec=P.solve, rmatvec=lambda v: P.solve(v, trans="T"))
        cond1 = spla.norm(A, 1) * spla.onenormest(Pinv)
        fwd_tol = max(1e-10, 20 * cond1 * np.finfo(float).eps)
        Anorm = spla.norm(A, np.inf)
        for Yo in outs:
            for j in range(r[k]):
                y = Yo[k][:, j][inv]
                back = np.abs(A @ y - xk[:, j]).max() / (Anorm * np.abs(y).max() + np.abs(xk[:, j]).max())
                assert back <= 1e-12, (k, j, back)
                err = np.linalg.norm(y - ref[:, j]) / np.linalg.norm(ref[:, j])
                assert err <= fwd_tol, (k, j, err, cond1)
        for Yo in outs[1:]:
            for j in range(r[k]):
                d = np.linalg.norm(Yo[k][:, j] - Yh[k][:, j]) / np.linalg.norm(Yh[k][:, j])
                assert d <= fwd_tol, (k, j, d)
    sub.close()
    return Yh


@pytest.mark.parametrize("tol", [3e-2, 1e-12])
def test_truncate_matches_svd_truncation(tol):
    """lrfsi_truncate on mixed (non-orthonormal) factors against the exact SVD
    truncation of their product.  Two error sources are allowed:
    * the Cholesky-QR representation X = Q R reproduces X V^T to about
      eps cond(X) |X| |V| (cond(X) ~ 1e5 here);
    * the Jacobi SVD leaves columns below 1e-2 tol of the largest unrotated
      (they lie below what the truncation keeps): the kept part can move by
      up to 1e-2 tol sqrt(n) sigma_1.
    tol = 3e-2 cuts subset 0 by the tolerance and subset 1 by the cap;
    tol = 1e-12 lets the caps cut both, where only the first source counts."""
    lm, om, perm, subs = _two_subsets(20, 4)
    mu = np.concatenate([s[0] for s in subs])
    nu = np.concatenate([s[1] for s in subs])
    xt = _dev(np.stack([s[2][perm] for s in subs]))
    sizes = [len(s[0]) for s in subs]
    caps = [6, 3]
    sub = lrfsi.Subsets(lm, xt, mu, nu, sizes, caps)
    rng = np.random.default_rng(2)
    p = [7, 10]
    ld = 10
    X = np.zeros((2, lm.M, ld))
    V = np.zeros((sum(sizes), ld))
    expect, bound = [], []
    eps = np.finfo(float).eps
    # spectra 10^(-j/2) (gaps of 3.2x)
    for k, m in enumerate(sizes):
        A, _ = np.linalg.qr(rng.standard_normal((lm.M, p[k])))
        Bm, _ = np.linalg.qr(rng.standard_normal((m, min(p[k], m))))
        n = min(p[k], m)
        s = 10.0 ** (-np.arange(n) / 2)
        Xk = A[:, :n] * s
        # mix the factors (X_k V_k^T is the same product, the factors are not
        # orthonormal): an orthogonal matrix times singular values in [1/2, 2]
        Qg, _ = np.linalg.qr(rng.standard_normal((p[k], p[k])))
        G = np.diag(np.geomspace(0.5, 2.0, n)) @ Qg[:n]
        Xm = Xk @ G
        Vm = Bm @ np.linalg.pinv(G).T
        X[k, :, :p[k]] = Xm
        o = sum(sizes[:k])
        V[o:o + m, :p[k]] = Vm
        expect.append(Xk @ Bm.T)
        bound.append(100 * eps * np.linalg.cond(Xm) * np.linalg.norm(Xm, 2) * np.linalg.norm(Vm, 2)
                     + 1e-2 * tol * np.sqrt(n) * s[0])
    ldo = 9
    U = torch.zeros(2 * lm.M * ldo, dtype=torch.float64, device=DEV)
    Vo = torch.zeros(sum(sizes) * ldo, dtype=torch.float64, device=DEV)
    Xd, Vd = _dev(X.reshape(-1)), _dev(V)   # kept alive across the call
    # the binding keeps the p and cap arrays alive during the call (a bare
    # np.array(...).ctypes.data temporary is freed before the library reads it)
    ranks = lrfsi.lrfsi_truncate(sub, Xd, ld, Vd, ld, p, tol, caps, U, ldo, Vo, ldo)
    Uh = U.cpu().numpy().reshape(2, lm.M, ldo)
    Vh = Vo.cpu().numpy().reshape(sum(sizes), ldo)
    for k, m in enumerate(sizes):
        P = expect[k]
        ref = lowrank.truncate(P, tol, caps[k])
        sv = np.linalg.svd(P, compute_uv=False)
        r_ref = lowrank.truncation_rank(sv, tol, caps[k])
        o = sum(sizes[:k])
        Uk = Uh[k][:, :ranks[k]]
        got = Uk @ Vh[o:o + m, :ranks[k]].T
        assert ranks[k] == r_ref, (k, ranks[k], r_ref, np.linalg.svd(got, compute_uv=False), sv)
        assert np.abs(got - ref).max() <= bound[k], (k, np.abs(got - ref).max(), bound[k])
        assert np.abs(Uk.T @ Uk - np.eye(ranks[k])).max() <= 1e-12
    sub.close()


def test_residual_entry_point_matches_oracle():
    lm, om, perm, subs = _two_subsets(20, 4, sizes=(9,))
    mu, nu, xt = subs[0]
    m = len(mu)
    rng = np.random.default_rng(3)
    r, ld = 4, 5
    Uh = np.zeros((lm.M, ld))
    Uh[:, :r] = 1e-3 * rng.standard_normal((lm.M, r)) * np.abs(om.bD[perm]).max()
    Vh = np.zeros((m, ld))
    Vh[:, :r] = rng.standard_normal((m, r))
    rel = lrfsi.lrfsi_residual(lm, _dev(xt[perm]), _dev(Uh), ld, _dev(Vh), ld, r, _dev(mu), _dev(nu), m)
    inv = np.argsort(perm)
    X = (xt[perm][:, None] + Uh[:, :r] @ Vh[:, :r].T)[inv]
    ref = algorithm1.relative_residuals(om, X, mu, nu)
    assert np.allclose(rel, ref, rtol=1e-10, atol=0.0), (rel, ref)
    # r = 0: the median solution for every column
    rel0 = lrfsi.lrfsi_residual(lm, _dev(xt[perm]), _dev(Uh), ld, _dev(Vh), ld, 0, _dev(mu), _dev(nu), m)
    ref0 = algorithm1.relative_residuals(om, np.repeat(xt[:, None], m, 1), mu, nu)
    # the median column's residual is at rounding level (~1e-13): compared absolutely
    assert np.allclose(rel0, ref0, rtol=1e-10, atol=1e-10)


def _recording_truncate(gaps):
    orig = lowrank.truncate

    def T(X, tol, cap):
        s = np.linalg.svd(X, compute_uv=False)
        r = lowrank.truncation_rank(s, tol, cap)
        if 0 < r < len(s) and s[r - 1] > 0:
            gaps.append((s[r - 1] - s[r]) / s[r - 1])
        return orig(X, tol, cap)
    return T


@pytest.mark.parametrize("solver", ["chebyshev", "gmres"])
def test_truncated_solver_parity_at_benchmark_settings(monkeypatch, solver):
    lm, om, perm, subs = _two_subsets(20, 4, sizes=(24,), seed=11)
    mu, nu, xt = subs[0]
    m = len(mu)
    cap, tol, c, d = 10, 1e-8, 0.65, 1.0
    J0, Jmu, Jnu = fsi.affine_jacobian(om, xt)
    R0, Rmu, Rnu = fsi.affine_residual(om, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu, nu)
    mb, nb = params.midpoint_parameters(mu, nu)
    gaps = []
    monkeypatch.setattr(lowrank, "truncate", _recording_truncate(gaps))
    kw = dict(iters=6, cycles=2, tol=tol, rank_cap=cap)
    if solver == "gmres":
        So = lowrank.gmres_T_scaled(J0, Jmu, Jnu, B, mu, nu, mb, nb, **kw)
    else:
        So = lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mu, nu, mb, nb, c, d, **kw)
    So = So[perm]
    assert gaps and min(gaps) >= 1e-6, min(gaps)
    sub = lrfsi.Subsets(lm, _dev(xt[perm]), mu, nu, [m], [cap])
    UB = _dev(np.stack([R0, Rmu, Rnu], 1)[perm])
    VB = _dev(-np.stack([np.ones(m), mu, nu], 1))
    U = torch.zeros(lm.M * cap, dtype=torch.float64, device=DEV)
    V = torch.zeros(m * cap, dtype=torch.float64, device=DEV)
    opt = lrfsi.cheb_options(c, d, iters=6, cycles=2, rank_cap=cap, tol=tol, solver=solver)
    fn = lrfsi.lrfsi_gmresT if solver == "gmres" else lrfsi.lrfsi_chebyshevT
    ranks, _ = fn(sub, UB, 3, VB, 3, [3], opt, U, cap, V, cap)
    r = int(ranks[0])
    S = U.cpu().numpy().reshape(lm.M, cap)[:, :r] @ V.cpu().numpy().reshape(m, cap)[:, :r].T
    scale = np.linalg.norm(So, axis=0).max()
    errs = [np.linalg.norm(S[:, j] - So[:, j]) / scale for j in range(m)]
    assert max(errs) <= 1e-8, (solver, max(errs), min(gaps))
    sub.close()


def test_error_paths_reported_not_trapped():
    lm = lrfsi.Mesh(20, 4)
    bD = torch.tensor(lm.dirichlet(), dtype=torch.float64, device=DEV)
    # host parameters that are not finite: rejected before any launch
    X = bD.repeat(2, 1)
    for bad in (np.nan, np.inf):
        with pytest.raises(lrfsi.LrfsiError) as e:
            lrfsi.lrfsi_newton_median(lm, X, np.array([7e5, bad]), np.array([3e-3, 3e-3]), 1e-8, 5)
        assert e.value.code == lrfsi.EINVAL
        with pytest.raises(lrfsi.LrfsiError) as e:
            lrfsi.Subsets(lm, X, np.array([7e5, 8e5, bad]), np.full(3, 3e-3), [3], [3])
        assert e.value.code == lrfsi.EINVAL
    # Newton limit: one step from b_D cannot reach 1e-12
    X = bD.repeat(1, 1)
    it, res, st = lrfsi.lrfsi_newton_median(lm, X, np.array([7e5]), np.array([3e-3]), 1e-12, 1, allow_noconv=True)
    assert st == lrfsi.ENOCONV and it[0] == 1 and np.isfinite(res[0])
    # a NaN state: the LU pivot search flags the NaN pivot as singular
    Xn = torch.full((1, lm.M), float("nan"), dtype=torch.float64, device=DEV)
    with pytest.raises(lrfsi.LrfsiError) as e:
        lrfsi.Subsets(lm, Xn, np.array([7e5, 8e5]), np.full(2, 3e-3), [2], [2])
    assert e.value.code == lrfsi.ESINGULAR
    # the context stays usable: a normal call afterwards succeeds
    it, res, st = lrfsi.lrfsi_newton_median(lm, X, np.array([7e5]), np.array([3e-3]), 1e-8, 30)
    assert st == 0 and res[0] <= 1e-8
