"""CUDA path vs the oracle, element by element, through the C ABI.

Tolerances: assembly and residuals are sums of the same quadrature terms in a
different order, so they agree to a few ulps of the largest entry (1e-12
relative to the max-norm); solves and iterations are compared at 1e-10
relative per column (FP64 path), converged Newton solutions at 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import algorithm1, fsi, lowrank, newton, params  # noqa: E402
from paper_2008_10275_gb300 import build, inputs, lrfsi  # noqa: E402
from tests.gpu_common import lib_csr, perm_lib_to_oracle, rel_max  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


def _meshes(nx, ny):
    lm = lrfsi.Mesh(nx, ny)
    om = fsi.Mesh(fsi.Problem(nx, ny))
    perm = perm_lib_to_oracle(lm, om)
    return lm, om, perm


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("nx,ny", [(20, 4), (10, 2), (40, 8)])
def test_mesh_layout_matches_oracle(nx, ny):
    lm, om, perm = _meshes(nx, ny)
    assert lm.M == om.M
    assert np.array_equal(lm.dirichlet(), om.bD[perm])
    assert lm.nsolid == int(om.cell_solid.sum())


@pytest.mark.parametrize("nx,ny,seed", [(20, 4, 0), (40, 8, 1)])
def test_affine_assembly_parity(nx, ny, seed):
    lm, om, perm = _meshes(nx, ny)
    x = om.bD + inputs.random_state(om.M, seed, nq2=om.NQ2)
    xl = _dev(x[perm])
    J3 = torch.zeros(lm.nnz * 3, dtype=torch.float64, device=DEV)
    R3 = torch.zeros(lm.M * 3, dtype=torch.float64, device=DEV)
    lrfsi.lrfsi_assemble_affine(lm, xl, J3, R3)
    torch.cuda.synchronize()
    J3 = J3.cpu().numpy().reshape(-1, 3)
    R3 = R3.cpu().numpy().reshape(-1, 3)
    oJ = fsi.affine_jacobian(om, x)
    oR = fsi.affine_residual(om, x)
    for t in range(3):
        A = oJ[t][perm][:, perm].toarray()
        B = lib_csr(lm, J3[:, t]).toarray()
        assert rel_max(B, A) <= 1e-12, t
        assert rel_max(R3[:, t], oR[t][perm]) <= 1e-12, t


def test_residual_batch_parity_and_norms():
    lm, om, perm = _meshes(20, 4)
    rng = np.random.default_rng(5)
    m = 7
    X = np.stack([om.bD + inputs.random_state(om.M, 10 + j, nq2=om.NQ2) for j in range(m)], 1)
    mu = rng.uniform(*inputs.MU_RANGE, m)
    nu = rng.uniform(*inputs.NU_RANGE, m)
    Xl = _dev(X[perm])
    R = torch.zeros(lm.M * m, dtype=torch.float64, device=DEV)
    n2 = torch.zeros(m, dtype=torch.float64, device=DEV)
    lrfsi.lrfsi_residual_batch(lm, Xl, m, m, _dev(mu), _dev(nu), R, m, n2)
    R = R.cpu().numpy().reshape(lm.M, m)
    for j in range(m):
        ref = fsi.residual(om, X[:, j], mu[j], nu[j])
        assert rel_max(R[:, j], ref[perm]) <= 1e-12
        assert abs(n2[j].item() - np.dot(ref, ref)) <= 1e-12 * np.dot(ref, ref)


def test_newton_median_parity_batched():
    lm, om, perm = _meshes(20, 4)
    mus = np.array([5e5, 1.3e6, 2e6])
    nus = np.array([1e-3, 3e-3, 5e-3])
    K = len(mus)
    X = _dev(np.tile(om.bD[perm], (K, 1)))
    it, res, st = lrfsi.lrfsi_newton_median(lm, X, mus, nus, 1e-10, 30)
    Xh = X.cpu().numpy()
    for k in range(K):
        xo, ito, ro = newton.newton(om, mus[k], nus[k], eps=1e-10)
        assert res[k] <= 1e-10
        assert rel_max(Xh[k], xo[perm]) <= 1e-9
        # the same number of steps: both take full Newton steps on this problem
        assert abs(int(it[k]) - ito) <= 1


def _subset_problem(nx=20, ny=4, m=10, seed=3):
    lm, om, perm = _meshes(nx, ny)
    rng = np.random.default_rng(seed)
    mu = np.sort(rng.uniform(6e5, 1.2e6, m))
    nu = rng.uniform(2.5e-3, 3.5e-3, m)
    med = params.upper_median_position(m)
    xt, _, _ = newton.newton(om, mu[med], nu[med], eps=1e-11)
    return lm, om, perm, mu, nu, xt


def test_chebyshevT_parity_fp64():
    lm, om, perm, mu, nu, xt = _subset_problem()
    m = len(mu)
    J0, Jmu, Jnu = fsi.affine_jacobian(om, xt)
    R0, Rmu, Rnu = fsi.affine_residual(om, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu, nu)
    mb, nb = params.midpoint_parameters(mu, nu)
    c, d = 0.5, 1.0
    sub = lrfsi.Subsets(lm, _dev(xt[perm]), mu, nu, [m], [m])
    ld = m
    UB = _dev(np.stack([R0, Rmu, Rnu], 1)[perm])                     # M x 3
    VB = _dev(-np.stack([np.ones(m), mu, nu], 1))                     # m x 3
    U = torch.zeros(lm.M * ld, dtype=torch.float64, device=DEV)
    V = torch.zeros(m * ld, dtype=torch.float64, device=DEV)
    for cycles in (1, 3):
        opt = lrfsi.cheb_options(c, d, iters=6, cycles=cycles, rank_cap=m, tol=1e-13)
        ranks, stats = lrfsi.lrfsi_chebyshevT(sub, UB, 3, VB, 3, [3], opt, U, ld, V, ld)
        r = int(ranks[0])
        S = U.cpu().numpy().reshape(lm.M, ld)[:, :r] @ V.cpu().numpy().reshape(m, ld)[:, :r].T
        So = lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mu, nu, mb, nb, c, d, iters=6, cycles=cycles, tol=1e-13,
                                        rank_cap=m)
        So = So[perm]
        # per column, relative to the largest column: the upper-median column's
        # exact update is ~0 (x~ solves its problem), so its own norm is no scale
        scale = np.linalg.norm(So, axis=0).max()
        for j in range(m):
            err = np.linalg.norm(S[:, j] - So[:, j]) / scale
            assert err <= 1e-10, (cycles, j, err)


def test_subset_step_reaches_target_and_matches_oracle_residual():
    lm, om, perm, mu, nu, xt = _subset_problem(m=8)
    m = len(mu)
    sub = lrfsi.Subsets(lm, _dev(xt[perm]), mu, nu, [m], [m])
    U = torch.zeros(lm.M * m, dtype=torch.float64, device=DEV)
    V = torch.zeros(m * m, dtype=torch.float64, device=DEV)
    opt = lrfsi.cheb_options(0.5, 1.0, iters=6, cycles=2, rank_cap=m, tol=1e-10)
    ranks, rel, outer, st = lrfsi.lrfsi_subset_step(sub, opt, 1e-8, 20, U, m, V, m)
    assert st == 0 and rel.max() <= 1e-8
    r = int(ranks[0])
    X = xt[perm][:, None] + U.cpu().numpy().reshape(lm.M, m)[:, :r] @ V.cpu().numpy().reshape(m, m)[:, :r].T
    inv = np.argsort(perm)
    rr = algorithm1.relative_residuals(om, X[inv], mu, nu)
    assert np.allclose(rr, rel, rtol=1e-6, atol=1e-14)
    assert rr.max() <= 1e-8


def test_mixed_precision_subset_step_reaches_target():
    """Mixed mode (FP32 SpMM and residual GEMM inside the FP64 correction loop)
    reaches the same target; its result agrees with the FP64 path to the
    target's accuracy."""
    lm, om, perm, mu, nu, xt = _subset_problem(m=8)
    m = len(mu)
    out = {}
    for prec in (0, 1):
        sub = lrfsi.Subsets(lm, _dev(xt[perm]), mu, nu, [m], [m])
        U = torch.zeros(lm.M * m, dtype=torch.float64, device=DEV)
        V = torch.zeros(m * m, dtype=torch.float64, device=DEV)
        opt = lrfsi.cheb_options(0.5, 1.0, iters=6, cycles=3, rank_cap=m, tol=1e-10, eta=0.05, precision=prec)
        ranks, rel, outer, st = lrfsi.lrfsi_subset_step(sub, opt, 1e-8, 30, U, m, V, m)
        assert st == 0 and rel.max() <= 1e-8, (prec, rel.max())
        r = int(ranks[0])
        X = xt[perm][:, None] + U.cpu().numpy().reshape(lm.M, m)[:, :r] @ V.cpu().numpy().reshape(m, m)[:, :r].T
        rr = algorithm1.relative_residuals(om, X[np.argsort(perm)], mu, nu)
        assert rr.max() <= 1e-8
        out[prec] = X
    # both are solutions to relative residual 1e-8: their difference is small
    # against the Newton update itself
    upd = np.linalg.norm(out[0] - xt[perm][:, None])
    assert np.linalg.norm(out[1] - out[0]) <= 1e-5 * upd


@pytest.mark.parametrize("r", [1, 7, 40, 80])
def test_spmm_parity_fp64_and_fp32(r):
    """lrfsi_spmm against the oracle's affine operators times U: FP64 to 1e-12
    of the largest entry (same products, different order); FP32 (FP32 values,
    FP32 accumulation over <= ~50 terms per row) to 1e-5."""
    lm, om, perm = _meshes(20, 4)
    x = om.bD + inputs.random_state(om.M, 3, nq2=om.NQ2)
    J3 = torch.zeros(lm.nnz * 3, dtype=torch.float64, device=DEV)
    lrfsi.lrfsi_assemble_affine(lm, _dev(x[perm]), J3, None)
    oJ = fsi.affine_jacobian(om, x)
    Uh = np.random.default_rng(r).standard_normal((lm.M, r))
    ref = np.concatenate([(oJ[t][perm][:, perm] @ Uh) for t in range(3)], 1)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        U = torch.tensor(Uh, dtype=dt, device=DEV)
        Y = torch.full((lm.M, 3 * r), float("nan"), dtype=dt, device=DEV)
        J = J3 if dt == torch.float64 else J3.to(torch.float32)
        for _ in range(2):  # the first call of a rank bucket runs the autotuner
            lrfsi.lrfsi_spmm(lm, J, U, r, r, Y, 3 * r)
            torch.cuda.synchronize()
            got = Y.double().cpu().numpy()
            for t in range(3):
                blk = slice(t * r, (t + 1) * r)
                assert rel_max(got[:, blk], ref[:, blk]) <= tol, (str(dt), t)
    v, ms = lrfsi.spmm_tuning(0, (r + 15) // 16 if r < 128 else 8)
    assert 0 <= v < 9 and ms[v] > 0


def test_chebyshevT_parity_uneven_subsets_batched():
    """Three subsets of uneven size and rank cap advance in the same launches;
    each matches its own oracle solve (1e-10 per column, relative to the
    subset's largest column)."""
    lm, om, perm = _meshes(20, 4)
    rng = np.random.default_rng(17)
    sizes = [5, 12, 9]
    K = len(sizes)
    mus, nus, xts = [], [], []
    for q, m in enumerate(sizes):
        mu = np.sort(rng.uniform(6e5 + 2e5 * q, 8e5 + 2e5 * q, m))
        nu = rng.uniform(2.5e-3, 3.5e-3, m)
        med = params.upper_median_position(m)
        xt, _, _ = newton.newton(om, mu[med], nu[med], eps=1e-11)
        mus.append(mu); nus.append(nu); xts.append(xt)
    mu_all, nu_all = np.concatenate(mus), np.concatenate(nus)
    ld = max(sizes)
    sub = lrfsi.Subsets(lm, _dev(np.stack([x[perm] for x in xts])), mu_all, nu_all, sizes, sizes)
    UB = torch.zeros(K * lm.M * 3, dtype=torch.float64, device=DEV)
    VB = torch.zeros(sum(sizes) * 3, dtype=torch.float64, device=DEV)
    o = 0
    for q, m in enumerate(sizes):
        R0, Rmu, Rnu = fsi.affine_residual(om, xts[q])
        UB[q * lm.M * 3:(q + 1) * lm.M * 3] = _dev(np.stack([R0, Rmu, Rnu], 1)[perm]).reshape(-1)
        VB[o * 3:(o + m) * 3] = _dev(-np.stack([np.ones(m), mus[q], nus[q]], 1)).reshape(-1)
        o += m
    U = torch.zeros(K * lm.M * ld, dtype=torch.float64, device=DEV)
    V = torch.zeros(sum(sizes) * ld, dtype=torch.float64, device=DEV)
    c, d = 0.5, 1.0
    opt = lrfsi.cheb_options(c, d, iters=6, cycles=2, rank_cap=ld, tol=1e-13)
    ranks, _ = lrfsi.lrfsi_chebyshevT(sub, UB, 3, VB, 3, [3] * K, opt, U, ld, V, ld)
    Uh, Vh = U.cpu().numpy(), V.cpu().numpy()
    o = 0
    for q, m in enumerate(sizes):
        r = int(ranks[q])
        Uq = Uh[q * lm.M * ld:(q + 1) * lm.M * ld].reshape(lm.M, ld)[:, :r]
        Vq = Vh[o * ld:(o + m) * ld].reshape(m, ld)[:, :r]
        S = Uq @ Vq.T
        J0, Jmu, Jnu = fsi.affine_jacobian(om, xts[q])
        R0, Rmu, Rnu = fsi.affine_residual(om, xts[q])
        B = lowrank.rhs(R0, Rmu, Rnu, mus[q], nus[q])
        mb, nb = params.midpoint_parameters(mus[q], nus[q])
        So = lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mus[q], nus[q], mb, nb, c, d, iters=6, cycles=2, tol=1e-13,
                                        rank_cap=m)[perm]
        scale = np.linalg.norm(So, axis=0).max()
        for j in range(m):
            err = np.linalg.norm(S[:, j] - So[:, j]) / scale
            assert err <= 1e-10, (q, j, err)
        o += m
