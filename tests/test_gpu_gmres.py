"""GMREST on the GPU (``lrfsi_gmresT``; ``lrfsi_subset_step`` with solver 1)
against the oracle's ``lowrank.gmres_T_scaled``, through the C ABI.

Tolerance as for ChebyshevT: at truncation tolerance 1e-13 with the rank cap
equal to the subset size (an exact bound on the rank of any M x m_k matrix)
both sides compute the same iterates up to rounding, so every column agrees
to 1e-10 relative to the subset's largest column."""
import numpy as np
import pytest

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


def _subsets(sizes, seed):
    lm = lrfsi.Mesh(20, 4)
    om = fsi.Mesh(fsi.Problem(20, 4))
    perm = perm_lib_to_oracle(lm, om)
    rng = np.random.default_rng(seed)
    mus, nus, xts = [], [], []
    for q, m in enumerate(sizes):
        mu = np.sort(rng.uniform(6e5 + 2e5 * q, 8e5 + 2e5 * q, m))
        nu = rng.uniform(2.5e-3, 3.5e-3, m)
        xt, _, _ = newton.newton(om, mu[params.upper_median_position(m)], nu[params.upper_median_position(m)],
                                 eps=1e-11)
        mus.append(mu)
        nus.append(nu)
        xts.append(xt)
    return lm, om, perm, mus, nus, xts


def _solve_gpu(lm, om, perm, mus, nus, xts, sizes, opt):
    K, ld = len(sizes), max(sizes)
    sub = lrfsi.Subsets(lm, _dev(np.stack([x[perm] for x in xts])), np.concatenate(mus), np.concatenate(nus),
                        sizes, sizes)
    UB = torch.zeros(K * lm.M * 3, dtype=torch.float64, device=DEV)
    VB = torch.zeros(sum(sizes) * 3, dtype=torch.float64, device=DEV)
    o = 0
    for q, m in enumerate(sizes):
        R3 = fsi.affine_residual(om, xts[q])
        UB[q * lm.M * 3:(q + 1) * lm.M * 3] = _dev(np.stack(R3, 1)[perm]).reshape(-1)
        VB[o * 3:(o + m) * 3] = _dev(-np.stack([np.ones(m), mus[q], nus[q]], 1)).reshape(-1)
        o += m
    U = torch.zeros(K * lm.M * ld, dtype=torch.float64, device=DEV)
    V = torch.zeros(sum(sizes) * ld, dtype=torch.float64, device=DEV)
    ranks, stats = lrfsi.lrfsi_gmresT(sub, UB, 3, VB, 3, [3] * K, opt, U, ld, V, ld)
    sub.close()
    Uh, Vh = U.cpu().numpy(), V.cpu().numpy()
    out, o = [], 0
    for q, m in enumerate(sizes):
        r = int(ranks[q])
        Uq = Uh[q * lm.M * ld:(q + 1) * lm.M * ld].reshape(lm.M, ld)[:, :r]
        Vq = Vh[o * ld:(o + m) * ld].reshape(m, ld)[:, :r]
        out.append(Uq @ Vq.T)
        o += m
    return out, stats


def _oracle(om, perm, mu, nu, xt, **kw):
    J0, Jmu, Jnu = fsi.affine_jacobian(om, xt)
    R0, Rmu, Rnu = fsi.affine_residual(om, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu, nu)
    mb, nb = params.midpoint_parameters(mu, nu)
    return lowrank.gmres_T_scaled(J0, Jmu, Jnu, B, mu, nu, mb, nb, **kw)[perm]


def _assert_columns(S, So, tol, tag):
    scale = np.linalg.norm(So, axis=0).max()
    for j in range(S.shape[1]):
        err = np.linalg.norm(S[:, j] - So[:, j]) / scale
        assert err <= tol, (tag, j, err)


@pytest.mark.parametrize("iters,cycles", [(6, 1), (6, 2), (3, 3)])
def test_gmresT_parity_fp64(iters, cycles):
    sizes = [10]
    lm, om, perm, mus, nus, xts = _subsets(sizes, 3)
    opt = lrfsi.cheb_options(0.0, 0.0, iters=iters, cycles=cycles, rank_cap=10, tol=1e-13)
    (S,), stats = _solve_gpu(lm, om, perm, mus, nus, xts, sizes, opt)
    assert stats[0]["steps"] == iters * cycles
    So = _oracle(om, perm, mus[0], nus[0], xts[0], iters=iters, cycles=cycles, tol=1e-13, rank_cap=10)
    _assert_columns(S, So, 1e-10, (iters, cycles))


def test_gmresT_parity_uneven_subsets_batched():
    """Three subsets of uneven size and rank cap advance in the same launches
    (grouped Gram products, SpMM, block-LU solves and truncations); each
    matches its own oracle solve."""
    sizes = [5, 12, 9]
    lm, om, perm, mus, nus, xts = _subsets(sizes, 17)
    opt = lrfsi.cheb_options(0.0, 0.0, iters=4, cycles=2, rank_cap=12, tol=1e-13)
    S, stats = _solve_gpu(lm, om, perm, mus, nus, xts, sizes, opt)
    for q, m in enumerate(sizes):
        So = _oracle(om, perm, mus[q], nus[q], xts[q], iters=4, cycles=2, tol=1e-13, rank_cap=m)
        _assert_columns(S[q], So, 1e-10, q)


def test_gmresT_eta_stops_early_like_the_oracle():
    """With eta the Arnoldi loop ends once the least-squares residual is below
    eta ||B||_F, and a cycle is skipped once the true residual is: the GPU
    takes fewer steps than iters x cycles and still matches the oracle run
    with the same eta."""
    sizes = [10]
    lm, om, perm, mus, nus, xts = _subsets(sizes, 5)
    opt = lrfsi.cheb_options(0.0, 0.0, iters=6, cycles=4, rank_cap=10, tol=1e-13, eta=1e-6)
    (S,), stats = _solve_gpu(lm, om, perm, mus, nus, xts, sizes, opt)
    assert stats[0]["steps"] < 24
    So = _oracle(om, perm, mus[0], nus[0], xts[0], iters=6, cycles=4, tol=1e-13, rank_cap=10, eta=1e-6)
    _assert_columns(S, So, 1e-9, "eta")


@pytest.mark.parametrize("precision", [0, 1])
def test_subset_step_with_gmrest_reaches_target(precision):
    """Algorithm 1's subset step with GMREST as the low-rank solver (FP64, and
    mixed: the inner residual in FP32) reaches relative residual 1e-8 in every
    column; the oracle's residual of the returned columns agrees."""
    sizes = [8]
    lm, om, perm, mus, nus, xts = _subsets(sizes, 3)
    mu, nu, xt = mus[0], nus[0], xts[0]
    m = len(mu)
    sub = lrfsi.Subsets(lm, _dev(xt[perm]), mu, nu, [m], [m])
    U = torch.zeros(lm.M * m, dtype=torch.float64, device=DEV)
    V = torch.zeros(m * m, dtype=torch.float64, device=DEV)
    opt = lrfsi.cheb_options(0.0, 0.0, iters=6, cycles=2, rank_cap=m, tol=1e-10, eta=0.05, precision=precision,
                             solver="gmres")
    ranks, rel, outer, st = lrfsi.lrfsi_subset_step(sub, opt, 1e-8, 20, U, m, V, m)
    sub.close()
    assert st == 0 and rel.max() <= 1e-8, (precision, rel.max())
    r = int(ranks[0])
    X = xt[perm][:, None] + U.cpu().numpy().reshape(lm.M, m)[:, :r] @ V.cpu().numpy().reshape(m, m)[:, :r].T
    rr = algorithm1.relative_residuals(om, X[np.argsort(perm)], mu, nu)
    assert np.allclose(rr, rel, rtol=1e-6, atol=1e-14)
    assert rr.max() <= 1e-8


def test_chebyshev_after_gmrest_on_one_handle():
    """GMREST widens the handle's concatenation buffers on first use; a
    ChebyshevT solve on the same handle afterwards still matches its oracle."""
    sizes = [10]
    lm, om, perm, mus, nus, xts = _subsets(sizes, 3)
    mu, nu, xt = mus[0], nus[0], xts[0]
    m = len(mu)
    sub = lrfsi.Subsets(lm, _dev(xt[perm]), mu, nu, [m], [m])
    R0, Rmu, Rnu = fsi.affine_residual(om, xt)
    UB = _dev(np.stack([R0, Rmu, Rnu], 1)[perm])
    VB = _dev(-np.stack([np.ones(m), mu, nu], 1))
    U = torch.zeros(lm.M * m, dtype=torch.float64, device=DEV)
    V = torch.zeros(m * m, dtype=torch.float64, device=DEV)
    lrfsi.lrfsi_gmresT(sub, UB, 3, VB, 3, [3], lrfsi.cheb_options(0.0, 0.0, iters=6, cycles=1, rank_cap=m, tol=1e-13),
                       U, m, V, m)
    ranks, _ = lrfsi.lrfsi_chebyshevT(sub, UB, 3, VB, 3, [3],
                                      lrfsi.cheb_options(0.5, 1.0, iters=6, cycles=2, rank_cap=m, tol=1e-13),
                                      U, m, V, m)
    sub.close()
    r = int(ranks[0])
    S = U.cpu().numpy().reshape(lm.M, m)[:, :r] @ V.cpu().numpy().reshape(m, m)[:, :r].T
    J0, Jmu, Jnu = fsi.affine_jacobian(om, xt)
    B = lowrank.rhs(R0, Rmu, Rnu, mu, nu)
    mb, nb = params.midpoint_parameters(mu, nu)
    So = lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mu, nu, mb, nb, 0.5, 1.0, iters=6, cycles=2, tol=1e-13,
                                    rank_cap=m)[perm]
    _assert_columns(S, So, 1e-10, "cheb after gmres")
