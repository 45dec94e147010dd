"""Degenerate cases and argument checks of the subset solvers through the C ABI.

* A one-parameter subset: the mean-based preconditioner at the range midpoint
  is the exact Jacobian J(x~; mu, nu), so P^{-1} F = I.  GMREST returns the
  Newton step (Eq. (newtonstep_vectornot1)) after one Arnoldi step (the
  orthogonalised vector vanishes); ChebyshevT converges to it at its
  polynomial rate.  Both match their oracle runs.
* A zero right-hand side: both solvers return rank 0 and leave the output
  factors untouched.
* Rank cap 1: every truncation keeps one singular triple; with the gaps of
  this case (sigma_2 / sigma_1 <= 0.68 at every truncation, checked in the
  oracle) the rank-1 iterates agree with the oracle's SVD truncation to 1e-9.
* Invalid sizes and options are rejected with LRFSI_EINVAL before any launch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fsi, lowrank, newton, params  # noqa: E402
from paper_2008_10275_gb300 import build, lrfsi  # noqa: E402
from tests.gpu_common import perm_lib_to_oracle  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


@pytest.fixture(scope="module")
def case():
    lm = lrfsi.Mesh(20, 4)
    om = fsi.Mesh(fsi.Problem(20, 4))
    perm = perm_lib_to_oracle(lm, om)
    rng = np.random.default_rng(3)
    mu = np.sort(rng.uniform(6e5, 8e5, 6))
    nu = rng.uniform(2.5e-3, 3.5e-3, 6)
    xt, _, _ = newton.newton(om, mu[params.upper_median_position(6)], nu[params.upper_median_position(6)],
                             eps=1e-11)
    return lm, om, perm, mu, nu, xt


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _run(lm, om, perm, xt, mu, nu, cap, opt, solver, UB=None, fill=0.0):
    m = len(mu)
    sub = lrfsi.Subsets(lm, _dev(xt[perm]), mu, nu, [m], [cap])
    if UB is None:
        UB = _dev(np.stack(fsi.affine_residual(om, xt), 1)[perm])
    VB = _dev(-np.stack([np.ones(m), mu, nu], 1))
    U = torch.full((lm.M * cap,), fill, dtype=torch.float64, device=DEV)
    V = torch.full((m * cap,), fill, dtype=torch.float64, device=DEV)
    fn = lrfsi.lrfsi_gmresT if solver == "gmres" else lrfsi.lrfsi_chebyshevT
    ranks, stats = fn(sub, UB, 3, VB, 3, [3], opt, U, cap, V, cap)
    sub.close()
    r = int(ranks[0])
    Uh, Vh = U.cpu().numpy().reshape(lm.M, cap), V.cpu().numpy().reshape(m, cap)
    return r, Uh, Vh, stats[0]


def _oracle(om, perm, xt, mu, nu, solver, **kw):
    J0, Jmu, Jnu = fsi.affine_jacobian(om, xt)
    B = lowrank.rhs(*fsi.affine_residual(om, xt), mu, nu)
    mb, nb = params.midpoint_parameters(mu, nu)
    if solver == "gmres":
        return lowrank.gmres_T_scaled(J0, Jmu, Jnu, B, mu, nu, mb, nb, **kw)[perm]
    return lowrank.chebyshev_T_scaled(J0, Jmu, Jnu, B, mu, nu, mb, nb, 0.5, 1.0, **kw)[perm]


@pytest.mark.parametrize("solver", ["chebyshev", "gmres"])
def test_single_parameter_subset_is_a_newton_step(case, solver):
    lm, om, perm, mu, nu, xt = case
    mu1, nu1 = mu[:1], nu[:1]        # linearised at another parameter's solution: a real update
    opt = lrfsi.cheb_options(0.5, 1.0, iters=6, cycles=2, rank_cap=1, tol=1e-13)
    r, Uh, Vh, st = _run(lm, om, perm, xt, mu1, nu1, 1, opt, solver)
    assert r == 1
    S = Uh[:, :1] @ Vh[:, :1].T
    So = _oracle(om, perm, xt, mu1, nu1, solver, iters=6, cycles=2, tol=1e-13, rank_cap=1)
    assert np.linalg.norm(S - So) <= 1e-10 * np.linalg.norm(So)
    bf = lowrank.brute_force(om, xt, mu1, nu1)[perm]
    err = np.linalg.norm(S - bf) / np.linalg.norm(bf)
    assert err <= (1e-9 if solver == "gmres" else 1e-5), err


@pytest.mark.parametrize("solver", ["chebyshev", "gmres"])
def test_zero_right_hand_side_gives_rank_zero(case, solver):
    lm, om, perm, mu, nu, xt = case
    opt = lrfsi.cheb_options(0.5, 1.0, iters=6, cycles=2, rank_cap=6, tol=1e-8)
    UB0 = torch.zeros(lm.M * 3, dtype=torch.float64, device=DEV)
    r, Uh, Vh, st = _run(lm, om, perm, xt, mu, nu, 6, opt, solver, UB=UB0, fill=7.0)
    assert r == 0 and st["steps"] == 0
    assert np.all(Uh == 7.0) and np.all(Vh == 7.0)


@pytest.mark.parametrize("solver", ["chebyshev", "gmres"])
def test_rank_cap_one_matches_truncated_oracle(case, solver):
    lm, om, perm, mu, nu, xt = case
    opt = lrfsi.cheb_options(0.5, 1.0, iters=6, cycles=2, rank_cap=1, tol=1e-8)
    r, Uh, Vh, st = _run(lm, om, perm, xt, mu, nu, 1, opt, solver)
    assert r == 1
    S = Uh[:, :1] @ Vh[:, :1].T
    So = _oracle(om, perm, xt, mu, nu, solver, iters=6, cycles=2, tol=1e-8, rank_cap=1)
    assert np.linalg.norm(S - So) <= 1e-9 * np.linalg.norm(So), np.linalg.norm(S - So) / np.linalg.norm(So)


def test_invalid_arguments_are_rejected(case):
    lm, om, perm, mu, nu, xt = case
    x = _dev(xt[perm])
    with pytest.raises(lrfsi.LrfsiError) as e:
        lrfsi.Subsets(lm, x, mu, nu, [0], [4])                    # empty subset
    assert e.value.code == lrfsi.EINVAL
    with pytest.raises(lrfsi.LrfsiError) as e:
        lrfsi.Subsets(lm, x, mu, nu, [6], [0])                    # rank cap 0
    assert e.value.code == lrfsi.EINVAL
    sub = lrfsi.Subsets(lm, x, mu, nu, [6], [6])
    UB = torch.zeros(lm.M * 3, dtype=torch.float64, device=DEV)
    VB = torch.zeros(6 * 3, dtype=torch.float64, device=DEV)
    U = torch.zeros(lm.M * 6, dtype=torch.float64, device=DEV)
    V = torch.zeros(6 * 6, dtype=torch.float64, device=DEV)
    bad = [
        (lrfsi.lrfsi_chebyshevT, lrfsi.cheb_options(1.0, 1.0, rank_cap=6), 6),     # c >= d
        (lrfsi.lrfsi_chebyshevT, lrfsi.cheb_options(0.5, 1.0, iters=0, rank_cap=6), 6),
        (lrfsi.lrfsi_gmresT, lrfsi.cheb_options(0.0, 0.0, cycles=0, rank_cap=6), 6),
        (lrfsi.lrfsi_gmresT, lrfsi.cheb_options(0.0, 0.0, tol=-1.0, rank_cap=6), 6),
        (lrfsi.lrfsi_gmresT, lrfsi.cheb_options(0.0, 0.0, rank_cap=6), 5),         # ldu, ldv < R_k
    ]
    for fn, opt, ld in bad:
        with pytest.raises(lrfsi.LrfsiError) as e:
            fn(sub, UB, 3, VB, 3, [3], opt, U, ld, V, ld)
        assert e.value.code == lrfsi.EINVAL
    opt = lrfsi.cheb_options(0.5, 1.0, rank_cap=6)
    opt.solver = 2                                                  # no such solver
    Ut = torch.zeros(lm.M * 6, dtype=torch.float64, device=DEV)
    with pytest.raises(lrfsi.LrfsiError) as e:
        lrfsi.lrfsi_subset_step(sub, opt, 1e-6, 2, Ut, 6, V, 6)
    assert e.value.code == lrfsi.EINVAL
    sub.close()
