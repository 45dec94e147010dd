"""Adaptive refinement of the subsets on the GPU (the product driver
``algorithm1.adaptive`` through the C ABI) against the oracle's
``algorithm1_adaptive`` (reading of Sec. 5, "Alternative ways to cluster the
parameter set"): the same refined subsets and medians, the same columns
(1e-8 of the largest update), and with chord corrections after the
refinement every column meets the target, confirmed by the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import algorithm1 as oa, fsi  # noqa: E402
from paper_2008_10275_gb300 import algorithm1, build, lrfsi  # noqa: E402
from tests.gpu_common import perm_lib_to_oracle  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


def _case():
    lm = lrfsi.Mesh(20, 4)
    om = fsi.Mesh(fsi.Problem(20, 4))
    mu_v, nu_v = np.linspace(5e5, 2e6, 4), np.linspace(1e-3, 5e-3, 2)
    L = algorithm1.grid_layout(mu_v, nu_v, 1, 8)
    return lm, om, perm_lib_to_oracle(lm, om), L


def _dense(res, M):
    cols = []
    for r in res:
        cols.append((r["xt"][:, None] + r["U"] @ r["V"].T).cpu().numpy())
    return np.concatenate(cols, 1)


def test_adaptive_matches_oracle_refinement():
    lm, om, perm, L = _case()
    opt = lrfsi.cheb_options(0.65, 1.0, iters=6, cycles=4, rank_cap=8, tol=1e-13)
    res = algorithm1.adaptive(lm, L, opt, target=0.0, max_levels=2, max_outer=0, eps_N=1e-9)
    oopt = oa.Options(K=1, eps_N=1e-9, c=0.65, d=1.0, iters=6, cycles=4, truncated=False, warm_start=False)
    Xo, subs = oa.algorithm1_adaptive(om, L.mu, L.nu, oopt, target=0.0, max_levels=2)
    assert [(r["start"], r["size"]) for r in res] == [(a, n) for a, n, _ in subs]
    X = _dense(res, lm.M)[np.argsort(perm)]
    upd = np.abs(Xo - om.bD[:, None]).max()
    assert np.abs(X - Xo).max() <= 1e-8 * upd


def test_adaptive_then_corrections_reach_target():
    lm, om, perm, L = _case()
    opt = lrfsi.cheb_options(0.65, 1.0, iters=6, cycles=2, rank_cap=8, tol=1e-10, eta=0.05)
    res = algorithm1.adaptive(lm, L, opt, target=1e-8, max_levels=1, max_outer=30, eps_N=1e-9)
    X = _dense(res, lm.M)[np.argsort(perm)]
    rr = oa.relative_residuals(om, X, L.mu, L.nu)
    assert rr.max() <= 1e-8, rr.max()
    got = np.concatenate([r["relres"] for r in res])
    assert np.allclose(got, rr, rtol=1e-6, atol=1e-12)
