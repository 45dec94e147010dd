"""The theta-scheme time step (Sec. 4.3) on the GPU against the oracle
(``oracle/timedep.py``), through the C ABI.

* lrfsi_mass_fluid: the fluid velocity mass A_t^f on the pattern (1e-13 of
  its largest entry).
* lrfsi_newton_theta: the time-step Newton solution of two problems (1e-9).
* lrfsi_subset_step_theta: one subset time step (Eq. (timedep_matrix1)) and a
  second step from the first: every column reaches the target, the oracle's
  R_theta of the GPU's columns confirms it, and the columns match the
  oracle's subset time step (1e-7 of the update, both at the same target).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import algorithm1, fsi, params, timedep  # noqa: E402
from paper_2008_10275_gb300 import build, lrfsi  # noqa: E402
from tests.gpu_common import lib_csr, perm_lib_to_oracle  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


@pytest.fixture(scope="module")
def meshes():
    lm = lrfsi.Mesh(20, 4)
    om = fsi.Mesh(fsi.Problem(20, 4))
    return lm, om, perm_lib_to_oracle(lm, om)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def test_mass_matrix(meshes):
    lm, om, perm = meshes
    Mv = torch.zeros(lm.nnz, dtype=torch.float64, device=DEV)
    lrfsi.lrfsi_mass_fluid(lm, Mv)
    A = lib_csr(lm, Mv.cpu().numpy()).toarray()
    ref = timedep.mass_fluid(om)[perm][:, perm].toarray()
    assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()


def test_newton_theta(meshes):
    lm, om, perm = meshes
    mus, nus = np.array([7e5, 1.4e6]), np.array([2.5e-3, 4e-3])
    theta, dt = 0.6, 0.02
    Xp = np.stack([om.bD, om.bD])
    X = _dev(Xp[:, perm])
    it, res, st = lrfsi.lrfsi_newton_theta(lm, X, _dev(Xp[:, perm]), mus, nus, theta, dt, 1e-10, 30)
    Xh = X.cpu().numpy()
    for k in range(2):
        xo, ito, ro = timedep.newton_theta(om, Xp[k], mus[k], nus[k], theta, dt, eps=1e-10)
        assert res[k] <= 1e-10
        assert np.abs(Xh[k] - xo[perm]).max() <= 1e-9 * np.abs(xo).max()


def test_subset_time_steps(meshes):
    lm, om, perm = meshes
    inv = np.argsort(perm)
    mu_k = np.repeat(np.linspace(7e5, 9e5, 3), 2)
    nu_k = np.tile(np.array([3.0e-3, 3.4e-3]), 3)
    m = len(mu_k)
    theta, dt, target = 0.6, 0.02, 1e-8
    med = params.upper_median_position(m)
    Xprev = np.repeat(om.bD[:, None], m, 1)          # oracle order
    opt = lrfsi.cheb_options(0.5, 1.0, iters=6, cycles=3, rank_cap=m, tol=1e-12, eta=0.05)
    oopt = algorithm1.Options(c=0.5, d=1.0, iters=6, cycles=3, truncated=False)
    for step in range(2):
        xt, _, _ = timedep.newton_theta(om, Xprev[:, med], mu_k[med], nu_k[med], theta, dt, eps=1e-11)
        # the GPU's own median step from the GPU's previous state
        Xg = _dev(Xprev[perm, med][None])
        lrfsi.lrfsi_newton_theta(lm, Xg, _dev(Xprev[perm, med][None]), mu_k[med:med + 1], nu_k[med:med + 1], theta,
                                 dt, 1e-11, 30)
        assert np.abs(Xg[0].cpu().numpy() - xt[perm]).max() <= 1e-9 * np.abs(xt).max()
        sub = lrfsi.Subsets(lm, Xg, mu_k, nu_k, [m], [m], theta=theta, dt=dt)
        U = torch.zeros(lm.M * m, dtype=torch.float64, device=DEV)
        V = torch.zeros(m * m, dtype=torch.float64, device=DEV)
        ranks, rel, outer, st = lrfsi.lrfsi_subset_step_theta(sub, opt, _dev(Xprev[perm]), m, target, 30, U, m, V, m)
        sub.close()
        assert st == 0 and rel.max() <= target, (step, rel.max())
        r = int(ranks[0])
        X = Xg[0].cpu().numpy()[:, None] + U.cpu().numpy().reshape(lm.M, m)[:, :r] @ V.cpu().numpy().reshape(m, m)[:, :r].T
        X = X[inv]
        rr = timedep.relative_residuals_theta(om, X, Xprev, mu_k, nu_k, theta, dt)
        assert rr.max() <= target and np.allclose(rr, rel, rtol=1e-6, atol=1e-12), (step, rr, rel)
        Xo, _, rro = timedep.subset_step_theta(om, xt, Xprev, mu_k, nu_k, theta, dt, oopt, target=target)
        upd = np.abs(Xo - Xprev).max()
        assert np.abs(X - Xo).max() <= 1e-7 * upd, step
        Xprev = X
