"""Full-size parity on sampled outputs: the 400-parameter workload on the 80x16
mesh (M = 22629, 4 subsets of 100, rank cap 40) in the launch configuration
the benchmark times (Chebyshev c = 0.65, d = 1, 6 steps x 2 cycles, eta 0.05,
target 1e-6; FP64, mixed, and FP64 with GMREST as the low-rank solver).  The
oracle cannot run the whole method at this size in a test,
so it checks what it can compute one by one: the Newton solution of one
median parameter, and the nonlinear relative residual of sampled columns of
the GPU result (the definition of the reported metric, Sec. 5.1.2), which must
equal the GPU's own residual and lie below the target."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import algorithm1, fsi, newton  # noqa: E402
from paper_2008_10275_gb300 import algorithm1 as a1, build, inputs, lrfsi  # noqa: E402
from tests.gpu_common import perm_lib_to_oracle, rel_max  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


@pytest.fixture(scope="module")
def fullsize():
    W = inputs.WORKLOADS["medium"]
    lm = lrfsi.Mesh(W.nx, W.ny)
    om = fsi.Mesh(fsi.Problem(W.nx, W.ny))
    perm = perm_lib_to_oracle(lm, om)
    L = a1.workload_layout(W)
    mus, nus = L.mu, L.nu
    K, R, m = L.K, W.rank_cap, L.m
    sizes, medians = L.sizes.tolist(), L.medians.tolist()
    bD = torch.tensor(lm.dirichlet(), device=DEV)
    X = bD.repeat(K, 1)
    it, res, st = lrfsi.lrfsi_newton_median(lm, X, mus[medians], nus[medians], 1e-8, 30)
    assert st == 0 and np.all(res <= 1e-8)
    out = {}
    for variant, precision, solver in (("fp64", 0, "chebyshev"), ("mixed", 1, "chebyshev"), ("gmrest", 0, "gmres")):
        sub = lrfsi.Subsets(lm, X, mus, nus, sizes, [R] * K)
        U = torch.zeros(K * lm.M * R, dtype=torch.float64, device=DEV)
        V = torch.zeros(m * R, dtype=torch.float64, device=DEV)
        opt = lrfsi.cheb_options(0.65, 1.0, iters=6, cycles=2, rank_cap=R, tol=W.tol, eta=0.05, precision=precision,
                                 solver=solver)
        ranks, rel, outer, st = lrfsi.lrfsi_subset_step(sub, opt, 1e-6, 40, U, R, V, R)
        sub.close()
        out[variant] = (ranks, rel, st, U.cpu().numpy(), V.cpu().numpy())
    return dict(W=W, lm=lm, om=om, perm=perm, mus=mus, nus=nus, K=K, R=R, m=m, sizes=sizes, medians=medians,
                X=X.cpu().numpy(), out=out)


def test_fullsize_median_newton_matches_oracle(fullsize):
    f = fullsize
    q = 1
    med = f["medians"][q]
    xo, _, _ = newton.newton(f["om"], f["mus"][med], f["nus"][med], eps=1e-8)
    assert rel_max(f["X"][q], xo[f["perm"]]) <= 1e-7


@pytest.mark.parametrize("variant", ["fp64", "mixed", "gmrest"])
def test_fullsize_sampled_columns_residual_matches_oracle(fullsize, variant):
    f = fullsize
    ranks, rel, st, U, V = f["out"][variant]
    assert st == 0 and rel.max() <= 1e-6
    M, R, mloc = f["lm"].M, f["R"], f["m"] // f["K"]
    inv = np.argsort(f["perm"])
    rng = np.random.default_rng(7)
    cols = sorted(set([0, mloc - 1, f["m"] - 1] + list(rng.choice(f["m"], 9, replace=False))))
    for i in cols:
        q = i // mloc
        r = int(ranks[q])
        Uq = U[q * M * R:(q + 1) * M * R].reshape(M, R)[:, :r]
        vi = V[i * R:(i + 1) * R][:r]
        x = f["X"][q] + Uq @ vi
        ro = algorithm1.relative_residuals(f["om"], x[inv][:, None], f["mus"][i:i + 1], f["nus"][i:i + 1])[0]
        assert ro <= 1e-6, (variant, i, ro)
        assert ro == pytest.approx(rel[i], rel=1e-6, abs=1e-13), (variant, i, ro, rel[i])
