"""Concurrent groups of subsets (algorithm1.Runner(groups=G)): the K subsets
are independent (Sec. 2), so solving them as G contiguous groups, each with
its own handle, stream and host thread, must give what one handle over all K
gives -- the same correction counts, ranks within one, and residuals and
solutions that differ only by the rounding of differently batched launches.

The medium workload (20 x 20 grid on the 80 x 16 channel, 4 subsets of 100,
rank cap 40, FP64; the fixed Chebyshev interval c = 0.65, d = 1 is the one set
for this mesh); the groups split it 2 + 2 (balanced by m_k R_k).  Bars: the
dense solutions to 1e-9 of their largest entry (far below the 1e-6 residual
target, far above rounding; measured 1e-15), and the relative residuals to
atol 1e-9: the operator's solid block is ~1e6 times its fluid block, so a
solution that differs by rounding (1e-15 of its largest entry) moves a
residual of 1e-7 by ~1e-10 (measured 1.6e-10).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_10275_gb300 import algorithm1, build, inputs, lrfsi  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


def test_concurrent_groups_match_one_handle():
    W = inputs.WORKLOADS["medium"]
    mesh = lrfsi.Mesh(W.nx, W.ny)
    L = algorithm1.workload_layout(W)
    opt = lrfsi.cheb_options(0.65, 1.0, iters=6, cycles=2, rank_cap=W.rank_cap, tol=W.tol, eta=0.05)
    out = {}
    for G in (1, 2):
        run = algorithm1.Runner(mesh, L, opt, target=1e-6, device=DEV, groups=G)
        assert run.groups == G
        res = run.step()
        torch.cuda.synchronize()
        assert res["status"] == 0 and res["relres"].max() <= 1e-6, (G, res["relres"].max())
        out[G] = (res, run.dense(res).cpu().numpy())
    (r1, X1), (r2, X2) = out[1], out[2]
    assert list(r1["outer"]) == list(r2["outer"])
    # a rank at the truncation's boundary may differ by one (rounding of other batches)
    assert np.abs(np.asarray(r1["ranks"]) - np.asarray(r2["ranks"])).max() <= 1
    assert np.allclose(r1["relres"], r2["relres"], rtol=0, atol=1e-9)
    scale = np.abs(X1).max()
    assert np.abs(X1 - X2).max() <= 1e-9 * scale
