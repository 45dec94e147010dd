"""The allocation-free residual entry point (lrfsi_residual_batch_noalloc).

Callers whose device memory belongs to their own pool allocator or a fixed
budget cannot let the library allocate.  This file checks, through the C ABI,
that the allocation-free variant returns the same residual block and column
norms as lrfsi_residual_batch on two calls in a row with different inputs
(the shared scratch keeps the previous call's partial sums, which must not
leak into the next result), with padded leading dimensions, and without the
norms.  It is named to be collected last so that a run stopping at the first
failure has run every other test already.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fsi  # noqa: E402
from paper_2008_10275_gb300 import build, inputs, lrfsi  # noqa: E402
from tests.gpu_common import perm_lib_to_oracle  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


@pytest.mark.parametrize("pad_x,pad_r", [(0, 0), (3, 5)])
def test_noalloc_residual_matches_allocating_entry_point_twice(pad_x, pad_r):
    dev = "cuda:0"
    lm = lrfsi.Mesh(20, 4)
    om = fsi.Mesh(fsi.Problem(20, 4))
    perm = perm_lib_to_oracle(lm, om)
    for call, (m, seed) in enumerate(((7, 11), (12, 23))):
        rng = np.random.default_rng(seed)
        ldx, ldr = m + pad_x, m + pad_r
        X = np.full((lm.M, ldx), 1e300)   # padding columns must never be read into a result
        X[:, :m] = np.stack([om.bD + inputs.random_state(om.M, seed + j, nq2=om.NQ2) for j in range(m)], 1)[perm]
        Xd = torch.tensor(np.ascontiguousarray(X), device=dev)
        mu = torch.tensor(rng.uniform(*inputs.MU_RANGE, m), device=dev)
        nu = torch.tensor(rng.uniform(*inputs.NU_RANGE, m), device=dev)
        R_ref = torch.zeros(lm.M * ldr, dtype=torch.float64, device=dev)
        n_ref = torch.zeros(m, dtype=torch.float64, device=dev)
        lrfsi.lrfsi_residual_batch(lm, Xd, ldx, m, mu, nu, R_ref, ldr, n_ref)
        R = torch.full((lm.M * ldr,), float("nan"), dtype=torch.float64, device=dev)
        n2 = torch.full((m,), float("nan"), dtype=torch.float64, device=dev)
        lrfsi.lrfsi_residual_batch_noalloc(lm, Xd, ldx, m, mu, nu, R, ldr, n2)
        torch.cuda.synchronize()
        Rv, Rr = R.view(lm.M, ldr)[:, :m], R_ref.view(lm.M, ldr)[:, :m]
        scale = float(Rr.abs().max())
        assert float((Rv - Rr).abs().max()) <= 1e-12 * scale, call
        assert torch.allclose(n2, n_ref, rtol=1e-12, atol=0.0), call
        # the residual alone (no norms): the scratch is not touched
        R2 = torch.full((lm.M * ldr,), float("nan"), dtype=torch.float64, device=dev)
        lrfsi.lrfsi_residual_batch_noalloc(lm, Xd, ldx, m, mu, nu, R2, ldr, None)
        torch.cuda.synchronize()
        assert float((R2.view(lm.M, ldr)[:, :m] - Rr).abs().max()) <= 1e-12 * scale, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lm = lrfsi.Mesh(20, 4)  # M = 1581: ceil(M / 256) = 7 partial sums per column
    m = (1 << 21) // 7 + 1  # 7 m > 2^21
    # the size check precedes every launch, so these buffers are never read
    buf = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    with pytest.raises(lrfsi.LrfsiError):
        lrfsi.lrfsi_residual_batch_noalloc(lm, buf, m, m, buf, buf, buf, m, buf)
