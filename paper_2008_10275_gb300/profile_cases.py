"""Small, self-contained cases of the hot kernels for profiling (ncu) and
timing outside the full step.

    python -m paper_2008_10275_gb300.profile_cases lu       # K block-LU factorisations (subset preconditioners)
    python -m paper_2008_10275_gb300.profile_cases trunc    # median Newton + two correction steps (truncations)
    python -m paper_2008_10275_gb300.profile_cases spmm     # FP64 and FP32 SpMM of the affine operators
    python -m paper_2008_10275_gb300.profile_cases large    # 320 x 64 mesh: SpMM, block LU, solve, one ChebyshevT step
    python -m paper_2008_10275_gb300.profile_cases ndsolve  # preconditioner solves, 40 right-hand sides, both paths

Each case builds the 80 x 16 channel mesh (M = 22629) with the seeded
parameters of the 400-parameter workload, runs the case twice (the first run
warms up) and prints the CUDA-event time of the second run.  The large case
uses the 320 x 64 mesh (M = 351621) and one subset of the first 100
parameters of the 50 x 50 grid (rank cap 80), timed once each.
"""
from __future__ import annotations

import sys

import numpy as np


def _setup():
    import torch
    from . import build, inputs, lrfsi
    if not torch.cuda.is_available():
        raise SystemExit("profile cases need a CUDA GPU")
    build.build()
    lrfsi.load()
    from . import algorithm1
    W = inputs.WORKLOADS["medium"]
    mesh = lrfsi.Mesh(W.nx, W.ny)
    L = algorithm1.workload_layout(W)
    return torch, lrfsi, W, mesh, L.mu, L.nu


def _timed(torch, fn, reps=1):
    """CUDA-event time of one call (mean over reps back-to-back calls, after a
    warm-up call)."""
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def case_lu():
    torch, lrfsi, W, mesh, mus, nus = _setup()
    K = W.K
    bD = torch.tensor(mesh.dirichlet(), device="cuda:0")
    X = bD.repeat(K, 1)
    sizes = [len(mus) // K] * K

    def run():
        s = lrfsi.Subsets(mesh, X, mus, nus, sizes, [W.rank_cap] * K)
        s.close()

    ms, _ = _timed(torch, run)
    print(f"lu: {K} subset preconditioners (assembly, equilibration, block LU) {ms:.2f} ms")


def case_trunc():
    torch, lrfsi, W, mesh, mus, nus = _setup()
    K, R, m = W.K, W.rank_cap, len(mus)
    sizes = [m // K] * K
    med = [k * (m // K) + (m // K) // 2 for k in range(K)]
    bD = torch.tensor(mesh.dirichlet(), device="cuda:0")
    U = torch.zeros(K * mesh.M * R, dtype=torch.float64, device="cuda:0")
    V = torch.zeros(m * R, dtype=torch.float64, device="cuda:0")
    opt = lrfsi.cheb_options(0.65, 1.0, iters=6, cycles=2, rank_cap=R, tol=W.tol, eta=0.05)

    def run():
        X = bD.repeat(K, 1)
        lrfsi.lrfsi_newton_median(mesh, X, mus[med], nus[med], 1e-8, 30)
        sub = lrfsi.Subsets(mesh, X, mus, nus, sizes, [R] * K)
        out = lrfsi.lrfsi_subset_step(sub, opt, 1e-6, 2, U, R, V, R)
        sub.close()
        return out

    ms, (ranks, rel, outer, st) = _timed(torch, run)
    print(f"trunc: Newton + two correction steps {ms:.2f} ms, ranks {ranks.tolist()}, max rel {rel.max():.2e}")


def case_spmm():
    torch, lrfsi, W, mesh, mus, nus = _setup()
    R = W.rank_cap
    rng = np.random.default_rng(0)
    x = torch.tensor(mesh.dirichlet(), device="cuda:0")
    J3 = torch.zeros(3 * mesh.nnz, dtype=torch.float64, device="cuda:0")
    lrfsi.lrfsi_assemble_affine(mesh, x, J3, None)
    Uh = rng.standard_normal((mesh.M, R))
    for dt in (torch.float64, torch.float32):
        U = torch.tensor(Uh, dtype=dt, device="cuda:0")
        Y = torch.zeros(mesh.M, 3 * R, dtype=dt, device="cuda:0")
        J = J3 if dt == torch.float64 else J3.to(torch.float32)
        ms, _ = _timed(torch, lambda: lrfsi.lrfsi_spmm(mesh, J, U, R, R, Y, 3 * R), reps=50)
        by = mesh.nnz * (3 * J.element_size() + 4) + (mesh.M + 1) * 4 + U.numel() * U.element_size() \
            + Y.numel() * Y.element_size()
        v, tms = lrfsi.spmm_tuning(0 if dt == torch.float64 else 1, min((R + 15) // 16, 8))
        print(f"spmm {str(dt)[6:]}: r = {R} {ms * 1e3:.1f} us, {by / (ms * 1e-3) / 1e9:.0f} GB/s "
              f"(shape {v}, tuned ms {[round(float(t), 4) for t in tms]})")


def case_ndsolve():
    """The K preconditioner solves P_k^{-1} X of the medium workload (nested
    dissection, subset operators at b_D) with 40 right-hand sides, on the
    tensor-core sweeps (path 1) and on the FP64 sweeps (path 0)."""
    torch, lrfsi, W, mesh, mus, nus = _setup()
    K = W.K
    bD = torch.tensor(mesh.dirichlet(), device="cuda:0")
    sizes = [len(mus) // K] * K
    sub = lrfsi.Subsets(mesh, bD.repeat(K, 1), mus, nus, sizes, [W.rank_cap] * K)
    ld = 40
    gen = torch.Generator(device="cuda:0").manual_seed(3)
    X = torch.randn(K * mesh.M * ld, dtype=torch.float64, device="cuda:0", generator=gen)
    Y = torch.zeros_like(X)
    prev = lrfsi.gram_path()
    for path in (1, 0):
        lrfsi.gram_path(path)
        ms, _ = _timed(torch, lambda: lrfsi.lrfsi_precond_apply(sub, X, ld, ld, Y, ld))
        print(f"ndsolve path {path}: {K} problems x {ld} columns {ms:.3f} ms")
    lrfsi.gram_path(prev)
    sub.close()


def case_large():
    import json
    import torch
    from . import build, inputs, lrfsi
    if not torch.cuda.is_available():
        raise SystemExit("profile cases need a CUDA GPU")
    build.build()
    lrfsi.load()
    dev = "cuda:0"
    W = inputs.WORKLOADS["large"]
    mesh = lrfsi.Mesh(W.nx, W.ny)
    from . import algorithm1
    L = algorithm1.workload_layout(W)
    mus, nus = L.mu[:100], L.nu[:100]
    R, m = W.rank_cap, 100
    out = {"mesh": f"{W.nx}x{W.ny}", "M": mesh.M, "nnz": mesh.nnz, "slabs": mesh.nslab, "slab_max": mesh.nmax}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    bD = torch.tensor(mesh.dirichlet(), device=dev)
    # SpMM at r = R
    J3 = torch.zeros(3 * mesh.nnz, dtype=torch.float64, device=dev)
    lrfsi.lrfsi_assemble_affine(mesh, bD, J3, None)
    Uh = np.random.default_rng(0).standard_normal((mesh.M, R))
    for dt in (torch.float64, torch.float32):
        U = torch.tensor(Uh, dtype=dt, device=dev)
        Y = torch.zeros(mesh.M, 3 * R, dtype=dt, device=dev)
        J = J3 if dt == torch.float64 else J3.to(torch.float32)
        ms, _ = _timed(torch, lambda: lrfsi.lrfsi_spmm(mesh, J, U, R, R, Y, 3 * R), reps=10)
        by = mesh.nnz * (3 * J.element_size() + 4) + (mesh.M + 1) * 4 + U.numel() * U.element_size() \
            + Y.numel() * Y.element_size()
        out[f"spmm_{str(dt)[6:]}"] = {"us": ms * 1e3, "GBs": by / (ms * 1e-3) / 1e9,
                                       "TFLOPs": 6.0 * mesh.nnz * R / (ms * 1e-3) / 1e12}
    del J3
    # median Newton: two steps from b_D (two block-LU factorisations in single-solve mode)
    med = m // 2
    X = bD.repeat(1, 1)
    e0, e1 = ev(), ev()
    torch.cuda.synchronize(); e0.record()
    it, res, st = lrfsi.lrfsi_newton_median(mesh, X, mus[med:med + 1], nus[med:med + 1], 1e-8, 2,
                                            allow_noconv=True)
    e1.record(); torch.cuda.synchronize()
    out["newton_2_steps_ms"] = e0.elapsed_time(e1)
    out["newton_residual_after_2"] = float(res[0])
    # subset operators + preconditioner (assembly, equilibration, block LU keeping the inverses)
    e0, e1 = ev(), ev()
    e0.record()
    sub = lrfsi.Subsets(mesh, X, mus, nus, [m], [R])
    e1.record(); torch.cuda.synchronize()
    out["subset_create_ms"] = e0.elapsed_time(e1)
    # preconditioner solve with r = R right-hand sides (block-LU factors read once)
    Xr = torch.tensor(np.random.default_rng(1).standard_normal((mesh.M, R)), device=dev)
    Yr = torch.zeros(mesh.M, R, dtype=torch.float64, device=dev)
    ms, _ = _timed(torch, lambda: lrfsi.lrfsi_precond_apply(sub, Xr.clone(), R, R, Yr, R), reps=3)
    nb2 = mesh.nmax ** 2
    lu_bytes = 8.0 * nb2 * (3 * mesh.nslab - 2)
    out["precond_solve"] = {"ms": ms, "GBs": lu_bytes / (ms * 1e-3) / 1e9,
                            "TFLOPs": 2.0 * R * nb2 * (3 * mesh.nslab - 2) / (ms * 1e-3) / 1e12}
    # one ChebyshevT iteration on the subset's rank-3 Newton right-hand side
    R3 = torch.zeros(mesh.M * 3, dtype=torch.float64, device=dev)
    lrfsi.lrfsi_assemble_affine(mesh, X[0], None, R3)
    VB = torch.tensor(-np.stack([np.ones(m), mus, nus], 1), device=dev)
    U = torch.zeros(mesh.M * R, dtype=torch.float64, device=dev)
    V = torch.zeros(m * R, dtype=torch.float64, device=dev)
    for iters in (1, 3):
        opt = lrfsi.cheb_options(0.65, 1.0, iters=iters, cycles=1, rank_cap=R, tol=W.tol)
        e0, e1 = ev(), ev()
        torch.cuda.synchronize(); e0.record()
        ranks, st = lrfsi.lrfsi_chebyshevT(sub, R3, 3, VB, 3, [3], opt, U, R, V, R)
        e1.record(); torch.cuda.synchronize()
        out[f"chebyshevT_{iters}_iter_ms"] = e0.elapsed_time(e1)
        out[f"chebyshevT_{iters}_iter_rel_lin_res"] = st[0]["rel_lin_res"]
    out["chebyshevT_ms_per_step"] = (out["chebyshevT_3_iter_ms"] - out["chebyshevT_1_iter_ms"]) / 2
    sub.close()
    print(json.dumps(out))


if __name__ == "__main__":
    {"lu": case_lu, "trunc": case_trunc, "spmm": case_spmm, "large": case_large,
     "ndsolve": case_ndsolve}[sys.argv[1]]()
