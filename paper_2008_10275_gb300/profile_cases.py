"""Small, self-contained cases of the hot kernels for profiling (ncu) and
timing outside the full step.

    python -m paper_2008_10275_gb300.profile_cases lu       # K block-LU factorisations (subset preconditioners)
    python -m paper_2008_10275_gb300.profile_cases trunc    # median Newton + two correction steps (truncations)
    python -m paper_2008_10275_gb300.profile_cases spmm     # FP64 and FP32 SpMM of the affine operators

Each case builds the 80 x 16 channel mesh (M = 22629) with the seeded
parameters of the 400-parameter workload, runs the case twice (the first run
warms up) and prints the CUDA-event time of the second run.
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
    W = inputs.WORKLOADS["medium"]
    mesh = lrfsi.Mesh(W.nx, W.ny)
    mus, nus = inputs.workload_parameters(W)
    return torch, lrfsi, W, mesh, mus, nus


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


if __name__ == "__main__":
    {"lu": case_lu, "trunc": case_trunc, "spmm": case_spmm}[sys.argv[1]]()
