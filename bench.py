#!/usr/bin/env python
"""Benchmark: parameter solves per second of Algorithm 1 to a nonlinear
relative residual <= 1e-6 in every parameter column, on one GB300 per rank.

One step = the whole hot path over the workload's parameter set: batched
Newton for the K upper-median problems (from b_D), the K subset operators and
mean-based preconditioners (assembly, equilibration, block LU), and the
subset Newton step solved by the truncated preconditioned Chebyshev iteration
with nonlinear-residual corrections until every column meets the target.
The line also carries the same step with the mixed-precision inner residual
("mixed") and with the truncated GMRES as the low-rank solver ("gmrest").

--impl reference times the CPU oracle (the paper's "standard Newton":
consecutive per-parameter Newton with a sparse direct solve) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2008_10275_gb300 import inputs, multi  # noqa: E402

METRIC = "parameter solves/sec to nonlinear rel. residual 1e-6"
EPS_N = 1e-6                 # median Newton stopping tolerance ||R||_2 (the paper's epsilon_N, Sec. 5)


def fp64_peak(dev, n=4096, reps=10):
    """Measured FP64 rate of this GPU: a cuBLAS DGEMM n^3 (torch.matmul on
    float64), best of ``reps`` by CUDA events (the FP64 counterpart of the
    bf16 GEMM peak measured for the pool)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    c = a @ b
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12, f"cuBLAS DGEMM {n}^3 measured in this run (best of {reps})"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                parts = [p.strip() for p in out.stdout.strip().split(",")]
                if len(parts) == 7:
                    self.samples.append(parts)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_reference(workload, n_sample, procs=1):
    """The oracle's standard Newton (Sec. 5.1.2) on the first n_sample
    parameters of the workload, in a fresh process; with procs > 1 the sample
    is split into procs consecutive chunks solved by spawned single-threaded
    worker processes (each chunk warm-started along its own parameters), and
    the wall time includes their start-up and mesh construction."""
    code = f"""
import sys, time, json, multiprocessing as mp, numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import fsi, newton
from paper_2008_10275_gb300 import inputs
from oracle import params
W = inputs.WORKLOADS[{workload!r}]
mu_v, nu_v = inputs.workload_values(W)
if W.seed is None:
    mus, nus = params.ordered_grid(mu_v, nu_v, W.nu_fastest)
else:
    o = params.order_set(mu_v, nu_v)
    mus, nus = mu_v[o], nu_v[o]
n, p = {n_sample}, {procs}
if p == 1:
    m = fsi.Mesh(fsi.Problem(W.nx, W.ny))
    t = time.perf_counter()
    X, steps, norms = newton.standard_newton(m, mus[:n], nus[:n], eps={EPS_N!r})
    dt = time.perf_counter() - t
else:
    work = [(W.nx, W.ny, mus[n * k // p:n * (k + 1) // p], nus[n * k // p:n * (k + 1) // p], {EPS_N!r})
            for k in range(p)]
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(p) as pool:
        steps = sum(pool.starmap(newton.standard_newton_problem, work, chunksize=1))
    dt = time.perf_counter() - t
print(json.dumps(dict(seconds=dt, steps=int(steps), n=n, procs=p)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_algorithm1(workload, n_sample, c=0.65, d=1.0, eta=0.05, target=1e-6):
    """The oracle's own Algorithm 1 (Sec. 4; dense truncated ChebyshevT with
    the workload's rank cap and tolerance) on the first n_sample parameters as
    one subset: the median's Newton solve, then the subset step with chord
    corrections until every column is <= target; one thread, fresh process."""
    code = f"""
import sys, time, json, numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import algorithm1, fsi, newton, params
from paper_2008_10275_gb300 import inputs
W = inputs.WORKLOADS[{workload!r}]
mu_v, nu_v = inputs.workload_values(W)
if W.seed is None:
    mus, nus = params.ordered_grid(mu_v, nu_v, W.nu_fastest)
else:
    o = params.order_set(mu_v, nu_v)
    mus, nus = mu_v[o], nu_v[o]
mu, nu = mus[:{n_sample}], nus[:{n_sample}]
m = fsi.Mesh(fsi.Problem(W.nx, W.ny))
opt = algorithm1.Options(K=1, rank_cap=W.rank_cap, tol=W.tol, c={c!r}, d={d!r}, iters=6, cycles=2, eta={eta!r})
t = time.perf_counter()
med = params.upper_median_position(len(mu))
xt, it, r = newton.newton(m, mu[med], nu[med], eps={EPS_N!r})
X, k, rr = algorithm1.subset_step_to_target(m, xt, mu, nu, opt, {target!r})
dt = time.perf_counter() - t
print(json.dumps(dict(seconds=dt, n=len(mu), newton=int(it), corrections=int(k), max_relres=float(rr.max()))))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args, rank, world):
    """The oracle's standard Newton on all host cores: every step solves a
    bounded sample of 2 parameters per core (consecutive chunks, one
    single-threaded process per core)."""
    if rank != 0:
        return 0
    W = inputs.WORKLOADS[args.workload]
    cores = host_cores()
    n = 2 * cores
    vals = []
    last = None
    for i in range(args.warmup + args.steps):
        r = cpu_reference(args.workload, n, procs=cores)
        if i >= args.warmup:
            vals.append(r["n"] / r["seconds"])
        last = r
    v = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "params/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * last["seconds"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W.name, "mesh": f"{W.nx}x{W.ny}", "sample_params": n},
        "cpu_baseline": {"value": v, "unit": "params/s", "cores": cores, "kind": "oracle",
                         "sample": f"standard Newton (eps {EPS_N:g}) on the first {n} parameters, {cores} "
                                   f"single-threaded processes of {n // cores} consecutive parameters each, "
                                   f"start-up included"},
        "e2e": {"value": v, "unit": "params/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args, rank, world):
    """The learned-start workload: an MLP trained on 500 method-generated
    solutions (Latin hypercube parameters, 5 subsets of 100) starts both the
    median Newton iterations and the subset steps for 2000 held-out uniform
    parameters (20 subsets of 100, nu_f-major order).  Three arms on the same
    parameters: the plain FP64 method (median Newton from b_D, subset step
    from the median solution), the learned start in FP64, and the learned
    start with the mixed-precision inner residual (the line's value)."""
    import torch
    from paper_2008_10275_gb300 import algorithm1, build, lrfsi
    build.build()
    lrfsi.load()
    dev = "cuda:0"
    W = inputs.WORKLOADS["learned"]
    mesh = lrfsi.Mesh(W.nx, W.ny)
    M, R = mesh.M, W.rank_cap
    bD = torch.tensor(mesh.dirichlet(), dtype=torch.float64, device=dev)
    opts = [lrfsi.cheb_options(args.c, args.d, iters=6, cycles=2, rank_cap=R, tol=W.tol, precision=pr, eta=args.eta)
            for pr in (0, 1)]

    from concurrent.futures import ThreadPoolExecutor
    streams = [torch.cuda.Stream(device=dev) for _ in range(max(1, args.streams))]
    pool = ThreadPoolExecutor(max_workers=max(1, args.streams))

    def layout(mus, nus, K):
        Ly = algorithm1.set_layout(mus, nus, K=K, rank_cap=R)  # nu_f-major, mu fastest
        return Ly.mu, Ly.nu, Ly.sizes.tolist(), Ly.medians.tolist()

    def solve(mus, nus, K, ls=None, precision=0):
        """Method on (mus, nus): returns dense solutions (M x m) and stats."""
        opt = opts[precision]
        mus, nus, sizes, medians = layout(mus, nus, K)
        m = len(mus)
        X = bD.repeat(K, 1)
        if ls is not None:  # learned start of the median Newton iterations
            ls.start(mus[medians], nus[medians], X)
        it, res, _ = lrfsi.lrfsi_newton_median(mesh, X, mus[medians], nus[medians], EPS_N, 30)
        U = torch.zeros(K * M * R, dtype=torch.float64, device=dev)
        V = torch.zeros(m * R, dtype=torch.float64, device=dev)
        if ls is not None:
            k = ls.k
            U0 = torch.zeros(K * M * (k + 1), dtype=torch.float64, device=dev)
            V0 = torch.zeros(m * (k + 1), dtype=torch.float64, device=dev)
            ls.factors(sizes, mus, nus, X, U0, V0)
        # the subset steps in concurrent groups (contiguous, balanced by m_k R_k),
        # each with its own handle, stream and host thread, as Runner(groups=...)
        G = max(1, min(args.streams, K))
        first = [int(x) for x in lrfsi.lrfsi_partition(np.asarray(sizes, np.int64) * R, G)]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
        ready = torch.cuda.Event()
        ready.record()

        def run(g):
            k0, k1 = first[g], first[g + 1]
            c0, c1 = int(offs[k0]), int(offs[k1])
            s = streams[g]
            s.wait_event(ready)
            with torch.cuda.stream(s):
                sub = lrfsi.Subsets(mesh, X[k0:k1], mus[c0:c1], nus[c0:c1], sizes[k0:k1], [R] * (k1 - k0),
                                    stream=s.cuda_stream)
                try:
                    Ug, Vg = U[k0 * M * R:k1 * M * R], V[c0 * R:c1 * R]
                    if ls is None:
                        rk, rl, ou, st_ = lrfsi.lrfsi_subset_step(sub, opt, args.target, args.max_outer, Ug, R, Vg, R,
                                                                  stream=s.cuda_stream)
                        return rk, rl, ou, np.zeros(c1 - c0, np.int32), st_
                    kk = ls.k + 1
                    return lrfsi.lrfsi_subset_step_init(sub, opt, args.target, args.max_outer,
                                                        U0[k0 * M * kk:k1 * M * kk], kk, V0[c0 * kk:c1 * kk], kk, kk,
                                                        Ug, R, Vg, R, stream=s.cuda_stream)
                finally:
                    sub.close()

        outs = list(pool.map(run, range(G)))
        cur = torch.cuda.current_stream()
        for s in streams[:G]:
            cur.wait_stream(s)
        ranks = np.concatenate([o[0] for o in outs])
        rel = np.concatenate([o[1] for o in outs])
        outer = np.concatenate([o[2] for o in outs])
        fb = np.concatenate([o[3] for o in outs])
        st = next((int(o[4]) for o in outs if int(o[4]) != 0), 0)
        cols, o = [], 0
        for q in range(K):
            r = int(ranks[q])
            Uq = U[q * M * R:(q + 1) * M * R].view(M, R)[:, :r].contiguous()
            Vtq = V[o * R:(o + sizes[q]) * R].view(sizes[q], R)[:, :r].T.contiguous()
            Xq = X[q][:, None].repeat(1, sizes[q]).contiguous()
            if r > 0:   # the library's FP64 GEMM: X_q = x~_q 1^T + U_q V_q^T
                lrfsi.lrfsi_gemm(M, sizes[q], r, Uq, r, Vtq, sizes[q], Xq, sizes[q], 1.0, 1.0, tensor=False)
            cols.append(Xq)
            o += sizes[q]
        return torch.cat(cols, 1), dict(newton_steps=int(it.sum()), newton_max=int(it.max()),
                                        outer=outer.tolist(), max_relres=float(rel.max()), status=int(st),
                                        fallbacks=int(fb.sum()))

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    # training data: the method itself on 500 Latin-hypercube parameters
    mu_t, nu_t = inputs.latin_hypercube(500, seed=W.seed + 1)
    ms_gen, (Xt, st_t) = timed(lambda: solve(mu_t, nu_t, 5))
    mu_ts, nu_ts, _, _ = layout(mu_t, nu_t, 5)
    k = 64
    ls = lrfsi.LearnedStart(mesh, k=k, seed=W.seed)
    Xtrain = Xt.T.contiguous()  # problem-major
    ms_fit, loss = timed(lambda: ls.fit(Xtrain, mu_ts, nu_ts, epochs=12000, lr=2e-3))
    # evaluation on 2000 held-out parameters
    mu_e, nu_e = inputs.workload_values(W)
    for _ in range(max(1, args.warmup)):
        solve(mu_e[:200], nu_e[:200], 2)
        solve(mu_e[:200], nu_e[:200], 2, ls)
        solve(mu_e[:200], nu_e[:200], 2, ls, 1)
    ms_plain, (Xp, st_p) = timed(lambda: solve(mu_e, nu_e, W.K))
    ms_l64, (Xl64, st_l64) = timed(lambda: solve(mu_e, nu_e, W.K, ls))
    ms_learn, (Xl, st_l) = timed(lambda: solve(mu_e, nu_e, W.K, ls, 1))
    diff = float(torch.linalg.norm(Xl - Xp) / torch.linalg.norm(Xp - bD[:, None]))
    diff64 = float(torch.linalg.norm(Xl64 - Xp) / torch.linalg.norm(Xp - bD[:, None]))
    m = len(mu_e)
    line = {
        "metric": METRIC, "value": m / (ms_learn * 1e-3), "unit": "params/s", "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": ms_learn, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": W.name, "mesh": f"{W.nx}x{W.ny}", "M": M, "params": m, "subsets": W.K, "rank_cap": R,
                   "train": "500 method solutions at Latin-hypercube parameters", "pod_rank": k,
                   "mlp": "2-128-128-64 GELU, BF16 weights", "concurrent_groups": max(1, args.streams)},
        "learned_mixed": {**st_l, "ms": ms_learn, "params_per_s": m / (ms_learn * 1e-3)},
        "learned_fp64": {**st_l64, "ms": ms_l64, "params_per_s": m / (ms_l64 * 1e-3)},
        "plain_fp64": {**st_p, "ms": ms_plain, "params_per_s": m / (ms_plain * 1e-3)},
        "speedup_learned_mixed_vs_plain_fp64": ms_plain / ms_learn,
        "speedup_learned_fp64_vs_plain_fp64": ms_plain / ms_l64,
        "rel_diff_learned_mixed_vs_plain_fp64_solution_update": diff,
        "rel_diff_learned_fp64_vs_plain_fp64_solution_update": diff64,
        "train": {"generate_ms": ms_gen, "fit_ms": ms_fit, "final_loss": loss, "epochs": 12000,
                  "generate_status": st_t["status"], "generate_max_relres": st_t["max_relres"]},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="medium")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--c", type=float, default=0.65)
    ap.add_argument("--d", type=float, default=1.0)
    ap.add_argument("--target", type=float, default=1e-6)
    ap.add_argument("--max-outer", type=int, default=40)
    ap.add_argument("--ref-sample", type=int, default=4)
    ap.add_argument("--eta", type=float, default=0.05)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-gmres", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--streams", type=int, default=2,
                    help="groups of subsets run concurrently, each on its own stream and host thread")
    args = ap.parse_args()

    rank, world, local = multi.rank_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "learned":
        if rank != 0:
            return 0
        return run_learned(args, rank, world)

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the lrfsi library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2008_10275_gb300 import algorithm1, build, lrfsi
    build.build()
    lrfsi.load()
    dev = f"cuda:{local}"
    W = inputs.WORKLOADS[args.workload]
    # one workload for the whole job: `world` copies of the configuration's
    # shape, its subsets dealt out to the processes in contiguous blocks
    # balanced by m_k R_k; one gather of the results to process 0 per step
    job = algorithm1.workload_layout(W, replicas=world)
    first = algorithm1.partition(job, world)
    L = job.part(int(first[rank]), int(first[rank + 1]))
    m, K = L.m, L.K
    mesh = lrfsi.Mesh(W.nx, W.ny)
    bD = torch.tensor(mesh.dirichlet(), dtype=torch.float64, device=dev)
    R = int(job.caps.max())

    opt_mixed = lrfsi.cheb_options(args.c, args.d, iters=6, cycles=2, rank_cap=R, tol=W.tol, precision=1,
                                   eta=args.eta)
    opt = lrfsi.cheb_options(args.c, args.d, iters=6, cycles=2, rank_cap=R, tol=W.tol, precision=args.precision,
                             eta=args.eta)
    opt_gmres = lrfsi.cheb_options(args.c, args.d, iters=6, cycles=2, rank_cap=R, tol=W.tol, precision=0,
                                   eta=args.eta, solver="gmres")
    # subsets solved together: all of them, or groups of W.group (memory of the large mesh)
    gsz = W.group or K
    runs = [algorithm1.Runner(mesh, L.part(a, min(a + gsz, K)), opt, target=args.target, max_outer=args.max_outer,
                              eps_N=EPS_N, device=dev, groups=args.streams) for a in range(0, K, gsz)]
    run = runs[0]
    U, V = run.U, run.V
    mus, nus = L.mu, L.nu

    def step(mu_h, nu_h, o=None):
        res_all, off = [], 0
        for rn in runs:
            mg = rn.layout.m
            res_all.append(rn.step(mu_h[off:off + mg], nu_h[off:off + mg], o))
            off += mg
        res = dict(xt=torch.cat([r["xt"] for r in res_all]), ranks=np.concatenate([r["ranks"] for r in res_all]),
                   relres=np.concatenate([r["relres"] for r in res_all]),
                   outer=np.concatenate([r["outer"] for r in res_all]),
                   newton_iters=np.concatenate([r["newton_iters"] for r in res_all]),
                   status=min(r["status"] for r in res_all))
        if dist is not None:
            packed = multi.pack(res["xt"], U, V, res["ranks"], res["relres"], mesh.M, R)
            multi.gather_results(job, first, rank, world, packed, mesh.M, R, dist, device=dev)
        return dict(newton_iters=res["newton_iters"].tolist(), ranks=res["ranks"].tolist(),
                    outer=res["outer"].tolist(), max_relres=float(res["relres"].max()) if m else 0.0,
                    status=res["status"], xt=res["xt"], parts=res_all)

    def dense_solution(info):
        return torch.cat([rn.dense(p) for rn, p in zip(runs, info["parts"])], 1)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    peak64, peak64_src = fp64_peak(dev)
    info = None
    for _ in range(args.warmup):
        info = step(mus, nus)
    stream = torch.cuda.current_stream()
    L0, H0 = lrfsi.kernel_launches(), lrfsi.host_launches()
    lrfsi.truncation_counters(reset=True)
    barrier()
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            info = step(mus, nus)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (lrfsi.kernel_launches() - L0) / args.steps
    host_launches = (lrfsi.host_launches() - H0) / args.steps
    trunc_counts = lrfsi.truncation_counters()
    ms = multi.max_over_ranks(ms, dist, dev)
    value = job.m / (ms * 1e-3)

    X64 = dense_solution(info)
    mixed = None
    if not args.no_mixed:
        # the mixed-precision path (FP32 SpMM / residual GEMM inside the FP64 correction loop)
        step(mus, nus, opt_mixed)
        barrier()
        e4 = torch.cuda.Event(enable_timing=True)
        e5 = torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        for _ in range(args.steps):
            info_m = step(mus, nus, opt_mixed)
        e5.record(stream)
        barrier()
        ms_m = e4.elapsed_time(e5) / args.steps
        Xm = dense_solution(info_m)
        diff = float(torch.linalg.norm(Xm - X64) / torch.linalg.norm(X64 - bD[:, None]))
        # where the mixed step spends its time (one more step with per-launch events)
        lrfsi.stats_reset()
        lrfsi.timing(True)
        step(mus, nus, opt_mixed)
        torch.cuda.synchronize()
        ksm = lrfsi.kernel_stats()
        lrfsi.timing(False)
        mixed = {"value": job.m / (ms_m * 1e-3), "ms_per_step": ms_m, "max_relres": info_m["max_relres"],
                 "status": info_m["status"], "outer": info_m["outer"],
                 "rel_diff_vs_fp64_solution_update": diff,
                 "per_class_ms": {k: round(v["ms"], 3) for k, v in ksm.items() if v["ms"] > 0},
                 "spmm_fp32_gbs": (ksm["spmm_fp32"]["bytes"] / (ksm["spmm_fp32"]["ms"] * 1e-3) / 1e9
                                   if ksm["spmm_fp32"]["ms"] > 0 else None)}

    gmres = None
    if not args.no_gmres:
        # the same Algorithm 1 with GMREST as the low-rank solver (FP64)
        step(mus, nus, opt_gmres)
        barrier()
        e6 = torch.cuda.Event(enable_timing=True)
        e7 = torch.cuda.Event(enable_timing=True)
        e6.record(stream)
        for _ in range(args.steps):
            info_g = step(mus, nus, opt_gmres)
        e7.record(stream)
        barrier()
        ms_g = e6.elapsed_time(e7) / args.steps
        Xg = dense_solution(info_g)
        diff_g = float(torch.linalg.norm(Xg - X64) / torch.linalg.norm(X64 - bD[:, None]))
        lrfsi.stats_reset()
        lrfsi.timing(True)
        step(mus, nus, opt_gmres)
        torch.cuda.synchronize()
        ksg = lrfsi.kernel_stats()
        lrfsi.timing(False)
        gmres = {"value": job.m / (ms_g * 1e-3), "ms_per_step": ms_g, "max_relres": info_g["max_relres"],
                 "status": info_g["status"], "outer": info_g["outer"], "ranks": info_g["ranks"],
                 "rel_diff_vs_chebyshev_solution_update": diff_g,
                 "per_class_ms": {k: round(v["ms"], 3) for k, v in ksg.items() if v["ms"] > 0}}

    # end to end through the public API: host parameter arrays in, factors and
    # relative residuals back to host memory every step
    h2d = 2 * m * 8
    d2h = (K * mesh.M * R + m * R) * 8 + m * 8
    barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        mu_host = np.array(mus, copy=True)
        nu_host = np.array(nus, copy=True)
        step(mu_host, nu_host)
        for rn in runs:
            Uh = rn.U.cpu()
            Vh = rn.V.cpu()
    e3.record(stream)
    barrier()
    ms_e2e = e2.elapsed_time(e3) / args.steps
    ms_e2e = multi.max_over_ranks(ms_e2e, dist, dev)

    # roofline of the dominant kernel class: one more step with per-launch events
    lrfsi.stats_reset()
    lrfsi.timing(True)
    step(mus, nus)
    torch.cuda.synchronize()
    ks = lrfsi.kernel_stats()
    lrfsi.timing(False)
    # block_lu and lu_solve are timed regions that contain GEMM launches, so
    # they overlap gemm_fp64 and are not candidates for the dominant kernel
    dom = max((k for k in ks if k not in lrfsi.REGION_CLASSES), key=lambda k: ks[k]["ms"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    d = ks[dom]
    tc = ks.get("tc_mma")
    if dom in lrfsi.TENSOR_CLASSES and tc and tc["ms"] > 0:
        # FP64 products by error-free splitting: the dominant kernels are the
        # slice products (k_oz_gemm, k_oz_gram), BF16 MMA FLOPs issued over
        # their own launch time against the measured BF16 peak
        bf = peaks.get("bf16_tflops", 1900.0)
        achieved = tc["flops"] / (tc["ms"] * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf, "unit": "TFLOP/s", "frac": achieved / bf,
                "traffic": None, "kernel": "k_oz_gemm, k_oz_gram, k_oz_ndgemm (class %s)" % dom,
                "peak_source": "of measured (bf16 burst)" if "bf16_tflops" in peaks else "of fallback",
                "fp64_equiv_tflops": round(d["flops"] / (d["ms"] * 1e-3) / 1e12, 4)}
    elif dom in ("gemm_fp64", "gram_fp64", "trunc_small", "trunc_svd", "lu_panel", "lu_trsm", "fe_assembly"):
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                "frac": achieved / peak64, "traffic": None, "kernel": dom, "peak_source": peak64_src,
                "peak_nominal_fp64": 1.25,
                "peak_fp64_from_bf16": round(peaks["bf16_tflops"] * 1.25 / 2250.0, 4) if "bf16_tflops" in peaks
                else None}
    else:
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": dom, "peak_source": "of measured" if "hbm_gbs" in peaks else "of fallback"}
    # DRAM traffic per launch of the dominant kernel from an ncu capture of the
    # profile case (python -m paper_2008_10275_gb300.profile_cases trunc; the
    # summary under profiles/ names the command): dram__bytes_read.sum +
    # dram__bytes_write.sum of one launch; None for kernels not captured since
    # their last change
    traffic = {"trunc_svd": (117248, "k_trunc_svd, ncu on the truncation profile case (80x16, 4 subsets, the 10th "
                                     "launch): DRAM read 117,248 B, write 0; its inputs are L2-resident work arrays")}
    if dom in traffic:
        roof["traffic"], roof["traffic_source"] = traffic[dom]
    roof["per_class_ms"] = {k: round(v["ms"], 3) for k, v in ks.items()}
    # algorithmic FP rate per class (TFLOP/s over its own launch time) and launches
    roof["per_class_tflops"] = {k: round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 4)
                                for k, v in ks.items() if v["ms"] > 0 and v["flops"] > 0}
    # (tensor-core classes: FP64-equivalent rates, above the FP64 roof by design)
    roof["per_class_frac_fp64"] = {k: round(v / peak64, 4) for k, v in roof["per_class_tflops"].items()
                                   if not k.endswith("fp32") and k not in lrfsi.TENSOR_CLASSES and k != "tc_mma"}
    roof["per_class_launches"] = {k: int(v["launches"]) for k, v in ks.items() if v["launches"] > 0}
    # the tensor-core slice products (k_oz_gram, k_oz_gemm): BF16 MMA FLOPs issued
    # over their own launch time, against the measured BF16 peak
    if tc and tc["ms"] > 0 and tc["flops"] > 0:
        bf = peaks.get("bf16_tflops")
        tflops = tc["flops"] / (tc["ms"] * 1e-3) / 1e12
        roof["tensor"] = {"bound": "tensor", "kernels": "k_oz_gram, k_oz_gemm, k_oz_ndgemm", "achieved": round(tflops, 2),
                          "peak": bf, "unit": "TFLOP/s", "frac": round(tflops / bf, 4) if bf else None,
                          "ms": round(tc["ms"], 3), "launches": int(tc["launches"]),
                          "peak_source": "of measured (bf16 burst)" if bf else None}
    spmm = ks["spmm_fp64"]
    spmm_gbs = spmm["bytes"] / (spmm["ms"] * 1e-3) / 1e9 if spmm["ms"] > 0 else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            r = cpu_reference(args.workload, args.ref_sample)
            cpu = {"value": r["n"] / r["seconds"], "unit": "params/s", "cores": 1, "kind": "oracle",
                   "sample": f"standard Newton (eps {EPS_N:g}) on the first {args.ref_sample} of {m} parameters, "
                             f"{r['steps']} Newton steps, {r['seconds']:.1f} s"}
            ra = cpu_algorithm1(args.workload, 20, c=args.c, d=args.d, eta=args.eta, target=args.target)
            cpu["algorithm1"] = {"value": ra["n"] / ra["seconds"], "unit": "params/s", "cores": 1,
                                 "sample": f"the oracle's Algorithm 1 (dense truncated ChebyshevT, rank cap "
                                           f"{W.rank_cap}, tol {W.tol:g}) on the first {ra['n']} parameters as one "
                                           f"subset: median Newton ({ra['newton']} steps), subset step and "
                                           f"{ra['corrections']} chord corrections to max relres "
                                           f"{ra['max_relres']:.1e}, {ra['seconds']:.1f} s"}
            cores = host_cores()
            if cores > 1:  # the same method on every host core, 2 parameters per core
                ra = cpu_reference(args.workload, 2 * cores, procs=cores)
                cpu["all_cores"] = {"value": ra["n"] / ra["seconds"], "unit": "params/s", "cores": cores,
                                    "sample": f"the first {ra['n']} parameters in {cores} single-threaded processes, "
                                              f"{ra['steps']} Newton steps, {ra['seconds']:.1f} s wall incl. start-up"}
        except Exception as ex:  # reported, not fatal
            cpu = {"value": None, "unit": "params/s", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "params/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f64+f32", "data": "synthetic",
            "config": {"workload": W.name, "mesh": f"{W.nx}x{W.ny}", "M": mesh.M, "nnz": mesh.nnz, "params": m,
                       "subsets": K, "rank_cap": R, "tol": W.tol, "cheb": [args.c, args.d, 6, 2],
                       "target_relres": args.target, "l2": "working set (block-LU factors) larger than L2",
                       "parallelism": (f"{world} rank(s); the job's {job.K} subsets in contiguous blocks "
                                       f"balanced by m_k R_k, one gather of the results to rank 0 per step"
                                       if world > 1 else "1 rank"),
                       "concurrent_groups": runs[0].groups},
            "clocks": clk.summary(),
            "e2e": {"value": job.m / (ms_e2e * 1e-3), "unit": "params/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "host_launches": int(host_launches),
            "roofline": roof,
            "spmm_gbs": spmm_gbs,
            "cpu_baseline": cpu,
            "result": {**{k: v for k, v in info.items() if k not in ("xt", "parts")}, "truncation": trunc_counts},
            "mixed": mixed,
            "gmrest": gmres,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
