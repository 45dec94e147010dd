"""Algorithm 1 (Sec. 4) driven through the C ABI.

The parameter bookkeeping -- the little-endian order of a grid (Sec. 3.3,
Def. 1), the contiguous subsets of Eq. (clustering1) and their upper medians
-- is done by the library's host entry points (lrfsi_order_grid,
lrfsi_order_set, lrfsi_cluster, lrfsi_medians); this module only holds the
result (``Layout``) and sequences the device calls of one run (``Runner``):

1. the K upper-median problems by the batched Newton iteration
   (lrfsi_newton_median, from b_D; Sec. 3.2),
2. the K subset operators and mean-based preconditioners at the median
   solutions (lrfsi_subset_create; Sec. 3.4, Sec. 4.2),
3. the subset Newton step on factors with corrections until every column's
   relative residual (Sec. 5.1.2) meets the target (lrfsi_subset_step).

Every arithmetic step runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs, lrfsi


@dataclasses.dataclass
class Layout:
    """An ordered parameter set split into subsets."""
    mu: np.ndarray          # ordered shear moduli (m)
    nu: np.ndarray          # ordered viscosities (m)
    sizes: np.ndarray       # m_k (K)
    offsets: np.ndarray     # first position of each subset (K)
    medians: np.ndarray     # global position of each subset's upper median (K)
    caps: np.ndarray        # rank cap R_k of each subset (K)

    @property
    def m(self):
        return int(len(self.mu))

    @property
    def K(self):
        return int(len(self.sizes))

    def columns(self, k):
        """Positions of subset k's parameters."""
        return slice(int(self.offsets[k]), int(self.offsets[k] + self.sizes[k]))

    def part(self, k0, k1):
        """The layout of subsets k0 .. k1 - 1 alone (positions re-based)."""
        a = int(self.offsets[k0]) if k0 < self.K else self.m
        b = int(self.offsets[k1 - 1] + self.sizes[k1 - 1]) if k1 > k0 else a
        sizes = self.sizes[k0:k1].copy()
        offs, med = lrfsi.lrfsi_medians(sizes) if len(sizes) else (np.zeros(0, np.int32), np.zeros(0, np.int32))
        return Layout(self.mu[a:b].copy(), self.nu[a:b].copy(), sizes, offs[:len(sizes)], med[:len(sizes)],
                      self.caps[k0:k1].copy())

    def weights(self):
        """Work of each subset step, m_k R_k (the balance of a split over processes)."""
        return self.sizes.astype(np.int64) * self.caps.astype(np.int64)


def grid_layout(mu_values, nu_values, K, rank_cap, nu_fastest=False):
    """Def. 1 order of the grid, Eq. (clustering1) subsets, upper medians."""
    mu, nu = lrfsi.lrfsi_order_grid(mu_values, nu_values, nu_fastest)
    sizes, offs, med = lrfsi.lrfsi_cluster(len(mu), K)
    return Layout(mu, nu, sizes, offs, med, np.full(K, rank_cap, np.int32))


def set_layout(mu, nu, K=None, rank_cap=None, sizes=None, caps=None):
    """An unstructured set ordered by lrfsi_order_set, then split into K equal
    subsets (Eq. (clustering1)) or into the given uneven sizes."""
    perm = lrfsi.lrfsi_order_set(mu, nu)
    mu, nu = np.asarray(mu, np.float64)[perm], np.asarray(nu, np.float64)[perm]
    if sizes is None:
        sizes, offs, med = lrfsi.lrfsi_cluster(len(mu), K)
    else:
        sizes = np.asarray(sizes, np.int32)
        if int(sizes.sum()) != len(mu):
            raise ValueError("subset sizes must add up to the number of parameters")
        offs, med = lrfsi.lrfsi_medians(sizes)
    caps = np.full(len(sizes), rank_cap, np.int32) if caps is None else np.asarray(caps, np.int32)
    return Layout(mu, nu, np.asarray(sizes, np.int32), offs, med, caps)


def workload_layout(W, replicas=1):
    """The layout of a seeded workload (``inputs.WORKLOADS``); ``replicas``
    copies of its shape for a job on several GPUs (grid: replicas x more shear
    moduli and subsets; random: replicas x more draws and subsets)."""
    mu, nu = inputs.workload_values(W, replicas)
    if W.seed is None:
        return grid_layout(mu, nu, W.K * replicas, W.rank_cap, W.nu_fastest)
    if W.subset_sizes:
        return set_layout(mu, nu, sizes=list(W.subset_sizes) * replicas, caps=list(W.rank_caps) * replicas)
    return set_layout(mu, nu, K=W.K * replicas, rank_cap=W.rank_cap)


def partition(layout, nproc):
    """Contiguous blocks of subsets per process, balanced by m_k R_k
    (lrfsi_partition): process p owns subsets first[p] .. first[p + 1] - 1."""
    return lrfsi.lrfsi_partition(layout.weights(), nproc)


def group_bounds(layout, groups):
    """Contiguous groups of subsets balanced by m_k R_k (``partition``): one
    (first subset, end subset, first column, end column) per group."""
    first = [int(x) for x in partition(layout, groups)]
    out = []
    for g in range(groups):
        k0, k1 = first[g], first[g + 1]
        c0 = int(layout.offsets[k0]) if k0 < layout.K else layout.m
        c1 = int(layout.offsets[k1]) if k1 < layout.K else layout.m
        out.append((k0, k1, c0, c1))
    return out


class Runner:
    """One run of Algorithm 1 over a layout on the current device.

    ``groups`` > 1 splits the K subsets into that many contiguous groups,
    balanced by m_k R_k (``partition``), each with its own handle, CUDA stream
    and host thread: the subsets are independent (Sec. 2), and the groups'
    phases overlap on the GPU -- the small dense factorisations of one group's
    truncations (a few SMs each) beside another group's solves and products."""

    def __init__(self, mesh, layout, opt, target=1e-6, max_outer=40, eps_N=1e-6, newton_max_it=30,
                 device="cuda:0", groups=1):
        import torch
        self.torch = torch
        self.mesh, self.layout, self.opt = mesh, layout, opt
        self.target, self.max_outer, self.eps_N, self.newton_max_it = target, max_outer, eps_N, newton_max_it
        self.device = device
        self.bD = torch.tensor(mesh.dirichlet(), dtype=torch.float64, device=device)
        self.R = int(layout.caps.max()) if layout.K else 0
        self.U = torch.zeros(max(layout.K * mesh.M * self.R, 1), dtype=torch.float64, device=device)
        self.V = torch.zeros(max(layout.m * self.R, 1), dtype=torch.float64, device=device)
        self.groups = max(1, min(int(groups), layout.K)) if layout.K else 1
        self.bounds = None
        if self.groups > 1:
            from concurrent.futures import ThreadPoolExecutor
            self.bounds = group_bounds(layout, self.groups)
            self.streams = [torch.cuda.Stream(device=device) for _ in range(self.groups)]
            # persistent threads: each keeps its own GEMM workspace in the library
            self.pool = ThreadPoolExecutor(max_workers=self.groups)

    def _subset_step(self, X, mu, nu, opt):
        """The subset step of every subset (one handle, or one per group on its
        own stream and thread); returns ranks, relres, outer, status."""
        L, torch = self.layout, self.torch
        if self.groups == 1:
            sub = lrfsi.Subsets(self.mesh, X, mu, nu, L.sizes, L.caps)
            try:
                ranks, rel, outer, st = lrfsi.lrfsi_subset_step(sub, opt, self.target, self.max_outer,
                                                                self.U, self.R, self.V, self.R)
            finally:
                sub.close()
            return ranks, rel, outer, int(st)
        M, R = self.mesh.M, self.R
        ready = torch.cuda.Event()
        ready.record()  # the median solutions X on the current stream

        def run(g):
            k0, k1, c0, c1 = self.bounds[g]
            s = self.streams[g]
            s.wait_event(ready)
            with torch.cuda.stream(s):
                sub = lrfsi.Subsets(self.mesh, X[k0:k1], mu[c0:c1], nu[c0:c1], L.sizes[k0:k1], L.caps[k0:k1],
                                    stream=s.cuda_stream)
                try:
                    return lrfsi.lrfsi_subset_step(sub, opt, self.target, self.max_outer,
                                                   self.U[k0 * M * R:k1 * M * R], R, self.V[c0 * R:c1 * R], R,
                                                   stream=s.cuda_stream)
                finally:
                    sub.close()

        out = list(self.pool.map(run, range(self.groups)))
        cur = torch.cuda.current_stream()
        for s in self.streams:
            cur.wait_stream(s)
        ranks = np.concatenate([o[0] for o in out])
        rel = np.concatenate([o[1] for o in out])
        outer = np.concatenate([o[2] for o in out])
        st = next((int(o[3]) for o in out if int(o[3]) != 0), 0)
        return ranks, rel, outer, st

    def step(self, mu=None, nu=None, opt=None):
        """Algorithm 1 on the layout's parameters (or on host arrays ``mu``,
        ``nu`` of the same shape).  Returns a dict: xt (K x M device tensor of
        median solutions), ranks, relres (m), outer corrections, Newton
        iterations and the status of the subset step."""
        L = self.layout
        mu = L.mu if mu is None else mu
        nu = L.nu if nu is None else nu
        med = L.medians
        X = self.bD.repeat(L.K, 1)
        it, res, _ = lrfsi.lrfsi_newton_median(self.mesh, X, mu[med], nu[med], self.eps_N, self.newton_max_it)
        ranks, rel, outer, st = self._subset_step(X, mu, nu, opt or self.opt)
        return dict(xt=X, ranks=ranks, relres=rel, outer=outer, newton_iters=it, status=int(st))

    def factors(self, k, ranks):
        """(U_k, V_k) views of subset k's factors (M x r_k, m_k x r_k)."""
        L, M, R = self.layout, self.mesh.M, self.R
        r = int(ranks[k])
        Uk = self.U[k * M * R:(k + 1) * M * R].view(M, R)[:, :r]
        sl = L.columns(k)
        Vk = self.V[sl.start * R:sl.stop * R].view(int(L.sizes[k]), R)[:, :r]
        return Uk, Vk

    def dense(self, result):
        """The dense approximation X^k = x~_k 1^T + U_k V_k^T of every subset (M x m),
        formed by the library's FP64 GEMM."""
        torch = self.torch
        cols = []
        for k in range(self.layout.K):
            Uk, Vk = self.factors(k, result["ranks"])
            mk = int(self.layout.sizes[k])
            Xk = result["xt"][k][:, None].repeat(1, mk).contiguous()
            r = Uk.shape[1]
            if r > 0:
                Uc, Vtc = Uk.contiguous(), Vk.T.contiguous()
                lrfsi.lrfsi_gemm(self.mesh.M, mk, r, Uc, r, Vtc, mk, Xk, mk, 1.0, 1.0, tensor=False)
            cols.append(Xk)
        return torch.cat(cols, 1)


def solve_subsets(mesh, mu, nu, subsets, caps, opt, target, max_outer, eps_N=1e-6, device="cuda:0"):
    """Algorithm 1 on the given contiguous subsets [(start, size)] of the
    ordered parameters (mu, nu) in one batch: the upper-median Newton
    solutions, the subset operators and preconditioners, and the subset step
    with at most ``max_outer`` chord corrections.  Returns one dict per subset:
    start, size, xt, U (M x r), V (size x r), relres."""
    import torch
    sizes = np.array([n for _, n in subsets], np.int32)
    mu_s = np.concatenate([mu[a:a + n] for a, n in subsets])
    nu_s = np.concatenate([nu[a:a + n] for a, n in subsets])
    offs, med = lrfsi.lrfsi_medians(sizes)
    K = len(subsets)
    bD = torch.tensor(mesh.dirichlet(), dtype=torch.float64, device=device)
    X = bD.repeat(K, 1)
    lrfsi.lrfsi_newton_median(mesh, X, mu_s[med[:K]], nu_s[med[:K]], eps_N, 30)
    R = int(max(caps))
    sub = lrfsi.Subsets(mesh, X, mu_s, nu_s, sizes, caps)
    U = torch.zeros(K * mesh.M * R, dtype=torch.float64, device=device)
    V = torch.zeros(int(sizes.sum()) * R, dtype=torch.float64, device=device)
    try:
        ranks, rel, outer, st = lrfsi.lrfsi_subset_step(sub, opt, target, max_outer, U, R, V, R)
    finally:
        sub.close()
    out = []
    for k, (a, n) in enumerate(subsets):
        r = int(ranks[k])
        o = int(offs[k])
        out.append(dict(start=a, size=n, xt=X[k].clone(), U=U[k * mesh.M * R:(k + 1) * mesh.M * R].view(mesh.M, R)[:, :r],
                        V=V[o * R:(o + n) * R].view(n, R)[:, :r], relres=rel[o:o + n].copy(),
                        outer=int(outer[k])))
    return out


def adaptive(mesh, layout, opt, target, min_size=1, max_levels=3, max_outer=40, eps_N=1e-6, device="cuda:0"):
    """Algorithm 1 with adaptively refined subsets (reading of Sec. 5,
    "Alternative ways to cluster the parameter set"): after the subset step,
    every subset whose largest relative residual is above ``target`` and that
    has at least 2 * min_size parameters is split into its two halves
    (Eq. (clustering1) with K = 2 on the subset), each solved again from its
    own upper median, for at most ``max_levels`` levels; subsets still above
    the target then take chord corrections (at most ``max_outer``).  Returns
    the list of per-subset results (see solve_subsets), in parameter order."""
    cap = int(layout.caps.max())
    subs = [(int(a), int(n)) for a, n in zip(layout.offsets, layout.sizes)]

    def batch(items, outer):
        res = []
        for i in range(0, len(items), 32):   # at most 32 subsets per handle
            chunk = items[i:i + 32]
            res += solve_subsets(mesh, layout.mu, layout.nu, chunk, [min(cap, n) for _, n in chunk], opt, target,
                                 outer, eps_N, device)
        return res

    res = {(r["start"], r["size"]): r for r in batch(subs, 0)}
    for _ in range(max_levels):
        refine = [s for s in subs if res[s]["relres"].max() > target and s[1] >= 2 * min_size]
        if not refine:
            break
        halves = []
        for s in refine:
            a, n = s
            halves += [(a, n // 2), (a + n // 2, n - n // 2)]
        for r in batch(halves, 0):
            res[(r["start"], r["size"])] = r
        nxt = []
        for s in subs:
            if s in refine:
                nxt += [(s[0], s[1] // 2), (s[0] + s[1] // 2, s[1] - s[1] // 2)]
            else:
                nxt.append(s)
        subs = nxt
    late = [s for s in subs if res[s]["relres"].max() > target]
    if late and max_outer > 0:
        for r in batch(late, max_outer):
            res[(r["start"], r["size"])] = r
    return [res[s] for s in subs]
