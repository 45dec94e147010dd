"""Process-group plumbing for runs on several GPUs of one node.

Algorithm 1's subsets are independent (Sec. 2: the K subset problems can be
solved in parallel), so a job on N processes deals whole subsets out: process
p solves the contiguous block of subsets that ``algorithm1.partition``
assigns it (balanced by m_k R_k), with no exchange during the solve.  At the
end one gather brings every subset's result -- the median solution x~^k, the
factors U_k, V_k, the ranks and the per-column relative residuals -- to
process 0.  The other collectives are a barrier around the timed region and
the maximum of the per-process times.
"""
from __future__ import annotations

import os

import numpy as np


def rank_env():
    """(rank, world, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest ``value`` over all processes (``value`` itself without a
    process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def packed_length(layout, k0, k1, M, R):
    """Doubles in the packed result of subsets k0 .. k1 - 1: per subset x~ (M),
    U (M x R), its rank (1); then V (m_part x R) and the relative residuals
    (m_part)."""
    K = k1 - k0
    m = int(layout.sizes[k0:k1].sum())
    return K * (M + M * R + 1) + m * (R + 1)


def pack(xt, U, V, ranks, relres, M, R):
    """One flat FP64 tensor of a process's results (the layout of
    ``packed_length``); xt is K x M, U holds K blocks of M x R, V m x R."""
    import torch
    K = int(xt.shape[0])
    dev = xt.device
    parts = []
    for k in range(K):
        parts += [xt[k].reshape(-1), U[k * M * R:(k + 1) * M * R],
                  torch.tensor([float(ranks[k])], dtype=torch.float64, device=dev)]
    m = len(relres)
    parts += [V[:m * R], torch.as_tensor(np.asarray(relres, np.float64), device=dev)]
    return torch.cat([p.to(torch.float64) for p in parts])


def unpack(buf, sizes, M, R):
    """Inverse of ``pack`` for subsets of the given sizes: dict with xt
    (K x M), U (K x M x R), ranks (K), V (m x R), relres (m)."""
    K = len(sizes)
    m = int(np.sum(sizes))
    step = M + M * R + 1
    blocks = buf[:K * step].view(K, step) if K else buf[:0].view(0, step)
    out = dict(xt=blocks[:, :M], U=blocks[:, M:M + M * R].reshape(K, M, R),
               ranks=blocks[:, -1].round().long())
    o = K * step
    out["V"] = buf[o:o + m * R].view(m, R)
    out["relres"] = buf[o + m * R:o + m * R + m]
    return out


def gather_results(layout, first, rank, world, packed, M, R, dist, device="cpu"):
    """Gather every process's packed results to process 0 (one collective:
    the buffers are padded to the longest process's length).  Returns, on
    process 0, the list of unpacked results per process (subsets
    first[p] .. first[p + 1] - 1); None elsewhere."""
    import torch
    lens = [packed_length(layout, int(first[p]), int(first[p + 1]), M, R) for p in range(world)]
    assert packed.numel() == lens[rank]
    Lmax = max(lens)
    buf = torch.zeros(Lmax, dtype=torch.float64, device=device)
    buf[:lens[rank]] = packed
    bufs = [torch.zeros(Lmax, dtype=torch.float64, device=device) for _ in range(world)] if rank == 0 else None
    dist.gather(buf, bufs, dst=0)
    if rank != 0:
        return None
    return [unpack(bufs[p][:lens[p]], layout.sizes[int(first[p]):int(first[p + 1])], M, R) for p in range(world)]
