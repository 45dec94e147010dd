"""Process-group plumbing for runs on several GPUs of one node.

Algorithm 1's subsets and parameter sets are independent, so processes never
exchange solver data: each one solves its own parameters
(``inputs.workload_parameters``) and the only collectives are a barrier around
the timed region and the maximum of the per-process times."""
from __future__ import annotations

import os


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
