"""The host side of runs on several GPUs, on CPU with the gloo backend and two
processes: every process gets a workload of the same shape on its own strip
of the parameter box, and the timing reduction takes the maximum."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2008_10275_gb300 import inputs, multi  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, lr = multi.rank_env()
    assert (r, w, lr) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        W = inputs.WORKLOADS["medium"]
        mu, nu = inputs.workload_parameters(W, r, w)
        gathered = [torch.zeros(2, len(mu), dtype=torch.float64) for _ in range(w)]
        dist.all_gather(gathered, torch.tensor(np.stack([mu, nu])))
        ms = multi.max_over_ranks(10.0 + rank, dist)
        dist.barrier()
        if rank == 0:
            out.put((np.stack([g.numpy() for g in gathered]), ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_parameters_and_reduce_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    params, ms = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ms == 11.0
    W = inputs.WORKLOADS["medium"]
    n = len(W.mu_values) * len(W.nu_values)
    assert params.shape == (world, 2, n)
    for r in range(world):
        lo, hi = inputs.rank_strip(r, world)
        assert np.all(params[r, 0] >= lo - 1e-9) and np.all(params[r, 0] <= hi + 1e-9)
        assert np.all((params[r, 1] >= inputs.NU_RANGE[0]) & (params[r, 1] <= inputs.NU_RANGE[1]))
    # the same grid shape on every rank, different parameters
    assert not np.allclose(params[0, 0], params[1, 0])
    assert np.array_equal(params[0, 1], params[1, 1])


def test_one_process_keeps_the_workload_grid():
    W = inputs.WORKLOADS["medium"]
    mu, nu = inputs.workload_parameters(W)
    assert np.array_equal(np.unique(mu), np.array(W.mu_values))
    assert np.array_equal(np.unique(nu), np.array(W.nu_values))
    # little endian: mu varies fastest
    assert mu[1] != mu[0] and nu[1] == nu[0]
    assert multi.max_over_ranks(3.5) == 3.5
