"""The host side of runs on several GPUs, on CPU with the gloo backend and two
processes: one job's subsets are dealt out by the library's partitioner
(contiguous blocks balanced by m_k R_k), every process packs its results
(median solutions, factors, ranks, relative residuals), and one gather brings
them to process 0, which must find every subset exactly once with the values
its owner produced.  The timing reduction takes the maximum."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2008_10275_gb300 import algorithm1, build, inputs, lrfsi, multi  # noqa: E402

M, R = 37, 5   # a stand-in state size and rank cap (the gather does not depend on them)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_results(layout, k0, k1):
    """Deterministic per-subset values that identify their subset and position."""
    K = k1 - k0
    xt = torch.stack([torch.arange(M, dtype=torch.float64) + 1000.0 * (k0 + q) for q in range(K)]) if K else \
        torch.zeros(0, M, dtype=torch.float64)
    U = torch.cat([torch.full((M * R,), float(k0 + q), dtype=torch.float64) for q in range(K)]) if K else \
        torch.zeros(0, dtype=torch.float64)
    a = int(layout.offsets[k0]) if K else 0
    m = int(layout.sizes[k0:k1].sum())
    V = torch.arange(m * R, dtype=torch.float64) + 10.0 * a
    ranks = [min(int(layout.caps[k0 + q]), 3 + (k0 + q) % 3) for q in range(K)]
    rel = np.linspace(1e-7, 9e-7, m) + a
    return xt, U, V, ranks, rel


def _worker(rank, world, port, workload, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, lr = multi.rank_env()
    assert (r, w, lr) == (rank, world, rank)
    lrfsi.load()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        job = algorithm1.workload_layout(inputs.WORKLOADS[workload], replicas=world)
        first = algorithm1.partition(job, world)
        k0, k1 = int(first[rank]), int(first[rank + 1])
        packed = multi.pack(*_fake_results(job, k0, k1), M, R)
        parts = multi.gather_results(job, first, rank, world, packed, M, R, dist)
        ms = multi.max_over_ranks(10.0 + rank, dist)
        dist.barrier()
        if rank == 0:
            out.put((first.tolist(), [{k: v.numpy() for k, v in p.items()} for p in parts], ms))
        else:
            assert parts is None
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("workload", ["medium", "batched"])
def test_two_ranks_partition_and_gather(workload):
    build.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, workload, q)) for r in range(world)]
    for p in procs:
        p.start()
    first, parts, ms = q.get(timeout=180)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ms == 11.0
    job = algorithm1.workload_layout(inputs.WORKLOADS[workload], replicas=world)
    # contiguous, complete, balanced by m_k R_k
    assert first[0] == 0 and first[-1] == job.K and first[0] < first[1] < first[2]
    w = job.weights()
    loads = [int(w[first[p]:first[p + 1]].sum()) for p in range(world)]
    assert max(loads) - min(loads) <= int(w.max())
    # every subset arrives once, with its owner's values
    seen = []
    for p in range(world):
        k0, k1 = first[p], first[p + 1]
        xt, U, V, ranks, rel = _fake_results(job, k0, k1)
        g = parts[p]
        assert g["xt"].shape == (k1 - k0, M) and g["U"].shape == (k1 - k0, M, R)
        m = int(job.sizes[k0:k1].sum())
        assert g["V"].shape == (m, R) and g["relres"].shape == (m,)
        assert np.array_equal(g["xt"], xt.numpy())
        assert np.array_equal(g["U"].reshape(-1), U.numpy())
        assert np.array_equal(g["V"].reshape(-1), V.numpy())
        assert g["ranks"].tolist() == ranks
        assert np.array_equal(g["relres"], rel)
        seen += list(range(k0, k1))
    assert seen == list(range(job.K))


def test_one_process_owns_the_whole_job():
    build.build()
    lrfsi.load()
    job = algorithm1.workload_layout(inputs.WORKLOADS["medium"])
    assert algorithm1.partition(job, 1).tolist() == [0, job.K]
    assert multi.max_over_ranks(3.5) == 3.5
    xt, U, V, ranks, rel = _fake_results(job, 0, job.K)
    g = multi.unpack(multi.pack(xt, U, V, ranks, rel, M, R), job.sizes, M, R)
    assert np.array_equal(g["xt"].numpy(), xt.numpy()) and g["ranks"].tolist() == ranks
