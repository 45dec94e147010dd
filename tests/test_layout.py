"""Algorithm 1's parameter bookkeeping in the library (lrfsi_order_grid,
lrfsi_order_set, lrfsi_cluster, lrfsi_medians, lrfsi_partition; host-only
entry points, so these run without a GPU).

* Sec. 3.3, Examples 1 and 2 (tests/golden/clustering_example.json): the
  subsets of the 4 x 5 grid for K = 3 and their upper medians.
* The layouts of the seeded workloads equal the oracle's bookkeeping
  (``oracle.params``: Def. 1 order, Eq. (clustering1), upper median).
* The split over processes is contiguous, covers every subset once and
  minimises the largest block weight (brute force over all splits).
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import params
from paper_2008_10275_gb300 import algorithm1, build, inputs, lrfsi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "clustering_example.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lrfsi.load()


def test_paper_examples_1_and_2():
    g = json.load(open(GOLDEN))
    m1, m2, K = g["m1"], g["m2"], g["K"]
    # the grid of 1-based indices, ordered by the library
    i1, i2 = lrfsi.lrfsi_order_grid(np.arange(1, m1 + 1), np.arange(1, m2 + 1))
    sizes, offs, med = lrfsi.lrfsi_cluster(m1 * m2, K)
    got = [[[int(i1[p]), int(i2[p])] for p in range(o, o + s)] for o, s in zip(offs, sizes)]
    assert got == g["subsets"]
    assert [[int(i1[p]), int(i2[p])] for p in med] == g["upper_medians"]


@pytest.mark.parametrize("name", ["small", "medium", "batched", "large", "learned"])
def test_workload_layouts_match_the_oracle_bookkeeping(name):
    W = inputs.WORKLOADS[name]
    L = algorithm1.workload_layout(W)
    mu_v, nu_v = inputs.workload_values(W)
    if W.seed is None:
        mu, nu = params.ordered_grid(mu_v, nu_v, W.nu_fastest)
        sizes = params.cluster_sizes(len(mu), W.K)
    else:
        o = params.order_set(mu_v, nu_v)
        mu, nu = mu_v[o], nu_v[o]
        sizes = list(W.subset_sizes) if W.subset_sizes else params.cluster_sizes(len(mu), W.K)
    assert np.array_equal(L.mu, mu) and np.array_equal(L.nu, nu)
    assert L.sizes.tolist() == sizes
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    assert L.offsets.tolist() == offs.tolist()
    assert L.medians.tolist() == [int(o + params.upper_median_position(s)) for o, s in zip(offs, sizes)]
    caps = list(W.rank_caps) if W.rank_caps else [W.rank_cap] * W.K
    assert L.caps.tolist() == caps


def test_small_workload_cut_runs_along_mu():
    L = algorithm1.workload_layout(inputs.WORKLOADS["small"])
    a, b = L.columns(0), L.columns(1)
    assert L.mu[a].max() < L.mu[b].min()


def test_order_set_ties_and_errors():
    mu = np.array([3.0, 1.0, 2.0, 1.0, 5.0])
    nu = np.array([1.0, 2.0, 1.0, 2.0, 0.5])
    assert lrfsi.lrfsi_order_set(mu, nu).tolist() == [4, 2, 0, 1, 3]   # equal pairs 1, 3 keep input order
    with pytest.raises(lrfsi.LrfsiError):
        lrfsi.lrfsi_order_set(np.array([1.0, np.nan]), np.array([1.0, 2.0]))
    with pytest.raises(lrfsi.LrfsiError):
        lrfsi.lrfsi_cluster(3, 4)
    with pytest.raises(lrfsi.LrfsiError):
        lrfsi.lrfsi_medians([3, 0, 2])


def _best_split(w, n):
    K = len(w)
    best = None
    for cuts in itertools.combinations(range(1, K), min(n, K) - 1):
        b = [0, *cuts, K]
        worst = max(sum(w[b[i]:b[i + 1]]) for i in range(len(b) - 1))
        best = worst if best is None else min(best, worst)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_partition_is_contiguous_complete_and_optimal(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 10))
    n = int(rng.integers(1, 5))
    w = rng.integers(1, 100, K).astype(np.int64)
    first = lrfsi.lrfsi_partition(w, n)
    assert first[0] == 0 and first[-1] == K and np.all(np.diff(first) >= 0)
    blocks = [w[first[p]:first[p + 1]] for p in range(n)]
    if K >= n:
        assert all(len(b) > 0 for b in blocks)
    assert max(int(b.sum()) for b in blocks) == _best_split(w.tolist(), n)


def test_layout_part_and_job_split():
    W = inputs.WORKLOADS["medium"]
    job = algorithm1.workload_layout(W, replicas=2)
    assert job.K == 8 and job.m == 800
    first = algorithm1.partition(job, 2)
    assert first.tolist() == [0, 4, 8]
    p1 = job.part(4, 8)
    assert p1.K == 4 and p1.m == 400 and p1.offsets.tolist() == [0, 100, 200, 300]
    assert p1.medians.tolist() == [50, 150, 250, 350]
    assert np.array_equal(p1.mu, job.mu[400:]) and np.array_equal(p1.nu, job.nu[400:])


@pytest.mark.parametrize("name,groups", [("medium", 2), ("medium", 4), ("batched", 2), ("batched", 3), ("large", 2)])
def test_group_bounds_cover_the_layout_contiguously(name, groups):
    """The groups that Runner(groups=G) solves concurrently: contiguous blocks of
    whole subsets, every subset and every parameter column in exactly one group,
    the columns of a group those of its subsets, and the heaviest group (m_k
    R_k) within one subset of the mean."""
    L = algorithm1.workload_layout(inputs.WORKLOADS[name])
    b = algorithm1.group_bounds(L, groups)
    assert len(b) == groups
    assert b[0][0] == 0 and b[0][2] == 0 and b[-1][1] == L.K and b[-1][3] == L.m
    for (k0, k1, c0, c1), nxt in zip(b, b[1:] + [None]):
        assert k0 < k1  # no empty group while K >= groups
        assert c0 == int(L.offsets[k0]) and c1 - c0 == int(L.sizes[k0:k1].sum())
        if nxt is not None:
            assert nxt[0] == k1 and nxt[2] == c1
    # balance: the heaviest block of an optimal contiguous split exceeds the
    # mean by less than one subset (a greedy fill at the mean reaches it)
    w = L.weights()
    heaviest = max(int(w[k0:k1].sum()) for k0, k1, _, _ in b)
    assert heaviest <= w.sum() / groups + w.max()
