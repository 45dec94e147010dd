"""The seeded workload descriptions and draws (paper_2008_10275_gb300/inputs.py):
sizes, ranges and determinism (the module holds no ordering rule)."""
import numpy as np

from paper_2008_10275_gb300 import inputs


def test_box_and_grid_workloads():
    for name in ("small", "medium", "large"):
        W = inputs.WORKLOADS[name]
        mu, nu = inputs.workload_values(W)
        assert (len(mu), len(nu)) == (len(W.mu_values), len(W.nu_values))
        assert mu.min() == inputs.MU_RANGE[0] and mu.max() == inputs.MU_RANGE[1]
        assert nu.min() == inputs.NU_RANGE[0] and nu.max() == inputs.NU_RANGE[1]
        assert np.all(np.diff(mu) > 0) and np.all(np.diff(nu) > 0)
    # replicas refine the viscosities over the same range
    W = inputs.WORKLOADS["medium"]
    mu4, nu4 = inputs.workload_values(W, replicas=4)
    assert len(nu4) == 4 * len(W.nu_values) and np.array_equal(mu4, np.array(W.mu_values))
    assert nu4[0] == inputs.NU_RANGE[0] and nu4[-1] == inputs.NU_RANGE[1]


def test_batched_workload_sizes_and_caps():
    W = inputs.WORKLOADS["batched"]
    assert len(W.subset_sizes) == W.K == 16 and sum(W.subset_sizes) == W.n_random == 1000
    assert min(W.subset_sizes) >= 8 and max(W.subset_sizes) <= 64
    assert len(W.rank_caps) == 16 and max(W.rank_caps) == 60 and min(W.rank_caps) == 20
    assert list(W.rank_caps) == sorted(W.rank_caps, reverse=True)
    assert inputs.uneven_sizes() == inputs.uneven_sizes()  # seeded


def test_random_workloads_are_seeded_and_in_the_box():
    for name in ("batched", "learned"):
        W = inputs.WORKLOADS[name]
        a = inputs.workload_values(W)
        b = inputs.workload_values(W)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert len(a[0]) == W.n_random
        assert np.all((a[0] >= inputs.MU_RANGE[0]) & (a[0] <= inputs.MU_RANGE[1]))
        assert np.all((a[1] >= inputs.NU_RANGE[0]) & (a[1] <= inputs.NU_RANGE[1]))
    mu, nu = inputs.latin_hypercube(50, seed=3)
    # one sample per stratum in each coordinate
    for v, (lo, hi) in ((mu, inputs.MU_RANGE), (nu, inputs.NU_RANGE)):
        strata = np.floor((v - lo) / (hi - lo) * 50).astype(int)
        assert sorted(strata.tolist()) == list(range(50))


def test_mlp_init_layout():
    sizes = (2, 128, 128, 64)
    p = inputs.mlp_init(sizes, seed=0)
    n = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    assert p.dtype == np.float32 and p.size == n
    assert np.array_equal(p, inputs.mlp_init(sizes, seed=0))
    assert not np.array_equal(p, inputs.mlp_init(sizes, seed=1))
    # biases zero, weights He-scaled
    o = 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        w = p[o:o + a * b]; o += a * b
        assert abs(w.std() - np.sqrt(2.0 / a)) < 0.25 * np.sqrt(2.0 / a)
        assert np.all(p[o:o + b] == 0); o += b


def test_random_state_magnitudes():
    M, nq2 = 1581, 369
    x = inputs.random_state(M, 5, nq2=nq2)
    assert np.array_equal(x, inputs.random_state(M, 5, nq2=nq2))
    assert np.abs(x[:2 * nq2]).max() < 0.3 * 6 and np.abs(x[2 * nq2:4 * nq2]).max() < 1e-3 * 6
    assert np.abs(x[4 * nq2:]).std() > 10.0
