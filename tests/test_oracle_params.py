"""Pins of the parameter bookkeeping against the paper's worked examples
(Sec. 3.3, Examples 1 and 2; Sec. 3.4 column <-> parameter map)."""
import json
import os

import numpy as np

from oracle import params

GOLD = os.path.join(os.path.dirname(__file__), "golden", "clustering_example.json")


def test_example_1_subsets_and_example_2_medians():
    g = json.load(open(GOLD))
    order = params.little_endian_order(g["m1"], g["m2"])
    subs = params.clusters(order, g["K"])
    assert [[list(p) for p in s] for s in subs] == g["subsets"]
    med = [list(s[params.upper_median_position(len(s))]) for s in subs]
    assert med == g["upper_medians"]


def test_cluster_sizes_rule():
    assert params.cluster_sizes(20, 3) == [6, 6, 8]
    assert params.cluster_sizes(5000, 50) == [100] * 50
    assert params.cluster_sizes(1000, 16) == [62] * 15 + [70]
    for m in range(1, 40):
        for K in range(1, m + 1):
            s = params.cluster_sizes(m, K)
            assert sum(s) == m and len(s) == K and all(x == m // K for x in s[:-1])


def test_column_parameter_map_matches_order():
    m1, m2 = 7, 3
    order = params.little_endian_order(m1, m2)
    for p, pair in enumerate(order, start=1):
        assert params.column_parameter_index(p, m1) == pair


def test_upper_median_small_sets():
    assert [params.upper_median_position(n) + 1 for n in (1, 2, 3, 4, 5, 6, 8)] == [1, 2, 2, 3, 3, 4, 5]


def test_diagonal_and_midpoint():
    mu = np.array([1.0, 3.0, 2.0]); nu = np.array([5.0, 4.0, 6.0])
    Dmu, Dnu, Dmum, Dnum = params.diagonal_matrices(mu, nu, 1.5, 0.5)
    assert np.allclose(np.diag(Dmum), mu - 1.5) and np.allclose(np.diag(Dnum), nu - 0.5)
    assert params.midpoint_parameters(mu, nu) == (2.0, 5.0)
    g = json.load(open(GOLD))
    order = params.little_endian_order(g["m1"], g["m2"])
    s1 = params.clusters(order, 3)[0]
    mu1 = np.array([p[0] for p in s1]); nu1 = np.array([p[1] for p in s1])
    corners = {tuple(s1[i]) for i in params.corner_parameters(mu1, nu1)}
    assert corners == {(1, 1), (4, 1), (1, 2)}
