"""Pins of the oracle's adaptive refinement of the subsets (reading of Sec. 5,
"Alternative ways to cluster the parameter set"; CPU only).

* A target that no subset meets refines every subset at every level: L levels
  from K subsets give exactly the subsets and the columns of Algorithm 1 with
  K 2^L subsets when the sizes halve evenly (the halves follow Eq.
  (clustering1)).
* A target that every subset meets refines nothing: the result is Algorithm 1.
* Refinement never raises a column's subset's largest residual here, and the
  largest residual over all columns falls with the levels (the paper's
  observation for K = 50, 100, 200).
"""
import numpy as np
import pytest

from oracle import algorithm1, fsi


@pytest.fixture(scope="module")
def case():
    mesh = fsi.Mesh(fsi.Problem(20, 4))
    mus = np.tile(np.linspace(5e5, 2e6, 4), 2)
    nus = np.repeat(np.linspace(1e-3, 5e-3, 2), 4)
    opt = algorithm1.Options(K=1, eps_N=1e-9, c=0.65, d=1.0, iters=6, cycles=2, truncated=False,
                             warm_start=False)
    return mesh, mus, nus, opt


def test_split_rule():
    assert algorithm1.split_subset(3, 7) == [(3, 3), (6, 4)]
    assert algorithm1.split_subset(0, 2) == [(0, 1), (1, 1)]


def test_refining_everything_equals_more_subsets(case):
    mesh, mus, nus, opt = case
    Xa, subs = algorithm1.algorithm1_adaptive(mesh, mus, nus, opt, target=0.0, max_levels=2)
    opt4 = algorithm1.Options(**{**opt.__dict__, "K": 4})
    X4, info = algorithm1.algorithm1(mesh, mus, nus, opt4)
    assert [s[2] for s in subs] == info["medians"]
    assert [s[1] for s in subs] == [2, 2, 2, 2]
    assert np.abs(Xa - X4).max() <= 1e-9 * np.abs(X4).max()


def test_met_target_refines_nothing(case):
    mesh, mus, nus, opt = case
    Xa, subs = algorithm1.algorithm1_adaptive(mesh, mus, nus, opt, target=10.0, max_levels=3)
    X1, info = algorithm1.algorithm1(mesh, mus, nus, opt)
    assert len(subs) == 1 and subs[0][2] == info["medians"][0]
    assert np.abs(Xa - X1).max() <= 1e-12 * np.abs(X1).max()


def test_levels_lower_the_largest_residual(case):
    mesh, mus, nus, opt = case
    worst = []
    for lv in (0, 1, 2):
        X, subs = algorithm1.algorithm1_adaptive(mesh, mus, nus, opt, target=0.0, max_levels=lv)
        worst.append(algorithm1.relative_residuals(mesh, X, mus, nus).max())
    assert worst[0] > worst[1] > worst[2], worst
