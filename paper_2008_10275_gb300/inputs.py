"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds workload descriptions and random draws only -- none of the
method's arithmetic (no ordering rule, clustering, assembly or solver).  The
workloads are 2D stand-ins for the paper's 3D experiment (Sec. 5): the
channel [0, 2] x [0, 0.4] with the flap [0.6, 0.7] x [0, 0.2], rho_f = 1e3,
lambda_s = 2e6, parabolic inflow of mean 0.2, shear moduli in [5e5, 2e6] and
kinematic viscosities in [1e-3, 5e-3].
"""
from __future__ import annotations

import dataclasses

import numpy as np

MU_RANGE = (5.0e5, 2.0e6)
NU_RANGE = (1.0e-3, 5.0e-3)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    mu_values: tuple | None = None     # grid: the m1 shear moduli
    nu_values: tuple | None = None     # grid: the m2 viscosities
    nu_fastest: bool = False           # grid ordering axis (False = little endian, mu fastest)
    K: int = 1
    rank_cap: int = 20
    tol: float = 1e-8
    seed: int | None = None            # random parameters instead of a grid
    n_random: int = 0
    subset_sizes: tuple | None = None  # explicit uneven subset sizes (batched workload)
    rank_caps: tuple | None = None
    group: int | None = None           # subsets solved together on one GPU (memory), None = all


def _lin(lo_hi, n):
    return tuple(np.linspace(lo_hi[0], lo_hi[1], n).tolist())


def uneven_sizes(total=1000, n=16, seed=0):
    """Sizes of n uneven subsets summing to ``total``: 15 subsets of 64 and
    one of 40 placed at a seeded position (8..64 with a sum of 1000 over 16
    subsets leaves no room for more spread)."""
    rng = np.random.default_rng(seed)
    sizes = [64] * n
    sizes[int(rng.integers(n))] = total - 64 * (n - 1)
    return tuple(sizes)


WORKLOADS = {
    "small": Workload("channel20x4_fp64_100", 20, 4, _lin(MU_RANGE, 10), _lin(NU_RANGE, 10),
                      nu_fastest=True, K=2, rank_cap=20),
    "medium": Workload("channel80x16_400", 80, 16, _lin(MU_RANGE, 20), _lin(NU_RANGE, 20),
                       K=4, rank_cap=40),
    "batched": Workload("channel80x16_random1000_16uneven", 80, 16, K=16, seed=0, n_random=1000,
                        subset_sizes=uneven_sizes(), rank_caps=tuple(int(round(60 - 40 * j / 15)) for j in range(16))),
    "large": Workload("channel320x64_2500", 320, 64, _lin(MU_RANGE, 50), _lin(NU_RANGE, 50),
                      K=25, rank_cap=80, group=5),
    "learned": Workload("channel80x16_learned2000", 80, 16, seed=1, n_random=2000, K=20, rank_cap=40),
}


def uniform_parameters(n, seed):
    """n parameters drawn uniformly from the shear-modulus x viscosity box."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(*MU_RANGE, size=n)
    nu = rng.uniform(*NU_RANGE, size=n)
    return mu, nu


def latin_hypercube(n, seed):
    """n parameters by Latin hypercube sampling of the same box."""
    rng = np.random.default_rng(seed)
    u = (np.stack([rng.permutation(n), rng.permutation(n)], 1) + rng.uniform(size=(n, 2))) / n
    mu = MU_RANGE[0] + (MU_RANGE[1] - MU_RANGE[0]) * u[:, 0]
    nu = NU_RANGE[0] + (NU_RANGE[1] - NU_RANGE[0]) * u[:, 1]
    return mu, nu


def random_state(M, seed, scales=(0.3, 1e-3, 50.0), nq2=None):
    """A seeded random state vector (for assembly parity tests): velocity,
    deformation and pressure entries with the given magnitudes.  ``nq2`` is
    the number of Q2 nodes (the first 4 nq2 entries are v, u)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(M)
    if nq2 is not None:
        x[:2 * nq2] *= scales[0]
        x[2 * nq2:4 * nq2] *= scales[1]
        x[4 * nq2:] *= scales[2]
    return x


def mlp_init(sizes=(2, 128, 128, 64), seed=0):
    """Seeded initial parameters of the learned-start MLP, packed as the
    library expects (per layer: W_l (n_{l+1} x n_l, row-major), then b_l):
    He-normal weights, zero biases, FP32."""
    rng = np.random.default_rng(seed)
    parts = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        parts.append((rng.standard_normal((n_out, n_in)) * np.sqrt(2.0 / n_in)).astype(np.float32).ravel())
        parts.append(np.zeros(n_out, np.float32))
    return np.concatenate(parts)


def workload_values(W, replicas=1):
    """The parameter values of workload ``W``, unordered: for a grid the m1
    shear moduli and the m2 viscosities (``replicas`` > 1 refines the
    viscosities to replicas * m2 values over the same range: a job of that
    many copies of the workload's shape, for runs on several GPUs; in the
    little-endian order every subset then still holds whole rows of m1 shear
    moduli); for a random workload the n seeded draws from the box."""
    if W.seed is not None:
        rng = np.random.default_rng(W.seed)
        n = W.n_random * replicas
        return rng.uniform(*MU_RANGE, n), rng.uniform(*NU_RANGE, n)
    nu = np.array(W.nu_values)
    if replicas > 1:
        nu = np.linspace(nu[0], nu[-1], replicas * len(nu))
    return np.array(W.mu_values), nu
