"""Parameter set bookkeeping (oracle).  TEST INFRASTRUCTURE ONLY.

Sec. 3.3: little-endian order (Def. 1), clustering into K contiguous subsets
(Eq. (clustering1)), upper median index (Def. "Upper Median Index", Ex. 2);
Sec. 3.4: diagonal matrices D_mu^k, D_nu^k; Sec. 3.4 end: column p of the
global approximation <-> (mu^{((p-1) mod m1)+1}, nu^{ceil(p/m1)});
Sec. 4.4: the four-parameter little-endian order.
Indices in this module are 1-based where the paper's are, and say so.
"""
from __future__ import annotations

import numpy as np


def little_endian_order(m1, m2):
    """All multi-indices (i1, i2), 1-based, sorted by the key i1 + (i2-1) m1
    (Def. 1): mu index runs fastest."""
    pairs = [(i1, i2) for i1 in range(1, m1 + 1) for i2 in range(1, m2 + 1)]
    return sorted(pairs, key=lambda t: t[0] + (t[1] - 1) * m1)


def little_endian_order4(m1, m2, m3, m4):
    """All multi-indices (i1, i2, i3, i4), 1-based, sorted by the key
    i1 + (i2-1) m1 + (i3-1) m1 m2 + (i4-1) m1 m2 m3 (Sec. 4.4, "Clustering"):
    the mu index runs fastest, then nu, lambda, rho."""
    tuples = [(a, b, c, d) for a in range(1, m1 + 1) for b in range(1, m2 + 1)
              for c in range(1, m3 + 1) for d in range(1, m4 + 1)]
    return sorted(tuples, key=lambda t: t[0] + (t[1] - 1) * m1 + (t[2] - 1) * m1 * m2 + (t[3] - 1) * m1 * m2 * m3)


def order_set(mu, nu):
    """Order of a scattered parameter set (reading: the little-endian order of
    Def. 1 carried over from grids): sorted by nu, then by mu, equal pairs in
    input order.  Returns the permutation (0-based)."""
    return np.lexsort((np.asarray(mu, float), np.asarray(nu, float)))


def ordered_grid(mu_values, nu_values, nu_fastest=False):
    """The grid mu_values x nu_values as two arrays in Def. 1's order (mu
    index fastest), or with the nu index fastest."""
    if nu_fastest:
        pairs = [(b, a) for a, b in little_endian_order(len(nu_values), len(mu_values))]
    else:
        pairs = little_endian_order(len(mu_values), len(nu_values))
    mu = np.array([mu_values[i - 1] for i, _ in pairs], float)
    nu = np.array([nu_values[j - 1] for _, j in pairs], float)
    return mu, nu


def affine_midpoints(*coeffs):
    """Midpoints of the ranges of the subset's affine coefficients (the
    mean-based preconditioner's coefficients, reading of Sec. 4.2 applied to
    every coefficient; for four parameters they are mu, nu rho, lambda, rho)."""
    return tuple(0.5 * (np.min(c) + np.max(c)) for c in coeffs)


def cluster_sizes(m, K):
    """|I_k| = floor(m/K) for k < K and the remainder for k = K (Eq. (clustering1))."""
    if K < 1 or m < K:
        raise ValueError("need 1 <= K <= m")
    base = m // K
    return [base] * (K - 1) + [m - (K - 1) * base]


def clusters(ordered, K):
    """Split an ordered list of parameter indices into K contiguous subsets."""
    out, start = [], 0
    for s in cluster_sizes(len(ordered), K):
        out.append(list(ordered[start:start + s]))
        start += s
    return out


def upper_median_position(n):
    """0-based position of the upper median of an ordered set of n elements
    (the element at 1-based position floor(n/2) + 1)."""
    if n < 1:
        raise ValueError("empty subset")
    return n // 2


def column_parameter_index(p, m1):
    """Column p (1-based) of the little-endian global approximation belongs to
    (mu index, nu index) = (((p-1) mod m1) + 1, ceil(p / m1)) (Sec. 3.4)."""
    return ((p - 1) % m1) + 1, -(-p // m1)


def diagonal_matrices(mu_k, nu_k, mu_ref=0.0, nu_ref=0.0):
    """D_mu^k, D_nu^k and the shifted D_{mu-}^k = D_mu^k - mu_s I,
    D_{nu-}^k = D_nu^k - nu_f I (Sec. 3.4, Def. "Diagonal Matrices")."""
    Dmu = np.diag(np.asarray(mu_k, dtype=np.float64))
    Dnu = np.diag(np.asarray(nu_k, dtype=np.float64))
    I = np.eye(len(mu_k))
    return Dmu, Dnu, Dmu - mu_ref * I, Dnu - nu_ref * I


def midpoint_parameters(mu_k, nu_k):
    """Parameters of the mean-based preconditioner P_T^k (Sec. 4.2): the
    midpoint of the subset's parameter ranges (reading of the shifted
    definition, which adds back the reference values)."""
    mu_k, nu_k = np.asarray(mu_k), np.asarray(nu_k)
    return 0.5 * (mu_k.min() + mu_k.max()), 0.5 * (nu_k.min() + nu_k.max())


def corner_parameters(mu_k, nu_k):
    """The subset's 'corner' parameters used to estimate the Chebyshev
    interval (Sec. 5.1.1, reading: mu at the subset's min or max and nu at the
    subset's min or max)."""
    mu_k, nu_k = np.asarray(mu_k), np.asarray(nu_k)
    sel = ((mu_k == mu_k.min()) | (mu_k == mu_k.max())) & ((nu_k == nu_k.min()) | (nu_k == nu_k.max()))
    return np.flatnonzero(sel)
