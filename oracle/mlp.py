"""Learned initial guess (oracle): MLP, its gradients, Adam, POD basis.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Not a method of the paper: a serving-style start for the median Newton
iteration of Algorithm 1.  A multilayer perceptron maps the two scaled
parameters (mu_s, nu_f) -> 128 -> 128 -> k coefficients (GELU after the two
hidden layers); the start is x0 = s * (Phi c) + offset with Phi a rank-k POD
basis of method-generated solutions, s the per-field scale of the snapshots
and the Dirichlet rows overwritten with b_D.

Numerics of the CUDA path it checks: weights stored in BF16 (rounded to
nearest even), biases and all accumulation in FP32.  ``forward``/``backward``
take a ``dtype`` so the same definitions run in FP64 (finite-difference
checks) and FP32 (parity with the GPU).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT1_2 = np.sqrt(0.5)


def bf16_round(w):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    w = np.asarray(w, dtype=np.float32)
    u = w.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def gelu(x):
    """GELU in its exact erf form: x Phi(x) = 0.5 x (1 + erf(x / sqrt 2))."""
    return 0.5 * x * (1.0 + erf(x * SQRT1_2))


def gelu_grad(x):
    """d/dx of the exact GELU: Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x * SQRT1_2)) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def init_params(sizes=(2, 128, 128, 64), seed=0):
    """He-style normal initialisation (seeded); biases zero.  W_l is (out, in)."""
    rng = np.random.default_rng(seed)
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        W = (rng.standard_normal((n_out, n_in)) * np.sqrt(2.0 / n_in)).astype(np.float32)
        params += [W, np.zeros(n_out, np.float32)]
    return params


def forward(params, Z, dtype=np.float32, bf16=True):
    """Z: (B, 2).  Returns the output (B, k) and the cache for backward."""
    Ws = [bf16_round(p) if (bf16 and i % 2 == 0) else p for i, p in enumerate(params)]
    Ws = [np.asarray(p, dtype) for p in Ws]
    a = np.asarray(Z, dtype)
    cache = []
    nl = len(Ws) // 2
    for l in range(nl):
        W, b = Ws[2 * l], Ws[2 * l + 1]
        z = a @ W.T + b
        cache.append((a, z))
        a = gelu(z) if l < nl - 1 else z
    return a, (Ws, cache)


def loss(Y, T):
    """Mean squared error over batch and outputs."""
    return float(np.mean((Y - T) ** 2))


def backward(cache, Y, T):
    """Gradients of the mean squared error w.r.t. every parameter (same order
    as params), evaluated with the weights the forward pass used."""
    Ws, layers = cache
    B, k = Y.shape
    g = 2.0 * (Y - T) / (B * k)
    grads = [None] * len(Ws)
    nl = len(layers)
    for l in range(nl - 1, -1, -1):
        a, z = layers[l]
        if l < nl - 1:
            g = g * gelu_grad(z)
        grads[2 * l] = g.T @ a
        grads[2 * l + 1] = g.sum(axis=0)
        g = g @ Ws[2 * l]
    return grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place (Kingma and Ba, 2015); state = (m, v, t)."""
    m, v, t = state
    t += 1
    for i, (p, g) in enumerate(zip(params, grads)):
        m[i] = b1 * m[i] + (1 - b1) * g
        v[i] = b2 * v[i] + (1 - b2) * g * g
        mh = m[i] / (1 - b1 ** t)
        vh = v[i] / (1 - b2 ** t)
        params[i] = (p - lr * mh / (np.sqrt(vh) + eps)).astype(p.dtype)
    return params, (m, v, t)


def pod_basis(X, k):
    """Rank-k POD of the snapshot columns X (M x n): the leading left singular
    vectors Phi (M x k) and coefficients C = Phi^T X (k x n)."""
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    Phi = U[:, :k]
    return Phi, Phi.T @ X, s


def scale_params(mu, nu, mu_range, nu_range):
    """Map the parameter box to [-1, 1]^2."""
    mu = np.asarray(mu, float)
    nu = np.asarray(nu, float)
    z0 = 2.0 * (mu - mu_range[0]) / (mu_range[1] - mu_range[0]) - 1.0
    z1 = 2.0 * (nu - nu_range[0]) / (nu_range[1] - nu_range[0]) - 1.0
    return np.stack([z0, z1], axis=1)
