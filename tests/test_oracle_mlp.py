"""Pins of the learned-start oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: the BF16 grid, the closed form of GELU and its
derivative, central finite differences of the loss in FP64, the first Adam
step, and the Eckart-Young optimality of the POD."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_bf16_round_grid_and_ties():
    # BF16 keeps 8 significant bits: the spacing above 1 is 2^-7.
    one = np.float32(1.0)
    assert mlp.bf16_round(np.float32(1 + 2.0 ** -7)) == np.float32(1 + 2.0 ** -7)
    # halfway between 1 and 1 + 2^-7 ties to the even neighbour 1
    assert mlp.bf16_round(np.float32(1 + 2.0 ** -8)) == one
    # halfway between 1 + 2^-7 and 1 + 2^-6 ties to even 1 + 2^-6
    assert mlp.bf16_round(np.float32(1 + 3 * 2.0 ** -8)) == np.float32(1 + 2.0 ** -6)
    # just above the tie rounds up
    assert mlp.bf16_round(np.float32(1 + 2.0 ** -8 + 2.0 ** -20)) == np.float32(1 + 2.0 ** -7)
    # signs and exact values survive; relative error bounded by 2^-9
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32)
    y = mlp.bf16_round(x)
    assert np.all(np.sign(y) == np.sign(x))
    assert np.max(np.abs(y - x) / np.abs(x)) <= 2.0 ** -8 + 1e-12
    assert np.all(mlp.bf16_round(y) == y)
    assert np.all((y.view(np.uint32) & 0xFFFF) == 0)


def test_gelu_closed_form_and_derivative():
    x = np.linspace(-6, 6, 241)
    # GELU(x) = x * Phi(x) with the standard normal CDF
    assert np.allclose(mlp.gelu(x), x * norm.cdf(x), atol=1e-15, rtol=1e-14)
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu(10.0) - 10.0) < 1e-12 and abs(mlp.gelu(-10.0)) < 1e-12
    h = 1e-5
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(x))) < 1e-9
    # derivative closed form: Phi(x) + x phi(x)
    assert np.allclose(mlp.gelu_grad(x), norm.cdf(x) + x * norm.pdf(x), atol=1e-14)


def test_backward_matches_central_differences_fp64():
    rng = np.random.default_rng(3)
    sizes = (2, 7, 5, 4)
    params = [p.astype(np.float64) for p in mlp.init_params(sizes, seed=4)]
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]  # nonzero biases
    Z = rng.uniform(-1, 1, (6, 2))
    T = rng.standard_normal((6, 4))
    Y, cache = mlp.forward(params, Z, dtype=np.float64, bf16=False)
    grads = mlp.backward(cache, Y, T)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(params, Z, np.float64, False)[0], T)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(params, Z, np.float64, False)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            g = grads[pi].ravel()[idx]
            assert abs(fd - g) <= 1e-7 * max(1.0, abs(fd)), (pi, idx, fd, g)


def test_forward_linear_special_case():
    # With one hidden unit pattern removed (all-zero hidden weights) the output
    # is the last bias: the net reduces to a constant.
    sizes = (2, 3, 3, 2)
    params = mlp.init_params(sizes, seed=1)
    params[0][:] = 0
    params[1][:] = 0
    params[2][:] = 0
    params[3][:] = 0
    params[5][:] = np.array([0.5, -2.0], np.float32)
    Y, _ = mlp.forward(params, np.ones((4, 2)), np.float64, bf16=True)
    assert np.all(Y == np.array([0.5, -2.0]))


def test_first_adam_step_is_signed_learning_rate():
    # After one step from zero moments the bias-corrected update is
    # -lr * g / (|g| + eps), i.e. -lr sign(g) for |g| >> eps.
    g = [np.array([3.0, -2e-3, 5e2]), np.array([[-1.0]])]
    p = [np.zeros(3), np.zeros((1, 1))]
    state = ([np.zeros(3), np.zeros((1, 1))], [np.zeros(3), np.zeros((1, 1))], 0)
    p, state = mlp.adam_step(p, g, state, lr=0.01)
    assert np.allclose(p[0], -0.01 * np.sign(g[0]), rtol=1e-5)
    assert np.allclose(p[1], 0.01)
    assert state[2] == 1


def test_pod_is_best_rank_k():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((60, 8)) @ np.diag(2.0 ** -np.arange(8)) @ rng.standard_normal((8, 30))
    k = 3
    Phi, C, s = mlp.pod_basis(X, k)
    assert np.allclose(Phi.T @ Phi, np.eye(k), atol=1e-13)
    err = np.linalg.norm(X - Phi @ C)
    # Eckart-Young: the error is the tail of the singular values
    assert err == pytest.approx(np.sqrt(np.sum(s[k:] ** 2)), rel=1e-10)
    # exact for data of rank <= k
    X3 = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 20))
    P3, C3, _ = mlp.pod_basis(X3, 3)
    assert np.linalg.norm(X3 - P3 @ C3) < 1e-12 * np.linalg.norm(X3)


def test_scale_params_maps_box_corners():
    z = mlp.scale_params([5e5, 2e6, 1.25e6], [1e-3, 5e-3, 3e-3], (5e5, 2e6), (1e-3, 5e-3))
    assert np.allclose(z, [[-1, -1], [1, 1], [0, 0]])
