"""Pins of the MLP oracle (CPU): central finite differences of the loss, and
the closed form of a network whose only path is one linear unit."""
import numpy as np

from oracle import mlp as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, H, n = 5, 7, 23
    p = rng.normal(0, 0.5, M.n_params(n_in, H))
    X = rng.normal(size=(n, n_in)); t = rng.normal(size=n)
    loss, g = M.loss_grad(p, X, t, H)
    eps = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p); e[k] = eps
        fd[k] = (M.loss_grad(p + e, X, t, H)[0] - M.loss_grad(p - e, X, t, H)[0]) / (2 * eps)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-8)


def test_one_unit_linear_closed_form():
    # H = 1, every pre-activation positive: y = w3 (W2 (W1 x + b1) + b2) + b3
    n_in, H = 2, 1
    W1, b1, W2, b2, w3, b3 = np.array([[0.5, 0.25]]), np.array([1.0]), np.array([[2.0]]), np.array([0.5]), \
        np.array([3.0]), 0.1
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])
    X = np.array([[1.0, 2.0], [2.0, 0.0]]); t = np.array([10.0, 9.0])
    y = M.forward(p, X, H)
    assert np.allclose(y, [3 * (2 * (0.5 + 0.5 + 1) + 0.5) + 0.1, 3 * (2 * (1.0 + 1) + 0.5) + 0.1])
    loss, g = M.loss_grad(p, X, t, H)
    r = y - t
    assert np.isclose(loss, np.mean(r ** 2))
    # d loss / d b3 = mean 2 r ; d loss / d w3 = mean 2 r h2
    h2 = 2 * (X @ W1.T + b1)[:, 0] + 0.5
    assert np.isclose(g[-1], np.mean(2 * r))
    assert np.isclose(g[-2], np.mean(2 * r * h2))


def test_adam_first_step_is_sign_times_lr():
    p = np.array([1.0, -2.0, 3.0]); g = np.array([0.3, -0.01, 0.0])
    p1, m, v = M.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    # bias-corrected first step: lr * g / (|g| + eps)
    assert np.allclose(p1, p - 0.1 * np.sign(g) * (np.abs(g) / (np.abs(g) + 1e-8)))
