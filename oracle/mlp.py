"""FP64 numpy oracle of the learned schedule model's network (test infrastructure only).

Network n_in -> H -> H -> 1 with ReLU, parameters in one flat vector laid
out [W1 (H x n_in), b1 (H), W2 (H x H), b2 (H), w3 (H), b3]; loss = mean
squared error; Adam as defined by Kingma & Ba (2015), Algorithm 1.  Pinned by
central finite differences and by the closed form of a one-unit linear case
(tests/test_oracle_mlp.py).
"""
import numpy as np


def unpack(p, n_in, H):
    p = np.asarray(p, dtype=np.float64)
    k = 0
    W1 = p[k:k + H * n_in].reshape(H, n_in); k += H * n_in
    b1 = p[k:k + H]; k += H
    W2 = p[k:k + H * H].reshape(H, H); k += H * H
    b2 = p[k:k + H]; k += H
    w3 = p[k:k + H]; k += H
    b3 = p[k]
    return W1, b1, W2, b2, w3, b3


def n_params(n_in, H):
    return H * n_in + H + H * H + H + H + 1


def forward(p, X, H):
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(p, X.shape[1], H)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3


def loss_grad(p, X, t, H):
    """Mean squared error and its gradient by the chain rule, layer by layer."""
    X = np.asarray(X, dtype=np.float64); t = np.asarray(t, dtype=np.float64)
    n, n_in = X.shape
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, H)
    a1 = X @ W1.T + b1; h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2; h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    r = y - t
    loss = np.mean(r * r)
    dy = 2.0 * r / n
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    da2 = np.outer(dy, w3) * (a2 > 0)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * (a1 > 0)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g


def adam(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
