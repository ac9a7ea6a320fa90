"""FP64 forward/backward of the order-proposal network.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; the network is an addition. It reads
u = [q; c], the query and its nearest cluster centroid, and proposes a
dimension visit order for PDX-BOND:
    h = relu(W1 u + b1)          W1: [H][2D], b1: [H]
    y = W2 h + b2                W2: [D][H],  b2: [D]
The training loss is the mean squared error against a target t (per-dimension
trace scores), L = sum((y - t)^2) / (B * D) over a batch of B rows.

Written with plain matrix products in float64. It is checked against central
finite differences in tests, so that a transposed or dropped term in the
analytic backward fails.
"""
from __future__ import annotations

import numpy as np


def forward(W1, b1, W2, b2, U):
    U = np.asarray(U, np.float64)
    Z = U @ np.asarray(W1, np.float64).T + b1
    H = np.maximum(Z, 0.0)
    Y = H @ np.asarray(W2, np.float64).T + b2
    return Y, H, Z


def loss(W1, b1, W2, b2, U, T):
    Y, _, _ = forward(W1, b1, W2, b2, U)
    B, D = Y.shape
    return float(((Y - T) ** 2).sum() / (B * D))


def backward(W1, b1, W2, b2, U, T):
    """Gradients of loss() w.r.t. (W1, b1, W2, b2)."""
    U = np.asarray(U, np.float64)
    Y, H, Z = forward(W1, b1, W2, b2, U)
    B, D = Y.shape
    dY = 2.0 * (Y - np.asarray(T, np.float64)) / (B * D)
    dW2 = dY.T @ H
    db2 = dY.sum(axis=0)
    dH = dY @ np.asarray(W2, np.float64)
    dZ = dH * (Z > 0)
    dW1 = dZ.T @ U
    db1 = dZ.sum(axis=0)
    return dW1, db1, dW2, db2


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), in place; t counts from 1."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= beta1
        mm += (1 - beta1) * g
        vv *= beta2
        vv += (1 - beta2) * g * g
        mhat = mm / (1 - beta1 ** t)
        vhat = vv / (1 - beta2 ** t)
        p -= lr * mhat / (np.sqrt(vhat) + eps)


def order_from_scores(y):
    """Visit order: dimensions by decreasing score, ties to the lower index."""
    y = np.asarray(y)
    return np.lexsort((np.arange(y.shape[-1]), -y))


def learned_order(q, mu, y):
    """Learned visit order: decreasing (q_j - mu_j)^2 + s_q y_j with
    s_q = mean_j (q_j - mu_j)^2 (the network y corrects the distance-to-means
    heuristic, in units of s_q)."""
    q = np.asarray(q, np.float64)
    h = (q - np.asarray(mu, np.float64)) ** 2
    return order_from_scores(h + h.mean() * np.asarray(y, np.float64))


def trace_targets(q, X, mu):
    """Residual target for one query: mean over the rows of X (vectors the
    plain search pruned) of (q_j - x_j)^2, minus (q_j - mu_j)^2, divided by
    s_q = mean_j (q_j - mu_j)^2."""
    q = np.asarray(q, np.float64)
    X = np.asarray(X, np.float64)
    h = (q - np.asarray(mu, np.float64)) ** 2
    return (((X - q) ** 2).mean(axis=0) - h) / h.mean()
