"""Pins of the FP64 network oracle: the analytic backward equals central
finite differences of the loss for every parameter tensor, the forward agrees
with a per-example loop, and an Adam step on a separable problem lowers the
loss."""
import numpy as np

from oracle import mlp as M


def _params(rng, D=5, H=7):
    W1 = rng.standard_normal((H, 2 * D)) * 0.5
    b1 = rng.standard_normal(H) * 0.1
    W2 = rng.standard_normal((D, H)) * 0.5
    b2 = rng.standard_normal(D) * 0.1
    return W1, b1, W2, b2


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    W1, b1, W2, b2 = _params(rng)
    U = rng.standard_normal((6, 10))
    T = rng.standard_normal((6, 5))
    grads = M.backward(W1, b1, W2, b2, U, T)
    eps = 1e-6
    for pi, p in enumerate((W1, b1, W2, b2)):
        num = np.zeros_like(p)
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            ix = it.multi_index
            old = p[ix]
            p[ix] = old + eps
            lp = M.loss(W1, b1, W2, b2, U, T)
            p[ix] = old - eps
            lm = M.loss(W1, b1, W2, b2, U, T)
            p[ix] = old
            num[ix] = (lp - lm) / (2 * eps)
        np.testing.assert_allclose(grads[pi], num, rtol=1e-6, atol=1e-9)


def test_forward_per_example_loop():
    rng = np.random.default_rng(1)
    W1, b1, W2, b2 = _params(rng)
    U = rng.standard_normal((4, 10))
    Y, _, _ = M.forward(W1, b1, W2, b2, U)
    for r in range(4):
        h = [max(0.0, sum(W1[i, j] * U[r, j] for j in range(10)) + b1[i]) for i in range(7)]
        y = [sum(W2[o, i] * h[i] for i in range(7)) + b2[o] for o in range(5)]
        np.testing.assert_allclose(Y[r], y, rtol=1e-12)


def test_adam_lowers_loss():
    rng = np.random.default_rng(2)
    W1, b1, W2, b2 = _params(rng, D=4, H=16)
    U = rng.standard_normal((64, 8))
    T = np.abs(U[:, :4]) + 0.5 * U[:, 4:]          # a learnable target
    params = [W1, b1, W2, b2]
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    l0 = M.loss(*params, U, T)
    for t in range(1, 301):
        M.adam_step(params, M.backward(*params, U, T), m, v, t, lr=1e-2)
    assert M.loss(*params, U, T) < 0.2 * l0


def test_order_from_scores():
    assert M.order_from_scores(np.array([0.5, 2.0, 2.0, -1.0])).tolist() == [1, 2, 0, 3]
