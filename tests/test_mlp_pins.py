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


def test_adam_two_steps_hand_worked():
    # tests/golden/ads_bsa_worked.json "adam": two steps worked out by hand
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ads_bsa_worked.json")))["adam"]
    p = [np.array([g["p0"]])]
    m = [np.zeros(1)]
    v = [np.zeros(1)]
    for t, (gr, want) in enumerate(zip(g["grads"], g["p_after"]), start=1):
        M.adam_step(p, [np.array([gr])], m, v, t, lr=g["lr"])
        assert abs(p[0][0] - want) < 1e-6


def test_adam_constant_gradient_moves_lr_per_step():
    # with bias correction, a constant gradient g gives m_hat = g and
    # v_hat = g^2 at every step, so each step moves exactly lr against sign(g)
    # (up to eps); without the correction the first step would be 3.16 lr
    p = [np.array([0.0, 1.0, -2.0])]
    g = np.array([0.3, -7.0, 0.5])
    m, v = [np.zeros(3)], [np.zeros(3)]
    for t in range(1, 6):
        M.adam_step(p, [g], m, v, t, lr=0.01)
        np.testing.assert_allclose(p[0], np.array([0.0, 1.0, -2.0]) - 0.01 * t * np.sign(g), rtol=0, atol=1e-8)


def test_adam_is_gradient_scale_invariant():
    rng = np.random.default_rng(3)
    g1, g2 = rng.standard_normal(5), rng.standard_normal(5)
    out = []
    for s in (1.0, 1000.0):
        p, m, v = [np.ones(5)], [np.zeros(5)], [np.zeros(5)]
        M.adam_step(p, [s * g1], m, v, 1, lr=0.05)
        M.adam_step(p, [s * g2], m, v, 2, lr=0.05)
        out.append(p[0].copy())
    np.testing.assert_allclose(out[0], out[1], rtol=0, atol=1e-7)
