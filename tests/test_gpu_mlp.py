"""The order-proposal network on the GPU: forward and backward against the
FP64 oracle (itself pinned by finite differences), training, trace targets,
and the learned visit order. Its searches stay exact (FP64 oracle), and it
visits fewer values than the distance-to-means heuristic on data whose
per-dimension spread the heuristic cannot see."""
import numpy as np
import pytest

import pdx_synth
from oracle import mlp as M
from oracle import quant as Q
from tests._parity import check_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx
    return pdx


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def _split(p, D, H):
    W1 = p[:H * 2 * D].reshape(H, 2 * D)
    b1 = p[H * 2 * D:H * 2 * D + H]
    W2 = p[H * 2 * D + H:H * 2 * D + H + D * H].reshape(D, H)
    b2 = p[H * 2 * D + H + D * H:]
    return [a.astype(np.float64) for a in (W1, b1, W2, b2)]


def test_forward_backward_match_oracle(P, torch):
    D, H = 40, 48
    net = P.Mlp(D, H, seed=11)
    rng = np.random.default_rng(0)
    p = net.get_params()
    p[H * 2 * D:H * 2 * D + H] = rng.standard_normal(H) * 0.1      # non-zero biases
    p[-D:] = rng.standard_normal(D) * 0.1
    net.set_params(p)
    W1, b1, W2, b2 = _split(p, D, H)
    U = rng.standard_normal((70, 2 * D)).astype(np.float32)
    T = rng.standard_normal((70, D)).astype(np.float32)
    Ud, Td = torch.from_numpy(U).cuda(), torch.from_numpy(T).cuda()
    Y = net.forward(Ud).cpu().numpy()
    Yo, _, _ = M.forward(W1, b1, W2, b2, U)
    np.testing.assert_allclose(Y, Yo, rtol=1e-5, atol=1e-5)
    # BF16 inference weights: the oracle with the same rounding of W1, W2
    Yb = net.forward(Ud, bf16=True).cpu().numpy()
    Ybo, _, _ = M.forward(Q.bf16_round(W1.astype(np.float32)), b1, Q.bf16_round(W2.astype(np.float32)), b2, U)
    np.testing.assert_allclose(Yb, Ybo, rtol=1e-4, atol=1e-4)
    g, loss = net.backward(Ud, Td)
    go = np.concatenate([a.ravel() for a in M.backward(W1, b1, W2, b2, U, T)])
    assert abs(loss - M.loss(W1, b1, W2, b2, U, T)) <= 1e-5 * abs(loss)
    assert np.abs(g - go).max() <= 1e-5 * np.abs(go).max()


def test_adam_steps_match_oracle(P, torch):
    # three full-batch Adam steps of the GPU trainer (adam_kernel) against the
    # oracle's backward + adam_step (itself pinned by hand-worked steps). Where
    # a gradient entry is near 0 its step depends on the FP32 rounding of g
    # (the step is about lr * sign(g) early on), so those entries only get
    # the bound |step| <= lr per step.
    D, H, B, lr, steps = 24, 32, 256, 1e-3, 3
    net = P.Mlp(D, H, seed=12)
    rng = np.random.default_rng(4)
    p0 = net.get_params()
    p0[H * 2 * D:H * 2 * D + H] = rng.standard_normal(H) * 0.1
    net.set_params(p0)
    U = rng.standard_normal((B, 2 * D)).astype(np.float32)
    T = rng.standard_normal((B, D)).astype(np.float32)
    net.train(torch.from_numpy(U).cuda(), torch.from_numpy(T).cuda(), epochs=steps, batch=B, lr=lr, seed=3)
    got = net.get_params().astype(np.float64)
    params = _split(p0, D, H)
    m = [np.zeros_like(a) for a in params]
    v = [np.zeros_like(a) for a in params]
    gmin = None
    for t in range(1, steps + 1):
        g = M.backward(*params, U, T)
        flat = np.abs(np.concatenate([a.ravel() for a in g]))
        gmin = flat if gmin is None else np.minimum(gmin, flat)
        M.adam_step(params, g, m, v, t, lr=lr)
    want = np.concatenate([a.ravel() for a in params])
    clear = gmin > 1e-3 * gmin.max()
    assert clear.mean() > 0.9
    np.testing.assert_allclose(got[clear], want[clear], rtol=0, atol=2e-3 * lr * steps)
    assert np.all(np.abs(got - p0.astype(np.float64)) <= lr * steps * 1.01)


def test_training_lowers_loss(P, torch):
    D = 16
    rng = np.random.default_rng(1)
    U = rng.standard_normal((4096, 2 * D)).astype(np.float32)
    T = (np.abs(U[:, :D]) - 0.5 * U[:, D:]).astype(np.float32)     # a learnable target
    net = P.Mlp(D, 64, seed=2)
    Ud, Td = torch.from_numpy(U).cuda(), torch.from_numpy(T).cuda()
    _, l0 = net.backward(Ud, Td)
    l1 = net.train(Ud, Td, epochs=30, batch=128, lr=3e-3)
    _, l2 = net.backward(Ud, Td)
    assert l2 < 0.1 * l0, (l0, l1, l2)


def test_trace_targets_match_oracle(P, torch):
    x, q = pdx_synth.hetero_mixture(3000, 24, 7, n_centres=8)
    ix = P.pdx_build_layout(torch.from_numpy(x).cuda(), partition_size=1000)
    rng = np.random.default_rng(2)
    ids = rng.integers(0, 3000, size=(7, 33)).astype(np.int64)
    t = P.pdx_order_targets(ix, torch.from_numpy(q).cuda(), torch.from_numpy(ids).cuda()).cpu().numpy()
    mu = x.astype(np.float64).mean(axis=0)
    for r in range(7):
        np.testing.assert_allclose(t[r], M.trace_targets(q[r], x[ids[r]], mu), rtol=1e-3, atol=1e-4)


def test_learned_order_exact_and_gain(P, torch):
    n, d = 60000, 128
    x, q = pdx_synth.hetero_mixture(n, d, 1400, n_centres=32)
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    ivf = P.pdx_ivf_build(xd, nlist=32, kmeans_iters=4)
    cent = torch.from_numpy(ivf.copy_out("centroids")).cuda()
    ix = P.pdx_build_layout(xd, partition_size=10000)
    qtr, qte = qd[:1200].contiguous(), qd[1200:].contiguous()
    # traces of the plain method: vectors it ranked just behind the top-k,
    # and a sample of the vectors it pruned
    _, ids = P.pdx_search_exact(ix, qtr, 10 + 48)
    rnd = torch.from_numpy(np.random.default_rng(3).integers(0, n, size=(1200, 160))).cuda()
    tgt = P.pdx_order_targets(ix, qtr, torch.cat([ids[:, 10:], rnd], dim=1).contiguous())
    u = P.pdx_mlp_inputs(qtr, cent)
    net = P.Mlp(d, 256, seed=4)
    net.train(u, tgt, epochs=40, batch=128, lr=1e-3)
    dh, ih, sh = P.pdx_search_exact(ix, qte, 10, stats=True)
    dl, il, sl = P.pdx_search_exact(ix, qte, 10, stats=True, order="learned", mlp=net, mlp_centroids=cent)
    torch.cuda.synchronize()
    check_topk(x, q[1200:], 10, dl, il)
    assert np.array_equal(il.cpu().numpy(), ih.cpu().numpy())
    # the trained correction visits fewer values than the heuristic alone
    assert sl["values_visited"] < 0.9 * sh["values_visited"], (sl, sh)


def test_learned_order_argument_errors(P, torch):
    x, q = pdx_synth.iid_normal(500, 16, 3)
    ix = P.pdx_build_layout(torch.from_numpy(x).cuda())
    cent = torch.zeros((4, 16), device="cuda")
    wrong = P.Mlp(8, 16)
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(ix, torch.from_numpy(q).cuda(), 5, order="learned", mlp=wrong, mlp_centroids=cent)
