"""Pins of the FP64 surrogate reference (oracle/mpnn.py).

The reference's gradients come from autograd of its forward; they are
pinned by central finite differences. Its forward is pinned by properties
fixed by the definition: permutation equivariance, batching additivity of
disjoint graphs, an isolated receiver reducing to the encoder-processor-
decoder chain without messages, a layer's message sum taken apart edge by
edge, and the hydrostatic split of its inputs (a state at rest gives zero
potential differences on every edge).
"""
import numpy as np
import pytest
import torch

from oracle import mpnn


def _graph(n=40, dim=2, seed=0, deg=5):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, size=(n, dim))
    recv, send = [], []
    for i in range(n):
        js = rng.choice(np.delete(np.arange(n), i), size=deg, replace=False)
        recv += [i] * deg
        send += list(js)
    recv, send = np.array(recv), np.array(send)
    r = x[send] - x[recv]
    node = rng.normal(size=(n, dim + 3))
    du = node[send, :dim] - node[recv, :dim]
    dphi = node[send, dim + 1:dim + 2] - node[recv, dim + 1:dim + 2]
    edge = np.concatenate([r / 0.1, np.linalg.norm(r, axis=1, keepdims=True) / 0.1, du, dphi], axis=1)
    return node, recv, send, edge


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_matches_central_differences(dim):
    node, recv, send, edge = _graph(n=12, dim=dim, seed=dim, deg=4)
    theta = mpnn.init_params(dim, seed=1).astype(np.float64)
    theta += np.random.default_rng(2).normal(scale=0.05, size=theta.shape)
    dout = np.random.default_rng(3).normal(size=(node.shape[0], dim + 1))
    g = mpnn.grad_np(theta, dim, node, recv, send, edge, dout)
    f = lambda th: float((mpnn.forward_np(th, dim, node, recv, send, edge) * dout).sum())
    idx = np.random.default_rng(4).choice(theta.size, size=40, replace=False)
    for k in idx:
        e = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[k] += e
        tm[k] -= e
        fd = (f(tp) - f(tm)) / (2 * e)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_permutation_equivariance():
    node, recv, send, edge = _graph(n=30, seed=5)
    theta = mpnn.init_params(2, seed=3)
    out = mpnn.forward_np(theta, 2, node, recv, send, edge)
    perm = np.random.default_rng(9).permutation(node.shape[0])
    inv = np.argsort(perm)
    out_p = mpnn.forward_np(theta, 2, node[perm], inv[recv], inv[send], edge)
    assert np.allclose(out_p, out[perm], rtol=1e-12, atol=1e-12)


def test_disjoint_graphs_batch_additively():
    a = _graph(n=20, seed=1)
    b = _graph(n=15, seed=2)
    theta = mpnn.init_params(2, seed=4)
    oa = mpnn.forward_np(theta, 2, *a)
    ob = mpnn.forward_np(theta, 2, *b)
    node = np.concatenate([a[0], b[0]])
    recv = np.concatenate([a[1], b[1] + 20])
    send = np.concatenate([a[2], b[2] + 20])
    edge = np.concatenate([a[3], b[3]])
    o = mpnn.forward_np(theta, 2, node, recv, send, edge)
    assert np.allclose(o[:20], oa, atol=1e-12) and np.allclose(o[20:], ob, atol=1e-12)


def test_isolated_receiver_has_no_messages():
    """A node that receives no edge gets a = 0 in every layer: its output is
    dec(h_L) with h_{l+1} = h_l + MLP_n([h_l, 0]), independent of the rest."""
    node, recv, send, edge = _graph(n=20, seed=6)
    keep = recv != 0
    recv, send, edge = recv[keep], send[keep], edge[keep]
    theta = mpnn.init_params(2, seed=5)
    out = mpnn.forward_np(theta, 2, node, recv, send, edge)
    node2 = node.copy()
    node2[1:] += 3.0
    out2 = mpnn.forward_np(theta, 2, node2, recv, send, edge)
    assert np.array_equal(out[0], out2[0])
    assert not np.allclose(out[1:], out2[1:])


def test_parameter_count_and_layout():
    assert mpnn.num_params(2) == mpnn.init_params(2).size
    P = mpnn.unflatten(torch.zeros(mpnn.num_params(3), dtype=torch.float64), 3)
    assert P["mp0_e"][0].shape == (8 + 64 + 32, 64) and P["dec"][2].shape == (64, 4)
    assert P["enc_n"][0].shape == (6, 64) and "enc_e" not in P
    # 2D: encoder 5*64+64+64*64+64, per layer edge (6+64+32)*64+64+64*64+64 and
    # node 128*64+64+64*64+64, decoder 64*64+64+64*3+3
    assert mpnn.num_params(2) == 4544 + 3 * (10752 + 12416) + 4355


def test_message_sum_taken_apart_edge_by_edge():
    """One layer's aggregate m_i = sum_j MLP_e([g_ij, h_i, h_j[:32]]),
    evaluated here edge by edge with explicit loops and numpy for a one-layer
    network: the decoder input must equal h + MLP_n([h, m]). Catches a wrong
    sender or receiver gather, a missing sum, a residual on the messages and
    the wrong half of the sender's state."""
    dim = 2
    node, recv, send, edge = _graph(n=9, dim=dim, seed=11, deg=3)
    theta = mpnn.init_params(dim, seed=7, layers=1).astype(np.float64)
    theta += np.random.default_rng(8).normal(scale=0.1, size=theta.shape)
    P = {k: tuple(t.numpy() for t in v)
         for k, v in mpnn.unflatten(torch.as_tensor(theta), dim, layers=1).items()}

    def silu(z):
        return z / (1.0 + np.exp(-z))

    def mlp(x, p):
        return silu(x @ p[0] + p[1]) @ p[2] + p[3]

    h = mlp(node, P["enc_n"])
    m = np.zeros_like(h)
    for e in range(recv.size):
        i, j = recv[e], send[e]
        m[i] += mlp(np.concatenate([edge[e], h[i], h[j][:32]]), P["mp0_e"])
    h1 = h + mlp(np.concatenate([h, m], axis=1), P["mp0_n"])
    want = mlp(h1, P["dec"])
    with torch.no_grad():
        got = mpnn.forward(torch.as_tensor(theta), dim, torch.as_tensor(node), torch.as_tensor(recv),
                           torch.as_tensor(send), torch.as_tensor(edge), layers=1).numpy()
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_graph_and_features_by_hand():
    """Receivers are the fluid particles, senders everything within 2h; the
    features follow their definitions, worked out by hand for four particles
    (h = 0.13): fluid 0 at (0.5, 0.5), fluid 1 at (0.6, 0.5), a dummy 2 at
    (0.5, 0.3) and fluid 3 at (0.9, 0.5), out of everyone's reach."""
    import math

    from paper_2608_22269_gb300 import scenes as S
    p = S.default_params(2, dx=0.1, c0=10.0)                  # G = (0, -9.81)
    x = np.array([[0.5, 0.6, 0.5, 0.9], [0.5, 0.5, 0.3, 0.5]])
    u = np.array([[0.1, -0.2, 0.05, 0.0], [0.3, 0.0, -0.1, 0.0]])
    phi = np.array([2.0, 1.5, 4.0, 0.0])
    typ = np.array([0, 0, 1, 0], dtype=np.uint8)
    mean = np.array([0.1, -0.1, 0.0, 1.0], dtype=np.float32)
    std = np.array([0.5, 0.25, 0.001, 2.0], dtype=np.float32)
    estd = np.array([0.4, 0.8], dtype=np.float32)
    H = 0.7                                                    # water height of the split
    recv, send, node_in, edge_in = mpnn.graph_and_features(p, x, u, phi, typ, mean, std, estd, H)
    assert recv.tolist() == [0, 0, 1, 1] and send.tolist() == [1, 2, 0, 2]
    h = 0.13
    m, sd = mean.astype(np.float64), std.astype(np.float64)  # the FP32 values the library holds
    es = estd.astype(np.float64)
    # phi' = phi - (G.x + |G| H) = phi - 9.81 (H - y)
    phip = [phi[k] - 9.81 * (H - x[1, k]) for k in range(4)]
    for k in range(4):
        rho = 1000.0 * math.exp(phi[k] / 100.0)  # linear EOS, C0 = 10
        want = [(u[0, k] - m[0]) / sd[0], (u[1, k] - m[1]) / sd[1], (rho / 1000.0 - 1.0) / sd[2],
                (phip[k] - m[3]) / sd[3], 1.0 if k == 2 else 0.0]
        assert np.array_equal(node_in[k], mpnn.bf16_round(np.array(want)).astype(np.float64))
    for e, (i, j) in enumerate([(0, 1), (0, 2), (1, 0), (1, 2)]):
        rx, ry = x[0, j] - x[0, i], x[1, j] - x[1, i]
        want = [rx / h, ry / h, math.hypot(rx, ry) / h, (u[0, j] - u[0, i]) / es[0],
                (u[1, j] - u[1, i]) / es[0], (phip[j] - phip[i]) / es[1]]
        assert np.allclose(edge_in[e], mpnn.bf16_round(np.array(want)), rtol=0, atol=1e-12), e


def test_hydrostatic_state_has_no_potential_differences():
    """At rest with phi = G.x + |G| H (the hydrostatic state of Eq. eqSol as
    the scenes write it) every edge's potential input vanishes and every
    node's phi' is zero, whatever the positions: the split removes the
    hydrostatic part exactly (up to the rounding of phi itself)."""
    from paper_2608_22269_gb300 import scenes as S
    sc = S.jitter(S.dam_break_2d(dx=0.02, width=0.8, column=(0.3, 0.2)), 0.2, seed=3)
    f = sc.type == 0
    phi = 9.81 * (sc.water_height - sc.x[1])               # at the jittered positions
    mean = np.zeros(4, np.float32)
    std = np.ones(4, np.float32)
    recv, send, node_in, edge_in = mpnn.graph_and_features(sc.params, sc.x, sc.u, phi, sc.type, mean,
                                                           std, np.ones(2, np.float32), sc.water_height)
    assert recv.size > 1000
    assert np.abs(edge_in[:, 5]).max() <= 1e-14 and np.abs(node_in[f, 3]).max() <= 1e-14


def _bf(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _forward_bf16(theta, dim, node_in, recv, send, edge_in):
    """The network with activations rounded to BF16 where the CUDA kernels
    round them (encoder and node-MLP hidden layers, states h, the message
    layer's halved first-layer terms, its SiLU input and output, and m), sums
    in FP64 where the kernels accumulate in FP32 (the message sum is kept in
    FP32 and enters W2 as a BF16 high and low part, so it is never rounded to
    BF16), exact tanh where they use the hardware approximation: a model of
    the kernels' arithmetic, used only to bound the error that BF16 alone
    causes."""
    P = {k: tuple(t.numpy() for t in v) for k, v in mpnn.unflatten(torch.as_tensor(theta), dim).items()}

    def silu(z):
        return z / (1.0 + np.exp(-z))

    w1, b1, w2, b2 = P["enc_n"]
    h = _bf(_bf(silu(node_in @ w1 + b1)) @ w2 + b2)
    n, kg = h.shape[0], edge_in.shape[1]
    for layer in range(mpnn.LAYERS):
        we1, be1, we2, be2 = P[f"mp{layer}_e"]
        wg, wr, ws = _bf(0.5 * we1[:kg]), _bf(0.5 * we1[kg:kg + 64]), _bf(0.5 * we1[kg + 64:])
        pr = _bf(h @ wr + 0.5 * be1)
        u = _bf(_bf(edge_in @ wg + h[send][:, :mpnn.SEND] @ ws) + pr[recv])
        sm = _bf(u + _bf(u * _bf(np.tanh(u))))          # silu(2u) = u + u tanh u
        acc = np.zeros((n, 64))
        np.add.at(acc, recv, sm)                        # sum_j silu W2 = (sum_j silu) W2 in exact arithmetic
        cnt = np.bincount(recv, minlength=n).astype(np.float64)
        m = _bf(acc @ we2 + cnt[:, None] * be2)
        wn1, bn1, wn2, bn2 = P[f"mp{layer}_n"]
        h = _bf(h + _bf(silu(np.c_[h, m] @ wn1 + bn1)) @ wn2 + bn2)
    wd1, bd1, wd2, bd2 = P["dec"]
    return _bf(silu(h @ wd1 + bd1)) @ wd2 + bd2


def test_bf16_error_of_the_trained_2d_network():
    """The committed 2D weights on a dam-break column at rest (about 8,000
    fluid particles): the BF16 model of the kernels' arithmetic deviates
    from the FP64 reference by a few per cent of the largest normalised
    output. The trained network's horizontal acceleration at rest is a small
    residual of larger activations, so its BF16 error is well above the
    ~1 % of a random network; the full-size GPU check of the trained
    network (tests/test_gpu_fullsize.py) takes its 5e-2 bound from this."""
    import os

    from oracle import oracle as O
    from paper_2608_22269_gb300 import surrogate as SG
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    z = np.load(os.path.join(root, "paper_2608_22269_gb300", "data", "surrogate_2d.npz"))
    nm, ns, es = (np.asarray(z[k], dtype=np.float32) for k in ("node_mean", "node_std", "edge_std"))
    sc = SG.dam_scene(0.45, 0.3, 8000)
    p = sc.params
    u, phi = O.dummy_update(p, sc.x, sc.u, sc.phi, sc.type, sc.normal, 0.0)
    recv, send, node_in, edge_in = mpnn.graph_and_features(p, sc.x, u, phi, sc.type, nm, ns, es, sc.water_height)
    th = mpnn.round_weights_bf16(z["params"], 2)
    ref = mpnn.forward_np(th, 2, node_in, recv, send, edge_in)
    em = _forward_bf16(th, 2, node_in, recv, send, edge_in)
    f = sc.type == 0
    rel = np.abs(em[f] - ref[f]).max() / np.abs(ref[f]).max()
    print("BF16 model against FP64, trained 2D network:", rel)
    assert 0.005 < rel < 0.05
