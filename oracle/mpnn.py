"""FP64 reference of the message-passing surrogate (test infrastructure only).

Plain PyTorch CPU float64 statement of the network that the CUDA surrogate
kernels evaluate in BF16 with FP32 accumulation; gradients come from
autograd of this forward and are pinned by central finite differences in
the tests. Only the tests may import this module. The paper has no learned
part: this network is the surrogate of the pair pass that the rollouts use
between plain re-anchoring steps.

Network (dimension d, hidden H = 64, three message-passing layers):
  hydrostatic split  phi'_i = phi_i - phi_hs(x_i), phi_hs(x) = G.x + |G| H
                     (G the constant body force, H the scene's water height;
                     the same split as the mixed path), so that at rest the
                     potential input carries only the departure from balance
  node input  f_i = (U_i, rho_i/rho0 - 1, phi'_i) minus node_mean over
              node_std, then the dummy flag                              (d + 3)
  edge input  g_ij = ((x_j - x_i)/h, |x_j - x_i|/h, (U_j - U_i)/s_U, (phi'_j - phi'_i)/s_phi)
              for receiver i, sender j (2d + 2; s_U, s_phi the edge scales)
  MLP(x) = W2 silu(W1 x + b1) + b2 (weights stored input-major: x @ W)
  h = MLP_enc(f)
  per layer: m_i = sum_j MLP_e([g_ij, h_i, h_j[:32]]);  h <- h + MLP_n([h_i, m_i])
  (a sender contributes the first 32 of its 64 state features)
  output y_i = MLP_dec(h_i)  (d + 1: normalised DU/Dt and Dphi/Dt)
No state is kept per edge: every layer's messages are formed from the edge
inputs g_ij and the node states. Edges: every fluid receiver i with every
particle j within 2h (dummies only send). Loss: mean over fluid particles and
output components of the squared difference to the normalised targets.

Flat parameter layout (shared with the CUDA library): blocks in the order
node encoder, (edge MLP, node MLP) per layer, decoder; each block W1 [in][H],
b1 [H], W2 [H][out], b2 [out], row-major; the edge MLP's W1 rows are the
2d + 2 edge inputs, then h_i (64 rows), then h_j[:32] (32 rows).
"""
from __future__ import annotations

import numpy as np
import torch

HIDDEN = 64
LAYERS = 3
SEND = 32   # sender features in a message


def block_dims(dim: int, hidden: int = HIDDEN, layers: int = LAYERS):
    fn, fe, fo = dim + 3, 2 * dim + 2, dim + 1
    dims = [("enc_n", fn, hidden)]
    for l in range(layers):
        dims += [(f"mp{l}_e", fe + hidden + SEND, hidden), (f"mp{l}_n", 2 * hidden, hidden)]
    dims.append(("dec", hidden, fo))
    return dims


def num_params(dim: int, hidden: int = HIDDEN, layers: int = LAYERS) -> int:
    return sum(i * hidden + hidden + hidden * o + o for _, i, o in block_dims(dim, hidden, layers))


def unflatten(theta: torch.Tensor, dim: int, hidden: int = HIDDEN, layers: int = LAYERS):
    out, k = {}, 0
    for name, i, o in block_dims(dim, hidden, layers):
        w1 = theta[k:k + i * hidden].view(i, hidden); k += i * hidden
        b1 = theta[k:k + hidden]; k += hidden
        w2 = theta[k:k + hidden * o].view(hidden, o); k += hidden * o
        b2 = theta[k:k + o]; k += o
        out[name] = (w1, b1, w2, b2)
    assert k == theta.numel()
    return out


def init_params(dim: int, seed: int = 0, hidden: int = HIDDEN, layers: int = LAYERS) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases; the last
    layer of every processor MLP is scaled by 0.1 so that the residual updates
    start small (the edge MLP's by a further 1/8: its outputs are summed over
    the receiver's neighbours)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, i, o in block_dims(dim, hidden, layers):
        s1, s2 = 1.0 / np.sqrt(i), 1.0 / np.sqrt(hidden)
        if name.startswith("mp"):
            s2 *= 0.1
        if name.endswith("_e"):
            s2 /= 8.0
        parts += [rng.uniform(-s1, s1, i * hidden), np.zeros(hidden),
                  rng.uniform(-s2, s2, hidden * o), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


def _mlp(x, p):
    w1, b1, w2, b2 = p
    return torch.nn.functional.silu(x @ w1 + b1) @ w2 + b2


def forward(theta, dim, node_in, recv, send, edge_in, hidden=HIDDEN, layers=LAYERS):
    """node_in (N, d+3), recv/send (E,) int64, edge_in (E, 2d+2) -> (N, d+1)."""
    P = unflatten(theta, dim, hidden, layers)
    h = _mlp(node_in, P["enc_n"])
    for l in range(layers):
        msg = _mlp(torch.cat([edge_in, h[recv], h[send][:, :SEND]], dim=1), P[f"mp{l}_e"])
        m = torch.zeros(h.shape, dtype=h.dtype).index_add(0, recv, msg)
        h = h + _mlp(torch.cat([h, m], dim=1), P[f"mp{l}_n"])
    return _mlp(h, P["dec"])


def hydrostatic_potential(params, x, water_height):
    """phi_hs(x) = G.x + |G| H with the constant body force G of the scene."""
    d = int(params["dim"])
    g = np.asarray(params["g"][:d], dtype=np.float64)
    return g @ np.asarray(x, dtype=np.float64)[:d] + np.linalg.norm(g) * water_height


def graph_and_features(params, x, u, phi, typ, node_mean, node_std, edge_std, water_height,
                       row=None, col=None):
    """Edges and network inputs of a particle state, by the definitions above.

    u and phi are the stage's values (wall particles after their update from
    the nearest fluid particle); row/col is the oracle's neighbour CSR of x
    (computed here when None). Receivers are the fluid particles in ascending
    index, each with its neighbours within 2h in ascending index as senders.
    Node inputs: (U, rho/rho0 - 1, phi') minus node_mean over node_std, then
    the dummy flag; edge inputs: ((x_j - x_i)/h, |x_j - x_i|/h,
    (U_j - U_i)/s_U, (phi'_j - phi'_i)/s_phi) with (s_U, s_phi) = edge_std.
    Both are rounded to BF16, the precision the network reads them in.
    Returns recv, send (int64), node_in (N, d + 3) and edge_in (E, 2d + 2) as
    float64."""
    from . import oracle as O
    d = int(params["dim"])
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    typ = np.asarray(typ)
    mean = np.asarray(node_mean, dtype=np.float64)
    std = np.asarray(node_std, dtype=np.float64)
    es = np.asarray(edge_std, dtype=np.float64)
    if row is None:
        row, col = O.neighbors(params, x)
    fl = np.nonzero(typ == 0)[0]
    cnt = (row[fl + 1] - row[fl]).astype(np.int64)
    E = int(cnt.sum())
    recv = np.repeat(fl, cnt).astype(np.int64)
    start = np.repeat(row[fl], cnt)
    within = np.arange(E, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    send = np.asarray(col, dtype=np.int64)[start + within]
    h = params["h_over_dx"] * params["dx"]
    rho = O.density(params, phi)
    phip = phi - hydrostatic_potential(params, x, water_height)
    raw = np.r_[u[:d], (rho / params["rho0"] - 1.0)[None], phip[None]]
    node_in = np.c_[((raw - mean[:d + 2, None]) / std[:d + 2, None]).T, (typ != 0).astype(np.float64)]
    r = x[:d, send] - x[:d, recv]
    edge_in = np.c_[(r / h).T, np.sqrt((r * r).sum(axis=0)) / h,
                    ((u[:d, send] - u[:d, recv]) / es[0]).T, (phip[send] - phip[recv]) / es[1]]
    return (recv, send, bf16_round(node_in).astype(np.float64),
            bf16_round(edge_in).astype(np.float64))


def loss(out, target, fluid):
    d = out[fluid] - target[fluid]
    return (d * d).mean()


def as_t(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64)


def forward_np(theta, dim, node_in, recv, send, edge_in):
    with torch.no_grad():
        return forward(as_t(theta), dim, as_t(node_in), torch.as_tensor(recv, dtype=torch.int64),
                       torch.as_tensor(send, dtype=torch.int64), as_t(edge_in)).numpy()


def grad_np(theta, dim, node_in, recv, send, edge_in, dout):
    """Gradient of sum(dout * out) with respect to the flat parameters."""
    th = as_t(theta).clone().requires_grad_(True)
    out = forward(th, dim, as_t(node_in), torch.as_tensor(recv, dtype=torch.int64),
                  torch.as_tensor(send, dtype=torch.int64), as_t(edge_in))
    (out * as_t(dout)).sum().backward()
    return th.grad.numpy()


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even) and back, as the
    surrogate stores weights and activations."""
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def round_weights_bf16(theta: np.ndarray, dim: int, hidden: int = HIDDEN, layers: int = LAYERS) -> np.ndarray:
    """Weights (W1, W2 of every block) rounded to bfloat16, biases unchanged:
    the parameters exactly as the BF16 kernels use them."""
    out = np.asarray(theta, dtype=np.float64).copy()
    k = 0
    for _, i, o in block_dims(dim, hidden, layers):
        for size, is_w in ((i * hidden, True), (hidden, False), (hidden * o, True), (o, False)):
            if is_w:
                out[k:k + size] = bf16_round(out[k:k + size])
            k += size
    return out
