"""CPU oracle of the learned edge-MLP prior (float64 numpy): forward, loss and backward.

TEST INFRASTRUCTURE ONLY (imported by tests/ and nothing in the product path).  The paper
has no learned component; the model below is this project's definition of the learned prior
that feeds LSD, and the GPU kernels implement the same definition in BF16 with FP32
accumulation.  Its backward pass is pinned by finite differences
(tests/test_oracle_prior.py).

Model, for a check matrix H (m x n) with edges (c, v), hidden width Hd, R rounds:
    sigma_c = 1 - 2 s_c                        (syndrome bit as +-1)
    h_v^0  = relu(lambda_v * a0 + a1)          (lambda_v: channel-prior LLR)
    h_c^0  = sigma_c * u0 + u1
    for t = 0 .. R-1:
        h_v^{t+1} = h_v^t + sum_{c in N(v)} MLP_cv([h_c^t, h_v^t, sigma_c])
        h_c^{t+1} = h_c^t + sum_{v in N(c)} MLP_vc([h_v^{t+1}, h_c^t, sigma_c])
    LLR_v = lambda_v + w_o . h_v^R + b_o
    MLP(x) = W2 relu(W1 x + b1) + b2,   W1: Hd x (2 Hd + 1),  W2: Hd x Hd
    loss = mean over shots and v of  softplus(LLR_v) - (1 - e_v) LLR_v
           (binary cross-entropy of P(e_v = 1) = sigmoid(-LLR_v))
The MLP weights are shared by the R rounds, one MLP per message direction.

Flat parameter order (the C ABI uses the same): a0, a1, u0, u1,
W1_cv, b1_cv, W2_cv, b2_cv, W1_vc, b1_vc, W2_vc, b2_vc, w_o, b_o.
"""
from __future__ import annotations

import numpy as np


def param_shapes(hd: int = 32):
    din = 2 * hd + 1
    return [("a0", (hd,)), ("a1", (hd,)), ("u0", (hd,)), ("u1", (hd,)),
            ("W1_cv", (hd, din)), ("b1_cv", (hd,)), ("W2_cv", (hd, hd)), ("b2_cv", (hd,)),
            ("W1_vc", (hd, din)), ("b1_vc", (hd,)), ("W2_vc", (hd, hd)), ("b2_vc", (hd,)),
            ("w_o", (hd,)), ("b_o", (1,))]


def num_params(hd: int = 32) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(hd)))


def unflatten(theta, hd: int = 32):
    out, off = {}, 0
    for name, shp in param_shapes(hd):
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[off:off + k], dtype=np.float64).reshape(shp)
        off += k
    return out


def flatten(p, hd: int = 32):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel()
                           for name, _ in param_shapes(hd)])


class Graph:
    """Edges of H in row-major order with one-hot scatter matrices."""

    def __init__(self, h):
        h = np.asarray(h, dtype=np.uint8)
        self.m, self.n = h.shape
        self.ec, self.ev = np.nonzero(h)
        E = self.ec.size
        self.Sc = np.zeros((self.m, E))  # check <- edge
        self.Sv = np.zeros((self.n, E))  # variable <- edge
        self.Sc[self.ec, np.arange(E)] = 1.0
        self.Sv[self.ev, np.arange(E)] = 1.0


def _mlp_fwd(x, W1, b1, W2, b2):
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    return z1, a1, a1 @ W2.T + b2


def forward(g: Graph, theta, syndromes, lam, rounds: int = 4, hd: int = 32):
    """Returns (LLR [B][n], cache for backward)."""
    p = unflatten(theta, hd)
    s = np.atleast_2d(np.asarray(syndromes, dtype=np.float64))
    B = s.shape[0]
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), (B, g.n))
    sig = 1.0 - 2.0 * s                                          # [B][m]
    zv0 = lam[..., None] * p["a0"] + p["a1"]                     # [B][n][hd]
    hv = np.maximum(zv0, 0.0)
    hc = sig[..., None] * p["u0"] + p["u1"]                      # [B][m][hd]
    sig_e = sig[:, g.ec][..., None]                              # [B][E][1]
    cache = dict(p=p, sig=sig, sig_e=sig_e, zv0=zv0, lam=lam, steps=[])
    for _ in range(rounds):
        x1 = np.concatenate([hc[:, g.ec], hv[:, g.ev], sig_e], axis=-1)
        z1a, a1a, m1 = _mlp_fwd(x1, p["W1_cv"], p["b1_cv"], p["W2_cv"], p["b2_cv"])
        hv_new = hv + np.einsum("ve,beh->bvh", g.Sv, m1)
        x2 = np.concatenate([hv_new[:, g.ev], hc[:, g.ec], sig_e], axis=-1)
        z1b, a1b, m2 = _mlp_fwd(x2, p["W1_vc"], p["b1_vc"], p["W2_vc"], p["b2_vc"])
        hc_new = hc + np.einsum("ce,beh->bch", g.Sc, m2)
        cache["steps"].append((x1, z1a, a1a, x2, z1b, a1b))
        hv, hc = hv_new, hc_new
    llr = lam + hv @ p["w_o"] + p["b_o"][0]
    cache["hv"] = hv
    return llr, cache


def loss_and_dllr(llr, errors):
    """Mean binary cross-entropy and its gradient w.r.t. the LLRs."""
    e = np.asarray(errors, dtype=np.float64)
    sp = np.logaddexp(0.0, llr)                                  # softplus
    loss = np.mean(sp - (1.0 - e) * llr)
    sig = 1.0 / (1.0 + np.exp(-llr))
    dllr = (sig - (1.0 - e)) / llr.size
    return loss, dllr


def _mlp_bwd(dm, x, z1, a1, W1, W2):
    """Gradients of MLP(x) = W2 relu(W1 x + b1) + b2 given dL/dMLP = dm (rows over edges)."""
    dW2 = np.einsum("beh,bej->hj", dm, a1)
    db2 = dm.sum(axis=(0, 1))
    da1 = dm @ W2
    dz1 = da1 * (z1 > 0)
    dW1 = np.einsum("beh,bej->hj", dz1, x)
    db1 = dz1.sum(axis=(0, 1))
    dx = dz1 @ W1
    return dx, dW1, db1, dW2, db2


def backward(g: Graph, cache, dllr, rounds: int = 4, hd: int = 32):
    """Gradient of the loss w.r.t. the flat parameter vector."""
    p = cache["p"]
    grads = {name: np.zeros(shp) for name, shp in param_shapes(hd)}
    grads["w_o"] = np.einsum("bv,bvh->h", dllr, cache["hv"])
    grads["b_o"] = np.array([dllr.sum()])
    dhv = dllr[..., None] * p["w_o"]                             # dL/dh_v^R
    dhc = np.zeros((dllr.shape[0], g.m, hd))                     # dL/dh_c^R
    for t in reversed(range(rounds)):
        x1, z1a, a1a, x2, z1b, a1b = cache["steps"][t]
        # h_c^{t+1} = h_c^t + Sc m2(x2);  x2 = [h_v^{t+1}, h_c^t, sigma]
        dm2 = dhc[:, g.ec]
        dx2, dW1, db1, dW2, db2 = _mlp_bwd(dm2, x2, z1b, a1b, p["W1_vc"], p["W2_vc"])
        grads["W1_vc"] += dW1
        grads["b1_vc"] += db1
        grads["W2_vc"] += dW2
        grads["b2_vc"] += db2
        dhv = dhv + np.einsum("ve,beh->bvh", g.Sv, dx2[..., :hd])
        dhc = dhc + np.einsum("ce,beh->bch", g.Sc, dx2[..., hd:2 * hd])
        # h_v^{t+1} = h_v^t + Sv m1(x1);  x1 = [h_c^t, h_v^t, sigma]
        dm1 = dhv[:, g.ev]
        dx1, dW1, db1, dW2, db2 = _mlp_bwd(dm1, x1, z1a, a1a, p["W1_cv"], p["W2_cv"])
        grads["W1_cv"] += dW1
        grads["b1_cv"] += db1
        grads["W2_cv"] += dW2
        grads["b2_cv"] += db2
        dhc = dhc + np.einsum("ce,beh->bch", g.Sc, dx1[..., :hd])
        dhv = dhv + np.einsum("ve,beh->bvh", g.Sv, dx1[..., hd:2 * hd])
    # h_v^0 = relu(lam a0 + a1),  h_c^0 = sigma u0 + u1
    dzv0 = dhv * (cache["zv0"] > 0)
    grads["a0"] = np.einsum("bvh,bv->h", dzv0, cache["lam"])
    grads["a1"] = dzv0.sum(axis=(0, 1))
    grads["u0"] = np.einsum("bch,bc->h", dhc, cache["sig"])
    grads["u1"] = dhc.sum(axis=(0, 1))
    return flatten(grads, hd)


def loss_and_grad(h, theta, syndromes, errors, lam, rounds: int = 4, hd: int = 32):
    g = Graph(h)
    llr, cache = forward(g, theta, syndromes, lam, rounds, hd)
    loss, dllr = loss_and_dllr(llr, errors)
    return loss, backward(g, cache, dllr, rounds, hd), llr
