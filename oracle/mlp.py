"""ORACLE - test infrastructure, not part of the product.

FP64 numpy reference of the direction-policy network used by the CUDA
library: a multilayer perceptron 6 -> 32 -> 32 -> K with ReLU hidden layers,
parameters packed as W1[32][6], b1[32], W2[32][32], b2[32], W3[K][32], b3[K].

  forward(p, x, k)                  outputs [n, k]
  loss_grad(p, x, t, w, k, kind)    weighted loss and its analytic gradient
                                    (kind 0: softmax cross-entropy with class
                                    targets; kind 1: squared error), weights
                                    normalised by their sum
  adam(p, g, m, v, t, ...)          one Adam step (Kingma and Ba, ICLR 2015)
  forward_fp16_weights(p, x, k)     the inference path: weights rounded to
                                    float16, sums in float32

The analytic gradient is pinned by central finite differences of loss() in
the tests (FP64).
"""
from __future__ import annotations

import numpy as np

IN, H = 6, 32


def param_count(k: int) -> int:
    return H * IN + H + H * H + H + k * H + k


def unpack(p, k):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + k * H].reshape(k, H); o += k * H
    b3 = p[o:o + k]; o += k
    assert o == len(p)
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def init(k: int, seed: int = 0) -> np.ndarray:
    """He-style random initialisation (seeded)."""
    r = np.random.default_rng(seed)
    W1 = r.normal(0, np.sqrt(2 / IN), (H, IN))
    W2 = r.normal(0, np.sqrt(2 / H), (H, H))
    W3 = r.normal(0, np.sqrt(1 / H), (k, H))
    return pack(W1, np.zeros(H), W2, np.zeros(H), W3, np.zeros(k))


def forward(p, x, k, return_hidden=False):
    W1, b1, W2, b2, W3, b3 = unpack(p, k)
    x = np.asarray(x, np.float64).reshape(-1, IN)
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0)
    out = a2 @ W3.T + b3
    if return_hidden:
        return out, (x, z1, a1, z2, a2)
    return out


def loss(p, x, t, w, k, kind):
    out = forward(p, x, k)
    n = out.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, np.float64)
    ws = w / w.sum()
    t = np.asarray(t, np.float64)
    if kind == 0:
        m = out.max(axis=1, keepdims=True)
        lse = (m + np.log(np.exp(out - m).sum(axis=1, keepdims=True)))[:, 0]
        return float(np.sum(ws * (lse - out[np.arange(n), t.astype(int)])))
    r = out[:, 0] - t
    return float(np.sum(ws * r * r))


def loss_grad(p, x, t, w, k, kind):
    """(loss, gradient) by backpropagation written out layer by layer."""
    W1, b1, W2, b2, W3, b3 = unpack(p, k)
    out, (x, z1, a1, z2, a2) = forward(p, x, k, return_hidden=True)
    n = out.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, np.float64)
    ws = w / w.sum()
    t = np.asarray(t, np.float64)
    if kind == 0:
        m = out.max(axis=1, keepdims=True)
        e = np.exp(out - m)
        prob = e / e.sum(axis=1, keepdims=True)
        ti = t.astype(int)
        L = float(np.sum(ws * (np.log(e.sum(axis=1)) + m[:, 0] - out[np.arange(n), ti])))
        d_out = prob.copy()
        d_out[np.arange(n), ti] -= 1.0
        d_out *= ws[:, None]
    else:
        r = out[:, 0] - t
        L = float(np.sum(ws * r * r))
        d_out = (2 * ws * r)[:, None]
    gW3 = d_out.T @ a2
    gb3 = d_out.sum(axis=0)
    d_a2 = d_out @ W3
    d_z2 = d_a2 * (z2 > 0)
    gW2 = d_z2.T @ a1
    gb2 = d_z2.sum(axis=0)
    d_a1 = d_z2 @ W2
    d_z1 = d_a1 * (z1 > 0)
    gW1 = d_z1.T @ x
    gb1 = d_z1.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def forward_fp16_weights(p, x, k=2):
    """Inference reference: parameters rounded to float16, arithmetic in float32."""
    q = np.asarray(p, np.float32).astype(np.float16).astype(np.float32)
    W1, b1, W2, b2, W3, b3 = (a.astype(np.float32) for a in unpack(q, k))
    x = np.asarray(x, np.float32).reshape(-1, IN)
    a1 = np.maximum(x @ W1.T + b1, 0)
    a2 = np.maximum(a1 @ W2.T + b2, 0)
    return a2 @ W3.T + b3
