"""Learned best-so-far proposal network, written out in FP64 (test infrastructure only).

Not in the paper: the network only proposes where the approximate search (Sec. 3.3) should
look, so it never changes an answer. Shape: PAA (16) -> 256 -> 256 -> 4096 logits, exact GELU
after the two hidden layers, softmax cross-entropy over 4096 buckets (bucket = the first 12
bits of the interleaved iSAX key = first bit of segments 0..11), AdamW updates.

Parameters are a dict of numpy arrays: W1 [256][16], b1 [256], W2 [256][256], b2 [256],
W3 [4096][256], b3 [4096] (out x in, as the library stores them).
"""
from __future__ import annotations

import math

import numpy as np

SHAPES = {"W1": (256, 16), "b1": (256,), "W2": (256, 256), "b2": (256,), "W3": (4096, 256), "b3": (4096,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(z):
    """Exact GELU: z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2))."""
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, x):
    """x [B][16] -> (logits [B][4096], cache)."""
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    logits = h2 @ params["W3"].T + params["b3"]
    return logits, (x, z1, h1, z2, h2)


def cross_entropy(logits, labels):
    """Mean softmax cross-entropy and its gradient with respect to the logits."""
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    s = e.sum(axis=1, keepdims=True)
    p = e / s
    B = logits.shape[0]
    loss = float(np.mean(np.log(s[:, 0]) + m[:, 0] - logits[np.arange(B), labels]))
    d = p.copy()
    d[np.arange(B), labels] -= 1.0
    return loss, d / B


def loss_and_grads(params, x, labels):
    logits, (x, z1, h1, z2, h2) = forward(params, x)
    loss, dl = cross_entropy(logits, labels)
    g = {}
    g["W3"] = dl.T @ h2
    g["b3"] = dl.sum(axis=0)
    dz2 = (dl @ params["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ params["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adamw_step(params, grads, state, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One AdamW update (decoupled weight decay on every parameter), t counted from 1."""
    out = {}
    for k in ORDER:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        out[k] = params[k] - lr * (mh / (np.sqrt(vh) + eps) + weight_decay * params[k])
    return out


def topr_of_logits(logits, r):
    """The r highest-scoring buckets of each row of a logit matrix [B][4096], best first; equal
    logits are ranked by lower bucket (a stable sort on the negated scores)."""
    logits = np.asarray(logits)
    order = np.argsort(-logits, axis=1, kind="stable")
    return order[:, :r]


def topr_buckets(params, x, r):
    """The r highest-scoring buckets per row of the network's logits (ties by lower bucket)."""
    logits, _ = forward(params, x)
    return topr_of_logits(logits, r)
