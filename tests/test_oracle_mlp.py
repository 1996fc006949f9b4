"""Pins of the MLP oracle: closed forms (GELU values, cross-entropy of uniform logits = ln 4096),
central finite differences of every gradient on a small net, and the AdamW update rule on a
one-parameter quadratic."""
import math

import numpy as np

from oracle import mlp


def small_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return {k: rng.standard_normal(s) * scale for k, s in mlp.SHAPES.items()}


def test_gelu_closed_form():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    phi = np.array([0.5 * math.erfc(-v / math.sqrt(2)) for v in z])
    assert np.allclose(mlp.gelu(z), z * phi, rtol=1e-15, atol=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


def test_uniform_logits_loss_is_ln_4096():
    p = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    x = np.random.default_rng(1).standard_normal((5, 16))
    loss, g = mlp.loss_and_grads(p, x, np.array([0, 7, 4095, 12, 2048]))
    assert abs(loss - math.log(4096)) < 1e-12
    # with zero weights only the output bias receives a gradient: (1/4096 - onehot) / B
    assert abs(g["b3"][0] - (5 / 4096 - 1) / 5) < 1e-15
    assert np.all(g["W1"] == 0) and np.all(g["W3"] == 0)


def test_gradients_match_central_differences():
    p = small_params(3)
    x = np.random.default_rng(4).standard_normal((6, 16))
    y = np.array([1, 4000, 77, 1, 2048, 333])
    _, g = mlp.loss_and_grads(p, x, y)
    rng = np.random.default_rng(5)
    h = 1e-6
    for k in mlp.ORDER:
        for _ in range(6):
            idx = tuple(int(rng.integers(0, d)) for d in p[k].shape)
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += h
            lp, _ = mlp.loss_and_grads(q, x, y)
            q[k][idx] -= 2 * h
            lm, _ = mlp.loss_and_grads(q, x, y)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, g[k][idx])


def test_adamw_first_step_is_signed_lr():
    # first AdamW step moves every parameter by lr * sign(g) (bias-corrected moments), minus decay
    p = {k: np.full(s, 2.0) for k, s in mlp.SHAPES.items()}
    g = {k: np.full(s, -3.0) for k, s in mlp.SHAPES.items()}
    out = mlp.adamw_step(p, g, {}, 1, lr=0.01, eps=0.0, weight_decay=0.1)
    assert np.allclose(out["W3"], 2.0 + 0.01 - 0.01 * 0.1 * 2.0)


def test_training_lowers_loss():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((64, 16))
    y = (np.abs(x[:, :12]) > 0.5).astype(int) @ (1 << np.arange(12))   # a learnable bucket rule
    p = small_params(9, 0.1)
    st = {}
    l0 = mlp.loss_and_grads(p, x, y)[0]
    for t in range(1, 31):
        _, g = mlp.loss_and_grads(p, x, y)
        p = mlp.adamw_step(p, g, st, t, lr=3e-3)
    assert mlp.loss_and_grads(p, x, y)[0] < 0.5 * l0


def test_topr_brute_force_with_ties():
    """Top-r buckets against a brute-force ordering by (score descending, bucket ascending), on
    logits with planted ties (equal scores, +0 and -0, a tie straddling the r-th place)."""
    rng = np.random.default_rng(11)
    L = rng.standard_normal((6, 4096)).astype(np.float32)
    L[0, [5, 900, 4095]] = 9.0                      # a three-way tie for first place
    L[1, :] = 0.0                                   # all tied: the lowest buckets win
    L[2, [3, 7]] = [0.0, -0.0]
    L[2, :] = np.minimum(L[2, :], 0.0)
    L[3, [10, 20, 30, 40]] = 5.0                    # tie across the r-th place (r = 3)
    L[4, ::2] = L[4, 1::2]                          # every even bucket ties with its right neighbour
    for r in (1, 3, 8):
        got = mlp.topr_of_logits(L, r)
        for b in range(L.shape[0]):
            want = sorted(range(4096), key=lambda i: (-float(L[b, i]), i))[:r]
            assert got[b].tolist() == want
    assert mlp.topr_of_logits(L, 3)[3].tolist() == [10, 20, 30]
    assert mlp.topr_of_logits(L, 3)[1].tolist() == [0, 1, 2]
    p = small_params(4)
    x = rng.standard_normal((3, 16))
    assert np.array_equal(mlp.topr_buckets(p, x, 4), mlp.topr_of_logits(mlp.forward(p, x)[0], 4))
