"""Element-wise error bounds for the proposal network's GPU forward pass and gradients.

The GPU evaluates the network of ``oracle.mlp`` with BF16 GEMM operands and FP32 everything else:
* every GEMM rounds both operands to BF16 when it stages them (unit roundoff ub = 2^-8; weights
  given as BF16 values are unchanged) and accumulates in FP32 on the tensor cores; the
  accumulation is bounded as if each of the K additions truncated (ua = 2^-23 per addition);
* bias adds, GELU and its derivative, softmax and the column sums run in FP32 (u = 2^-24) with
  erff/expf within 2 ulp and logf within 1 ulp (the CUDA math library's documented bounds);
* the FP64 PAA inputs are rounded to FP32 before the first GEMM.

Given the exact FP64 values of every intermediate (from ``oracle.mlp``), each function below
returns, element by element, an upper bound on |GPU value - exact value| that follows the data
flow of the GPU code: the error carried in by the operands, the rounding of the operands, and
the rounding of the operation. |gelu'| <= 1.13 and |gelu''| <= 0.8 carry an argument's error
through GELU and its derivative; a softmax input perturbed by at most E moves each probability
by a factor within [e^-2E, e^2E].
"""
from __future__ import annotations

import math

import numpy as np

from oracle import mlp

U = 2.0 ** -24
UB = 2.0 ** -8
UA = 2.0 ** -23
ULP2 = 2.0 ** -22          # 2 ulp of a value below 1 in magnitude, relative


def gamma(k, unit=UA):
    return k * unit / (1.0 - k * unit)


def rounded_operand(a, e, exact_bf16=False):
    """Error of a GEMM operand after BF16 staging, given the exact value a and carried error e."""
    if exact_bf16:
        return e
    return e + UB * (np.abs(a) + e)


def gemm_err(A, eA, B, eB, K, a_bf16=False, b_bf16=False):
    """Bound on |fl(A~ B~) - A B| for A [M][K], B [K][N] with carried errors eA, eB."""
    ea = rounded_operand(A, np.broadcast_to(np.asarray(eA, np.float64), A.shape), a_bf16)
    eb = rounded_operand(B, np.broadcast_to(np.asarray(eB, np.float64), B.shape), b_bf16)
    absA, absB = np.abs(A), np.abs(B)
    return ea @ (absB + eb) + absA @ eb + gamma(K) * ((absA + ea) @ (absB + eb))


def gelu_eval(z, h):
    """FP32 evaluation error of 0.5 z (1 + erff(z / sqrt 2)) at argument z (value h)."""
    az = np.abs(z)
    return 0.5 * az * (0.8 * U * az + ULP2 + 4 * U) + 2 * U * np.abs(h) + 1e-45


def gelu_grad_eval(z):
    az = np.abs(z)
    phi = np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    g = np.abs(mlp.gelu_grad(z))
    return 0.5 * (ULP2 + 0.8 * U * az + 2 * U) + az * phi * (U * az * az + ULP2 + 6 * U) + 2 * U * g


def forward_bounds(params, x):
    """Exact logits and intermediates of oracle.mlp.forward and the bound on each GPU value."""
    logits, (x, z1, h1, z2, h2) = mlp.forward(params, x)
    W1, W2, W3 = params["W1"].T, params["W2"].T, params["W3"].T
    ex = (U + UB + U * UB) * np.abs(x)                       # FP64 -> FP32 -> BF16 input
    e_z1 = gemm_err(x, ex, W1, 0.0, W1.shape[0], a_bf16=True, b_bf16=True) + U * (np.abs(z1) + 1e-30)
    e_h1 = 1.13 * e_z1 + gelu_eval(z1, h1)
    e_z2 = gemm_err(h1, e_h1, W2, 0.0, W2.shape[0], b_bf16=True) + U * np.abs(z2)
    e_h2 = 1.13 * e_z2 + gelu_eval(z2, h2)
    e_l = gemm_err(h2, e_h2, W3, 0.0, W3.shape[0], b_bf16=True) + U * np.abs(logits)
    cache = dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, logits=logits, e_z1=e_z1, e_h1=e_h1, e_z2=e_z2, e_h2=e_h2,
                 e_l=e_l)
    return logits, e_l, cache


def gradient_bounds(params, x, labels):
    """Exact loss/gradients of oracle.mlp.loss_and_grads and a bound on each GPU gradient."""
    _, e_l, c = forward_bounds(params, x)
    loss, grads = mlp.loss_and_grads(params, x, labels)
    logits = c["logits"]
    B, N = logits.shape
    m = logits.max(axis=1, keepdims=True)
    p = np.exp(logits - m)
    p /= p.sum(axis=1, keepdims=True)
    y = np.zeros_like(p)
    y[np.arange(B), labels] = 1.0
    D3 = (p - y) / B
    # logits perturbed by d (|d_j| <= e_j): p_i'/p_i = e^(d_i) / sum_j p_j e^(d_j) lies within
    # e^(+-(e_i + e^E S)), E = max_j e_j, S = sum_j p_j e_j (Jensen below, e^x <= 1 + x e^E above)
    E = e_l.max(axis=1, keepdims=True)
    S = (p * e_l).sum(axis=1, keepdims=True)
    span = (logits - m).__abs__().max(axis=1, keepdims=True) + 2 * E
    rel_eval = ULP2 + U * span + 40 * U                      # expf, argument, sum depth 32, 1/s, products
    rel = np.expm1(e_l + np.exp(E) * S)
    e_p = p * (rel + rel_eval * (1 + rel))
    e_D3 = (e_p + U * np.abs(p - y)) / B * (1 + 4 * U) + 2 * U * np.abs(D3)
    W2, W3 = params["W2"], params["W3"]
    g = {}
    # dW3 = D3^T h2 and db3 = column sums of D3
    g["W3"] = gemm_err(D3.T, e_D3.T, c["h2"], c["e_h2"], B)
    g["b3"] = e_D3.sum(axis=0) + gamma(B, U) * np.abs(D3).sum(axis=0)
    # dh2 = D3 W3, dz2 = dh2 * gelu'(z2)
    dh2 = D3 @ W3
    e_dh2 = gemm_err(D3, e_D3, W3, 0.0, N, b_bf16=True)
    gp2 = mlp.gelu_grad(c["z2"])
    e_gp2 = 0.8 * c["e_z2"] + gelu_grad_eval(c["z2"])
    dz2 = dh2 * gp2
    e_dz2 = e_dh2 * (np.abs(gp2) + e_gp2) + np.abs(dh2) * e_gp2 + U * (np.abs(dz2) + e_dh2 * e_gp2)
    g["W2"] = gemm_err(dz2.T, e_dz2.T, c["h1"], c["e_h1"], B)
    g["b2"] = e_dz2.sum(axis=0) + gamma(B, U) * np.abs(dz2).sum(axis=0)
    dh1 = dz2 @ W2
    e_dh1 = gemm_err(dz2, e_dz2, W2, 0.0, W2.shape[0], b_bf16=True)
    gp1 = mlp.gelu_grad(c["z1"])
    e_gp1 = 0.8 * c["e_z1"] + gelu_grad_eval(c["z1"])
    dz1 = dh1 * gp1
    e_dz1 = e_dh1 * (np.abs(gp1) + e_gp1) + np.abs(dh1) * e_gp1 + U * (np.abs(dz1) + e_dh1 * e_gp1)
    ex = U * np.abs(c["x"])                                  # FP32 input; the GEMM rounds it to BF16
    g["W1"] = gemm_err(dz1.T, e_dz1.T, c["x"], ex, B)
    g["b1"] = e_dz1.sum(axis=0) + gamma(B, U) * np.abs(dz1).sum(axis=0)
    return loss, grads, g
