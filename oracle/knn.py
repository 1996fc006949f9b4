"""Exact k-nearest-neighbour search by brute force (test infrastructure only).

Definition followed (ParIS+ Sec. 2.1 "Similarity Search"): the answer to a query S_q is the
series of the collection with the smallest Euclidean distance to it; ParIS+ reaches exactly
that answer (Sec. 3.3: every series that cannot be pruned is compared on its raw values).
Readings: ED = sqrt(sum_j (x_j - q_j)^2) (the paper's wording of ED is garbled); k-NN returns
the k rows with the smallest ED; equal distances are ordered by the lower row number.

"Smallest" is decided on the EXACT real value of sum_j (x_j - q_j)^2 of the fp32 inputs:
every fp32 number is an integer multiple of 2^-149, so the squared distance scaled by 2^298 is
an integer and Python computes it exactly. An FP64 pass screens the collection first; its
error is bounded by gamma_{n+2} (relative, every term is non-negative), and every row that the
bound cannot separate from the k-th best is re-ranked exactly.
"""
from __future__ import annotations

import math

import numpy as np

U64 = 2.0 ** -53
SCALE = 2.0 ** 149          # fp32 value * SCALE is an exact integer


def gamma(m: int, u: float = U64) -> float:
    return m * u / (1.0 - m * u)


def exact_sq_int(x_row: np.ndarray, q: np.ndarray) -> int:
    """sum_j (x_j - q_j)^2 * 2^298 as an exact Python int."""
    xs = (np.asarray(x_row, dtype=np.float32).astype(np.float64) * SCALE).tolist()
    qs = (np.asarray(q, dtype=np.float32).astype(np.float64) * SCALE).tolist()
    acc = 0
    for a, b in zip(xs, qs):
        d = int(a) - int(b)
        acc += d * d
    return acc


def exact_sq_float(x_row: np.ndarray, q: np.ndarray) -> float:
    """The exact squared distance rounded to FP64."""
    return math.ldexp(float(exact_sq_int(x_row, q)), -298)


def _rerank(X, q, rows, k):
    ex = [(exact_sq_int(X[r], q), int(r)) for r in rows]
    ex.sort()
    top = ex[:k]
    idx = np.array([r for _, r in top], dtype=np.int64)
    dist = np.array([math.sqrt(math.ldexp(float(e), -298)) for e, _ in top], dtype=np.float64)
    return idx, dist


def knn_one(X: np.ndarray, q: np.ndarray, k: int):
    """Exact k-NN of one query by direct FP64 differences + exact re-rank of near ties.

    Returns (rows [k] int64, distances [k] float64), ordered by (exact distance, row).
    """
    n = X.shape[1]
    d2 = ((X.astype(np.float64) - q.astype(np.float64)[None, :]) ** 2).sum(axis=1)
    g = gamma(n + 2)
    kth = np.partition(d2, k - 1)[k - 1]
    window = kth * (1.0 + g) / (1.0 - g) * (1.0 + 4 * U64)
    rows = np.nonzero(d2 <= window)[0]
    return _rerank(X, q, rows, k)


def knn(X: np.ndarray, Q: np.ndarray, k: int):
    """Exact k-NN for every query: (idx [nq][k], dist [nq][k])."""
    Q = np.atleast_2d(Q)
    out_i = np.empty((Q.shape[0], k), dtype=np.int64)
    out_d = np.empty((Q.shape[0], k), dtype=np.float64)
    for t in range(Q.shape[0]):
        out_i[t], out_d[t] = knn_one(X, Q[t], k)
    return out_i, out_d


def knn_chunked(row_source, n_rows: int, Q: np.ndarray, k: int, chunk: int = 1 << 18):
    """Exact k-NN over a collection too large for one FP64 copy.

    ``row_source(r0, r1)`` returns rows [r0, r1) as float32. Screening uses the GEMM form
    |x|^2 + |q|^2 - 2 x.q in FP64 whose error is at most 4(n+2)u(|x|^2 + |q|^2) per row; rows the
    bound cannot separate from the k-th best are re-ranked exactly.
    """
    Q = np.atleast_2d(Q).astype(np.float32)
    nq, n = Q.shape
    Qd = Q.astype(np.float64)
    qn = (Qd * Qd).sum(axis=1)
    # keep, per query, the rows whose screened distance may still reach the top k
    keep_rows = [np.empty(0, np.int64) for _ in range(nq)]
    keep_d = [np.empty(0, np.float64) for _ in range(nq)]
    keep_err = [np.empty(0, np.float64) for _ in range(nq)]
    c_err = 4.0 * (n + 2) * U64
    for r0 in range(0, n_rows, chunk):
        r1 = min(n_rows, r0 + chunk)
        Xd = np.asarray(row_source(r0, r1), dtype=np.float32).astype(np.float64)
        xn = (Xd * Xd).sum(axis=1)
        d2 = xn[None, :] + qn[:, None] - 2.0 * (Qd @ Xd.T)
        err = c_err * (xn[None, :] + qn[:, None])
        for t in range(nq):
            rows = np.concatenate((keep_rows[t], np.arange(r0, r1)))
            dd = np.concatenate((keep_d[t], d2[t]))
            ee = np.concatenate((keep_err[t], err[t]))
            kk = min(k, dd.size)
            ub = np.partition(dd + ee, kk - 1)[kk - 1]       # k-th smallest upper bound
            sel = np.nonzero(dd - ee <= ub)[0]
            keep_rows[t], keep_d[t], keep_err[t] = rows[sel], dd[sel], ee[sel]
    out_i = np.empty((nq, k), dtype=np.int64)
    out_d = np.empty((nq, k), dtype=np.float64)
    for t in range(nq):
        rows = np.sort(keep_rows[t])
        Xr = np.concatenate([np.asarray(row_source(int(r), int(r) + 1), dtype=np.float32) for r in rows])
        i, d = _rerank(Xr, Q[t], np.arange(rows.size), k)
        out_i[t], out_d[t] = rows[i], d
    return out_i, out_d
