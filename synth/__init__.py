"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only *generates inputs*; it holds none of the indexing or search arithmetic.
Both sides read the very same bytes: the tests copy these arrays to the GPU and hand the
same arrays to the oracle.

Workload recipe (ParIS+ Sec. 4, "Datasets"): a random-walk series starts with a draw from
N(0,1) and each later point adds a fresh N(0,1) step to the previous value. Series are
z-normalised (mean 0, population standard deviation 1, Sec. 2.1) in FP64 and stored as fp32.

Reproducibility: rows are produced in chunks of ``CHUNK`` rows; chunk ``c`` of a dataset with
seed ``s`` draws its normals from ``numpy.random.default_rng([s, c])`` in row-major order, so
every row is fixed by (seed, row index, length) alone, independent of the dataset size and of
how many worker threads fill it.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 65536


def _znorm_rows_inplace(x: np.ndarray) -> None:
    """z-normalise each row of a float64 array in place (population std)."""
    x -= x.mean(axis=1, keepdims=True)
    sd = np.sqrt((x * x).mean(axis=1, keepdims=True))
    x /= sd


def _walk_chunk(seed: int, chunk: int, rows: int, length: int) -> np.ndarray:
    x = np.random.default_rng([seed, chunk]).standard_normal((rows, length))
    np.cumsum(x, axis=1, out=x)
    _znorm_rows_inplace(x)
    return x


def random_walk(n_rows: int, length: int, seed: int, out: np.ndarray | None = None,
                threads: int | None = None, start_row: int = 0) -> np.ndarray:
    """Rows [0, n_rows) of the z-normalised random-walk dataset ``seed``; float32 [n_rows][length].

    ``out`` may be any writable float32 C-contiguous array of that shape (e.g. a numpy view of a
    pinned host tensor); chunks are filled by a thread pool (numpy releases the GIL). With
    ``start_row`` only rows [start_row, n_rows) of ``out`` are written (the rows before it are
    left as they are, e.g. already copied from a smaller collection of the same seed).
    """
    if out is None:
        out = np.empty((n_rows, length), dtype=np.float32)
    assert out.shape == (n_rows, length) and out.dtype == np.float32
    n_chunks = (n_rows + CHUNK - 1) // CHUNK
    first = start_row // CHUNK

    def fill(c: int) -> None:
        r0 = c * CHUNK
        r1 = min(n_rows, r0 + CHUNK)
        lo = max(r0, start_row)
        out[lo:r1] = _walk_chunk(seed, c, r1 - r0, length)[lo - r0:]

    threads = threads or min(32, os.cpu_count() or 1)
    if n_chunks - first <= 1 or threads == 1:
        for c in range(first, n_chunks):
            fill(c)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(fill, range(first, n_chunks)))
    return out


def walk_rows(rows: np.ndarray, length: int, seed: int) -> np.ndarray:
    """The given rows of dataset ``seed`` (regenerating only the chunks they live in)."""
    rows = np.asarray(rows, dtype=np.int64)
    out = np.empty((rows.size, length), dtype=np.float32)
    for c in np.unique(rows // CHUNK):
        sel = np.nonzero(rows // CHUNK == c)[0]
        need = int(rows[sel].max() - c * CHUNK + 1)
        blk = _walk_chunk(seed, int(c), need, length).astype(np.float32)
        out[sel] = blk[rows[sel] - c * CHUNK]
    return out


def noisy_queries(base_rows: np.ndarray, sigma, noise_seed) -> np.ndarray:
    """Queries formed from dataset rows by adding N(0, sigma^2) noise and re-z-normalising.

    ``sigma`` is a scalar or one value per query; the noise comes from
    ``default_rng(noise_seed)`` in row-major order.
    """
    base = np.asarray(base_rows, dtype=np.float64)
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64).reshape(-1, 1), (base.shape[0], 1))
    x = base + sig * np.random.default_rng(noise_seed).standard_normal(base.shape)
    _znorm_rows_inplace(x)
    return x.astype(np.float32)


# ----------------------------------------------------------------------------- named workloads
# Seeds and shapes of the synthetic workloads (random-walk, length-256 default).

def small_workload(n_rows: int = 100_000, length: int = 256, n_queries: int = 20):
    """100K x 256 dataset (seed 1) and 20 independent random-walk queries (seed 2)."""
    data = random_walk(n_rows, length, seed=1)
    queries = random_walk(n_queries, length, seed=2)
    return data, queries


def sigma_query_sources(n_rows: int, n_queries: int, seed: int = 3) -> np.ndarray:
    """Distinct dataset rows that noisy queries are made from."""
    return np.sort(np.random.default_rng(seed).choice(n_rows, n_queries, replace=False))


def sigma_queries(data_or_none, n_rows: int, length: int, n_per_sigma: int,
                  sigmas=(0.01, 0.1, 1.0), data_seed: int = 1):
    """``n_per_sigma`` noisy queries per sigma level: sources from ``default_rng(3)``, the
    noise of level k from ``default_rng([4, k])``. Returns (queries [S*n][len], sigma per query,
    source row per query)."""
    src = sigma_query_sources(n_rows, n_per_sigma)
    if data_or_none is not None:
        base = np.asarray(data_or_none[src])
    else:
        base = walk_rows(src, length, data_seed)
    qs, sg, sr = [], [], []
    for k, s in enumerate(sigmas):
        qs.append(noisy_queries(base, s, [4, k]))
        sg.append(np.full(len(src), s))
        sr.append(src)
    return np.concatenate(qs), np.concatenate(sg), np.concatenate(sr)


def mixed_sigma_queries(data_or_none, n_rows: int, length: int, n_queries: int,
                        lo: float = 0.01, hi: float = 2.0, seed: int = 5, data_seed: int = 1):
    """Queries with sigma ~ U[lo, hi] (``default_rng([seed, 0])``), sources
    ``default_rng([seed, 1])``, noise ``default_rng([seed, 2])``."""
    sig = np.random.default_rng([seed, 0]).uniform(lo, hi, n_queries)
    src = np.random.default_rng([seed, 1]).choice(n_rows, n_queries, replace=n_queries > n_rows)
    if data_or_none is not None:
        base = np.asarray(data_or_none[src])
    else:
        base = walk_rows(src, length, data_seed)
    return noisy_queries(base, sig, [seed, 2]), sig, src
