"""Helpers for the GPU parity tests (device selection and cached workloads)."""
import functools
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2009_00166_gb300 import _build, binding
    if not os.path.exists(binding.LIB_PATH):
        _build.build()
    return torch.device("cuda:0")


@functools.lru_cache(maxsize=None)
def small_dataset(n=100_000, length=256):
    import synth
    return synth.random_walk(n, length, seed=1)


def rw(n, length, seed):
    import synth
    return synth.random_walk(n, length, seed=seed)
