"""Host-side checks of the C ABI (no GPU): the library builds, loads, exports every entry point
declared in include/paris.h, computes the iSAX breakpoints bit-for-bit like the oracle's
independent N(0,1) quantile, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "paris.h")


@pytest.fixture(scope="module")
def L():
    from paper_2009_00166_gb300 import _build, binding
    if not os.path.exists(binding.LIB_PATH):
        _build.build()
    return binding.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(paris_[a-z0-9_]+)\s*\(", text)) - {"paris_alloc_fn", "paris_free_fn"})


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("card", [2, 4, 16, 256])
def test_breakpoints_bitwise_equal_oracle(L, card):
    from oracle import isax
    from paper_2009_00166_gb300 import paris_breakpoints
    got = paris_breakpoints(card)
    want = isax.breakpoints(card)
    assert got.tobytes() == want.tobytes()


def test_argument_errors_without_gpu(L):
    from paper_2009_00166_gb300 import binding
    out = C.c_void_p()
    x = np.zeros((4, 10), np.float32)
    # len not a multiple of w, bad card, bad w: rejected before any device call
    for (ln, w, card) in [(10, 3, 256), (10, 5, 3), (10, 0, 256), (10, 5, 512)]:
        st = L.paris_build(x.ctypes.data, 4, ln, w, card, None, C.byref(out))
        assert st == 1 and out.value is None
        assert binding.paris_last_error()
    assert L.paris_breakpoints(100, None) == 1
    assert "power of two" in binding.paris_last_error()
    assert L.paris_exact_knn(None, None, 1, 1, None, None, None) == 1
