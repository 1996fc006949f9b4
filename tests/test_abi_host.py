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


STRUCTS = {
    "paris_build_opts": ("BuildOpts", ["leaf_capacity", "bf16_shadow", "reserved"]),
    "paris_query_opts": ("QueryOpts", ["mode", "query_tile", "chunk", "precision", "seed", "reserved"]),
    "paris_query_stats": ("QueryStats", ["candidates", "refined", "contenders", "leaf_rows", "dense_queries",
                                         "ms_prep", "ms_descent", "ms_lbscan", "ms_refine", "ms_select", "ms_dense",
                                         "query_tile", "rescreens", "lb_lookups"]),
    "paris_knn_plan_stats": ("PlanStats", ["graph_kernels", "replays", "eager_runs", "captured", "query_tile"]),
    "paris_index_view": ("IndexView", ["n", "len", "w", "card", "leaf_capacity", "series", "keys_sorted",
                                       "rows_sorted"]),
}


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's sizes and field offsets (compiled with gcc)."""
    import shutil
    import subprocess
    from paper_2009_00166_gb300 import binding
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "paris.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, what, val = line.split()
        got[(cname, what)] = int(val)
    for cname, (pyname, fields) in STRUCTS.items():
        cls = getattr(binding, pyname)
        assert C.sizeof(cls) == got[(cname, "size")], cname
        for f in fields:
            assert getattr(cls, f).offset == got[(cname, f)], (cname, f)


def test_every_declared_function_has_a_signature(L):
    """The binding declares argument and result types for every entry point of the header."""
    for n in declared_functions():
        assert getattr(L, n).argtypes is not None, n
