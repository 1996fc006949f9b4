"""Compiles the CUDA/C++ sources of the library into ``libparis.so`` next to this file.

Every translation unit is compiled in parallel for sm_103a only (``-gencode
arch=compute_103a,code=sm_103a``), then linked with the static CUDA runtime.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_objs")
LIB = os.path.join(HERE, "libparis.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, jobs: int | None = None) -> str:
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    cu, cpp = _sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "paris.h"))
    cmds = []
    objs = []
    for f in cu:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OBJ, f + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            cmds.append([nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", *ARCH,
                         "-Xcompiler", "-fPIC", "-Xptxas", "-O3", "--expt-relaxed-constexpr"])
    for f in cpp:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OBJ, f + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            cmds.append([nvcc, "-c", src, "-o", obj, "-O2", "-std=c++17", "-Xcompiler",
                         "-fPIC,-ffp-contract=off"])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.returncode

    with ThreadPoolExecutor(jobs or max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        rcs = list(ex.map(run, cmds))
    if any(rcs):
        raise RuntimeError("compiling the CUDA library failed (see messages above)")
    if cmds or not os.path.exists(LIB):
        link = [nvcc, "-shared", *ARCH, "-o", LIB, *objs, "-cudart", "static"]
        if run(link):
            raise RuntimeError("linking libparis.so failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
