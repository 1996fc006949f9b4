"""ctypes marshalling for ``libparis.so`` (declarations in ``include/paris.h``)."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparis.so")

PARIS_MODE_PLAIN = 0
PARIS_MODE_BATCHED = 1
PARIS_REFINE_FP32 = 0
PARIS_REFINE_MIXED = 1
PARIS_SEED_DESCENT = 0
PARIS_SEED_LEARNED = 1
PARIS_SEED_ADAPTIVE = 2
SEED_MODEL_PARAMS = 1122816
SEED_MODEL_SHAPES = [("W1", (256, 16)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (4096, 256)),
                     ("b3", (4096,))]

_STATUS = {0: "PARIS_OK", 1: "PARIS_EINVAL", 2: "PARIS_ENOMEM", 3: "PARIS_ECUDA", 4: "PARIS_ETIMEOUT",
           5: "PARIS_EINTERNAL"}


class ParisError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class BuildOpts(C.Structure):
    _fields_ = [("leaf_capacity", C.c_int32), ("bf16_shadow", C.c_int32), ("series_on_host", C.c_int32),
                ("reserved", C.c_int32 * 5)]


class QueryOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("query_tile", C.c_int32), ("chunk", C.c_int32),
                ("precision", C.c_int32), ("seed", C.c_int32), ("no_leaf_pruning", C.c_int32),
                ("private_bsf", C.c_int32), ("reserved", C.c_int32 * 1)]


class QueryStats(C.Structure):
    _fields_ = [("candidates", C.c_int64), ("refined", C.c_int64), ("contenders", C.c_int64),
                ("leaf_rows", C.c_int64), ("dense_queries", C.c_int64), ("ms_prep", C.c_double),
                ("ms_descent", C.c_double), ("ms_lbscan", C.c_double), ("ms_refine", C.c_double),
                ("ms_select", C.c_double), ("ms_dense", C.c_double), ("query_tile", C.c_int32),
                ("rescreens", C.c_int32), ("lb_lookups", C.c_int64), ("pages_examined", C.c_int64),
                ("pages_kept", C.c_int64), ("bsf_updates", C.c_int64), ("list_rows", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PlanStats(C.Structure):
    _fields_ = [("graph_kernels", C.c_int64), ("replays", C.c_int64), ("eager_runs", C.c_int64),
                ("captured", C.c_int32), ("query_tile", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class IndexView(C.Structure):
    _fields_ = [("n", C.c_int64), ("len", C.c_int32), ("w", C.c_int32), ("card", C.c_int32),
                ("leaf_capacity", C.c_int32), ("series", C.c_void_p), ("keys_sorted", C.c_void_p),
                ("rows_sorted", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None


def lib():
    """The loaded ``libparis.so``; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libparis.so is missing ({LIB_PATH}); run paper_2009_00166_gb300._build.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, F32, VP = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_void_p
        sig = {
            "paris_build": ([P, I64, I32, I32, I32, VP, C.POINTER(VP)], I32),
            "paris_build_ex": ([P, I64, I32, I32, I32, C.POINTER(BuildOpts), VP, C.POINTER(VP)], I32),
            "paris_free": ([VP], None),
            "paris_exact_knn": ([VP, P, I64, I32, P, P, VP], I32),
            "paris_exact_knn_ex": ([VP, P, I64, I32, P, P, C.POINTER(QueryOpts), C.POINTER(QueryStats), VP], I32),
            "paris_knn_plan_create": ([VP, I64, I32, C.POINTER(QueryOpts), C.POINTER(VP)], I32),
            "paris_knn_plan_run": ([VP, P, P, P, VP], I32),
            "paris_knn_plan_info": ([VP, C.POINTER(PlanStats)], I32),
            "paris_knn_plan_free": ([VP], None),
            "paris_knn_plan_create_multi": ([C.POINTER(VP), I32, C.POINTER(C.c_int64), I32, C.POINTER(QueryOpts),
                                             C.POINTER(VP)], I32),
            "paris_knn_plan_run_multi": ([VP, C.POINTER(VP), C.POINTER(VP), C.POINTER(VP), VP], I32),
            "paris_exact_knn_multi": ([C.POINTER(VP), I32, C.POINTER(VP), C.POINTER(C.c_int64), I32, C.POINTER(VP),
                                       C.POINTER(VP), C.POINTER(QueryOpts), C.POINTER(QueryStats), VP], I32),
            "paris_last_error": ([], C.c_char_p),
            "paris_kernel_launches": ([], C.c_uint64),
            "paris_set_allocator": ([ALLOC_FN, FREE_FN, VP], I32),
            "paris_trim_memory": ([], I32),
            "paris_set_wait_limit": ([C.c_uint64], I32),
            "paris_index_describe": ([VP, C.POINTER(IndexView)], I32),
            "paris_breakpoints": ([I32, P], I32),
            "paris_export_sax": ([VP, P, VP], I32),
            "paris_encode": ([P, I64, I32, I32, I32, P, P, P, VP], I32),
            "paris_export_order": ([VP, P, P, VP], I32),
            "paris_build_adaptive_leaves": ([VP, VP], I32),
            "paris_adaptive_leaves_info": ([VP, C.POINTER(I64), C.POINTER(I64), C.POINTER(I32)], I32),
            "paris_adaptive_leaves_export": ([VP, P, P, VP], I32),
            "paris_approx_search": ([VP, P, I64, I32, P, P, VP], I32),
            "paris_lb_scan": ([VP, P, F32, P, P, I64, C.POINTER(I64), VP], I32),
            "paris_lb_scan_noalloc": ([VP, P, I64, P, P, P, I64, P, VP], I32),
            "paris_leaf_scan": ([VP, P, F32, P, C.POINTER(I64), VP], I32),
            "paris_approx_search_ex": ([VP, P, I64, I32, I32, P, P, VP], I32),
            "paris_seed_model_create": ([C.c_uint64, VP, C.POINTER(VP)], I32),
            "paris_seed_model_free": ([VP], None),
            "paris_seed_model_set_weights": ([VP, P, VP], I32),
            "paris_seed_model_get_weights": ([VP, P, VP], I32),
            "paris_seed_model_forward": ([VP, P, I64, P, VP], I32),
            "paris_seed_model_gradients": ([VP, P, P, I32, P, C.POINTER(F32), VP], I32),
            "paris_seed_model_topr": ([VP, P, I64, I32, P, VP], I32),
            "paris_seed_model_train": ([VP, P, P, I64, I32, I32, F32, F32, C.c_uint64, P, VP], I32),
            "paris_attach_seed_model": ([VP, VP, I32], I32),
            "paris_row_buckets": ([VP, P, I64, P, VP], I32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def paris_kernel_launches() -> int:
    return int(lib().paris_kernel_launches())


def paris_trim_memory():
    _check(lib().paris_trim_memory())


def paris_set_wait_limit(ns: int = 0):
    """Bound of the device-side waits in ns (0: the default 4 s)."""
    _check(lib().paris_set_wait_limit(int(ns)))


def paris_last_error() -> str:
    return lib().paris_last_error().decode()


def _check(status: int):
    if status != 0:
        raise ParisError(status, paris_last_error())


def _ptr(t) -> int | None:
    """Address of a torch tensor (device or host) or numpy array; None for None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        assert t.is_contiguous(), "tensors passed to the library must be contiguous"
        return t.data_ptr()
    import numpy as np
    a = t
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _stream(stream) -> int | None:
    import torch
    if stream is None:
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    return getattr(stream, "cuda_stream", stream)


@dataclass
class ParisIndex:
    """Handle returned by paris_build; keeps the borrowed series tensor alive."""
    handle: int
    n: int
    len: int
    w: int
    card: int
    series: object = None

    def free(self):
        if self.handle:
            lib().paris_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def paris_build_ex(series, w: int = 16, card: int = 256, leaf_capacity: int = 0, bf16_shadow: bool = False,
                   stream=None, series_on_host: bool = False) -> ParisIndex:
    """paris_build_ex: series is a contiguous [n][len] float32 tensor (device: borrowed; host: copied,
    or borrowed and read in place with series_on_host)."""
    n, length = int(series.shape[0]), int(series.shape[1])
    opts = BuildOpts(leaf_capacity=leaf_capacity, bf16_shadow=1 if bf16_shadow else 0,
                     series_on_host=1 if series_on_host else 0)
    out = C.c_void_p()
    _check(lib().paris_build_ex(_ptr(series), n, length, w, card, C.byref(opts), _stream(stream), C.byref(out)))
    return ParisIndex(out.value, n, length, w, card, series)


def paris_build(series, w: int = 16, card: int = 256, stream=None) -> ParisIndex:
    return paris_build_ex(series, w, card, 0, False, stream)


def paris_free(index: ParisIndex):
    index.free()


def paris_exact_knn_ex(index: ParisIndex, queries, k: int, out_idx=None, out_dist=None, mode: int = PARIS_MODE_PLAIN,
                       query_tile: int = 0, chunk: int = 0, precision: int = PARIS_REFINE_FP32,
                       seed: int = PARIS_SEED_DESCENT, want_stats: bool = False, stream=None,
                       leaf_pruning: bool = True, private_bsf: bool = False):
    """paris_exact_knn_ex: returns (idx [nq][k] int64, dist [nq][k] float32[, stats dict]).

    Outputs are allocated like the queries (same device) when not given.
    """
    import torch
    nq = int(queries.shape[0])
    dev = queries.device if hasattr(queries, "device") else torch.device("cpu")
    if out_idx is None:
        out_idx = torch.empty((nq, k), dtype=torch.int64, device=dev)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
    opts = QueryOpts(mode=mode, query_tile=query_tile, chunk=chunk, precision=precision, seed=seed,
                     no_leaf_pruning=0 if leaf_pruning else 1, private_bsf=1 if private_bsf else 0)
    stats = QueryStats()
    _check(lib().paris_exact_knn_ex(index.handle, _ptr(queries), nq, k, _ptr(out_idx), _ptr(out_dist),
                                    C.byref(opts), C.byref(stats) if want_stats else None, _stream(stream)))
    if want_stats:
        return out_idx, out_dist, stats.as_dict()
    return out_idx, out_dist


def paris_exact_knn_multi(indexes, queries, k: int, mode: int = PARIS_MODE_BATCHED, query_tile: int = 0,
                          chunk: int = 0, precision: int = PARIS_REFINE_FP32, seed: int = PARIS_SEED_DESCENT,
                          want_stats: bool = False, stream=None, leaf_pruning: bool = True):
    """paris_exact_knn_multi: one (idx [nq][k], dist [nq][k]) pair per collection[, stats dicts]."""
    import torch
    m = len(indexes)
    if len(queries) != m:
        raise ValueError("one query block per index")
    outs = []
    for q in queries:
        nq = int(q.shape[0])
        dev = q.device if hasattr(q, "device") else torch.device("cpu")
        outs.append((torch.empty((nq, k), dtype=torch.int64, device=dev),
                     torch.empty((nq, k), dtype=torch.float32, device=dev)))
    VPA = C.c_void_p * m
    hs = VPA(*[ix.handle for ix in indexes])
    qp = VPA(*[_ptr(q) for q in queries])
    nqs = (C.c_int64 * m)(*[int(q.shape[0]) for q in queries])
    oi = VPA(*[_ptr(o[0]) for o in outs])
    od = VPA(*[_ptr(o[1]) for o in outs])
    opts = QueryOpts(mode=mode, query_tile=query_tile, chunk=chunk, precision=precision, seed=seed,
                     no_leaf_pruning=0 if leaf_pruning else 1)
    stats = (QueryStats * m)()
    _check(lib().paris_exact_knn_multi(hs, m, qp, nqs, k, oi, od, C.byref(opts), stats if want_stats else None,
                                       _stream(stream)))
    if want_stats:
        return outs, [st.as_dict() for st in stats]
    return outs


class KnnPlan:
    """paris_knn_plan_*: a batch of exactly ``nq`` queries recorded once as a CUDA graph."""

    def __init__(self, index: ParisIndex, nq: int, k: int, mode: int = PARIS_MODE_BATCHED, query_tile: int = 0,
                 chunk: int = 0, precision: int = PARIS_REFINE_FP32, leaf_pruning: bool = True):
        self.index, self.nq, self.k = index, int(nq), int(k)
        opts = QueryOpts(mode=mode, query_tile=query_tile, chunk=chunk, precision=precision,
                         no_leaf_pruning=0 if leaf_pruning else 1)
        h = C.c_void_p()
        _check(lib().paris_knn_plan_create(index.handle, self.nq, self.k, C.byref(opts), C.byref(h)))
        self.handle = h

    def run(self, queries, out_idx=None, out_dist=None, stream=None):
        import torch
        dev = queries.device if hasattr(queries, "device") else torch.device("cpu")
        if out_idx is None:
            out_idx = torch.empty((self.nq, self.k), dtype=torch.int64, device=dev)
        if out_dist is None:
            out_dist = torch.empty((self.nq, self.k), dtype=torch.float32, device=dev)
        _check(lib().paris_knn_plan_run(self.handle, _ptr(queries), _ptr(out_idx), _ptr(out_dist), _stream(stream)))
        return out_idx, out_dist

    def info(self) -> dict:
        st = PlanStats()
        _check(lib().paris_knn_plan_info(self.handle, C.byref(st)))
        return st.as_dict()

    def free(self):
        if self.handle:
            lib().paris_knn_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class KnnPlanMulti(KnnPlan):
    """paris_knn_plan_create_multi: batches of nqs[c] queries per collection, one CUDA graph."""

    def __init__(self, indexes, nqs, k: int, query_tile: int = 0, chunk: int = 0,
                 precision: int = PARIS_REFINE_FP32, leaf_pruning: bool = True):
        m = len(indexes)
        self.indexes, self.nqs, self.k = list(indexes), [int(v) for v in nqs], int(k)
        opts = QueryOpts(mode=PARIS_MODE_BATCHED, query_tile=query_tile, chunk=chunk, precision=precision,
                         no_leaf_pruning=0 if leaf_pruning else 1)
        VPA = C.c_void_p * m
        h = C.c_void_p()
        _check(lib().paris_knn_plan_create_multi(VPA(*[ix.handle for ix in indexes]), m,
                                                 (C.c_int64 * m)(*self.nqs), self.k, C.byref(opts), C.byref(h)))
        self.handle = h

    def run(self, queries, stream=None):
        """queries: one [nq_c][len_c] tensor per collection; returns [(idx, dist)] per collection."""
        import torch
        m = len(self.indexes)
        outs = []
        for q, nq in zip(queries, self.nqs):
            dev = q.device if hasattr(q, "device") else torch.device("cpu")
            outs.append((torch.empty((nq, self.k), dtype=torch.int64, device=dev),
                         torch.empty((nq, self.k), dtype=torch.float32, device=dev)))
        VPA = C.c_void_p * m
        _check(lib().paris_knn_plan_run_multi(self.handle, VPA(*[_ptr(q) for q in queries]),
                                              VPA(*[_ptr(o[0]) for o in outs]), VPA(*[_ptr(o[1]) for o in outs]),
                                              _stream(stream)))
        return outs


def paris_exact_knn(index: ParisIndex, queries, k: int, out_idx=None, out_dist=None, stream=None):
    return paris_exact_knn_ex(index, queries, k, out_idx, out_dist, stream=stream)


def paris_index_describe(index: ParisIndex) -> dict:
    v = IndexView()
    _check(lib().paris_index_describe(index.handle, C.byref(v)))
    return {f: getattr(v, f) for f, _ in v._fields_}


def paris_breakpoints(card: int):
    import numpy as np
    out = np.empty(card - 1, dtype=np.float64)
    _check(lib().paris_breakpoints(card, out.ctypes.data))
    return out


def paris_export_sax(index: ParisIndex, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty((index.n, index.w), dtype=torch.uint8, device="cuda")
    _check(lib().paris_export_sax(index.handle, _ptr(out), _stream(stream)))
    return out


def paris_export_order(index: ParisIndex):
    """paris_export_order into host arrays: (keys_sorted uint64 [n], rows_sorted int64 [n])."""
    import numpy as np
    keys = np.empty(index.n, np.uint64)
    rows = np.empty(index.n, np.uint32)
    _check(lib().paris_export_order(index.handle, keys.ctypes.data, rows.ctypes.data, _stream(None)))
    return keys, rows.astype(np.int64)


def paris_build_adaptive_leaves(index: ParisIndex, stream=None):
    _check(lib().paris_build_adaptive_leaves(index.handle, _stream(stream)))


def paris_adaptive_leaves_info(index: ParisIndex) -> dict:
    nn, nl, d = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib().paris_adaptive_leaves_info(index.handle, C.byref(nn), C.byref(nl), C.byref(d)))
    return {"nodes": nn.value, "leaves": nl.value, "depth": d.value}


def paris_adaptive_leaves_export(index: ParisIndex):
    """(rows uint32 [n]: series row per leaf-order position, nodes int64 [n_nodes][5]:
    start, count, split segment or -1, bit-0 child or -1, bits per segment packed 4 bits each)."""
    import numpy as np
    info = paris_adaptive_leaves_info(index)
    rows = np.empty(index.n, np.uint32)
    nodes = np.empty((info["nodes"], 5), np.int64)
    _check(lib().paris_adaptive_leaves_export(index.handle, rows.ctypes.data, nodes.ctypes.data, _stream(None)))
    return rows, nodes


def paris_encode(series, w: int = 16, card: int = 256, want_paa: bool = False, stream=None):
    """paris_encode on a device [n][len] float32 tensor: (sax [n][w] uint8, key64 [n] int64 bits[, paa])."""
    import torch
    n, length = int(series.shape[0]), int(series.shape[1])
    sax = torch.empty((n, w), dtype=torch.uint8, device=series.device)
    key = torch.empty((n,), dtype=torch.int64, device=series.device)
    paa = torch.empty((n, w), dtype=torch.float64, device=series.device) if want_paa else None
    _check(lib().paris_encode(_ptr(series), n, length, w, card, _ptr(sax), _ptr(key), _ptr(paa), _stream(stream)))
    return (sax, key, paa) if want_paa else (sax, key)


def paris_approx_search(index: ParisIndex, queries, k: int = 1, seed_mode: int = PARIS_SEED_DESCENT, stream=None):
    """paris_approx_search(_ex): (leaf [nq][2] int64 sorted-position ranges, seed [nq] float32)."""
    import torch
    nq = int(queries.shape[0])
    leaf = torch.empty((nq, 2), dtype=torch.int64, device=queries.device)
    seed = torch.empty((nq,), dtype=torch.float32, device=queries.device)
    _check(lib().paris_approx_search_ex(index.handle, _ptr(queries), nq, k, seed_mode, _ptr(leaf), _ptr(seed),
                                        _stream(stream)))
    return leaf, seed


def paris_lb_scan(index: ParisIndex, query, threshold_sq: float, capacity: int | None = None, stream=None):
    """paris_lb_scan: (rows uint32-as-int64 [m], lb [m] float32, total count) for one query."""
    import torch
    cap = index.n if capacity is None else capacity
    rows = torch.empty((max(cap, 1),), dtype=torch.int32, device="cuda")
    lbs = torch.empty((max(cap, 1),), dtype=torch.float32, device="cuda")
    cnt = C.c_int64()
    _check(lib().paris_lb_scan(index.handle, _ptr(query), C.c_float(threshold_sq), _ptr(rows), _ptr(lbs), cap,
                               C.byref(cnt), _stream(stream)))
    m = min(cnt.value, cap)
    return rows[:m].to(torch.int64) & 0xFFFFFFFF, lbs[:m], cnt.value


PARIS_PAGE_ROWS = 256


def paris_leaf_scan(index: ParisIndex, query, threshold_sq: float, stream=None):
    """Leaf pruning of one device query: (bits, kept) -- device uint32 page bits of the index
    order (bit p: page p may hold a row that the lower-bound scan keeps) and their count."""
    import torch
    n = paris_index_describe(index)["n"]
    words = ((n + PARIS_PAGE_ROWS - 1) // PARIS_PAGE_ROWS + 31) // 32
    bits = torch.zeros(words, dtype=torch.int32, device=query.device)
    kept = C.c_int64()
    _check(lib().paris_leaf_scan(index.handle, _ptr(query), float(threshold_sq), _ptr(bits), C.byref(kept),
                                 _stream(stream)))
    return bits, kept.value


_alloc_keepalive = []


def paris_set_allocator(alloc_fn, free_fn, ctx=None):
    """Install ctypes-compatible allocation callbacks (or None, None for the default)."""
    if alloc_fn is None:
        _check(lib().paris_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return
    a, f = ALLOC_FN(alloc_fn), FREE_FN(free_fn)
    _alloc_keepalive[:] = [a, f]
    _check(lib().paris_set_allocator(a, f, ctx))


def use_torch_allocator():
    """Route the library's device scratch through PyTorch's caching allocator."""
    import torch

    def _a(nbytes, stream, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _f(ptr, _nbytes, _stream, _ctx):
        torch.cuda.caching_allocator_delete(ptr)

    paris_set_allocator(_a, _f)


class SeedModel:
    """Handle of a learned best-so-far proposal network (paris_seed_model_*)."""

    def __init__(self, init_seed: int = 0, stream=None):
        out = C.c_void_p()
        _check(lib().paris_seed_model_create(init_seed, _stream(stream), C.byref(out)))
        self.handle = out.value

    def free(self):
        if self.handle:
            lib().paris_seed_model_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def set_weights(self, params: dict):
        import numpy as np
        flat = np.concatenate([np.asarray(params[k], np.float32).ravel() for k, _ in SEED_MODEL_SHAPES])
        assert flat.size == SEED_MODEL_PARAMS
        _check(lib().paris_seed_model_set_weights(self.handle, flat.ctypes.data, _stream(None)))

    def get_weights(self) -> dict:
        import numpy as np
        flat = np.empty(SEED_MODEL_PARAMS, np.float32)
        _check(lib().paris_seed_model_get_weights(self.handle, flat.ctypes.data, _stream(None)))
        return _split(flat)

    def forward(self, paa):
        """paris_seed_model_forward on device FP64 PAA [m][16]: device logits [m][4096]."""
        import torch
        m = int(paa.shape[0])
        out = torch.empty((m, 4096), dtype=torch.float32, device=paa.device)
        _check(lib().paris_seed_model_forward(self.handle, _ptr(paa), m, _ptr(out), _stream(None)))
        return out

    def topr(self, paa, r: int):
        """paris_seed_model_topr on device FP64 PAA [m][16]: device int32 buckets [m][r]."""
        import torch
        m = int(paa.shape[0])
        out = torch.empty((m, r), dtype=torch.int32, device=paa.device)
        _check(lib().paris_seed_model_topr(self.handle, _ptr(paa), m, r, _ptr(out), _stream(None)))
        return out

    def gradients(self, paa, labels):
        import torch
        m = int(paa.shape[0])
        g = torch.empty(SEED_MODEL_PARAMS, dtype=torch.float32, device=paa.device)
        loss = C.c_float()
        _check(lib().paris_seed_model_gradients(self.handle, _ptr(paa), _ptr(labels), m, _ptr(g), C.byref(loss),
                                                _stream(None)))
        return float(loss.value), _split(g.cpu().numpy())

    def train(self, paa, labels, batch=256, epochs=1, lr=1e-3, weight_decay=0.0, order_seed=0):
        import numpy as np
        losses = np.zeros(max(epochs, 1), np.float32)
        _check(lib().paris_seed_model_train(self.handle, _ptr(paa), _ptr(labels), int(paa.shape[0]), batch, epochs,
                                            lr, weight_decay, order_seed, losses.ctypes.data, _stream(None)))
        return losses[:epochs]


def _split(flat):
    out, o = {}, 0
    for k, shp in SEED_MODEL_SHAPES:
        n = 1
        for d in shp:
            n *= d
        out[k] = flat[o:o + n].reshape(shp)
        o += n
    return out


def paris_attach_seed_model(index: ParisIndex, model, top_r: int = 3):
    _check(lib().paris_attach_seed_model(index.handle, model.handle if model is not None else None, top_r))
    index._seed_model = model


def paris_row_buckets(index: ParisIndex, rows):
    """12-bit key-prefix bucket of each row (numpy or device int64 rows)."""
    import numpy as np
    rows = np.ascontiguousarray(np.asarray(rows, np.int64))
    out = np.empty(rows.size, np.int32)
    _check(lib().paris_row_buckets(index.handle, rows.ctypes.data, rows.size, out.ctypes.data, _stream(None)))
    return out

