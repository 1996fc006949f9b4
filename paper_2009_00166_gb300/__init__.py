"""GB300 (sm_103a) ParIS+ exact similarity search: iSAX index build and exact k-NN.

A thin ctypes binding over the C ABI in ``include/paris.h`` (``libparis.so``). The Python
functions carry the C names and only marshal arguments: every step of the build and of the
queries runs in the library's CUDA kernels. PyTorch supplies device memory (tensors and, via
``paris_set_allocator``, the library's scratch) and streams.

The library must be built first (``paper_2009_00166_gb300._build.build()``); importing a
function that needs it raises ``RuntimeError`` when ``libparis.so`` is missing.
"""
from .binding import (  # noqa: F401
    PARIS_MODE_BATCHED,
    PARIS_MODE_PLAIN,
    PARIS_REFINE_FP32,
    PARIS_REFINE_MIXED,
    PARIS_SEED_DESCENT,
    PARIS_SEED_LEARNED,
    PARIS_SEED_ADAPTIVE,
    SeedModel,
    ParisError,
    ParisIndex,
    QueryStats,
    lib,
    paris_approx_search,
    paris_adaptive_leaves_export,
    paris_adaptive_leaves_info,
    paris_build_adaptive_leaves,
    paris_attach_seed_model,
    paris_breakpoints,
    paris_build,
    paris_build_ex,
    paris_encode,
    paris_exact_knn,
    paris_exact_knn_ex,
    paris_exact_knn_multi,
    KnnPlan,
    KnnPlanMulti,
    paris_export_order,
    paris_export_sax,
    paris_free,
    paris_index_describe,
    paris_kernel_launches,
    paris_lb_scan,
    paris_leaf_scan,
    paris_set_wait_limit,
    PARIS_PAGE_ROWS,
    paris_row_buckets,
    paris_last_error,
    paris_set_allocator,
    paris_trim_memory,
    use_torch_allocator,
)
