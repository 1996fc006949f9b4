/*
 * paris.h -- C ABI of a GB300 (sm_103a) implementation of the ParIS+ exact similarity-search
 * hot path: iSAX index build and exact k-NN query answering over z-normalised fp32 series.
 *
 * Paper: B. Peng, P. Fatourou, T. Palpanas, "ParIS+: Data Series Indexing on Multi-Core
 * Architectures". Section references below are to that paper.
 *
 * Conventions for every entry point
 *   - Returns a paris_status; nothing is thrown across the ABI. On failure a message is kept
 *     for the calling thread and returned by paris_last_error().
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are stream-ordered
 *     and return after the work completes unless stated otherwise.
 *   - "device or host" pointers are classified with cudaPointerGetAttributes; host buffers are
 *     staged through device memory by the library (pinned host memory copies fastest).
 *   - All arrays are dense and row-major. Series and queries must be finite fp32 values
 *     (PARIS_EINVAL otherwise) and are expected to be z-normalised (Sec. 2.1); the library
 *     does not normalise.
 *   - Device memory the library needs is taken from the allocator installed with
 *     paris_set_allocator (default: the library's own stream-ordered pool per device, whose
 *     freed blocks stay cached until paris_trim_memory).
 */
#ifndef PARIS_H
#define PARIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paris_index paris_index; /* opaque; owned by the caller after paris_build */

typedef enum paris_status {
  PARIS_OK = 0,
  PARIS_EINVAL = 1,    /* bad argument (shape, null pointer, non-finite value, k > n ...) */
  PARIS_ENOMEM = 2,    /* device or host allocation failed */
  PARIS_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error string) */
  PARIS_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  PARIS_EINTERNAL = 5, /* an internal capacity was exceeded (message says which) */
} paris_status;

/* ------------------------------------------------------------------------------------------
 * Index build (Sec. 2.2 iSAX; Alg. 2 ConvertToSAX; Sec. 3.1-3.2 index construction).
 *
 * For each series r: PAA_i = RN64(exact sum of segment i) / (len/w), i < w; iSAX symbol
 * sym_i = number of breakpoints beta_j = Phi^-1(j/card) (j = 1..card-1) that are <= PAA_i;
 * SAX[r] = the w symbols (the summary array of Alg. 2, indexed by position); the key is the
 * bit-plane interleave of the symbols (first plane = first bit of every segment = the ADS+ root
 * child) and the index orders rows by (top 64 key bits, row). The ADS+ leaves are the runs of
 * that order sharing a key prefix with at most leaf_capacity rows.
 *
 *   series  device or host, [n][len] fp32. Device series are BORROWED: keep them alive and
 *           unchanged until paris_free (refinement reads them). Host series are copied into
 *           an index-owned device array, in chunks that the encode pass consumes as they land.
 *   n       1 <= n < 2^32;  len >= 1;  1 <= w <= 16 with len % w == 0;
 *   card    alphabet size, a power of two in [2, 256] (256 = 8-bit symbols).
 *   out     receives the new index; *out is NULL on failure.
 * ---------------------------------------------------------------------------------------- */
paris_status paris_build(const float* series, int64_t n, int32_t len, int32_t w, int32_t card,
                         void* stream, paris_index** out);

typedef struct paris_build_opts {
  int32_t leaf_capacity; /* L: rows per approximate-search leaf; 0 = 2048; max 4096 */
  int32_t bf16_shadow;   /* 1: the encode pass also writes the BF16 copy of the series and the
                            row norms that PARIS_REFINE_MIXED screens with (otherwise they are
                            built by the first MIXED query); written by the encode pass only when
                            len is a multiple of 64, len <= 1024 and len / w <= 16 (otherwise
                            the first MIXED query builds it) */
  int32_t series_on_host; /* 1 (host series only): keep the series in host memory instead of copying
                             it to the device -- the collection may exceed HBM. The build streams
                             it through two 512 MB device staging buffers (a copy of one chunk
                             overlaps the encode of the other, the double-buffered loading of
                             Sec. 3.1-3.2); the summaries, keys, leaf envelopes and the optional
                             BF16 copy stay in device memory, while the approximate search,
                             refinement and exact re-rank read raw rows from host memory over the
                             CPU-GPU link. The series is BORROWED: keep it alive and unchanged
                             until paris_free. Pageable memory is registered with the driver for
                             the index's lifetime (pinned memory is used as it is). */
  int32_t reserved[5];   /* must be zero */
} paris_build_opts;

/* paris_build with options (opts may be NULL = defaults). */
paris_status paris_build_ex(const float* series, int64_t n, int32_t len, int32_t w, int32_t card,
                            const paris_build_opts* opts, void* stream, paris_index** out);

/* Releases the index and everything it owns. NULL-safe. Waits for the index's pending work. */
void paris_free(paris_index* idx);

/* ------------------------------------------------------------------------------------------
 * Exact k-NN (Sec. 3.3, Alg. 7-9): approximate search seeds the best-so-far (BSF); a
 * MINDIST_PAA_iSAX lower-bound scan over every summary keeps the rows that can still beat it
 * (Alg. 8); the kept rows are refined with early-abandoning Euclidean distance while the BSF
 * is lowered atomically (Alg. 9). The answer is the exact brute-force answer: the k rows with
 * the smallest Euclidean distance, ties ordered by the lower row number. Distances are decided
 * on their exact real values (near ties are re-ranked in exact integer arithmetic).
 *
 *   queries   device or host, [nq][len] fp32, len as built.
 *   nq        >= 0 (0 is a no-op);  1 <= k <= min(n, 1024).
 *   out_idx   device or host, [nq][k] int64: neighbour rows, ascending (distance, row).
 *   out_dist  device or host, [nq][k] fp32: their Euclidean distances (may be NULL).
 * ---------------------------------------------------------------------------------------- */
paris_status paris_exact_knn(const paris_index* idx, const float* queries, int64_t nq, int32_t k,
                             int64_t* out_idx, float* out_dist, void* stream);

enum {
  PARIS_MODE_PLAIN = 0,   /* one query per lower-bound pass, as in Alg. 7 */
  PARIS_MODE_BATCHED = 1, /* a tile of queries per pass over the summaries (one read per tile) */
};

enum {
  PARIS_REFINE_FP32 = 0,  /* every kept candidate is refined by an fp32 gather (Alg. 9) */
  PARIS_REFINE_MIXED = 1, /* queries whose lower bounds keep many rows are screened by BF16
                             tensor-core |q|^2+|x|^2-2q.x tiles (FP32 accumulation); only rows
                             within the proven BF16 error margin of the best-so-far are
                             re-checked in fp32. Same exact answers. k <= 16; the screening
                             needs len a multiple of 64 and at most 1024 (other shapes refine
                             every kept candidate as PARIS_REFINE_FP32 does). */
};

enum {
  PARIS_SEED_DESCENT = 0, /* the approximate search visits the query key's leaf (Sec. 3.3) */
  PARIS_SEED_LEARNED = 1, /* ... and the leaves of the attached model's top-r key buckets */
  PARIS_SEED_ADAPTIVE = 2, /* the query's leaf of the adaptive-split tree (paris_build_adaptive_leaves) */
};

typedef struct paris_query_opts {
  int32_t mode;        /* PARIS_MODE_*; default PLAIN */
  int32_t query_tile;  /* queries per pass in BATCHED mode; 0 = pick automatically */
  int32_t chunk;       /* queries whose candidate lists are resident at once; 0 = automatic */
  int32_t precision;   /* PARIS_REFINE_*; default FP32 */
  int32_t seed;        /* PARIS_SEED_*; default DESCENT */
  int32_t no_leaf_pruning; /* 0 (default): leaf pruning -- every page of 256 consecutive rows in
                              index order (rows sorted by key, so each page lies inside one ADS+
                              subtree) keeps the per-segment range of its symbols, and a row scan
                              visits only the pages whose MINDIST to the query (the distance to
                              that box of iSAX regions) passes the same test as a row; pages that
                              fail hold no row that could pass. 1: scan every summary (Alg. 8 as
                              printed). Same answers either way. */
  int32_t private_bsf; /* 0 (default): one best-so-far per query, shared through atomics, which
                          every refining warp re-reads before each distance (ParIS+, Alg. 9);
                          1: each warp refines against its own best-so-far, started from the
                          query's threshold when it takes up the query and published only when
                          it leaves it (the per-worker BSF of nb-ParIS+, Sec. 3.3.2), for the
                          ablation of BSF sharing. Same answers either way. */
  int32_t reserved[1]; /* must be zero */
} paris_query_opts;

typedef struct paris_query_stats {
  int64_t candidates;  /* rows kept by the lower-bound scans (sum over queries) */
  int64_t refined;     /* candidates whose raw series was read (refinement started) */
  int64_t contenders;  /* rows re-ranked exactly */
  int64_t leaf_rows;   /* rows visited by the approximate searches */
  int64_t dense_queries; /* queries screened by the BF16 tensor-core path */
  double ms_prep, ms_descent, ms_lbscan, ms_refine, ms_select; /* device time per phase */
  double ms_dense;     /* device time of the BF16 screening (MIXED) */
  int32_t query_tile;  /* queries per summary pass used by BATCHED mode (0 in PLAIN) */
  int32_t rescreens;   /* MIXED: repeated BF16 screenings of queries whose screened candidate list
                          overflowed (each repeat first lowers the query's threshold to the k-th
                          best candidate found; the call fails with EINTERNAL after 4 repeats) */
  int64_t lb_lookups;  /* BATCHED: lower-bound table lookups the scans performed (one per lane,
                          slot and pair of queries; early abandoning skips the rest) */
  int64_t pages_examined; /* leaf pruning: page lower bounds computed (pages x queries) */
  int64_t pages_kept;     /* ... of which passed (their rows were scanned for that query) */
  int64_t bsf_updates;    /* times refinement lowered a query's shared threshold */
  int64_t list_rows;      /* BATCHED with leaf pruning: rows tested one query at a time by the
                             list scan (queries whose kept pages fit a list of 32768 pages; the
                             others share tile passes, counted in lb_lookups) */
} paris_query_stats;

/* paris_exact_knn with options (NULL = defaults) and optional host stats (NULL = none). */
paris_status paris_exact_knn_ex(const paris_index* idx, const float* queries, int64_t nq,
                                int32_t k, int64_t* out_idx, float* out_dist,
                                const paris_query_opts* opts, paris_query_stats* stats,
                                void* stream);

/* Exact k-NN over several collections in one call (the paper's search, Sec. 3.3 and Alg. 7-9,
 * applied per collection): queries[c] ([nq[c]][len of idx[c]], row-major fp32, device or host)
 * are answered against idx[c] only, into out_idx[c] / out_dist[c] ([nq[c]][k], laid out and
 * ordered as in paris_exact_knn; out_dist may be NULL, or out_dist[c] NULL for a collection).
 * In BATCHED mode the lower-bound scans of all collections run as ONE launch per chunk round:
 * the collections' CTAs split the GPU in proportion to rows x query tiles, and each CTA streams
 * its collection's summaries (16 B per series whatever the series length). Lengths may differ
 * (e.g. 128, 256 and 1024); cardinalities must be equal. The query tile of the launch is
 * opts->query_tile, or the tuned tile of the collection with the most work. Other phases run
 * per collection on the same stream. 1 <= nidx <= 4. stats (NULL = none) points to nidx
 * records; the shared scan's device time is reported in each record's ms_lbscan.
 * Errors: EINVAL for a bad argument of any collection (nothing is run), otherwise as
 * paris_exact_knn_ex; the first failing collection's status is returned. */
paris_status paris_exact_knn_multi(const paris_index* const* idx, int32_t nidx,
                                   const float* const* queries, const int64_t* nq, int32_t k,
                                   int64_t* const* out_idx, float* const* out_dist,
                                   const paris_query_opts* opts, paris_query_stats* stats,
                                   void* stream);

/* ------------------------------------------------------------------------------------------
 * Captured batches: the batched search of Sec. 3.3 recorded ONCE as a CUDA graph for batches of
 * exactly nq queries against one index, then replayed per batch (no per-kernel launch cost and
 * no host round trip inside the batch). The plan owns device buffers for nq queries and
 * [nq][k] outputs; idx stays borrowed and must outlive the plan. The first run executes eagerly
 * (it also picks the query tile when opts->query_tile is 0) and records the graph; later runs
 * copy the queries in, replay the graph and copy the outputs out. Results are those of
 * paris_exact_knn_ex with the same options. A run whose tensor-core screening overflowed a
 * candidate list (MIXED) is redone eagerly, with the repeated screenings, before returning.
 * Descent seed only (PARIS_SEED_LEARNED: EINVAL). One thread at a time per plan.
 * ---------------------------------------------------------------------------------------- */
typedef struct paris_knn_plan paris_knn_plan;

typedef struct paris_knn_plan_stats {
  int64_t graph_kernels; /* kernels in the recorded graph (0 before the first run) */
  int64_t replays;       /* runs served by the graph */
  int64_t eager_runs;    /* runs executed eagerly (the first, and any that overflowed) */
  int32_t captured;      /* 1 once the graph exists */
  int32_t query_tile;    /* query tile of the batched scan */
} paris_knn_plan_stats;

/* nq >= 1; k, opts as paris_exact_knn_ex. Allocates the plan's buffers (and the BF16 shadow in
 * MIXED). Errors: EINVAL, ENOMEM, ECUDA. */
paris_status paris_knn_plan_create(const paris_index* idx, int64_t nq, int32_t k,
                                   const paris_query_opts* opts, paris_knn_plan** out);
/* queries: [nq][len] fp32, device or host; out_idx [nq][k] int64 and out_dist [nq][k] fp32
 * (NULL allowed), device or host. The call is ordered after earlier work on `stream` and later
 * work on `stream` waits for it; it returns once the outputs are written. */
paris_status paris_knn_plan_run(paris_knn_plan* plan, const float* queries, int64_t* out_idx,
                                float* out_dist, void* stream);
/* A captured plan over several collections: the multi-collection search of
 * paris_exact_knn_multi (Sec. 3.3 per collection; one batched scan launch per chunk round over
 * every collection, BATCHED mode only) recorded once as one CUDA graph for batches of exactly
 * nq[c] queries against idx[c] (1 <= nidx <= 4, nq[c] >= 0 with at least one query, equal
 * cardinalities). Runs take queries[c] ([nq[c]][len of idx[c]]) and write out_idx[c] /
 * out_dist[c] ([nq[c]][k]; out_dist or out_dist[c] may be NULL), device or host, with the
 * results and ordering guarantees of paris_exact_knn_multi. paris_knn_plan_run rejects such a
 * plan; paris_knn_plan_run_multi also runs single-collection plans (arrays of one). */
paris_status paris_knn_plan_create_multi(const paris_index* const* idx, int32_t nidx, const int64_t* nq,
                                         int32_t k, const paris_query_opts* opts, paris_knn_plan** out);
paris_status paris_knn_plan_run_multi(paris_knn_plan* plan, const float* const* queries,
                                      int64_t* const* out_idx, float* const* out_dist, void* stream);
paris_status paris_knn_plan_info(const paris_knn_plan* plan, paris_knn_plan_stats* out);
void paris_knn_plan_free(paris_knn_plan* plan); /* NULL-safe */

/* Number of GPU kernels the library has launched since it was loaded (all threads). */
uint64_t paris_kernel_launches(void);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char* paris_last_error(void);

/* ------------------------------------------------------------------------------------------
 * Memory: route the library's device allocations through the caller (e.g. a framework's
 * caching allocator). alloc returns NULL on failure. Passing NULL functions restores the
 * default. Not thread-safe with respect to concurrent library calls.
 * ---------------------------------------------------------------------------------------- */
/* By default the library allocates from its own stream-ordered pool per device, which keeps
 * freed blocks cached for later calls; paris_trim_memory returns the cached blocks of the
 * current device to the driver (it synchronises the device first). */
paris_status paris_trim_memory(void);

/* Bound, in nanoseconds, of every device-side wait of the pipelined kernels (the tensor-core
 * screening's waits between its copy, MMA and epilogue roles); 0 restores the default of 4 s;
 * above 60 s: EINVAL. When a wait expires the kernel stops issuing work, waits (at most 0.1 s
 * more) for its own copies and MMAs in flight, releases its tensor memory and returns; the call
 * then fails with PARIS_ETIMEOUT and the device stays usable. Process-wide; takes effect at
 * the next launch. */
paris_status paris_set_wait_limit(uint64_t ns);

typedef void* (*paris_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*paris_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
paris_status paris_set_allocator(paris_alloc_fn alloc, paris_free_fn free_fn, void* ctx);

/* ------------------------------------------------------------------------------------------
 * Inspection and step-level entry points: the same kernels the build and query paths run,
 * exposed so each step can be checked on its own.
 * ---------------------------------------------------------------------------------------- */
typedef struct paris_index_view {
  int64_t n;
  int32_t len, w, card, leaf_capacity;
  const float* series;          /* device-accessible [n][len] (device memory, or mapped host
                                   memory with series_on_host) */
  const uint64_t* keys_sorted;  /* device [n]: top 64 key bits in index order */
  const uint32_t* rows_sorted;  /* device [n]: rows in index order (key, row) */
} paris_index_view;

paris_status paris_index_describe(const paris_index* idx, paris_index_view* out);

/* Breakpoints beta_1..beta_{card-1} = Phi^-1(j/card) as FP64 (Wichura's AS241, 1988), host. */
paris_status paris_breakpoints(int32_t card, double* out_host);

/* The index's summary array as plain symbols, device [n][w] uint8 (Alg. 2: SAX[r]). */
paris_status paris_export_sax(const paris_index* idx, uint8_t* out_sax, void* stream);

/* The index order (Sec. 3.1-3.2 leaves as runs of the key order): keys_sorted (top 64 key bits)
 * and rows_sorted, copied to caller buffers (device or host, [n] each; either may be NULL). */
paris_status paris_export_order(const paris_index* idx, uint64_t* out_keys, uint32_t* out_rows,
                                void* stream);

/* Encode without building: device [n][len] series -> device SAX [n][w] uint8, device keys [n]
 * (top 64 interleaved key bits), and, if out_paa is not NULL, device PAA [n][w] FP64. */
paris_status paris_encode(const float* series, int64_t n, int32_t len, int32_t w, int32_t card,
                          uint8_t* out_sax, uint64_t* out_key64, double* out_paa, void* stream);

/* Approximate search with a seed mode (PARIS_SEED_*): as paris_approx_search; with
 * PARIS_SEED_LEARNED the seed also covers the leaves of the attached model's top-r buckets
 * (out_leaf still reports the query key's own leaf). */
paris_status paris_approx_search_ex(const paris_index* idx, const float* queries, int64_t nq, int32_t k,
                                    int32_t seed_mode, int64_t* out_leaf, float* out_seed_sq, void* stream);

/* Adaptive-split leaves (Sec. 2.2, ADS+): the tree in which a leaf holding more than the
 * index's leaf capacity splits into two children by adding one bit to the segment whose next
 * bit divides its series most evenly (smallest |n0 - n1|, lowest segment on ties; a split that
 * leaves one side empty is still made; a node whose segments all have every bit stays a leaf of
 * any size). Root children are the words of first bits of the w segments. Built level by level
 * on the device from the index's summaries (deterministic: the same tree on every run); the
 * series of each side keep their order, bit 0 first, so the leaves tile the "leaf order" of the
 * series depth first, starting from the index order. Needs 5 x 4 B per series of scratch during
 * the build and keeps 8 B per series plus 32 B per node. Rebuilding replaces the tree.
 * PARIS_SEED_ADAPTIVE then seeds the best-so-far from the query's leaf of this tree: its root
 * child is that of the query's first-bit word (an empty one is replaced by the next non-empty
 * word, else the last one), then its bits choose the children; an empty leaf is replaced by the
 * leaf holding the series at the empty leaf's start; a leaf with fewer than k series becomes the
 * k series of the leaf order from its start (moved left to fit), and one with more than
 * max(leaf capacity, k) series is cut to its first ones. With this seed, out_leaf of
 * paris_approx_search_ex reports leaf-order positions. Answers never depend on the seed. */
paris_status paris_build_adaptive_leaves(paris_index* idx, void* stream);
/* Size of the adaptive-split tree (any pointer may be NULL); EINVAL when none was built. */
paris_status paris_adaptive_leaves_info(const paris_index* idx, int64_t* n_nodes, int64_t* n_leaves,
                                        int32_t* depth);
/* Host copies of the tree: rows_host [n] (series row at each leaf-order position) and nodes_host
 * [n_nodes][5] int64 (first leaf-order position, number of series, split segment or -1 for a
 * leaf, index of the bit-0 child -- the bit-1 child follows it -- or -1, and the bits fixed per
 * segment, 4 bits each, segment i at bits 4i..4i+3). Root children come first, in increasing
 * first-bit word order. Either pointer may be NULL. */
paris_status paris_adaptive_leaves_export(const paris_index* idx, uint32_t* rows_host, int64_t* nodes_host,
                                          void* stream);

/* Approximate search alone (Sec. 3.3): per query, the sorted-position range [lo, hi) of its
 * leaf (device or host [nq][2] int64) and the seed -- the k-th smallest fp32 squared distance
 * among the leaf rows (device or host [nq] fp32, may be NULL). */
paris_status paris_approx_search(const paris_index* idx, const float* queries, int64_t nq,
                                 int32_t k, int64_t* out_leaf, float* out_seed_sq, void* stream);

/* Lower-bound scan alone (Alg. 8) for one query against a squared threshold: every row whose
 * conservative fp32 MINDIST^2 lower bound is <= threshold_sq is kept. Writes up to `capacity`
 * (row, lb_sq) pairs in no particular order to out_rows/out_lb (device) and the number of kept
 * rows (which may exceed capacity) to *out_count (host). */
paris_status paris_lb_scan(const paris_index* idx, const float* query, float threshold_sq,
                           uint32_t* out_rows, float* out_lb, int64_t capacity, int64_t* out_count,
                           void* stream);

/* Leaf pruning alone for one query against a squared threshold (Sec. 2.2 ADS+ leaves; the
 * MINDIST of Sec. 3.3.1 taken to a page's box of iSAX regions). The index order (rows sorted
 * by key, paris_export_order) is cut into pages of PARIS_PAGE_ROWS consecutive positions; page
 * p covers positions [p * PARIS_PAGE_ROWS, (p + 1) * PARIS_PAGE_ROWS). Bit p of out_bits
 * (device uint32 [(pages + 31) / 32], bit p % 32 of word p / 32) is set when the page's box
 * MINDIST^2 lower bound passes the row test of paris_lb_scan; a page that fails holds no row
 * that paris_lb_scan would keep. *out_kept (host) receives the number of set bits. */
#define PARIS_PAGE_ROWS 256
paris_status paris_leaf_scan(const paris_index* idx, const float* query, float threshold_sq, uint32_t* out_bits,
                             int64_t* out_kept, void* stream);

/* ------------------------------------------------------------------------------------------
 * Learned best-so-far proposal (not in the paper; it only chooses which extra leaves the
 * approximate search of Sec. 3.3 visits, so answers never change). An MLP maps a query's PAA
 * (16 values) through 256 -> 256 (exact GELU) to 4096 logits over 12-bit key-prefix buckets
 * (bucket = first 12 bits of the interleaved key = first bit of segments 0..11). BF16 weights
 * for the GEMMs (tensor cores, FP32 accumulation), FP32 master weights, softmax cross-entropy,
 * AdamW. Parameters travel as one FP32 host array in the order W1 [256][16], b1 [256],
 * W2 [256][256], b2 [256], W3 [4096][256], b3 [4096] (1,122,816 values).
 * ---------------------------------------------------------------------------------------- */
typedef struct paris_seed_model paris_seed_model;
#define PARIS_SEED_MODEL_PARAMS 1122816

/* Xavier-uniform weights from a splitmix64 stream seeded by init_seed, zero biases. */
paris_status paris_seed_model_create(uint64_t init_seed, void* stream, paris_seed_model** out);
void paris_seed_model_free(paris_seed_model* model); /* NULL-safe */
paris_status paris_seed_model_set_weights(paris_seed_model* model, const float* params_host, void* stream);
paris_status paris_seed_model_get_weights(const paris_seed_model* model, float* params_host, void* stream);
/* Inputs are PAA vectors as paris_encode writes them: device FP64 [m][16] (unused segments 0). */
/* logits (device [m][4096]) of device PAA inputs [m][16]. */
paris_status paris_seed_model_forward(const paris_seed_model* model, const double* paa, int64_t m, float* logits,
                                      void* stream);
/* The top_r (1..8) highest-scoring buckets of each input, best first, equal logits ranked by
 * lower bucket: the selection the learned proposal makes before the approximate search of
 * Sec. 3.3 visits those buckets' leaves (PARIS_SEED_LEARNED). paa device FP64 [m][16],
 * out_buckets device int32 [m][top_r]. Waits on `stream` before returning. */
paris_status paris_seed_model_topr(const paris_seed_model* model, const double* paa, int64_t m, int32_t top_r,
                                   int32_t* out_buckets, void* stream);
/* Mean cross-entropy of one batch (device paa [m][16], labels [m]) and its gradients (device
 * [PARIS_SEED_MODEL_PARAMS], parameter order above); *loss_host may be NULL. No update. */
paris_status paris_seed_model_gradients(const paris_seed_model* model, const double* paa, const int32_t* labels,
                                        int32_t m, float* grads, float* loss_host, void* stream);
/* `epochs` passes of AdamW (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay) over full
 * batches of `batch` pairs visited in a pseudo-random order drawn from order_seed;
 * loss_per_epoch (host [epochs], may be NULL) receives each epoch's mean loss. */
paris_status paris_seed_model_train(paris_seed_model* model, const double* paa, const int32_t* labels, int64_t m,
                                    int32_t batch, int32_t epochs, float lr, float weight_decay,
                                    uint64_t order_seed, float* loss_per_epoch, void* stream);
/* Lets PARIS_SEED_LEARNED queries on idx visit the leaves of the model's top_r buckets
 * (1 <= top_r <= 8). The model is borrowed: keep it alive while attached; NULL detaches. */
paris_status paris_attach_seed_model(paris_index* idx, const paris_seed_model* model, int32_t top_r);
/* Training labels: the 12-bit bucket of each given row (device or host rows [m], out [m]). */
paris_status paris_row_buckets(const paris_index* idx, const int64_t* rows, int64_t m, int32_t* out_buckets,
                               void* stream);

/* ------------------------------------------------------------------------------------------
 * Lower-bound scan without allocation. The paper has no counterpart: this entry point exists
 * for callers that cannot have the library allocate device memory while they run -- services
 * that reserve all their device memory up front and forbid allocation on the request path, or
 * hosts that hand a library only pre-existing buffers. It runs the same kernels as
 * paris_lb_scan, for nq queries, but calls no cudaMalloc, cudaFree or other allocating routine:
 * its scratch (each query's PAA, key and lower-bound table, the counters, a status word) lives
 * in one static device array of PARIS_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the
 * library holds until the process exits.
 *
 *   queries        device [nq][len] fp32 (as built).
 *   thresholds_sq  host [nq]: squared thresholds, one per query.
 *   out_rows/out_lb device [nq][capacity]: query q writes its first `capacity` kept rows (any
 *                  order) at offset q*capacity; capacity may be 0 (counts only).
 *   out_counts     host [nq]: number of kept rows per query (may exceed capacity).
 * Scratch limit: nq * (card*64 + 140) bytes (rounded up per array) must fit in the static
 * array; larger requests fail with PARIS_EINVAL and a message naming the limit.
 * Set-up: the first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Every call waits on `stream` before it returns: the per-query counts are copied back to the
 * host through a stack buffer.
 * Sharing: all calls share the one array and it keeps the previous call's contents (the call
 * clears what must start at zero). Calls that overlap on the GPU -- on different streams or
 * from different threads -- race on it and must not be issued.
 * ---------------------------------------------------------------------------------------- */
#define PARIS_NOALLOC_SCRATCH_BYTES (256 * 1024)
paris_status paris_lb_scan_noalloc(const paris_index* idx, const float* queries, int64_t nq,
                                   const float* thresholds_sq, uint32_t* out_rows, float* out_lb,
                                   int64_t capacity, int64_t* out_counts, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PARIS_H */
