// Query-path kernels of the GB300 ParIS+ library (host-side launch interface).
#pragma once
#include "internal.h"

namespace paris {

constexpr int kContCap = 512;   // exact re-rank contenders per query
constexpr int kLimbs = 20;      // 640-bit exact squared distances, least significant bit 2^-298
constexpr int kMaxLeaf = 4096;  // leaf capacity limit
constexpr int kDenseRetries = 4;  // repeated screenings of an overflowed list before giving up
constexpr int kPageRows = 256;    // index-order positions per leaf envelope (a multiple of 32)

// Per-call query state, all device pointers.
struct QueryState {
  int64_t nq = 0;
  int k = 1;
  const float* queries = nullptr;  // device [nq][len]
  double* qpaa = nullptr;          // [nq][16]
  uint64_t* qkey = nullptr;        // [nq]
  uint8_t* qsym = nullptr;         // [nq][16] iSAX symbols in segment order (0 past w); may be NULL
  float* qtable = nullptr;         // [nq][card][16] conservative MINDIST^2 contributions
  uint32_t* thr = nullptr;         // [nq] fp32 bits: prune/abandon threshold on squared ED
  unsigned long long* bsf = nullptr;  // [nq] packed (F bits << 32 | row), k = 1
  int64_t* leaf = nullptr;         // [nq][2]
  float* seed = nullptr;           // [nq]
  uint32_t* status = nullptr;      // [1]
  unsigned long long* counters = nullptr;  // [8]: candidates, refined, contenders, leaf rows, batched-scan
                                           // lookups, pages kept by the leaf pruning, list-scan rows,
                                           // shared best-so-far updates
  float cg = 1.f;                  // (1+gamma)/(1-gamma), rounded up, gamma = gamma_{len+2}
  const uint64_t* keys = nullptr;  // [nq][nk] approximate-search keys (NULL: qkey only)
  int nk = 1;
  int private_bsf = 0;             // refinement keeps a per-warp best-so-far (nb-ParIS+ ablation)
};

// Candidate lists of a chunk of queries [q0, q0 + qc).
struct ChunkState {
  int64_t q0 = 0;
  int qc = 0;
  int64_t cap = 0;                 // candidates per query
  uint32_t* count = nullptr;       // [qc]
  uint32_t* rows = nullptr;        // [qc][cap]
  float* lb = nullptr;             // [qc][cap]
  float* F = nullptr;              // [qc][cap], in the order of rows2
  uint32_t* rows2 = nullptr;       // [qc][cap] candidates reordered by lower-bound bucket
  float* lb2 = nullptr;            // [qc][cap]
  uint32_t* bucket = nullptr;      // [qc][32] bucket counts, then cursors
  uint32_t* packed = nullptr;      // [(qc+1)/2][card][16] FP16 pair tables of the batched scan
  uint32_t* prefix = nullptr;      // [qc + 1]
  uint32_t* kth = nullptr;         // [qc] fp32 bits of the k-th smallest F
  uint32_t* sel_hist = nullptr;    // [qc][2048]
  uint32_t* sel_state = nullptr;   // [qc][2]: prefix bits, remaining rank
  uint32_t* cont_count = nullptr;  // [qc]
  uint32_t* cont_rows = nullptr;   // [qc][kContCap]
  uint32_t* cont_limbs = nullptr;  // [qc][kContCap][kLimbs]
  uint32_t* pilot = nullptr;       // [2][qc] pilot-pass counts: kept rows, rows alive after 8 slots
  int* perm = nullptr;             // [qc] tile slot -> chunk query of the batched scan
  int* dslots = nullptr;           // [qc] chunk slots of the queries screened by the tensor cores
  int* dnd = nullptr;              // [1] number of such queries
  int* nover = nullptr;            // [1] screened lists that overflowed
  void* dqbf = nullptr;            // [dq_rows][len] BF16 query tiles of the screening
  float2* dqnm = nullptr;          // [dq_rows] (|q|^2, |q|) of those queries
  int64_t dq_rows = 0;             // qc rounded up to whole query tiles
  // leaf pruning (NULL pagebits: every page is scanned)
  uint32_t* pagebits = nullptr;    // [qc][page words]: bit p of query j = page p may hold a kept row
  uint32_t* page_list = nullptr;   // BATCHED: [qc][page list cap] kept pages per query; PLAIN: [npages]
  uint32_t* page_count = nullptr;  // [qc] kept pages per query (may exceed the list cap)
  uint32_t* item_prefix = nullptr; // [qc + 1] work items of the list scan
};

paris_status launch_query_prep(const paris_index* idx, const QueryState& qs, cudaStream_t st);
// adaptive: the leaves of the adaptive-split tree (paris_build_adaptive_leaves) in place of the
// fixed-order trie's.
paris_status launch_descent(const paris_index* idx, const QueryState& qs, cudaStream_t st, bool adaptive = false);
// Per query, the leaf-order range [lo, hi) of its adaptive-split leaf, into qs.leaf.
paris_status launch_adaptive_leaf(const paris_index* idx, const QueryState& qs, cudaStream_t st);
// Builds the adaptive-split tree of an index from its index-order summaries.
paris_status build_adaptive(paris_index* idx, cudaStream_t st);
// Host copies of the tree: series row per leaf-order position, and per node (start, count,
// split segment or -1, bit-0 child or -1, bits per segment packed 4 bits each).
paris_status export_adaptive(const paris_index* idx, uint32_t* rows_host, int64_t* nodes_host, cudaStream_t st);
paris_status launch_lbscan(const paris_index* idx, const QueryState& qs, int64_t q, uint32_t* count,
                           uint32_t* rows, float* lb, int64_t cap, uint32_t* status, int stop_on_overflow,
                           cudaStream_t st);
paris_status launch_lbscan_threshold(const paris_index* idx, const float* table, float thr,
                                     uint32_t* count, uint32_t* rows, float* lb, int64_t cap,
                                     uint32_t* status, cudaStream_t st);
// Leaf pruning (leaf.cu): index-order summaries and page envelopes (build), page lower bounds.
int64_t page_count(int64_t n);
int64_t page_words(int64_t n);
int64_t page_list_cap(int64_t n);  // kept pages a BATCHED query may list (more: tile scan)
paris_status build_leaf_envelopes(paris_index* idx, cudaStream_t st);
// Page bits of chunk queries [q0, q0 + nq) into bits ([nq][words], may be NULL), kept page counts into
// list_count [nq] and the first list_cap kept pages of each into lists [nq][list_cap] (may be
// NULL); bits and counts are zeroed first. With stop_over_cap, a query's pass may end as soon as
// its count passes list_cap (its bits and count are then partial; the count stays > list_cap).
paris_status launch_page_lb(const paris_index* idx, const QueryState& qs, int64_t q0, int64_t nq, uint32_t* bits,
                            uint32_t* lists, uint32_t* list_count, int64_t list_cap, cudaStream_t st,
                            bool stop_over_cap = false);
// The scan of the chunk's queries whose kept pages fit their lists (the others: tile scan).
paris_status launch_lbscan_lists(const paris_index* idx, const QueryState& qs, const ChunkState& cs,
                                 int stop_on_overflow, uint32_t* status, cudaStream_t st);
// The lower-bound scan of query q over the index-order pages in page_list (count on the device).
paris_status launch_lbscan_pages(const paris_index* idx, const QueryState& qs, int64_t q, const uint32_t* page_list,
                                 const uint32_t* page_count, uint32_t* count, uint32_t* rows, float* lb, int64_t cap,
                                 uint32_t* status, int stop_on_overflow, cudaStream_t st);
paris_status launch_refine(const paris_index* idx, const QueryState& qs, const ChunkState& cs,
                           cudaStream_t st);
// Batched lower-bound scan (batched.cu): one persistent launch for a chunk, tiles of qt queries.
constexpr int kNumQueryTiles = 6;
extern const int kQueryTiles[kNumQueryTiles];
bool query_tile_fits(int qt, int card);
paris_status launch_lbscan_batched(const paris_index* idx, const QueryState& qs, const ChunkState& cs, int qt,
                                   int stop_on_overflow, uint32_t* status, cudaStream_t st);
// Several collections (same cardinality) in one scan launch; their CTAs split the grid by work.
struct ScanJob {
  const paris_index* idx;
  const QueryState* qs;
  const ChunkState* cs;
  int stop;          // lists may overflow (MIXED refinement)
  uint32_t* status;  // the collection's device status word
};
constexpr int kMaxScanJobs = 4;
paris_status launch_lbscan_batched_multi(const ScanJob* jobs, int m, int qt, cudaStream_t st);

// Learned approximate-search keys (mlp.cu): [nq][r+1], own key first.
paris_status learned_keys(const paris_index* idx, const paris_seed_model* md, int r, const QueryState& qs,
                          uint64_t* keys, cudaStream_t st);
paris_status launch_row_buckets(const paris_index* idx, const int64_t* rows, int64_t m, int32_t* out,
                                uint32_t* status, cudaStream_t st);

// Mixed-precision screening (dense.cu).
bool dense_supported(const paris_index* idx, int k);
void dense_margins(int len, float* c1, float* c2);
paris_status ensure_shadow(paris_index* idx, cudaStream_t st);
// The shadow's buffers, for a build that writes them during the encode pass.
struct ShadowBufs {
  void* shadow = nullptr;   // [n][len] BF16
  float2* xnorm = nullptr;  // [n rounded up to 64] (|x|^2, |x|)
  float4* xtile = nullptr;  // [row tiles] norm ranges
};
bool dense_shape_ok(int len);
paris_status alloc_shadow(const paris_index* idx, ShadowBufs* out, cudaStream_t st);
void free_shadow_bufs(const paris_index* idx, ShadowBufs* b, cudaStream_t st);
paris_status finish_shadow(paris_index* idx, ShadowBufs* b, cudaStream_t st);
void release_shadow(paris_index* idx);
paris_status launch_dense(paris_index* idx, const QueryState& qs, const ChunkState& cs, uint32_t* overflow, int* nd_out,
                          cudaStream_t st);
paris_status tighten_overflowed(const QueryState& qs, const ChunkState& cs, int* nover, cudaStream_t st);
// Graph form of the above: adds the count of overflowed lists to cs.nover without reading it.
paris_status launch_tighten(const QueryState& qs, const ChunkState& cs, cudaStream_t st);
size_t dense_query_rows(int64_t qc);

paris_status launch_select(const paris_index* idx, const QueryState& qs, const ChunkState& cs,
                           int64_t* out_idx, float* out_dist, cudaStream_t st);

}  // namespace paris
