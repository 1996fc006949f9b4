// Adaptive-split ADS+ leaves (Sec. 2.2): the root has one child per word of first bits of the
// segments; a node holding more series than the leaf capacity becomes an inner node whose two
// children add one bit to one segment -- the segment whose next bit splits the node's series
// into the two most balanced parts. The approximate search (Sec. 3.3) then follows the query's
// bits down to a leaf.
//
// Data-parallel form: the tree is grown level by level over the series in index order (sorted
// by interleaved key, so every root child is already a run). At each level every oversized
// node, at once:
//   1. counts, per open segment, the series whose next bit is 1 (one pass over the positions of
//      the splitting nodes; warps whose 32 positions lie in one node add ballot counts);
//   2. picks the segment with the smallest |n0 - n1| (lowest index on ties) and appends its two
//      children (numbered by a prefix sum over the splitting nodes, so the numbering does not
//      depend on scheduling);
//   3. moves its series stably: bit 0 first, then bit 1 (ranks from a prefix sum of the bits).
// Leaves therefore tile the positions in depth-first order. Splits that leave one side empty are
// made as the rule says (the empty side is an empty leaf); a node whose segments have all their
// bits stays a leaf of any size.
#include <algorithm>
#include <vector>

#include "query.cuh"

namespace paris {

struct AdNode {
  int64_t start, count;  // leaf-order positions of the node's series
  uint64_t cards;        // bits fixed per segment: 4 bits each, segment i at bits 4i..4i+3
  int32_t seg;           // split segment; -1 for a leaf
  int32_t child0;        // bit-0 child (the bit-1 child follows it); -1 for a leaf
};

namespace {

constexpr int kAdThreads = 256;
constexpr int kAdMaxDepth = 16 * 8 + 1;  // a path fixes at most 8 bits of 16 segments

__device__ __forceinline__ int card_of(uint64_t cards, int i) { return (int)((cards >> (4 * i)) & 15u); }

// Symbol of segment i of the series at index-order position q (its summary is rotated by q mod 16).
__device__ __forceinline__ int sym_at(const uint4& v, int64_t q, int i) {
  const int slot = (i - (int)(q & 15)) & 15;
  const uint32_t word = slot < 4 ? v.x : (slot < 8 ? v.y : (slot < 12 ? v.z : v.w));
  return (int)((word >> (8 * (slot & 3))) & 0xffu);
}

__device__ __forceinline__ bool open_segment(uint64_t cards, int w, int bits) {
  for (int i = 0; i < w; ++i)
    if (card_of(cards, i) < bits) return true;
  return false;
}

__device__ __forceinline__ int64_t grid_start() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t grid_step() { return (int64_t)gridDim.x * blockDim.x; }

__global__ void ad_heads(const uint64_t* __restrict__ keys, int64_t n, int w, uint32_t* __restrict__ flag) {
  for (int64_t p = grid_start(); p < n; p += grid_step())
    flag[p] = (p == 0 || (keys[p] >> (64 - w)) != (keys[p - 1] >> (64 - w))) ? 1u : 0u;
}

// Root children: one per run of equal first-bit words; excl = exclusive prefix of the run heads.
__global__ void ad_roots(const uint64_t* __restrict__ keys, int64_t n, int w, int bits,
                         const uint32_t* __restrict__ excl, AdNode* __restrict__ nodes, int32_t* __restrict__ root_tab,
                         int32_t* __restrict__ nid, uint32_t* __restrict__ pos) {
  uint64_t cards = 0;
  for (int i = 0; i < 16; ++i) cards |= (uint64_t)(i < w ? 1 : bits) << (4 * i);
  for (int64_t p = grid_start(); p < n; p += grid_step()) {
    const uint64_t r = keys[p] >> (64 - w);
    const bool head = p == 0 || r != (keys[p - 1] >> (64 - w));
    const int32_t id = (int32_t)(excl[p] + (head ? 1u : 0u)) - 1;
    nid[p] = id;
    pos[p] = (uint32_t)p;
    if (head) {
      AdNode nd;
      nd.start = p;
      nd.count = 0;
      nd.cards = cards;
      nd.seg = -1;
      nd.child0 = -1;
      nodes[id] = nd;
      root_tab[r] = id;
    }
  }
}

__global__ void ad_root_counts(AdNode* __restrict__ nodes, int64_t nroot, int64_t n) {
  for (int64_t j = grid_start(); j < nroot; j += grid_step())
    nodes[j].count = (j + 1 < nroot ? nodes[j + 1].start : n) - nodes[j].start;
}

// flag[j] = node j holds more than L series and has a segment with a bit left to add.
__global__ void ad_mark(const AdNode* __restrict__ nodes, int64_t first, int64_t last, int64_t L, int w, int bits,
                        uint32_t* __restrict__ flag, unsigned long long* __restrict__ nsplit) {
  for (int64_t j = first + grid_start(); j < last; j += grid_step()) {
    const bool f = nodes[j].count > L && open_segment(nodes[j].cards, w, bits);
    flag[j] = f ? 1u : 0u;
    if (f) atomicAdd(nsplit, 1ull);
  }
}

// ones[j][i]: series of splitting node j whose next bit of segment i is 1.
__global__ void __launch_bounds__(kAdThreads) ad_hist(const uint32_t* __restrict__ pos, const int32_t* __restrict__ nid,
                                                      int64_t n, const uint32_t* __restrict__ flag,
                                                      const AdNode* __restrict__ nodes, const uint4* __restrict__ sax,
                                                      int w, int bits, uint32_t* __restrict__ ones) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = grid_start() >> 5, nw = grid_step() >> 5;
  for (int64_t base = gw * 32; base < n; base += nw * 32) {
    const int64_t p = base + lane;
    int node = -1;
    if (p < n) {
      const int nd = nid[p];
      if (flag[nd]) node = nd;
    }
    const bool act = node >= 0;
    if (!__any_sync(PARIS_FULL_MASK, act)) continue;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    uint64_t cards = 0;
    int64_t q = 0;
    if (act) {
      q = pos[p];
      v = sax[q];
      cards = nodes[node].cards;
    }
    const int node0 = __shfl_sync(PARIS_FULL_MASK, node, 0);
    const bool uniform = __all_sync(PARIS_FULL_MASK, node == node0);  // then node0 >= 0
    for (int i = 0; i < w; ++i) {
      const int c = act ? card_of(cards, i) : bits;
      const int b = c < bits ? ((sym_at(v, q, i) >> (bits - 1 - c)) & 1) : 0;
      if (uniform) {
        const int cnt = __popc(__ballot_sync(PARIS_FULL_MASK, b));
        if (lane == 0 && cnt) atomicAdd(&ones[(int64_t)node0 * 16 + i], (uint32_t)cnt);
      } else if (b) {
        atomicAdd(&ones[(int64_t)node * 16 + i], 1u);
      }
    }
  }
}

// The split of every splitting node: segment, then its two children at base + 2 * rank[j].
__global__ void ad_choose(AdNode* __restrict__ nodes, int64_t nnodes, const uint32_t* __restrict__ flag,
                          const uint32_t* __restrict__ rank, const uint32_t* __restrict__ ones, int w, int bits,
                          int64_t base) {
  for (int64_t j = grid_start(); j < nnodes; j += grid_step()) {
    if (!flag[j]) continue;
    const AdNode nd = nodes[j];
    int best = -1;
    int64_t best_bal = 0;
    for (int i = 0; i < w; ++i) {
      if (card_of(nd.cards, i) >= bits) continue;
      const int64_t o = ones[j * 16 + i];
      const int64_t bal = nd.count - 2 * o < 0 ? 2 * o - nd.count : nd.count - 2 * o;
      if (best < 0 || bal < best_bal) {
        best = i;
        best_bal = bal;
      }
    }
    const int64_t o1 = ones[j * 16 + best];
    const int32_t c0 = (int32_t)(base + 2 * (int64_t)rank[j]);
    AdNode a;
    a.start = nd.start;
    a.count = nd.count - o1;
    a.cards = nd.cards + (1ull << (4 * best));
    a.seg = -1;
    a.child0 = -1;
    AdNode b = a;
    b.start = nd.start + a.count;
    b.count = o1;
    nodes[c0] = a;
    nodes[c0 + 1] = b;
    nodes[j].seg = best;
    nodes[j].child0 = c0;
  }
}

__device__ __forceinline__ int split_bit(const AdNode& nd, const uint4* sax, int64_t q, int bits) {
  const int c = card_of(nd.cards, nd.seg);
  return (sym_at(sax[q], q, nd.seg) >> (bits - 1 - c)) & 1;
}

__global__ void ad_bits(const uint32_t* __restrict__ pos, const int32_t* __restrict__ nid, int64_t n,
                        const uint32_t* __restrict__ flag, const AdNode* __restrict__ nodes,
                        const uint4* __restrict__ sax, int bits, uint32_t* __restrict__ bit) {
  for (int64_t p = grid_start(); p < n; p += grid_step()) {
    const int nd = nid[p];
    bit[p] = flag[nd] ? (uint32_t)split_bit(nodes[nd], sax, pos[p], bits) : 0u;
  }
}

// Stable move of the splitting nodes' series: ones_before = ranks[p] - ranks[start] (exclusive
// prefix of the bits), the bit-0 side first.
__global__ void ad_scatter(const uint32_t* __restrict__ pos, const int32_t* __restrict__ nid, int64_t n,
                           const uint32_t* __restrict__ flag, const AdNode* __restrict__ nodes,
                           const uint4* __restrict__ sax, int bits, const uint32_t* __restrict__ ranks,
                           uint32_t* __restrict__ pos2, int32_t* __restrict__ nid2) {
  for (int64_t p = grid_start(); p < n; p += grid_step()) {
    const int ndi = nid[p];
    const uint32_t a = pos[p];
    if (!flag[ndi]) {
      pos2[p] = a;
      nid2[p] = ndi;
      continue;
    }
    const AdNode nd = nodes[ndi];
    const int b = split_bit(nd, sax, a, bits);
    const int64_t s = nd.start;
    const int64_t zeros = nodes[nd.child0].count;
    const int64_t ob = (int64_t)(ranks[p] - ranks[s]);
    const int64_t np = b ? s + zeros + ob : s + (p - s) - ob;
    pos2[np] = a;
    nid2[np] = nd.child0 + b;
  }
}

__global__ void ad_clear(uint32_t* __restrict__ flag, int64_t m) {
  for (int64_t j = grid_start(); j < m; j += grid_step()) flag[j] = 0u;
}

__global__ void ad_rows_kernel(const uint32_t* __restrict__ pos, const uint32_t* __restrict__ rows_sorted, int64_t n,
                               uint32_t* __restrict__ out) {
  for (int64_t p = grid_start(); p < n; p += grid_step()) out[p] = rows_sorted[pos[p]];
}

// One thread per query: root child of its first-bit word, then its bits down to a leaf.
__global__ void ad_leaf_kernel(const AdNode* __restrict__ nodes, const int32_t* __restrict__ root_tab,
                               const int32_t* __restrict__ leaf_of, const uint8_t* __restrict__ qsym,
                               const uint64_t* __restrict__ qkey, int64_t nq, int w, int bits, int64_t n, int Lp,
                               int k, int64_t* __restrict__ leaf_out) {
  for (int64_t q = grid_start(); q < nq; q += grid_step()) {
    int32_t node = root_tab[qkey[q] >> (64 - w)];
    for (int step = 0; step < kAdMaxDepth; ++step) {
      const AdNode nd = nodes[node];
      if (nd.seg < 0) break;
      const int c = card_of(nd.cards, nd.seg);
      node = nd.child0 + ((qsym[q * 16 + nd.seg] >> (bits - 1 - c)) & 1);
    }
    int64_t lo = nodes[node].start, cnt = nodes[node].count;
    if (cnt == 0) {  // an empty leaf: the leaf that holds the series at its start position
      const AdNode lf = nodes[leaf_of[lo < n ? lo : n - 1]];
      lo = lf.start;
      cnt = lf.count;
    }
    int64_t hi;
    if (cnt < k) {
      lo = lo < n - k ? lo : n - k;
      hi = lo + k;
    } else {
      hi = lo + (cnt > Lp ? (int64_t)Lp : cnt);
    }
    leaf_out[2 * q] = lo;
    leaf_out[2 * q + 1] = hi;
  }
}

int ad_grid(int64_t m) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t b = (m + kAdThreads - 1) / kAdThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * 8));
}

// Replaces a device array of `old_cap` entries of `elem` bytes by one of `want` entries that
// keeps its first `keep` entries.
paris_status grow(void** p, size_t elem, int64_t old_cap, int64_t keep, int64_t want, cudaStream_t st) {
  void* q = dev_alloc((size_t)want * elem, st);
  if (!q) return fail(PARIS_ENOMEM, "adaptive-split tree (%lld nodes)", (long long)want);
  if (*p && keep > 0) PARIS_CUDA(cudaMemcpyAsync(q, *p, (size_t)keep * elem, cudaMemcpyDeviceToDevice, st));
  if (*p) dev_free(*p, (size_t)old_cap * elem, st);
  *p = q;
  return PARIS_OK;
}

}  // namespace

void release_adaptive(paris_index* idx) {
  cudaStream_t st = nullptr;
  if (idx->ad_nodes) dev_free(idx->ad_nodes, (size_t)idx->ad_cap * sizeof(AdNode), st);
  if (idx->ad_root) dev_free(idx->ad_root, (size_t)4 << idx->w, st);
  if (idx->ad_rows) dev_free(idx->ad_rows, (size_t)idx->n * 4, st);
  if (idx->ad_leaf_of) dev_free(idx->ad_leaf_of, (size_t)idx->n * 4, st);
  idx->ad_nodes = nullptr;
  idx->ad_root = nullptr;
  idx->ad_rows = nullptr;
  idx->ad_leaf_of = nullptr;
  idx->ad_nnodes = idx->ad_cap = idx->ad_leaves = 0;
  idx->ad_depth = 0;
}

paris_status build_adaptive(paris_index* idx, cudaStream_t st) {
  release_adaptive(idx);
  const int64_t n = idx->n, L = idx->leaf_cap;
  const int w = idx->w, bits = idx->bits;
  const int64_t nroot_max = std::min<int64_t>(n, (int64_t)1 << w);
  DevBuf posb[2], nidb[2], bitb, cnt;
  for (int i = 0; i < 2; ++i)
    if (!posb[i].alloc((size_t)n * 4, st) || !nidb[i].alloc((size_t)n * 4, st))
      return fail(PARIS_ENOMEM, "adaptive-split build (%lld rows)", (long long)n);
  if (!bitb.alloc((size_t)n * 4, st) || !cnt.alloc(8, st)) return fail(PARIS_ENOMEM, "adaptive-split build");
  // owned results; on failure they are released with the index (or by the next build)
  void* root = dev_alloc((size_t)4 << w, st);
  void* rows = dev_alloc((size_t)n * 4, st);
  if (!root || !rows) {
    if (root) dev_free(root, (size_t)4 << w, st);
    if (rows) dev_free(rows, (size_t)n * 4, st);
    return fail(PARIS_ENOMEM, "adaptive-split build");
  }
  idx->ad_root = (int32_t*)root;
  idx->ad_rows = (uint32_t*)rows;
  // node arrays (grown as levels add nodes): the tree itself (owned by the index) and, per node,
  // the split flag, its rank among the splitting nodes and the 16 counts of ones
  void *nodes = nullptr, *flag = nullptr, *rank = nullptr, *ones = nullptr;
  int64_t cap = 0, fcap = 0, rcap = 0, ocap = 0, used = 0;
  auto free_work = [&]() {
    if (flag) dev_free(flag, (size_t)fcap * 4, st);
    if (rank) dev_free(rank, (size_t)rcap * 4, st);
    if (ones) dev_free(ones, (size_t)ocap * 64, st);
  };
  auto ensure = [&](int64_t want) -> paris_status {
    if (want <= cap) return PARIS_OK;
    const int64_t nc = std::max<int64_t>(want, cap * 2);
    PARIS_TRY(grow(&nodes, sizeof(AdNode), cap, used, nc, st));
    idx->ad_nodes = nodes;
    idx->ad_cap = cap = nc;
    PARIS_TRY(grow(&flag, 4, fcap, used, nc, st));
    fcap = nc;
    PARIS_TRY(grow(&rank, 4, rcap, 0, nc, st));
    rcap = nc;
    PARIS_TRY(grow(&ones, 64, ocap, 0, nc, st));
    ocap = nc;
    return PARIS_OK;
  };
  auto run = [&]() -> paris_status {
    const uint4* sax = (const uint4*)idx->sax_sorted;
    uint32_t* pos = posb[0].as<uint32_t>();
    int32_t* nid = nidb[0].as<int32_t>();
    uint32_t* pos2 = posb[1].as<uint32_t>();
    int32_t* nid2 = nidb[1].as<int32_t>();
    uint32_t* bitp = bitb.as<uint32_t>();  // run heads, then each level's split bits and their ranks
    // root children
    ad_heads<<<ad_grid(n), kAdThreads, 0, st>>>(idx->keys_sorted, n, w, bitp);
    PARIS_CUDA(cudaGetLastError());
    uint32_t last_head = 0, last_excl = 0;
    PARIS_CUDA(cudaMemcpyAsync(&last_head, bitp + n - 1, 4, cudaMemcpyDeviceToHost, st));
    PARIS_TRY(exclusive_scan(bitp, n, st));
    PARIS_CUDA(cudaMemcpyAsync(&last_excl, bitp + n - 1, 4, cudaMemcpyDeviceToHost, st));
    PARIS_CUDA(cudaStreamSynchronize(st));
    const int64_t nroot = (int64_t)last_excl + last_head;
    if (nroot < 1 || nroot > nroot_max) return fail(PARIS_EINTERNAL, "adaptive-split build: %lld root children", (long long)nroot);
    PARIS_TRY(ensure(std::max<int64_t>(2 * nroot, 1024)));
    used = nroot;
    PARIS_CUDA(cudaMemsetAsync(idx->ad_root, 0xff, (size_t)4 << w, st));
    ad_roots<<<ad_grid(n), kAdThreads, 0, st>>>(idx->keys_sorted, n, w, bits, bitp, (AdNode*)nodes, idx->ad_root,
                                                nid, pos);
    ad_root_counts<<<ad_grid(nroot), kAdThreads, 0, st>>>((AdNode*)nodes, nroot, n);
    // the root table: an empty first-bit word takes the next non-empty one, else the last one
    {
      std::vector<int32_t> tab((size_t)1 << w);
      PARIS_CUDA(cudaMemcpyAsync(tab.data(), idx->ad_root, tab.size() * 4, cudaMemcpyDeviceToHost, st));
      PARIS_CUDA(cudaStreamSynchronize(st));
      int32_t next = -1, last = -1;
      for (size_t e = tab.size(); e-- > 0;) {
        if (tab[e] >= 0) {
          next = tab[e];
          if (last < 0) last = tab[e];
        } else {
          tab[e] = next;
        }
      }
      for (auto& t : tab)
        if (t < 0) t = last;
      PARIS_CUDA(cudaMemcpyAsync(idx->ad_root, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
      PARIS_CUDA(cudaStreamSynchronize(st));  // tab is released at the end of this block
    }
    unsigned long long* nsplit_d = cnt.as<unsigned long long>();
    PARIS_CUDA(cudaMemsetAsync(nsplit_d, 0, 8, st));
    ad_mark<<<ad_grid(nroot), kAdThreads, 0, st>>>((const AdNode*)nodes, 0, nroot, L, w, bits, (uint32_t*)flag,
                                                   nsplit_d);
    unsigned long long nsplit = 0;
    PARIS_CUDA(cudaMemcpyAsync(&nsplit, nsplit_d, 8, cudaMemcpyDeviceToHost, st));
    PARIS_CUDA(cudaStreamSynchronize(st));
    int64_t nnodes = nroot, splits = 0;
    int level = 0;
    while (nsplit > 0) {
      if (level >= kAdMaxDepth) return fail(PARIS_EINTERNAL, "adaptive-split build: deeper than %d levels", kAdMaxDepth);
      used = nnodes;
      PARIS_TRY(ensure(nnodes + 2 * (int64_t)nsplit));
      uint32_t* fl = (uint32_t*)flag;
      PARIS_CUDA(cudaMemsetAsync(ones, 0, (size_t)nnodes * 64, st));
      ad_hist<<<ad_grid(n), kAdThreads, 0, st>>>(pos, nid, n, fl, (const AdNode*)nodes, sax, w, bits,
                                                 (uint32_t*)ones);
      PARIS_CUDA(cudaMemcpyAsync(rank, fl, (size_t)nnodes * 4, cudaMemcpyDeviceToDevice, st));
      PARIS_TRY(exclusive_scan((uint32_t*)rank, nnodes, st));
      ad_choose<<<ad_grid(nnodes), kAdThreads, 0, st>>>((AdNode*)nodes, nnodes, fl, (const uint32_t*)rank,
                                                        (const uint32_t*)ones, w, bits, nnodes);
      ad_bits<<<ad_grid(n), kAdThreads, 0, st>>>(pos, nid, n, fl, (const AdNode*)nodes, sax, bits, bitp);
      PARIS_TRY(exclusive_scan(bitp, n, st));
      ad_scatter<<<ad_grid(n), kAdThreads, 0, st>>>(pos, nid, n, fl, (const AdNode*)nodes, sax, bits, bitp, pos2,
                                                    nid2);
      std::swap(pos, pos2);
      std::swap(nid, nid2);
      ad_clear<<<ad_grid(nnodes), kAdThreads, 0, st>>>(fl, nnodes);
      PARIS_CUDA(cudaMemsetAsync(nsplit_d, 0, 8, st));
      const int64_t made = 2 * (int64_t)nsplit;
      ad_mark<<<ad_grid(made), kAdThreads, 0, st>>>((const AdNode*)nodes, nnodes, nnodes + made, L, w, bits, fl,
                                                    nsplit_d);
      PARIS_CUDA(cudaGetLastError());
      nnodes += made;
      used = nnodes;
      splits += (int64_t)nsplit;
      ++level;
      PARIS_CUDA(cudaMemcpyAsync(&nsplit, nsplit_d, 8, cudaMemcpyDeviceToHost, st));
      PARIS_CUDA(cudaStreamSynchronize(st));
    }
    ad_rows_kernel<<<ad_grid(n), kAdThreads, 0, st>>>(pos, idx->rows_sorted, n, idx->ad_rows);
    PARIS_CUDA(cudaGetLastError());
    // the leaf of every position: the last level's node ids (kept; the other buffer is freed)
    int32_t* leaf_of = (int32_t*)dev_alloc((size_t)n * 4, st);
    if (!leaf_of) return fail(PARIS_ENOMEM, "adaptive-split build");
    PARIS_CUDA(cudaMemcpyAsync(leaf_of, nid, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    idx->ad_leaf_of = leaf_of;
    idx->ad_nnodes = nnodes;
    idx->ad_leaves = nnodes - splits;
    idx->ad_depth = level + 1;
    note_launches(3 + 7 * level + 1);
    PARIS_CUDA(cudaStreamSynchronize(st));
    return PARIS_OK;
  };
  paris_status s = run();
  free_work();
  if (s != PARIS_OK) release_adaptive(idx);
  return s;
}

paris_status launch_adaptive_leaf(const paris_index* idx, const QueryState& qs, cudaStream_t st) {
  const int Lp = std::max(idx->leaf_cap, qs.k);
  ad_leaf_kernel<<<ad_grid(qs.nq), kAdThreads, 0, st>>>((const AdNode*)idx->ad_nodes, idx->ad_root, idx->ad_leaf_of,
                                                        qs.qsym, qs.qkey, qs.nq, idx->w, idx->bits, idx->n, Lp, qs.k,
                                                        qs.leaf);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status export_adaptive(const paris_index* idx, uint32_t* rows_host, int64_t* nodes_host, cudaStream_t st) {
  if (rows_host) PARIS_CUDA(cudaMemcpyAsync(rows_host, idx->ad_rows, (size_t)idx->n * 4, cudaMemcpyDefault, st));
  if (nodes_host) {
    std::vector<AdNode> h((size_t)idx->ad_nnodes);
    PARIS_CUDA(cudaMemcpyAsync(h.data(), idx->ad_nodes, h.size() * sizeof(AdNode), cudaMemcpyDeviceToHost, st));
    PARIS_CUDA(cudaStreamSynchronize(st));
    for (size_t j = 0; j < h.size(); ++j) {
      nodes_host[5 * j] = h[j].start;
      nodes_host[5 * j + 1] = h[j].count;
      nodes_host[5 * j + 2] = h[j].seg;
      nodes_host[5 * j + 3] = h[j].child0;
      nodes_host[5 * j + 4] = (int64_t)h[j].cards;
    }
  }
  PARIS_CUDA(cudaStreamSynchronize(st));
  return PARIS_OK;
}

}  // namespace paris
