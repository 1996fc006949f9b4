// Batched lower-bound scan (the batched form of Alg. 8): one persistent launch scans the
// summary array for a whole chunk of queries, a tile of QT queries at a time, so each pass over
// the 16-byte summaries serves QT queries.
//
// Each CTA keeps the tile's lower-bound tables in shared memory as FP16 pairs: one 32-bit word
// holds the entries of two queries for the same (symbol, segment), and the words of two pairs
// sit side by side, so one 64-bit lookup feeds four queries (two HADD2). A lane reads the
// segment its rotated summary slot names; a 64-bit access is served per half-warp, and the 16
// lanes of a half read 16 different segments of the same 128-byte region row, so the lookups
// are conflict-free with a single copy of the tables.
// Entries are rounded down to FP16 (and capped at 4000) so each stays below the exact
// contribution; the 16-term FP16 sum has relative error below 16 * 2^-11, so a row is kept when
// (sum * (1 - 2^-6)) <= threshold, and that scaled value is what is stored as its lower bound.
//
// Work order: the summaries are read in index order (rows sorted by their interleaved key, so
// the ADS+ leaves are contiguous). Each CTA owns a contiguous range of pages of kPageRows
// positions and every query tile passes over it, visiting only the pages that the leaf pruning
// kept for some active query of the tile (all pages without it); a tile with no kept page in the
// CTA's range does not even load its tables. Within a tile a warp checks its
// 32 rows after 4 and after 8 of the 16 slots and drops them as soon as no (row, query) partial
// sum is within its threshold; partial sums of non-negative terms never decrease, so the kept
// set and the stored bounds are unchanged.
//
// A pilot pass over every 128th row group first counts each query's kept rows; a query whose
// scaled count reaches 3/4 of its list capacity would overflow anyway and is handed to the
// tensor-core screening before the scan (only when overflow is allowed, i.e. MIXED refinement).
// The pilot's count of rows still within the threshold after 8 slots then orders the chunk's
// queries, so that a tile gathers queries whose scans abandon alike (one loose query no longer
// keeps eleven tight ones from abandoning).
#include <cuda_fp16.h>

#include <algorithm>

#include "query.cuh"

namespace paris {

namespace {

constexpr int kBThreads = 768;
constexpr int kBUnroll = 4;
constexpr float kHalfKeep = 1.0f - 1.0f / 64.0f;
constexpr float kHalfCap = 4000.0f;
constexpr int64_t kPilotStride = 128;  // the pilot pass reads every 128th group of 32 rows
constexpr double kPilotRoute = 0.75;  // routed when the scaled pilot count reaches 0.75 * capacity

__device__ __forceinline__ uint32_t pack_half2_rd(float a, float b) {
  __half ha = __float2half_rd(fminf(a, kHalfCap)), hb = __float2half_rd(fminf(b, kHalfCap));
  return (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
}

// Appends the kept rows of one query (warp-aggregated); stops writing once the list overflowed.
__device__ __forceinline__ void append_kept(bool keep, int64_t row, float lb, int lane, uint32_t* count,
                                            uint32_t* out_rows, float* out_lb, int64_t cap, bool& overflowed,
                                            uint32_t* status) {
  const uint32_t mk = __ballot_sync(PARIS_FULL_MASK, keep);
  if (!mk || overflowed) return;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(count, (uint32_t)__popc(mk));
  base = __shfl_sync(PARIS_FULL_MASK, base, 0);
  if (keep) {
    const uint32_t p = base + __popc(mk & ((1u << lane) - 1u));
    if ((int64_t)p < cap) {
      out_rows[p] = (uint32_t)row;
      out_lb[p] = lb;
    } else {
      atomicOr(status, DEV_CAND_OVERFLOW);
    }
  }
  if ((int64_t)base + __popc(mk) > cap) overflowed = true;
}

// FP16 pair tables of a chunk: word (pair p, entry e) = {T[a][e], T[b][e]} for the queries a, b
// in tile slots 2p and 2p + 1 (slot j holds query perm[j], or j without a permutation).
__global__ void pack_pairs_kernel(const float* __restrict__ qtable, int qc, int64_t entries, const int* __restrict__ perm,
                                  uint32_t* __restrict__ out) {
  const int64_t npairs = (qc + 1) / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npairs * entries;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / entries, e = i - p * entries;
    const int64_t sa = 2 * p, sb = sa + 1;
    const int64_t qa = perm ? perm[sa] : sa, qb = sb < qc ? (perm ? perm[sb] : sb) : 0;
    const float va = qtable[qa * entries + e];
    const float vb = sb < qc ? qtable[qb * entries + e] : 0.f;
    out[i] = pack_half2_rd(va, vb);
  }
}

// Copies the FP16 pair tables of query tile `qb` into shared memory (two copies per symbol row,
// one per half-warp) and returns the tile's FP32 thresholds in s_thr (-1: nothing kept).
// Shared-memory word of (pair p, symbol c, segment i): pairs 2r and 2r+1 form region r; two
// regions share each 256-byte symbol row of a 64 KB block (region r: block r/2, half r%2); in a
// region the two pairs' words of a segment are adjacent.
__host__ __device__ constexpr int table_word(int p, int c, int i) {
  return (p >> 2) * 16384 + c * 64 + ((p >> 1) & 1) * 32 + i * 2 + (p & 1);
}

// Copies the FP16 pair tables of query tile `qb` into shared memory and returns the tile's FP32
// thresholds in s_thr (-1: nothing kept).
template <int NP>
__device__ __forceinline__ void load_tile(const uint32_t* __restrict__ packed, int64_t entries, int qb, int qc,
                                          const uint32_t* __restrict__ thr, int64_t q0, const int* __restrict__ perm,
                                          const bool* active, uint32_t* s_tab, float* s_thr) {
  constexpr int QT = 2 * NP, NR = (NP + 1) / 2;
  const int npairs_chunk = (qc + 1) / 2;
  // one step: 4 segments of one symbol for both pairs of a region (two 16-byte stores)
  for (int64_t t = threadIdx.x; t < (int64_t)NR * entries / 4; t += blockDim.x) {
    const int r = (int)(t / (entries / 4));
    const int64_t rem = 4 * (t - (int64_t)r * (entries / 4));
    const int c = (int)(rem >> 4), i = (int)(rem & 15);
    const int pa = 2 * r, pb = 2 * r + 1;
    const int ga = qb / 2 + pa, gb = qb / 2 + pb;  // pair indices within the chunk
    const uint4 A = ga < npairs_chunk ? *reinterpret_cast<const uint4*>(packed + (int64_t)ga * entries + rem)
                                      : make_uint4(0u, 0u, 0u, 0u);
    const uint4 B = (pb < NP && gb < npairs_chunk)
                        ? *reinterpret_cast<const uint4*>(packed + (int64_t)gb * entries + rem)
                        : make_uint4(0u, 0u, 0u, 0u);
    const int w0 = table_word(pa, c, i);
    *reinterpret_cast<uint4*>(&s_tab[w0]) = make_uint4(A.x, B.x, A.y, B.y);
    *reinterpret_cast<uint4*>(&s_tab[w0 + 4]) = make_uint4(A.z, B.z, A.w, B.w);
  }
  if (threadIdx.x < QT) {
    const int q = qb + threadIdx.x;
    s_thr[threadIdx.x] = (q < qc && active[threadIdx.x]) ? __uint_as_float(thr[q0 + (perm ? perm[q] : q)]) : -1.0f;
  }
}

// FP16 thresholds per pair: keep iff sum <= thr / (1 - 2^-6), the bound rounded up so the kept
// set is a superset of the FP32 test's.
template <int NP>
__device__ __forceinline__ void tile_thresholds(const float* s_thr, __half2 (&thh)[NP]) {
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float ta = s_thr[2 * p], tb = s_thr[2 * p + 1];
    thh[p] = __halves2half2(ta < 0.f ? __float2half(-65504.f) : __float2half_ru(fminf(ta / kHalfKeep, 65504.f)),
                            tb < 0.f ? __float2half(-65504.f) : __float2half_ru(fminf(tb / kHalfKeep, 65504.f)));
    if (ta >= 65504.f * kHalfKeep) thh[p] = __halves2half2(__float2half(65504.f), __high2half(thh[p]));
    if (tb >= 65504.f * kHalfKeep) thh[p] = __halves2half2(__low2half(thh[p]), __float2half(65504.f));
  }
}

// Adds the FP16 pair entries of slots [K0, K1) of one row to the two summation chains of every
// pair (even slots to a0, odd slots to a1): one 64-bit lookup per slot and region.
template <int NP, int K0, int K1>
__device__ __forceinline__ void add_slots(const uint32_t (&wv)[4], const uint32_t (&offp)[8], uint32_t tab,
                                          __half2 (&a0)[NP], __half2 (&a1)[NP]) {
#pragma unroll
  for (int kk = K0; kk < K1; kk += 2) {
    const uint32_t sel0 = (4u + 0u) | ((uint32_t)(kk & 3) << 4) | (5u << 8) | (5u << 12);
    const uint32_t sel1 = (4u + 2u) | ((uint32_t)((kk + 1) & 3) << 4) | (5u << 8) | (5u << 12);
    const uint32_t ad0 = tab + __byte_perm(wv[kk >> 2], offp[kk >> 1], sel0);
    const uint32_t ad1 = tab + __byte_perm(wv[(kk + 1) >> 2], offp[kk >> 1], sel1);
#pragma unroll
    for (int r = 0; r < (NP + 1) / 2; ++r) {
      const uint32_t off = (uint32_t)((r >> 1) * 65536 + (r & 1) * 128);
      if (2 * r + 1 < NP) {
        uint32_t v0x, v0y, v1x, v1y;
        asm("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v0x), "=r"(v0y) : "r"(ad0 + off));
        asm("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v1x), "=r"(v1y) : "r"(ad1 + off));
        a0[2 * r] = __hadd2(a0[2 * r], *reinterpret_cast<__half2*>(&v0x));
        a0[2 * r + 1] = __hadd2(a0[2 * r + 1], *reinterpret_cast<__half2*>(&v0y));
        a1[2 * r] = __hadd2(a1[2 * r], *reinterpret_cast<__half2*>(&v1x));
        a1[2 * r + 1] = __hadd2(a1[2 * r + 1], *reinterpret_cast<__half2*>(&v1y));
      } else {  // a region holding one pair
        uint32_t v0, v1;
        asm("ld.shared.b32 %0, [%1];" : "=r"(v0) : "r"(ad0 + off));
        asm("ld.shared.b32 %0, [%1];" : "=r"(v1) : "r"(ad1 + off));
        a0[2 * r] = __hadd2(a0[2 * r], *reinterpret_cast<__half2*>(&v0));
        a1[2 * r] = __hadd2(a1[2 * r], *reinterpret_cast<__half2*>(&v1));
      }
    }
  }
}

// True when some lane's row may still be kept for some query of the tile. The partial sums only
// grow with further non-negative terms (round-to-nearest addition is monotone), so a partial sum
// above a threshold already decides the full sum's test.
template <int NP>
__device__ __forceinline__ bool warp_alive(bool rv, const __half2 (&a0)[NP], const __half2 (&a1)[NP],
                                           const __half2 (&thh)[NP]) {
  uint32_t m = 0u;
#pragma unroll
  for (int p = 0; p < NP; ++p) m |= __hle2_mask(__hadd2(a0[p], a1[p]), thh[p]);
  return __any_sync(PARIS_FULL_MASK, rv && m != 0u);
}

// Keep bits of one row: bit 2p (query 2p of the tile) and 2p + 1, sums left in `sum`. The warp
// gives up on its 32 rows after 4 and after 8 of the 16 slots once no (row, query) partial sum
// is within its threshold (returns 0 for every lane then).
template <int NP>
__device__ __forceinline__ uint32_t row_keep_bits(const uint4& word, bool rv, const uint32_t (&offp)[8], uint32_t tab,
                                                  const __half2 (&thh)[NP], __half2 (&sum)[NP], uint32_t& slots) {
  const uint32_t wv[4] = {word.x, word.y, word.z, word.w};
  __half2 a0[NP], a1[NP];  // two chains per pair: shorter latency
#pragma unroll
  for (int p = 0; p < NP; ++p) a0[p] = a1[p] = __floats2half2_rn(0.f, 0.f);
  add_slots<NP, 0, 4>(wv, offp, tab, a0, a1);
  slots += 4;
  if (!warp_alive<NP>(rv, a0, a1, thh)) return 0u;
  add_slots<NP, 4, 8>(wv, offp, tab, a0, a1);
  slots += 4;
  if (!warp_alive<NP>(rv, a0, a1, thh)) return 0u;
  add_slots<NP, 8, 16>(wv, offp, tab, a0, a1);
  slots += 8;
  uint32_t keepmask = 0u;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    sum[p] = __hadd2(a0[p], a1[p]);
    const uint32_t m = __hle2_mask(sum[p], thh[p]);
    keepmask |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * p);
  }
  return rv ? keepmask : 0u;
}

// Appends one row group's kept (row, query) pairs to the queries' lists; returns the updated
// overflow bits (bit q: the list of tile slot q passed its capacity). Kept out of line: it runs
// for few row groups, and inlining it into the unrolled scan loop crowds the instruction cache.
template <int NP>
__device__ __noinline__ uint32_t emit_row(uint32_t keepmask, uint32_t any, const uint32_t* sums, int64_t row, int lane,
                                         const int* s_qid, uint32_t* count, uint32_t* rows, float* lbs, int64_t cap,
                                         uint32_t ovf, uint32_t* status) {
  for (int p = 0; p < NP; ++p) {
    if (!((any >> (2 * p)) & 3u)) continue;
    const uint32_t sp = sums[p];
    const __half2 h2 = *reinterpret_cast<const __half2*>(&sp);
    const float lv[2] = {__low2float(h2) * kHalfKeep, __high2float(h2) * kHalfKeep};
    for (int j = 0; j < 2; ++j) {
      const int slot = 2 * p + j, q = s_qid[slot];
      bool o = (ovf >> slot) & 1u;
      append_kept(((keepmask >> slot) & 1u) != 0u, row, lv[j], lane, count + q, rows + (int64_t)q * cap,
                  lbs + (int64_t)q * cap, cap, o, status);
      ovf |= (o ? 1u : 0u) << slot;
    }
  }
  return ovf;
}

__device__ __forceinline__ void lane_offsets(int lane, uint32_t (&offp)[8]) {
#pragma unroll
  for (int m = 0; m < 8; ++m) {  // byte offset of the lane's segment in a region row, per slot
    uint32_t o0 = 8u * ((2 * m + lane) & 15);
    uint32_t o1 = 8u * ((2 * m + 1 + lane) & 15);
    offp[m] = o0 | (o1 << 16);
  }
}

// One collection's share of a batched scan launch: its summaries, the chunk's packed tables,
// thresholds and candidate lists, and the CTAs [cta0, cta0 + ncta) that split its rows.
struct ScanColl {
  const uint4* sax;      // index-order summaries (position p rotated by p mod 16)
  const uint32_t* pos_row;  // row of each index-order position
  const uint32_t* pagebits;  // [qc][words] kept pages per chunk query (NULL: every page)
  const uint32_t* page_count;  // [qc] kept pages per chunk query: those within list_cap take the list scan
  int64_t list_cap;
  int64_t words;
  int64_t n;
  const uint32_t* packed;
  const uint32_t* thr;
  int64_t q0;
  int qc, ntiles;
  uint32_t* count;
  uint32_t* rows;
  float* lb;
  int64_t cap;
  uint32_t* pilot;  // pilot counts (pilot launch only): kept rows [qc], then rows alive after 8 slots [qc]
  const int* perm;  // tile slot -> chunk query (NULL: slot j holds query j)
  int stop;         // lists may overflow (MIXED): overflowed queries leave the scan
  unsigned long long* lookups;  // table lookups performed (one per lane, slot and query pair)
  uint32_t* status;  // device status word of the collection's call
  int cta0, ncta;
};

constexpr int kMaxColl = 4;
static_assert(kMaxColl == kMaxScanJobs, "one scan descriptor per collection of a multi-collection call");

struct ScanWork {
  int ncoll;
  int card;
  int64_t stride;        // pilot: every stride-th row group
  ScanColl c[kMaxColl];
};

__device__ __forceinline__ int coll_of_block(const ScanWork& W) {
  int ci = 0;
  while (ci + 1 < W.ncoll && (int)blockIdx.x >= W.c[ci + 1].cta0) ++ci;
  return ci;
}

constexpr int kWinPages = 1024;  // pages per window of a CTA's range (the kept-page list in shared memory)

template <int NP>
__global__ void __launch_bounds__(kBThreads, 1) lbscan_batched_kernel(const __grid_constant__ ScanWork W) {
  constexpr int QT = 2 * NP;
  constexpr int kGpp = kPageRows / 32;  // 32-row groups per page
  extern __shared__ __align__(16) uint32_t s_tab[];  // region r (64 KB): pairs 2r, 2r+1
  __shared__ float s_thr[QT];
  __shared__ bool s_active[QT];
  __shared__ int s_qid[QT];  // chunk query of each tile slot
  __shared__ uint32_t s_pages[kWinPages];  // kept pages of the current window (any order)
  __shared__ int s_np;
  const ScanColl& C = W.c[coll_of_block(W)];
  const uint4* __restrict__ sax = C.sax;
  const int64_t n = C.n, cap = C.cap;
  const int qc = C.qc, stop_on_overflow = C.stop;
  uint32_t* __restrict__ count = C.count;
  uint32_t* __restrict__ status = C.status;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t offp[8];
  lane_offsets(lane, offp);
  const uint32_t tab = (uint32_t)__cvta_generic_to_shared(s_tab);
  // the CTA's range of index-order pages, in whole 32-page words
  const int64_t npages = (n + kPageRows - 1) / kPageRows;
  const int64_t nwords = (npages + 31) >> 5;
  const int64_t wper = (nwords + C.ncta - 1) / C.ncta;
  const int64_t pg0 = (int64_t)(blockIdx.x - C.cta0) * wper * 32, pg1 = min(npages, pg0 + wper * 32);
  const int64_t entries = (int64_t)W.card * 16;
  for (int tile = 0; tile < C.ntiles; ++tile) {
    const int qb = tile * QT;
    __syncthreads();  // the previous tile's tables and flags are no longer read
    bool act = false;
    if (threadIdx.x < QT) {  // one thread per tile slot
      const int q = threadIdx.x, qq = qb + q;
      const int qid = qq < qc ? (C.perm ? C.perm[qq] : qq) : 0;
      // a list whose count passed its capacity has flagged its overflow (or was handed to the
      // tensor-core screening beforehand): the query takes no further part in the scan; with
      // leaf pruning, a query whose kept pages fit its list is scanned by the list scan instead
      act = qq < qc && !(stop_on_overflow && (int64_t)__ldcg(count + qid) > cap) &&
            !(C.pagebits && (int64_t)C.page_count[qid] <= C.list_cap);
      s_active[q] = act;
      s_qid[q] = qid;
    }
    if (!__syncthreads_or(act)) continue;
    bool loaded = false;
    __half2 thh[NP];
    uint32_t ovf = 0u;   // bit q: the list of tile slot q passed its capacity
    uint32_t slots = 0;  // slots this warp looked up in this tile, per row group
    for (int64_t w0 = pg0; w0 < pg1; w0 += kWinPages) {
      const int64_t w1 = min(pg1, w0 + kWinPages);
      __syncthreads();  // the previous window's page list and count are no longer read
      if (threadIdx.x == 0) s_np = 0;
      __syncthreads();
      // pages of the window that some active query of the tile keeps (leaf pruning)
      for (int64_t wi = threadIdx.x; wi < (w1 - w0 + 31) >> 5; wi += blockDim.x) {
        const int64_t wd = (w0 >> 5) + wi;
        uint32_t u = 0u;
        if (C.pagebits) {
          for (int q = 0; q < QT; ++q)
            if (s_active[q]) u |= __ldg(C.pagebits + (int64_t)s_qid[q] * C.words + wd);
        } else {
          u = ~0u;
        }
        const int64_t lim = w1 - wd * 32;  // pages of this word inside the window
        if (lim < 32) u &= (1u << lim) - 1u;
        if (u) {
          int base = atomicAdd(&s_np, __popc(u));
          while (u) {
            const int b = __ffs(u) - 1;
            u &= u - 1u;
            s_pages[base++] = (uint32_t)(wd * 32 + b);
          }
        }
      }
      __syncthreads();
      const int np = s_np;
      if (np == 0) continue;
      if (!loaded) {
        load_tile<NP>(C.packed, entries, qb, qc, C.thr, C.q0, C.perm, s_active, s_tab, s_thr);
        __syncthreads();
        tile_thresholds<NP>(s_thr, thh);
        loaded = true;
      }
      const int64_t vgroups = (int64_t)np * kGpp;
      for (int64_t it = (int64_t)wib * kBUnroll; it < vgroups; it += (int64_t)nw * kBUnroll) {
        uint4 word[kBUnroll];
        int64_t pos[kBUnroll];
#pragma unroll
        for (int u = 0; u < kBUnroll; ++u) {
          const int64_t v = it + u;
          pos[u] = v < vgroups ? ((int64_t)s_pages[v / kGpp] * kGpp + v % kGpp) * 32 + lane : n;
          word[u] = pos[u] < n ? __ldcg(sax + pos[u]) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kBUnroll; ++u) {
          const bool rv = pos[u] < n;
          __half2 sum[NP];
          const uint32_t keepmask = row_keep_bits<NP>(word[u], rv, offp, tab, thh, sum, slots);
          const uint32_t any = __reduce_or_sync(PARIS_FULL_MASK, keepmask);
          if (any) {  // rare: some lane keeps this row for some query of the tile
            uint32_t sv[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) sv[p] = *reinterpret_cast<const uint32_t*>(&sum[p]);
            const uint32_t row = rv ? C.pos_row[pos[u]] : 0u;
            ovf = emit_row<NP>(keepmask, any, sv, row, lane, s_qid, count, C.rows, C.lb, cap, ovf, status);
          }
        }
        if (stop_on_overflow) {
          bool all = true;
#pragma unroll
          for (int q = 0; q < QT; ++q) all = all && (((ovf >> q) & 1u) || s_thr[q] < 0.f);
          if (all) break;
        }
      }
    }
    if (lane == 0 && C.lookups && slots) atomicAdd(C.lookups, (unsigned long long)slots * (NP * 32));
  }
}

// Pilot pass: counts, per query, the kept rows among every `stride`-th group of 32 rows (same
// test as the scan) and the rows still within the threshold after 8 of the 16 slots. The first
// count routes queries whose list would overflow to the tensor-core screening (MIXED); the
// second orders the chunk's queries so that tiles gather queries whose scans abandon alike.
template <int NP>
__global__ void __launch_bounds__(kBThreads, 1) pilot_kernel(const __grid_constant__ ScanWork W) {
  constexpr int QT = 2 * NP;
  extern __shared__ __align__(16) uint32_t s_tab[];
  __shared__ float s_thr[QT];
  __shared__ bool s_active[QT];
  __shared__ uint32_t s_cnt[2 * QT];
  const ScanColl& C = W.c[coll_of_block(W)];
  const int64_t n = C.n, stride = W.stride;
  const int qc = C.qc;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t offp[8];
  lane_offsets(lane, offp);
  const uint32_t tab = (uint32_t)__cvta_generic_to_shared(s_tab);
  const int64_t samples = (((n + 31) >> 5) + stride - 1) / stride;
  const int64_t per = (samples + C.ncta - 1) / C.ncta;
  const int64_t s0 = (int64_t)(blockIdx.x - C.cta0) * per, s1 = min(samples, s0 + per);
  const int64_t entries = (int64_t)W.card * 16;
  for (int tile = 0; tile < C.ntiles; ++tile) {
    const int qb = tile * QT;
    __syncthreads();
    // queries that the leaf pruning sends to the list scan need no pilot count (they are neither
    // routed nor placed in tiles): a tile of such queries only is skipped
    bool act = false;
    if (threadIdx.x < QT) {
      const int qq = qb + threadIdx.x;
      act = qq < qc && !(C.pagebits && (int64_t)C.page_count[qq] <= C.list_cap);
      s_active[threadIdx.x] = act;
    }
    if (!__syncthreads_or(act)) continue;
    load_tile<NP>(C.packed, entries, qb, qc, C.thr, C.q0, nullptr, s_active, s_tab, s_thr);
    if (threadIdx.x < 2 * QT) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    __half2 thh[NP];
    tile_thresholds<NP>(s_thr, thh);
    uint32_t cnt[QT], cnt8[QT];
#pragma unroll
    for (int q = 0; q < QT; ++q) cnt[q] = cnt8[q] = 0u;
    for (int64_t it = s0 + wib; it < s1; it += nw) {
      const int64_t row = it * stride * 32 + lane;
      const bool rv = row < n;
      const uint4 word = rv ? __ldcg(C.sax + row) : make_uint4(0u, 0u, 0u, 0u);
      const uint32_t wv[4] = {word.x, word.y, word.z, word.w};
      __half2 a0[NP], a1[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) a0[p] = a1[p] = __floats2half2_rn(0.f, 0.f);
      add_slots<NP, 0, 8>(wv, offp, tab, a0, a1);
      uint32_t m8 = 0u, mk = 0u;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const uint32_t m = __hle2_mask(__hadd2(a0[p], a1[p]), thh[p]);
        m8 |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * p);
      }
      m8 = rv ? m8 : 0u;
      // a pair dead after 8 slots stays dead (partial sums only grow): finish only when alive
      if (__any_sync(PARIS_FULL_MASK, m8 != 0u)) {
        add_slots<NP, 8, 16>(wv, offp, tab, a0, a1);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const uint32_t m = __hle2_mask(__hadd2(a0[p], a1[p]), thh[p]);
          mk |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * p);
        }
        mk = rv ? mk : 0u;
      }
#pragma unroll
      for (int q = 0; q < QT; ++q) {
        cnt[q] += __popc(__ballot_sync(PARIS_FULL_MASK, (mk >> q) & 1u));
        cnt8[q] += __popc(__ballot_sync(PARIS_FULL_MASK, (m8 >> q) & 1u));
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < QT; ++q) {
        if (cnt[q]) atomicAdd(&s_cnt[q], cnt[q]);
        if (cnt8[q]) atomicAdd(&s_cnt[QT + q], cnt8[q]);
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * QT) {
      const int q = threadIdx.x % QT, which = threadIdx.x / QT;
      if (qb + q < qc && s_cnt[threadIdx.x]) atomicAdd(C.pilot + which * qc + qb + q, s_cnt[threadIdx.x]);
    }
  }
}

// Tile order of a chunk: queries by rows alive after 8 slots in the pilot sample (ties by
// query), routed queries last. One block; rank by counting (qc <= 4096).
__global__ void __launch_bounds__(1024) order_kernel(const uint32_t* __restrict__ alive8,
                                                     const uint32_t* __restrict__ count, int qc, int64_t cap,
                                                     int stop, int* __restrict__ perm) {
  __shared__ unsigned long long key[4096];
  for (int q = threadIdx.x; q < qc; q += blockDim.x) {
    const bool routed = stop && (int64_t)count[q] > cap;
    key[q] = ((unsigned long long)(routed ? 0xffffffffu : alive8[q]) << 32) | (unsigned)q;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < qc; q += blockDim.x) {
    const unsigned long long k = key[q];
    int rank = 0;
    for (int j = 0; j < qc; ++j) rank += key[j] < k ? 1 : 0;
    perm[rank] = q;
  }
}

// Marks the queries whose kept pages exceed the list capacity as overflowed (count = cap + 1).
__global__ void page_route_kernel(const uint32_t* __restrict__ page_count, int qc, int64_t list_cap, int64_t cap,
                                  uint32_t* __restrict__ count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < qc && (int64_t)page_count[q] > list_cap) count[q] = (uint32_t)(cap + 1);
}

// Marks the queries whose scaled pilot count reaches `limit` as overflowed (count = cap + 1).
__global__ void pilot_route_kernel(const uint32_t* __restrict__ pilot, int qc, int64_t stride, double limit,
                                   int64_t cap, uint32_t* __restrict__ count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < qc && (double)pilot[q] * (double)stride >= limit) count[q] = (uint32_t)(cap + 1);
}

size_t batched_smem(int np, int card) {
  const int blocks = (np + 3) / 4;  // 64 KB blocks of 256-byte symbol rows, two regions each
  return (size_t)(blocks - 1) * 65536 + (size_t)card * 256;
}

int sm_count_b() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Splits `grid` CTAs (grid >= ncoll) among the collections in proportion to their work, at
// least one each.
void split_ctas(ScanWork& W, const double* work, int grid) {
  double total = 0.0;
  for (int c = 0; c < W.ncoll; ++c) total += work[c];
  int given = 0;
  for (int c = 0; c < W.ncoll; ++c) {
    W.c[c].ncta = std::max(1, total > 0.0 ? (int)(grid * work[c] / total) : grid / W.ncoll);
    given += W.c[c].ncta;
  }
  while (given > grid) {  // take from the collection holding the most CTAs
    int best = 0;
    for (int c = 1; c < W.ncoll; ++c)
      if (W.c[c].ncta > W.c[best].ncta) best = c;
    --W.c[best].ncta;
    --given;
  }
  while (given < grid) {  // give to the collection with the most work per CTA
    int best = 0;
    for (int c = 1; c < W.ncoll; ++c)
      if (work[c] / W.c[c].ncta > work[best] / W.c[best].ncta) best = c;
    ++W.c[best].ncta;
    ++given;
  }
  int off = 0;
  for (int c = 0; c < W.ncoll; ++c) {
    W.c[c].cta0 = off;
    off += W.c[c].ncta;
  }
}

template <int NP>
paris_status launch_np(const ScanJob* jobs, int m, cudaStream_t st) {
  const int card = jobs[0].idx->card;
  const size_t smem = batched_smem(NP, card);
  // set on every launch: the attribute is per device, and a cached flag would not be thread-safe
  PARIS_CUDA(cudaFuncSetAttribute(lbscan_batched_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  PARIS_CUDA(cudaFuncSetAttribute(pilot_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t entries = (int64_t)card * 16;
  const int sms = sm_count_b();
  ScanWork W{}, PW{};
  W.card = PW.card = card;
  W.stride = PW.stride = kPilotStride;
  double work[kMaxColl], pwork[kMaxColl];
  int pilot_of[kMaxColl];  // scan collection of each pilot collection
  int64_t groups_total = 0, pilot_samples = 0;
  bool any_tiles = false;
  auto pack = [&](const QueryState& qs, const ChunkState& cs, const int* perm) {
    pack_pairs_kernel<<<(unsigned)std::min<int64_t>(((cs.qc + 1) / 2 * entries + 255) / 256, 4096), 256, 0, st>>>(
        qs.qtable + cs.q0 * entries, cs.qc, entries, perm, cs.packed);
    note_launches(1);
  };
  for (int j = 0; j < m; ++j) {
    const paris_index* idx = jobs[j].idx;
    const QueryState& qs = *jobs[j].qs;
    const ChunkState& cs = *jobs[j].cs;
    const int64_t groups = (idx->n + 31) / 32;
    ScanColl C{};
    C.sax = reinterpret_cast<const uint4*>(idx->sax_sorted);
    C.pos_row = idx->rows_sorted;
    C.pagebits = cs.pagebits;
    C.page_count = cs.page_count;
    C.list_cap = page_list_cap(idx->n);
    C.words = page_words(idx->n);
    C.n = idx->n;
    C.packed = cs.packed;
    C.thr = qs.thr;
    C.q0 = cs.q0;
    C.qc = cs.qc;
    C.ntiles = (cs.qc + 2 * NP - 1) / (2 * NP);
    C.count = cs.count;
    C.rows = cs.rows;
    C.lb = cs.lb;
    C.cap = cs.cap;
    C.stop = jobs[j].stop;
    C.status = jobs[j].status;
    C.lookups = qs.counters + 4;
    const bool route = C.stop && cs.cap < idx->n;
    if (!(route && cs.pagebits)) pack(qs, cs, nullptr);  // FP16 tables of the tile scan
    if (route && cs.pagebits) {
      // with leaf pruning in MIXED refinement, every query whose kept pages do not fit its list
      // goes to the tensor-core screening (one pass of 2 len flops per row and query costs less
      // than scanning a fifth or more of the summaries and refining what it keeps); the others
      // take the list scan, so neither the pilot pass nor the tile scan has work
      page_route_kernel<<<(cs.qc + 255) / 256, 256, 0, st>>>(cs.page_count, cs.qc, C.list_cap, cs.cap, cs.count);
      note_launches(1);
      C.ntiles = 0;  // no query of this collection is left for the tile scan
    } else if (groups >= 64 * kPilotStride && (route || C.ntiles > 1)) {
      // the pilot pass: route lists that would overflow anyway (MIXED) and order the tiles
      C.pilot = cs.pilot;
      PARIS_CUDA(cudaMemsetAsync(cs.pilot, 0, (size_t)cs.qc * 8, st));
      const int64_t samples = (groups + kPilotStride - 1) / kPilotStride;
      pilot_of[PW.ncoll] = W.ncoll;
      PW.c[PW.ncoll] = C;
      pwork[PW.ncoll++] = (double)samples * C.ntiles;
      pilot_samples += samples;
    }
    W.c[W.ncoll] = C;
    work[W.ncoll++] = (double)groups * C.ntiles;
    groups_total += groups;
    any_tiles = any_tiles || C.ntiles > 0;
  }
  if (PW.ncoll > 0) {
    const int pgrid = (int)std::max<int64_t>(PW.ncoll, std::min<int64_t>(sms, pilot_samples / 64));
    split_ctas(PW, pwork, pgrid);
    pilot_kernel<NP><<<pgrid, kBThreads, smem, st>>>(PW);
    note_launches(1);
    for (int c = 0; c < PW.ncoll; ++c) {
      const ScanColl& C = PW.c[c];
      const ChunkState& cs = *jobs[pilot_of[c]].cs;
      if (C.stop && C.cap < C.n) {
        pilot_route_kernel<<<(C.qc + 255) / 256, 256, 0, st>>>(C.pilot, C.qc, kPilotStride,
                                                               kPilotRoute * (double)C.cap, C.cap, C.count);
        note_launches(1);
      }
      if (C.ntiles > 1 && C.qc <= 4096) {  // the ordering ranks at most 4096 queries in one block
        order_kernel<<<1, 1024, 0, st>>>(C.pilot + C.qc, C.count, C.qc, C.cap, C.stop, cs.perm);
        pack(*jobs[pilot_of[c]].qs, cs, cs.perm);
        W.c[pilot_of[c]].perm = cs.perm;
        note_launches(1);
      }
    }
    PARIS_CUDA(cudaGetLastError());
  }
  const int grid = (int)std::max<int64_t>(W.ncoll, std::min<int64_t>(sms, (groups_total + 63) / 64));
  if (any_tiles) {
    split_ctas(W, work, grid);
    lbscan_batched_kernel<NP><<<grid, kBThreads, smem, st>>>(W);
    note_launches(1);
    PARIS_CUDA(cudaGetLastError());
  }
  // the queries that the leaf pruning left with few pages: one work item per few pages each
  for (int j = 0; j < m; ++j)
    if (jobs[j].cs->pagebits) PARIS_TRY(launch_lbscan_lists(jobs[j].idx, *jobs[j].qs, *jobs[j].cs, jobs[j].stop,
                                                            jobs[j].status, st));
  return PARIS_OK;
}

}  // namespace

const int kQueryTiles[kNumQueryTiles] = {2, 4, 8, 12, 16, 24};

bool query_tile_fits(int qt, int card) { return batched_smem(qt / 2, card) <= 200 * 1024; }

paris_status launch_lbscan_batched_multi(const ScanJob* jobs, int m, int qt, cudaStream_t st) {
  if (m < 1 || m > kMaxScanJobs) return fail(PARIS_EINVAL, "between 1 and %d collections per batched scan", kMaxScanJobs);
  for (int j = 1; j < m; ++j)
    if (jobs[j].idx->card != jobs[0].idx->card)
      return fail(PARIS_EINVAL, "collections of one batched scan share the cardinality");
  switch (qt) {
    case 2: return launch_np<1>(jobs, m, st);
    case 4: return launch_np<2>(jobs, m, st);
    case 8: return launch_np<4>(jobs, m, st);
    case 12: return launch_np<6>(jobs, m, st);
    case 16: return launch_np<8>(jobs, m, st);
    case 24: return launch_np<12>(jobs, m, st);
    default: return fail(PARIS_EINVAL, "query_tile must be one of 2, 4, 8, 12, 16, 24 (got %d)", qt);
  }
}

paris_status launch_lbscan_batched(const paris_index* idx, const QueryState& qs, const ChunkState& cs, int qt,
                                   int stop_on_overflow, uint32_t* status, cudaStream_t st) {
  ScanJob job{idx, &qs, &cs, stop_on_overflow, status};
  return launch_lbscan_batched_multi(&job, 1, qt, st);
}

}  // namespace paris
