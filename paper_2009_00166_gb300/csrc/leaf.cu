// Leaf-level pruning over the ADS+ order (Sec. 2.2 ADS+ index; the tree's leaves let a search
// skip every series under a node whose iSAX region is too far from the query, the pruning that
// the MESSI follow-up of ParIS+ applies to in-memory leaves).
//
// The index orders rows by their interleaved key (the fixed-order trie of the ADS+ tree), so
// rows that share a key prefix are contiguous. The summaries are copied into that order, and
// every page of kPageRows consecutive positions gets an envelope: the smallest and largest
// symbol of each segment over the page's rows. A page always sits inside the trie node of its
// common key prefix, and its envelope is never wider than that node's iSAX region.
//
// The lower bound of a query against a page is the MINDIST of the query to the page's box of
// regions: per segment, the distance from the query's PAA to the nearest symbol region inside
// [lo, hi], i.e. the table entry of the symbol clamp(query symbol, lo, hi) (the entries of a
// segment grow with the distance of the symbol from the query's own symbol). Every row of the
// page has, per segment, a symbol inside [lo, hi], so its own table entry is at least the
// page's; the fp32 sum of the page's entries is then at most the fp32 sum of the row's in the
// same order (round-to-nearest addition is monotone), and a page that fails the row test
// (LB^2 * (1 - 2^-16) > threshold) holds no row that passes it.
#include <algorithm>

#include "query.cuh"

namespace paris {

namespace {

constexpr float kPageKeepScale = 1.0f - 1.0f / 65536.0f;  // the row scan's fp32 margin
constexpr int kPageThreads = 512;

// out byte j = in byte (j + k) mod 16 of a 16-byte vector (little-endian words)
__device__ __forceinline__ uint4 rot_bytes(uint4 v, int k) {
  k &= 15;
  const int q = k >> 2, r = (k & 3) * 8;
  const uint32_t w0 = v.x, w1 = v.y, w2 = v.z, w3 = v.w;
  const uint32_t a0 = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : w3;
  const uint32_t a1 = q == 0 ? w1 : q == 1 ? w2 : q == 2 ? w3 : w0;
  const uint32_t a2 = q == 0 ? w2 : q == 1 ? w3 : q == 2 ? w0 : w1;
  const uint32_t a3 = q == 0 ? w3 : q == 1 ? w0 : q == 2 ? w1 : w2;
  return make_uint4(__funnelshift_r(a0, a1, r), __funnelshift_r(a1, a2, r), __funnelshift_r(a2, a3, r),
                    __funnelshift_r(a3, a0, r));
}

// Summaries in index order: position p holds row rows_sorted[p]'s summary, its slots rotated by
// p mod 16 (slot j = segment (j + p) mod 16), as the scans expect.
__global__ void sorted_summaries_kernel(const uint4* __restrict__ sax, const uint32_t* __restrict__ rows_sorted,
                                        int64_t n, uint4* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t row = rows_sorted[p];
    out[p] = rot_bytes(__ldg(sax + row), (int)((p - (int64_t)row) & 15));  // slot j <- slot (j + p - row)
  }
}

// Envelope of every page: one warp per page. A lane reads positions lane, lane + 32, ... of the
// page, all rotated by lane mod 16, so it accumulates byte-wise minima and maxima in its own
// rotation and turns them into segment order once before the warp combines them.
__global__ void page_env_kernel(const uint4* __restrict__ sax_sorted, int64_t n, int64_t npages,
                                uint4* __restrict__ env) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t pg = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pg < npages; pg += warps) {
    uint4 lo = make_uint4(~0u, ~0u, ~0u, ~0u), hi = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int g = 0; g < kPageRows / 32; ++g) {
      const int64_t pos = pg * kPageRows + g * 32 + lane;
      if (pos < n) {
        const uint4 v = __ldg(sax_sorted + pos);
        lo = make_uint4(__vminu4(lo.x, v.x), __vminu4(lo.y, v.y), __vminu4(lo.z, v.z), __vminu4(lo.w, v.w));
        hi = make_uint4(__vmaxu4(hi.x, v.x), __vmaxu4(hi.y, v.y), __vmaxu4(hi.z, v.z), __vmaxu4(hi.w, v.w));
      }
    }
    // segment order: segment i sits in slot (i - rot) mod 16
    lo = rot_bytes(lo, 16 - (lane & 15));
    hi = rot_bytes(hi, 16 - (lane & 15));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo.x = __vminu4(lo.x, __shfl_xor_sync(PARIS_FULL_MASK, lo.x, o));
      lo.y = __vminu4(lo.y, __shfl_xor_sync(PARIS_FULL_MASK, lo.y, o));
      lo.z = __vminu4(lo.z, __shfl_xor_sync(PARIS_FULL_MASK, lo.z, o));
      lo.w = __vminu4(lo.w, __shfl_xor_sync(PARIS_FULL_MASK, lo.w, o));
      hi.x = __vmaxu4(hi.x, __shfl_xor_sync(PARIS_FULL_MASK, hi.x, o));
      hi.y = __vmaxu4(hi.y, __shfl_xor_sync(PARIS_FULL_MASK, hi.y, o));
      hi.z = __vmaxu4(hi.z, __shfl_xor_sync(PARIS_FULL_MASK, hi.z, o));
      hi.w = __vmaxu4(hi.w, __shfl_xor_sync(PARIS_FULL_MASK, hi.w, o));
    }
    if (lane == 0) {  // stored rotated by the page number, like a row's summary
      env[2 * pg] = rot_bytes(lo, (int)(pg & 15));
      env[2 * pg + 1] = rot_bytes(hi, (int)(pg & 15));
    }
  }
}

// Page lower bounds of one query per blockIdx.y, in two levels: super pages of 16 pages first
// (their envelopes cover their pages'), then the 32 pages of every word whose super pages
// passed. Lane l of a warp takes envelope 32 t + l, rotated by l mod 16; the query's symbols
// are rotated the same way once, so the clamped word is formed with byte-wise SIMD min/max and
// looked up in the query's fp32 table exactly like a row's summary (two copies of the table, one
// per half-warp, so the 32 lookups of a step fall in 32 different banks).
// Writes bit p of bits[q][words] for each kept page (the caller zeroes bits), counts the kept
// pages of each query in list_count[q] and lists the first list_cap of them in lists[q][].
constexpr int kPageAhead = 4;  // words of pages whose envelopes a warp loads together

__device__ __forceinline__ float box_lb(uint4 lo, uint4 hi, const uint4& sq, const uint32_t (&offp)[8], uint32_t tab) {
  const uint32_t wv[4] = {__vmaxu4(__vminu4(sq.x, hi.x), lo.x), __vmaxu4(__vminu4(sq.y, hi.y), lo.y),
                          __vmaxu4(__vminu4(sq.z, hi.z), lo.z), __vmaxu4(__vminu4(sq.w, hi.w), lo.w)};
  float lb = 0.f;
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) {
    const uint32_t sel = (4u + 2u * (kk & 1)) | ((uint32_t)(kk & 3) << 4) | (5u << 8) | (5u << 12);
    const uint32_t addr = tab + __byte_perm(wv[kk >> 2], offp[kk >> 1], sel);
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    lb += v;
  }
  return lb;
}

__device__ __forceinline__ void fp32_table_offsets(int lane, uint32_t (&offp)[8]) {
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const uint32_t o0 = 4u * (16u * (lane >> 4) + ((2 * m + lane) & 15));
    const uint32_t o1 = 4u * (16u * (lane >> 4) + ((2 * m + 1 + lane) & 15));
    offp[m] = o0 | (o1 << 16);
  }
}

__device__ __forceinline__ void load_fp32_table(const float* __restrict__ table, int card, float* s_tab) {
  for (int e = threadIdx.x; e < card * 16; e += blockDim.x) {
    const float v = table[e];
    const int c = e >> 4, i = e & 15;
    s_tab[c * 64 + i] = v;
    s_tab[c * 64 + 16 + i] = v;
  }
}

__global__ void __launch_bounds__(kPageThreads) page_lb_kernel(
    const uint4* __restrict__ senv, int64_t nsuper, const uint4* __restrict__ env, int64_t npages, int64_t words,
    const float* __restrict__ qtable, const uint8_t* __restrict__ qsym, const uint32_t* __restrict__ thr, int card,
    uint32_t* __restrict__ bits, uint32_t* __restrict__ lists, uint32_t* __restrict__ list_count, int64_t list_cap,
    unsigned long long* __restrict__ pages_kept, int stop_over_cap) {
  extern __shared__ __align__(16) float s_tab[];
  const int64_t q = blockIdx.y;
  load_fp32_table(qtable + q * (int64_t)card * 16, card, s_tab);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint4 sq = rot_bytes(*reinterpret_cast<const uint4*>(qsym + q * 16), lane & 15);
  const float t = __uint_as_float(thr[q]);
  uint32_t offp[8];
  fp32_table_offsets(lane, offp);
  __syncthreads();
  const uint32_t tab = (uint32_t)__cvta_generic_to_shared(s_tab);
  unsigned long long kept = 0;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t sw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; sw * 32 < nsuper; sw += nw) {
    // a query whose kept pages already exceed its list goes to the tensor-core screening: when
    // that is all the caller needs to know, its page pass ends here (one address per warp)
    if (stop_over_cap && (int64_t)__ldcg(list_count + q) > list_cap) break;
    const int64_t sp = sw * 32 + lane;
    const bool sval = sp < nsuper;
    const uint4 slo = sval ? __ldg(senv + 2 * sp) : make_uint4(0u, 0u, 0u, 0u);
    const uint4 shi = sval ? __ldg(senv + 2 * sp + 1) : make_uint4(0u, 0u, 0u, 0u);
    const float slb = box_lb(slo, shi, sq, offp, tab);
    const uint32_t ks = __ballot_sync(PARIS_FULL_MASK, sval && slb * kPageKeepScale <= t);
    // words of the 32 super pages: word 16 sw + j holds super pages 32 sw + 2j and 2j + 1
    uint32_t pw = (ks | (ks >> 1)) & 0x55555555u;
    while (pw) {
      // up to kPageAhead words of pages per round, their envelope loads in flight together
      int bs[kPageAhead];
#pragma unroll
      for (int a = 0; a < kPageAhead; ++a) {
        bs[a] = pw ? __ffs(pw) - 1 : -1;  // even: super page pair (b, b + 1)
        if (pw) pw &= pw - 1u;
      }
      uint4 lo[kPageAhead], hi[kPageAhead];
      bool valid[kPageAhead];
#pragma unroll
      for (int a = 0; a < kPageAhead; ++a) {
        const int b = bs[a];
        const int64_t pg = (sw * 16 + (b >> 1)) * 32 + lane;
        valid[a] = b >= 0 && ((ks >> (b + (lane >> 4))) & 1u) && pg < npages;
        lo[a] = valid[a] ? __ldg(env + 2 * pg) : make_uint4(0u, 0u, 0u, 0u);
        hi[a] = valid[a] ? __ldg(env + 2 * pg + 1) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int a = 0; a < kPageAhead; ++a) {
        const int b = bs[a];
        if (b < 0) break;  // warp-uniform
        const int64_t wd = sw * 16 + (b >> 1);
        const int64_t pg = wd * 32 + lane;
        const float lb = box_lb(lo[a], hi[a], sq, offp, tab);
        const bool keep = valid[a] && lb * kPageKeepScale <= t;
        const uint32_t m = __ballot_sync(PARIS_FULL_MASK, keep);
        if (!m) continue;
        if (lane == 0 && bits) bits[q * words + wd] = m;
        kept += __popc(m);
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(list_count + q, (uint32_t)__popc(m));
        base = __shfl_sync(PARIS_FULL_MASK, base, 0);
        const uint32_t at = base + __popc(m & ((1u << lane) - 1u));
        if (lists && keep && (int64_t)at < list_cap) lists[q * list_cap + at] = (uint32_t)pg;
      }
    }
  }
  if (lane == 0 && kept && pages_kept) atomicAdd(pages_kept, kept);
}

// Super-page envelopes: the per-segment min and max over 16 consecutive pages' envelopes.
__global__ void super_env_kernel(const uint4* __restrict__ env, int64_t npages, int64_t nsuper, uint4* __restrict__ senv) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsuper; s += (int64_t)gridDim.x * blockDim.x) {
    uint4 lo = make_uint4(~0u, ~0u, ~0u, ~0u), hi = make_uint4(0u, 0u, 0u, 0u);
    for (int j = 0; j < 16; ++j) {
      const int64_t pg = s * 16 + j;
      if (pg >= npages) break;
      const uint4 a = rot_bytes(env[2 * pg], 16 - (int)(pg & 15));  // to segment order
      const uint4 b = rot_bytes(env[2 * pg + 1], 16 - (int)(pg & 15));
      lo = make_uint4(__vminu4(lo.x, a.x), __vminu4(lo.y, a.y), __vminu4(lo.z, a.z), __vminu4(lo.w, a.w));
      hi = make_uint4(__vmaxu4(hi.x, b.x), __vmaxu4(hi.y, b.y), __vmaxu4(hi.z, b.z), __vmaxu4(hi.w, b.w));
    }
    senv[2 * s] = rot_bytes(lo, (int)(s & 15));
    senv[2 * s + 1] = rot_bytes(hi, (int)(s & 15));
  }
}

// Work items of the list scan: per chunk query, ceil(min(kept, list_cap) / kItemPages) items
// when its kept pages fit its list (the others go through the tile scan); prefix[qc] = total.
constexpr int kItemPages = 64;
__global__ void __launch_bounds__(1024) item_prefix_kernel(const uint32_t* __restrict__ list_count, int qc,
                                                            int64_t list_cap, uint32_t* __restrict__ prefix) {
  const uint64_t total = block_prefix(
      qc,
      [&](int j) {
        const uint32_t c = list_count[j];
        return (int64_t)c <= list_cap ? (uint64_t)((c + kItemPages - 1) / kItemPages) : 0ull;
      },
      [&](int j, uint64_t excl, uint64_t) { prefix[j] = (uint32_t)excl; });
  if (threadIdx.x == 0) prefix[qc] = (uint32_t)total;
}

constexpr int kListThreads = 512;
constexpr int kListStage = 64;
constexpr int kListAhead = 4;  // groups of 32 summaries whose loads a warp issues together

__device__ __forceinline__ void list_flush(uint32_t* s_row, float* s_lb, int nflush, int lane, uint32_t* count,
                                           uint32_t* out_rows, float* out_lb, int64_t cap, uint32_t* status) {
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(count, (uint32_t)nflush);
  base = __shfl_sync(PARIS_FULL_MASK, base, 0);
  for (int i = lane; i < nflush; i += 32) {
    const uint32_t p = base + i;
    if ((int64_t)p < cap) {
      out_rows[p] = s_row[i];
      out_lb[p] = s_lb[i];
    } else {
      atomicOr(status, DEV_CAND_OVERFLOW);
    }
  }
}

// The lower-bound scan of the chunk's queries whose kept pages fit their lists: work items of
// kItemPages kept pages of one query, a contiguous range of items per CTA (so consecutive items
// mostly share the query and its table); rows are tested exactly as in the one-query scan (fp32
// table, LB^2 * (1 - 2^-16) <= threshold) and kept rows appended to the query's candidate list.
__global__ void __launch_bounds__(kListThreads, 2) lbscan_list_kernel(
    const uint4* __restrict__ sax, const uint32_t* __restrict__ pos_row, int64_t n, const float* __restrict__ qtable,
    int card, const uint32_t* __restrict__ thr, const uint32_t* __restrict__ lists,
    const uint32_t* __restrict__ list_count, int64_t list_cap, const uint32_t* __restrict__ prefix, int qc,
    uint32_t* __restrict__ count, uint32_t* __restrict__ out_rows, float* __restrict__ out_lb, int64_t cap,
    uint32_t* __restrict__ status, int stop_on_overflow, unsigned long long* __restrict__ rows_tested) {
  extern __shared__ __align__(16) float s_tab[];
  __shared__ uint32_t s_stage_row[kListThreads / 32][kListStage];
  __shared__ float s_stage_lb[kListThreads / 32][kListStage];
  __shared__ int s_q, s_skip;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  constexpr int kGpp = kPageRows / 32;
  uint32_t offp[8];
  fp32_table_offsets(lane, offp);
  const uint32_t tab = (uint32_t)__cvta_generic_to_shared(s_tab);
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t* st_row = s_stage_row[wib];
  float* st_lb = s_stage_lb[wib];
  const int64_t total = prefix[qc];
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(total, i0 + per);
  int cur = -1;
  float t = 0.f;
  unsigned long long tested = 0;
  int qw = 0;  // thread 0: query of the current item (items of a CTA are consecutive)
  if (threadIdx.x == 0 && i0 < i1) {  // last j with prefix[j] <= i0
    int lo = 0, hi = qc;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)prefix[mid] <= i0) lo = mid; else hi = mid;
    }
    qw = lo;
  }
  for (int64_t item = i0; item < i1; ++item) {
    __syncthreads();  // the previous item's flags and table are no longer read
    if (threadIdx.x == 0) {
      while (qw + 1 < qc && (int64_t)prefix[qw + 1] <= item) ++qw;  // also skips queries without items
      s_q = qw;
      s_skip = stop_on_overflow && (int64_t)__ldcg(count + qw) > cap;
    }
    __syncthreads();
    const int q = s_q;
    if (q != cur) {
      load_fp32_table(qtable + (int64_t)q * card * 16, card, s_tab);
      t = __uint_as_float(thr[q]);
      cur = q;
    }
    __syncthreads();
    if (s_skip) continue;
    const int64_t j = item - prefix[q];
    const int64_t kept = min((int64_t)list_count[q], list_cap);
    const int64_t p0 = j * kItemPages, p1 = min(kept, p0 + kItemPages);
    const int64_t groups = (p1 - p0) * kGpp;
    const uint32_t* lst = lists + (int64_t)q * list_cap;
    uint32_t* qrows = out_rows + (int64_t)q * cap;
    float* qlb = out_lb + (int64_t)q * cap;
    int fill = 0;
    const int nw = blockDim.x >> 5;
    // kListAhead groups of 32 summaries per warp and round: their loads are in flight together
    for (int64_t g0 = wib; g0 < groups; g0 += (int64_t)kListAhead * nw) {
      int64_t pa[kListAhead];
      uint4 wa[kListAhead];
#pragma unroll
      for (int a = 0; a < kListAhead; ++a) {
        const int64_t g = g0 + (int64_t)a * nw;
        pa[a] = g < groups ? ((int64_t)lst[p0 + g / kGpp] * kGpp + g % kGpp) * 32 + lane : n;
      }
#pragma unroll
      for (int a = 0; a < kListAhead; ++a) wa[a] = pa[a] < n ? __ldcs(sax + pa[a]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int a = 0; a < kListAhead; ++a) {
        const int64_t pos = pa[a];
        const uint4 word = wa[a];
        const uint32_t wv[4] = {word.x, word.y, word.z, word.w};
        float lb = 0.f;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          const uint32_t sel = (4u + 2u * (kk & 1)) | ((uint32_t)(kk & 3) << 4) | (5u << 8) | (5u << 12);
          const uint32_t addr = tab + __byte_perm(wv[kk >> 2], offp[kk >> 1], sel);
          float v;
          asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
          lb += v;
        }
        const bool keep = pos < n && lb * kPageKeepScale <= t;
        tested += pos < n ? 1u : 0u;
        const uint32_t mk = __ballot_sync(PARIS_FULL_MASK, keep);
        if (mk) {
          if (keep) {
            const int p = fill + __popc(mk & lt_mask);
            st_row[p] = pos_row[pos];
            st_lb[p] = lb;
          }
          fill += __popc(mk);
          __syncwarp();
          if (fill >= 32) {
            list_flush(st_row, st_lb, 32, lane, count + q, qrows, qlb, cap, status);
            __syncwarp();
            if (lane < fill - 32) {
              st_row[lane] = st_row[32 + lane];
              st_lb[lane] = st_lb[32 + lane];
            }
            fill -= 32;
            __syncwarp();
          }
        }
      }
    }
    if (fill > 0) list_flush(st_row, st_lb, fill, lane, count + q, qrows, qlb, cap, status);
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) tested += __shfl_xor_sync(PARIS_FULL_MASK, tested, o);
  if (lane == 0 && tested) atomicAdd(rows_tested, tested);
}

int sm_count_leaf() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

int64_t page_count(int64_t n) { return (n + kPageRows - 1) / kPageRows; }
int64_t page_words(int64_t n) { return (page_count(n) + 31) / 32; }
int64_t page_list_cap(int64_t n) { return std::min<int64_t>(page_count(n), 32768); }

paris_status build_leaf_envelopes(paris_index* idx, cudaStream_t st) {
  const int64_t n = idx->n, npages = page_count(n), nsuper = (npages + 15) / 16;
  idx->npages = npages;
  idx->sax_sorted = (uint8_t*)dev_alloc((size_t)n * PARIS_SAX_BYTES, st);
  idx->env = (uint8_t*)dev_alloc((size_t)(npages + nsuper) * 32, st);
  if (!idx->sax_sorted || !idx->env) return fail(PARIS_ENOMEM, "index-order summaries and leaf envelopes");
  const int sms = sm_count_leaf();
  const int64_t g1 = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16);
  sorted_summaries_kernel<<<(unsigned)std::max<int64_t>(g1, 1), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(idx->sax), idx->rows_sorted, n, reinterpret_cast<uint4*>(idx->sax_sorted));
  const int64_t g2 = std::min<int64_t>((npages + 7) / 8, (int64_t)sms * 8);
  page_env_kernel<<<(unsigned)std::max<int64_t>(g2, 1), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(idx->sax_sorted), n, npages, reinterpret_cast<uint4*>(idx->env));
  uint4* senv = reinterpret_cast<uint4*>(idx->env) + 2 * npages;
  super_env_kernel<<<(unsigned)std::max<int64_t>((nsuper + 255) / 256, 1), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(idx->env), npages, nsuper, senv);
  note_launches(3);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status launch_page_lb(const paris_index* idx, const QueryState& qs, int64_t q0, int64_t nq, uint32_t* bits,
                            uint32_t* lists, uint32_t* list_count, int64_t list_cap, cudaStream_t st,
                            bool stop_over_cap) {
  if (nq <= 0) return PARIS_OK;
  if (!qs.qsym) return fail(PARIS_EINTERNAL, "query symbols were not prepared");
  const int64_t words = page_words(idx->n), npages = idx->npages, nsuper = (npages + 15) / 16;
  if (bits) PARIS_CUDA(cudaMemsetAsync(bits, 0, (size_t)nq * words * 4, st));
  PARIS_CUDA(cudaMemsetAsync(list_count, 0, (size_t)nq * 4, st));
  const size_t smem = (size_t)idx->card * 64 * sizeof(float);
  PARIS_CUDA(cudaFuncSetAttribute(page_lb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // one query: enough blocks to cover the super pages once; many queries: one block per query
  // (the table is loaded once per block and each warp walks many words)
  const int wpb = kPageThreads / 32;
  const int64_t sw = (nsuper + 31) / 32;
  const int64_t bx = nq == 1 ? std::max<int64_t>(1, (sw + wpb - 1) / wpb) : 1;
  dim3 grid((unsigned)bx, (unsigned)nq);
  const uint4* env = reinterpret_cast<const uint4*>(idx->env);
  page_lb_kernel<<<grid, kPageThreads, smem, st>>>(env + 2 * npages, nsuper, env, npages, words,
                                                  qs.qtable + q0 * (int64_t)idx->card * 16, qs.qsym + q0 * 16,
                                                  qs.thr + q0, idx->card, bits, lists, list_count, list_cap,
                                                  qs.counters + 5, stop_over_cap ? 1 : 0);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status launch_lbscan_lists(const paris_index* idx, const QueryState& qs, const ChunkState& cs,
                                 int stop_on_overflow, uint32_t* status, cudaStream_t st) {
  if (cs.qc <= 0) return PARIS_OK;
  const int64_t list_cap = page_list_cap(idx->n);
  item_prefix_kernel<<<1, 1024, 0, st>>>(cs.page_count, cs.qc, list_cap, cs.item_prefix);
  const size_t smem = (size_t)idx->card * 64 * sizeof(float);
  PARIS_CUDA(cudaFuncSetAttribute(lbscan_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = sm_count_leaf() * 2;
  lbscan_list_kernel<<<grid, kListThreads, smem, st>>>(
      reinterpret_cast<const uint4*>(idx->sax_sorted), idx->rows_sorted, idx->n,
      qs.qtable + cs.q0 * (int64_t)idx->card * 16, idx->card, qs.thr + cs.q0, cs.page_list, cs.page_count, list_cap,
      cs.item_prefix, cs.qc, cs.count, cs.rows, cs.lb, cs.cap, status, stop_on_overflow, qs.counters + 6);
  note_launches(2);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

}  // namespace paris
