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

// Page lower bounds of one query per blockIdx.y against every page. Lane l of a warp takes page
// 32 t + l, whose envelope is rotated by l mod 16; the query's symbols are rotated the same way
// once, so the clamped word is formed with byte-wise SIMD min/max and looked up in the query's
// fp32 table exactly like a row's summary (two copies of the table, one per half-warp, so the
// 32 lookups of a step fall in 32 different banks). Writes one bit per page (kept) to
// bits[q][words], and, when `list` is given (one query), appends the kept pages to it.
__global__ void __launch_bounds__(kPageThreads) page_lb_kernel(
    const uint4* __restrict__ env, int64_t npages, int64_t words, const float* __restrict__ qtable,
    const uint8_t* __restrict__ qsym, const uint32_t* __restrict__ thr, int card, uint32_t* __restrict__ bits,
    uint32_t* __restrict__ list, uint32_t* __restrict__ list_count, unsigned long long* __restrict__ pages_kept) {
  extern __shared__ __align__(16) float s_tab[];
  const int64_t q = blockIdx.y;
  const float* table = qtable + q * (int64_t)card * 16;
  for (int e = threadIdx.x; e < card * 16; e += blockDim.x) {
    const float v = table[e];
    const int c = e >> 4, i = e & 15;
    s_tab[c * 64 + i] = v;
    s_tab[c * 64 + 16 + i] = v;
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint4 sq = rot_bytes(*reinterpret_cast<const uint4*>(qsym + q * 16), lane & 15);
  const float t = __uint_as_float(thr[q]);
  uint32_t offp[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const uint32_t o0 = 4u * (16u * (lane >> 4) + ((2 * m + lane) & 15));
    const uint32_t o1 = 4u * (16u * (lane >> 4) + ((2 * m + 1 + lane) & 15));
    offp[m] = o0 | (o1 << 16);
  }
  __syncthreads();
  const uint32_t tab = (uint32_t)__cvta_generic_to_shared(s_tab);
  unsigned long long kept = 0;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wd = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; wd < words; wd += nw) {
    const int64_t pg = wd * 32 + lane;
    const bool valid = pg < npages;
    uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
    if (valid) {
      lo = __ldg(env + 2 * pg);
      hi = __ldg(env + 2 * pg + 1);
    }
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
    const bool keep = valid && lb * kPageKeepScale <= t;
    const uint32_t m = __ballot_sync(PARIS_FULL_MASK, keep);
    if (lane == 0) bits[q * words + wd] = m;
    kept += __popc(m);
    if (list && m) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(list_count, (uint32_t)__popc(m));
      base = __shfl_sync(PARIS_FULL_MASK, base, 0);
      if (keep) list[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)pg;
    }
  }
  if (lane == 0 && kept && pages_kept) atomicAdd(pages_kept, kept);
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

paris_status build_leaf_envelopes(paris_index* idx, cudaStream_t st) {
  const int64_t n = idx->n, npages = page_count(n);
  idx->npages = npages;
  idx->sax_sorted = (uint8_t*)dev_alloc((size_t)n * PARIS_SAX_BYTES, st);
  idx->env = (uint8_t*)dev_alloc((size_t)npages * 32, st);
  if (!idx->sax_sorted || !idx->env) return fail(PARIS_ENOMEM, "index-order summaries and leaf envelopes");
  const int sms = sm_count_leaf();
  const int64_t g1 = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16);
  sorted_summaries_kernel<<<(unsigned)std::max<int64_t>(g1, 1), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(idx->sax), idx->rows_sorted, n, reinterpret_cast<uint4*>(idx->sax_sorted));
  const int64_t g2 = std::min<int64_t>((npages + 7) / 8, (int64_t)sms * 8);
  page_env_kernel<<<(unsigned)std::max<int64_t>(g2, 1), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(idx->sax_sorted), n, npages, reinterpret_cast<uint4*>(idx->env));
  note_launches(2);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status launch_page_lb(const paris_index* idx, const QueryState& qs, int64_t q0, int64_t nq, uint32_t* bits,
                            uint32_t* list, uint32_t* list_count, cudaStream_t st) {
  if (nq <= 0) return PARIS_OK;
  if (!qs.qsym) return fail(PARIS_EINTERNAL, "query symbols were not prepared");
  const int64_t words = page_words(idx->n);
  const size_t smem = (size_t)idx->card * 64 * sizeof(float);
  PARIS_CUDA(cudaFuncSetAttribute(page_lb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // one query: enough blocks to cover the pages once; many queries: one block per query (the
  // table is loaded once per block and each warp walks many words)
  const int wpb = kPageThreads / 32;
  const int64_t bx = nq == 1 ? std::max<int64_t>(1, (words + wpb - 1) / wpb) : 1;
  dim3 grid((unsigned)bx, (unsigned)nq);
  page_lb_kernel<<<grid, kPageThreads, smem, st>>>(reinterpret_cast<const uint4*>(idx->env), idx->npages, words,
                                                  qs.qtable + q0 * (int64_t)idx->card * 16, qs.qsym + q0 * 16,
                                                  qs.thr + q0, idx->card, bits, list, list_count, qs.counters + 5);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

}  // namespace paris
