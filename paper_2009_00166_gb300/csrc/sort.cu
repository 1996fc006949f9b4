// Index build, step 2: order rows by (top 64 key bits, row) with a stable LSD radix sort.
// This replaces the paper's per-root-subtree receive buffers and leaf splitting (Alg. 2-3):
// a trie node of the ADS+ index is a run of this order sharing a key prefix.
#include "internal.h"

namespace paris {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_IPT = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;

// Per-block digit counts (one private histogram per warp, summed at the end).
__global__ void __launch_bounds__(RS_THREADS) radix_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                         int shift, uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t h[RS_WARPS][256];
  for (int w = 0; w < RS_WARPS; ++w) h[w][threadIdx.x] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int j = 0; j < RS_IPT; ++j) {
    int64_t i = base + j * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[warp][(uint32_t)(__ldcs(keys + i) >> shift) & 255u], 1u);
  }
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) c += h[w][threadIdx.x];
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = c;
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024); returns the total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& excl, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(PARIS_FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(PARIS_FULL_MASK, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;  // inclusive prefix of warp totals
  }
  __syncthreads();
  uint32_t before = warp ? s_warp[warp - 1] : 0u;
  uint32_t total = s_warp[nw - 1];
  excl = before + x - v;
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles(uint32_t* __restrict__ a, int64_t m,
                                                            uint32_t* __restrict__ sums) {
  __shared__ uint32_t s_warp[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  uint32_t v[SCAN_IPT], tot = 0;
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    v[j] = base + j < m ? a[base + j] : 0u;
    tot += v[j];
  }
  uint32_t excl;
  uint32_t total = block_exclusive_scan(tot, excl, s_warp);
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    if (base + j < m) a[base + j] = excl;
    excl += v[j];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_sums_single(uint32_t* __restrict__ sums, int64_t m) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < m; base += SCAN_THREADS) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < m ? sums[i] : 0u;
    uint32_t excl;
    uint32_t total = block_exclusive_scan(v, excl, s_warp);
    if (i < m) sums[i] = excl + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_add(uint32_t* __restrict__ a, int64_t m,
                                                          const uint32_t* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  uint32_t add = sums[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j)
    if (base + j < m) a[base + j] += add;
}

struct ScatterSmem {
  uint64_t key[RS_TILE];
  uint32_t row[RS_TILE];
  uint32_t wcnt[RS_WARPS][256];  // per-warp digit counts, then each warp's offset within its digit
  uint32_t start[256];
  uint32_t s_warp[32];
};

// One stable pass: each warp ranks a contiguous run of RS_IPT x 32 keys of the block's tile by
// digit (match_any groups the lanes of equal digit, a warp-private running count orders the
// rounds), one block-wide scan turns the per-warp counts into offsets, the tile is reordered by
// digit in shared memory and written out in runs of equal digit.
__global__ void __launch_bounds__(RS_THREADS) radix_scatter(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ rin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ rout, int64_t n, int shift, const uint32_t* __restrict__ offs, int nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem& S = *reinterpret_cast<ScatterSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const int64_t wbase = base + (int64_t)warp * (RS_IPT * 32);
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int q = 0; q < 8; ++q) S.wcnt[warp][lane * 8 + q] = 0u;
  uint64_t key[RS_IPT];
  uint32_t row[RS_IPT];
  uint32_t rank[RS_IPT];
#pragma unroll
  for (int j = 0; j < RS_IPT; ++j) {
    const int64_t i = wbase + j * 32 + lane;
    const bool valid = i < n;
    key[j] = valid ? kin[i] : 0ull;
    row[j] = valid ? (rin ? rin[i] : (uint32_t)i) : 0u;
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < RS_IPT; ++j) {
    const int64_t i = wbase + j * 32 + lane;
    const uint32_t d = i < n ? ((uint32_t)(key[j] >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(PARIS_FULL_MASK, d);
    const uint32_t before = d < 256u ? S.wcnt[warp][d] : 0u;
    rank[j] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (d < 256u && lane == __ffs(peers) - 1) S.wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int w2 = 0; w2 < RS_WARPS; ++w2) {
    const uint32_t c = S.wcnt[w2][t];
    S.wcnt[w2][t] = tot;
    tot += c;
  }
  uint32_t excl;
  const uint32_t total = block_exclusive_scan(tot, excl, S.s_warp);
  S.start[t] = excl;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RS_IPT; ++j) {
    const int64_t i = wbase + j * 32 + lane;
    if (i < n) {
      const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
      const uint32_t p = S.start[d] + S.wcnt[warp][d] + rank[j];
      S.key[p] = key[j];
      S.row[p] = row[j];
    }
  }
  __syncthreads();
  for (uint32_t p = t; p < total; p += RS_THREADS) {
    const uint64_t k = S.key[p];
    const uint32_t d = (uint32_t)(k >> shift) & 255u;
    const uint32_t o = offs[(int64_t)d * nblocks + blockIdx.x] + (p - S.start[d]);
    kout[o] = k;
    rout[o] = S.row[p];
  }
}

}  // namespace

paris_status exclusive_scan(uint32_t* a, int64_t m, cudaStream_t st) {
  int64_t tiles = (m + SCAN_TILE - 1) / SCAN_TILE;
  DevBuf sums;
  if (!sums.alloc((size_t)tiles * sizeof(uint32_t), st)) return fail(PARIS_ENOMEM, "scan scratch");
  scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(a, m, sums.as<uint32_t>());
  scan_sums_single<<<1, SCAN_THREADS, 0, st>>>(sums.as<uint32_t>(), tiles);
  scan_add<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(a, m, sums.as<uint32_t>());
  note_launches(3);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status radix_sort_index(uint64_t* keys, uint32_t* rows, int64_t n, cudaStream_t st) {
  if (n <= 1) {
    if (n == 1) PARIS_CUDA(cudaMemsetAsync(rows, 0, sizeof(uint32_t), st));
    return PARIS_OK;
  }
  const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
  const int64_t m = (int64_t)256 * nblocks;
  DevBuf kalt, ralt, hist;
  if (!kalt.alloc((size_t)n * 8, st) || !ralt.alloc((size_t)n * 4, st) || !hist.alloc((size_t)m * 4, st))
    return fail(PARIS_ENOMEM, "radix sort scratch (%lld rows)", (long long)n);
  // set on every call: the attribute is per device, and a cached flag would not be thread-safe
  PARIS_CUDA(cudaFuncSetAttribute(radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(ScatterSmem)));
  uint64_t* kbuf[2] = {keys, kalt.as<uint64_t>()};
  uint32_t* rbuf[2] = {rows, ralt.as<uint32_t>()};
  for (int pass = 0; pass < 8; ++pass) {
    int src = pass & 1, dst = src ^ 1;
    int shift = 8 * pass;
    radix_hist<<<nblocks, RS_THREADS, 0, st>>>(kbuf[src], n, shift, hist.as<uint32_t>(), nblocks);
    PARIS_CUDA(cudaGetLastError());
    PARIS_TRY(exclusive_scan(hist.as<uint32_t>(), m, st));
    radix_scatter<<<nblocks, RS_THREADS, sizeof(ScatterSmem), st>>>(
        kbuf[src], pass == 0 ? nullptr : rbuf[src], kbuf[dst], rbuf[dst], n, shift,
        hist.as<uint32_t>(), nblocks);
    note_launches(2);
    PARIS_CUDA(cudaGetLastError());
  }
  // 8 passes: the sorted data is back in (keys, rows)
  return PARIS_OK;
}

}  // namespace paris
