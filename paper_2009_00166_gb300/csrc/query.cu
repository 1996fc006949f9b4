// Query-path kernels: query preparation, approximate search, lower-bound scan with compaction,
// early-abandoning refinement with an atomic best-so-far, k-th selection and exact re-rank
// (ParIS+ Sec. 3.3, Alg. 7-9).
#include <math_constants.h>

#include <algorithm>

#include "query.cuh"

namespace paris {

namespace {

constexpr float kKeepScale = 1.0f - 1.0f / 65536.0f;  // LB^2 * (1 - 2^-16): fp32 LB error margin
constexpr int kDescentThreads = 256;
constexpr int kLbThreads = 512;
constexpr int kLbUnroll = 4;
constexpr int kRefineThreads = 256;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(PARIS_FULL_MASK, v, o);
  return v;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ __forceinline__ uint32_t up_scaled_bits(float f, float cg) {
  return __float_as_uint(__fmul_ru(f, cg));
}

// Query vector of one warp: lane holds float4 number lane + 32 t (vector path) .
template <int ITERS>
struct QVec {
  float4 v[ITERS];
  __device__ __forceinline__ void load(const float* q, int len, int lane) {
#pragma unroll
    for (int t = 0; t < ITERS; ++t) {
      int i4 = lane + 32 * t;
      v[t] = (4 * i4 < len) ? reinterpret_cast<const float4*>(q)[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
};

__device__ __forceinline__ float sq4(float4 a, float4 b, float acc) {
  float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
  acc = fmaf(d0, d0, acc);
  acc = fmaf(d1, d1, acc);
  acc = fmaf(d2, d2, acc);
  acc = fmaf(d3, d3, acc);
  return acc;
}

// fp32 squared Euclidean distance of one row to the warp's query, abandoning (returning +inf)
// once a prefix sum exceeds `abandon` (Alg. 9 refinement with early abandoning).
template <int ITERS>
__device__ __forceinline__ float warp_sq_dist_vec(const float* __restrict__ x, const QVec<ITERS>& q,
                                                  int len, int lane, float abandon) {
  // sweeps between abandon checks: rows of up to 256 values are loaded at once (one round trip)
  constexpr int CH = ITERS >= 4 ? ITERS / 4 : ITERS;
  float acc = 0.f;
#pragma unroll
  for (int t0 = 0; t0 < ITERS; t0 += CH) {
    float4 xv[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      int i4 = lane + 32 * (t0 + c);
      xv[c] = (4 * i4 < len) ? __ldcs(reinterpret_cast<const float4*>(x) + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) acc = sq4(xv[c], q.v[t0 + c], acc);
    if (t0 + CH < ITERS) {
      float part = warp_sum(acc);
      if (part > abandon) return CUDART_INF_F;
    }
  }
  float tot = warp_sum(acc);
  return tot > abandon ? CUDART_INF_F : tot;
}

// fp32 squared distances of R rows to the warp's query (no abandoning): all R rows' loads are
// issued before the first sum, so a warp keeps R rows in flight.
template <int ITERS, int R>
__device__ __forceinline__ void warp_sq_dist_rows(const float* const (&x)[R], const QVec<ITERS>& q, int len,
                                                  int lane, float (&out)[R]) {
  float4 xv[R][ITERS];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int t = 0; t < ITERS; ++t) {
      const int i4 = lane + 32 * t;
      xv[r][t] = (4 * i4 < len) ? __ldcs(reinterpret_cast<const float4*>(x[r]) + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < ITERS; ++t) acc = sq4(xv[r][t], q.v[t], acc);
    out[r] = warp_sum(acc);
  }
}

__device__ __forceinline__ float warp_sq_dist_scalar(const float* __restrict__ x, const float* __restrict__ q,
                                                     int len, int lane, float abandon) {
  float acc = 0.f;
  for (int j = lane; j < len; j += 32) {
    float d = x[j] - q[j];
    acc = fmaf(d, d, acc);
  }
  float tot = warp_sum(acc);
  return tot > abandon ? CUDART_INF_F : tot;
}

// ------------------------------------------------------------------------------ query prep
// PAA, symbols and key of each query (as in the build), and its lower-bound table:
// T[c][i] = (len/w) * d_i(c)^2, d_i(c) = distance from PAA_i to the interval of symbol c
// (Sec. 3.3.1: ABOVE / BELOW / IN), shrunk by a bound on the FP64 rounding of both PAA values
// and rounded down to fp32, so that every table sum stays below the exact MINDIST^2.
template <int SEGV>
__global__ void __launch_bounds__(256) prep_kernel(const float* __restrict__ queries, int64_t nq, RowShape sh,
                                                   int card, int bits, const uint64_t* __restrict__ beta_keys_g,
                                                   const double* __restrict__ beta_ext, double* __restrict__ qpaa,
                                                   uint64_t* __restrict__ qkey, float* __restrict__ qtable,
                                                   uint8_t* __restrict__ qsym, uint32_t* __restrict__ status) {
  __shared__ uint64_t beta_keys[255];
  __shared__ uint8_t sym_tab[kSymBuckets];
  for (int i = threadIdx.x; i < card - 1; i += blockDim.x) beta_keys[i] = beta_keys_g[i];
  __syncthreads();
  build_symbol_table(beta_keys, card, sym_tab);
  __syncthreads();
  const int lane = threadIdx.x & 31, half = lane >> 4, seg = lane & 15;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t pairs = (nq + 1) >> 1;
  for (int64_t pr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pr < pairs; pr += warps) {
    const int64_t q0 = 2 * pr;
    const bool has1 = q0 + 1 < nq;
    const float* row0 = queries + q0 * (int64_t)sh.len;
    double paa = 0.0;
    float fest = 0.f;
    if (!lane_segment_paa<SEGV>(row0, has1 ? row0 + sh.len : nullptr, sh, lane, paa, fest))
      atomicOr(status, DEV_NONFINITE);
    const int64_t q = q0 + half;
    const bool qv = half == 0 || has1;
    const int sym = (qv && seg < sh.w) ? symbol_of(paa, fest, beta_keys, sym_tab, card) : 0;
    const uint64_t key = warp_pair_key64(sym, lane, sh.w, bits);
    if (!qv) continue;
    qpaa[q * 16 + seg] = seg < sh.w ? paa : 0.0;
    if (qsym) qsym[q * 16 + seg] = (uint8_t)sym;  // 0 past w, like the summaries' unused slots
    if (seg == 0) qkey[q] = key;
  }
}

// The lower-bound table, one entry per thread: T[c][i] for queries blockIdx.y + j * gridDim.y; a block covers 16
// symbols of all 16 segments. Every FP64 value is held between its fp32 roundings down and up
// (the query's PAA per segment, the block's 17 region ends), and the distance from the PAA to
// region c is bounded from below in fp32 with rounding toward -inf: d = rd(lo- - P+) below the
// region, rd(P- - hi+) above it, 0 otherwise; T = rd(rd(d * d) * s) <= s * (exact distance)^2.
__global__ void __launch_bounds__(256) qtable_kernel(const double* __restrict__ qpaa, int64_t nq, int card, int w,
                                                     float scale, const double* __restrict__ beta_ext,
                                                     float* __restrict__ qtable) {
  __shared__ float2 s_p[16];  // PAA of each segment: (round down, round up)
  __shared__ float2 s_b[17];  // region ends c0 .. c0 + 16: (round down, round up)
  const int c0 = blockIdx.x * 16;
  const int e = c0 * 16 + threadIdx.x;
  const int cl = threadIdx.x >> 4, seg = threadIdx.x & 15;
  for (int64_t q = blockIdx.y; q < nq; q += gridDim.y) {  // the grid's y extent is capped at 65535
    __syncthreads();  // the previous query's values are no longer read
    if (threadIdx.x < 16) {
      const double P = qpaa[q * 16 + threadIdx.x];
      s_p[threadIdx.x] = make_float2(__double2float_rd(P), __double2float_ru(P));
    } else if (threadIdx.x < 33 && c0 + (int)threadIdx.x - 16 <= card) {
      const double b = beta_ext[c0 + threadIdx.x - 16];
      s_b[threadIdx.x - 16] = make_float2(__double2float_rd(b), __double2float_ru(b));
    }
    __syncthreads();
    if (e >= card * 16) continue;
    float val = 0.f;
    if (seg < w) {
      const float2 p = s_p[seg];
      const float lo = s_b[cl].x, hi = s_b[cl + 1].y;
      float d = 0.f;
      if (p.y < lo) d = __fsub_rd(lo, p.y);
      else if (p.x > hi) d = __fsub_rd(p.x, hi);
      val = __fmul_rd(__fmul_rd(d, d), scale);
    }
    qtable[q * (int64_t)card * 16 + e] = val;
  }
}

// --------------------------------------------------------------------- approximate search
__device__ int64_t cta_lower_bound(const uint64_t* __restrict__ keys, int64_t n, uint64_t x,
                                   int64_t* s_bounds) {
  const int t = threadIdx.x;
  if (t == 0) {
    s_bounds[0] = 0;
    s_bounds[1] = n;
  }
  __syncthreads();
  while (true) {
    int64_t lo = s_bounds[0], hi = s_bounds[1];
    if (hi - lo <= kDescentThreads) break;
    int64_t p = lo + ((hi - lo) * (t + 1)) / (kDescentThreads + 1);
    int pred = keys[p] < x;
    int cnt = __syncthreads_count(pred);
    if (t == cnt - 1) s_bounds[0] = p + 1;
    if (t == cnt) s_bounds[1] = p;
    __syncthreads();
  }
  int64_t lo = s_bounds[0], hi = s_bounds[1];
  int pred = (lo + t < hi) && keys[lo + t] < x;
  int cnt = __syncthreads_count(pred);
  return lo + cnt;
}

__device__ __forceinline__ int smem_lower_bound(const uint64_t* a, int m, uint64_t x) {
  int lo = 0;
  while (m > 0) {
    int h = m >> 1;
    if (a[lo + h] < x) {
      lo += h + 1;
      m -= h + 1;
    } else {
      m = h;
    }
  }
  return lo;
}
__device__ __forceinline__ int smem_upper_bound(const uint64_t* a, int m, uint64_t x) {
  int lo = 0;
  while (m > 0) {
    int h = m >> 1;
    if (a[lo + h] <= x) {
      lo += h + 1;
      m -= h + 1;
    } else {
      m = h;
    }
  }
  return lo;
}

// One CTA per query: for each of the query's nk keys (its own key first, then any learned
// bucket keys), find the leaf of the fixed-order trie that holds that key's position (Sec. 3.3
// approximate search); compute the distance to every series of the distinct leaves and seed the
// best-so-far with the k-th smallest. The leaf range reported is the own key's. With leaf_in
// (adaptive-split leaves, nk = 1) the leaf's range is given, in the order of rows_sorted.
template <int ITERS>
__global__ void __launch_bounds__(kDescentThreads) descent_kernel(
    const float* __restrict__ series, int64_t n, int len, int vec, const uint64_t* __restrict__ keys,
    const uint32_t* __restrict__ rows_sorted, int leaf_cap, int k, const float* __restrict__ queries,
    const uint64_t* __restrict__ qkeys, int nk, int64_t* __restrict__ leaf_out, float* __restrict__ seed_out,
    uint32_t* __restrict__ thr, unsigned long long* __restrict__ bsf, float cg,
    unsigned long long* __restrict__ counters, const int64_t* __restrict__ leaf_in) {
  extern __shared__ __align__(16) uint64_t s_mem[];
  const int Lp = max(leaf_cap, k);
  uint64_t* s_win = s_mem;               // [2 Lp + 1] keys of the window around a position
  uint64_t* s_buf = s_mem + (2 * Lp + 2);  // (F, row) pairs of all visited leaves
  __shared__ int64_t s_bounds[2];
  __shared__ int64_t s_lo[65], s_hi[65];
  __shared__ int s_best;
  __shared__ int64_t s_rng[16][2];
  __shared__ int s_dup;
  const int64_t q = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float* qp = queries + q * (int64_t)len;
  QVec<ITERS> qv;
  if (vec) qv.load(qp, len, lane);
  int filled = 0;
  for (int j = 0; j < nk; ++j) {
    int64_t lo, hi;
    if (leaf_in) {
      lo = leaf_in[2 * q];
      hi = leaf_in[2 * q + 1];
    } else {
    const uint64_t x = qkeys[q * nk + j];
    int64_t pos0 = cta_lower_bound(keys, n, x, s_bounds);
    const bool clamped = pos0 >= n;
    const int64_t pos = clamped ? n - 1 : pos0;
    const uint64_t anchor = keys[pos];
    const int64_t wa = max((int64_t)0, pos - Lp), wb = min(n, pos + Lp + 1);
    const int wn = (int)(wb - wa);
    for (int i = t; i < wn; i += blockDim.x) s_win[i] = keys[wa + i];
    if (t == 0) s_best = 65;
    __syncthreads();
    if (t <= 64) {
      uint64_t mask = t == 0 ? 0ull : (~0ull << (64 - t));
      int64_t lo = wa + smem_lower_bound(s_win, wn, anchor & mask);
      int64_t hi = wa + smem_upper_bound(s_win, wn, anchor | ~mask);
      bool inside = !(lo == wa && wa > 0) && !(hi == wb && wb < n);
      s_lo[t] = lo;
      s_hi[t] = hi;
      if (inside && hi - lo <= Lp) atomicMin(&s_best, t);
    }
    __syncthreads();
    const int best = s_best;
    if (best <= 64) {
      lo = s_lo[best];
      hi = s_hi[best];
      if (hi - lo < k) {
        lo = min(lo, n - k);
        hi = lo + k;
      }
    } else {
      // even the full key is shared by more than Lp rows: take the first Lp rows of that run
      int64_t start = clamped ? cta_lower_bound(keys, n, anchor, s_bounds) : pos;
      lo = start;
      hi = start + Lp;
    }
    }
    if (t == 0) {
      int dup = 0;
      for (int i = 0; i < j && i < 16; ++i) dup |= (s_rng[i][0] == lo && s_rng[i][1] == hi);
      if (j < 16) {
        s_rng[j][0] = lo;
        s_rng[j][1] = hi;
      }
      s_dup = dup;
      if (j == 0) {
        leaf_out[2 * q] = lo;
        leaf_out[2 * q + 1] = hi;
      }
    }
    __syncthreads();
    if (!s_dup) {
      const int m = (int)(hi - lo);
      const int nw = blockDim.x >> 5;
      if (vec) {
        // RR rows per warp and round, their loads in flight together
        constexpr int RR = ITERS >= 8 ? 1 : 8 / ITERS;
        for (int i0 = warp * RR; i0 < m; i0 += nw * RR) {
          uint32_t rw[RR];
          const float* xr[RR];
#pragma unroll
          for (int r = 0; r < RR; ++r) {
            rw[r] = rows_sorted[lo + min(i0 + r, m - 1)];
            xr[r] = series + (int64_t)rw[r] * len;
          }
          float F[RR];
          warp_sq_dist_rows<ITERS, RR>(xr, qv, len, lane, F);
          if (lane == 0)
#pragma unroll
            for (int r = 0; r < RR; ++r)
              if (i0 + r < m) s_buf[filled + i0 + r] = ((unsigned long long)__float_as_uint(F[r]) << 32) | rw[r];
        }
      } else {
        for (int i = warp; i < m; i += nw) {
          uint32_t row = rows_sorted[lo + i];
          const float* xr = series + (int64_t)row * len;
          float F = warp_sq_dist_scalar(xr, qp, len, lane, CUDART_INF_F);
          if (lane == 0) s_buf[filled + i] = ((unsigned long long)__float_as_uint(F) << 32) | row;
        }
      }
      filled += m;
    }
    __syncthreads();
  }
  int P2 = 1;
  while (P2 < filled) P2 <<= 1;
  for (int i = filled + t; i < P2; i += blockDim.x) s_buf[i] = ~0ull;
  __syncthreads();
  // bitonic sort of (F, row) pairs, ascending
  for (int size = 2; size <= P2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = t; i < (P2 >> 1); i += blockDim.x) {
        int p = 2 * i - (i & (stride - 1));
        int r = p + stride;
        bool asc = (p & size) == 0;
        uint64_t a = s_buf[p], b = s_buf[r];
        if ((a > b) == asc) {
          s_buf[p] = b;
          s_buf[r] = a;
        }
      }
      __syncthreads();
    }
  }
  if (t == 0) {
    uint64_t kth = s_buf[k - 1];
    float Fk = __uint_as_float((uint32_t)(kth >> 32));
    seed_out[q] = Fk;
    thr[q] = up_scaled_bits(Fk, cg);
    bsf[q] = s_buf[0];
    atomicAdd(&counters[3], (unsigned long long)filled);
  }
}

// ------------------------------------------------------------------ lower-bound scan (Alg. 8)
// One pass over the summary array for one query. Each lane owns one row of a 32-row group;
// the table is stored twice, symbol-major, so that the 16 lookups of a row never collide in
// a shared-memory bank: row r keeps its symbols rotated by r mod 16 (build), so at step k the
// 16 lanes of a half-warp read 16 different segments, and the two half-warps read different
// copies. A byte permute forms each lookup address from the symbol byte and a per-lane offset.
// Kept rows are staged per warp in shared memory and written out 32 at a time, so the global
// candidate counter sees one atomic per 32 kept rows.
constexpr int kStage = 64;  // staged (row, lb) pairs per warp

// Writes out nflush staged pairs; returns false once the list has overflowed its capacity.
__device__ __forceinline__ bool flush_stage(uint32_t* s_row, float* s_lb, int nflush, int lane,
                                            uint32_t* count, uint32_t* out_rows, float* out_lb, int64_t cap,
                                            uint32_t* status) {
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(count, (uint32_t)nflush);
  base = __shfl_sync(PARIS_FULL_MASK, base, 0);
  for (int i = lane; i < nflush; i += 32) {
    uint32_t p = base + i;
    if ((int64_t)p < cap) {
      out_rows[p] = s_row[i];
      out_lb[p] = s_lb[i];
    } else {
      atomicOr(status, DEV_CAND_OVERFLOW);
    }
  }
  return (int64_t)base + nflush <= cap;
}

// With a page list (leaf pruning), the pass visits only the 32-row groups of the listed pages of
// the index-order summaries and reports each kept position's row (pos_row).
__global__ void __launch_bounds__(kLbThreads, 2) lbscan_kernel(
    const uint4* __restrict__ sax, int64_t n, const float* __restrict__ table, int card,
    const uint32_t* __restrict__ thr_ptr, float thr_value, uint32_t* __restrict__ count,
    uint32_t* __restrict__ out_rows, float* __restrict__ out_lb, int64_t cap,
    uint32_t* __restrict__ status, int stop_on_overflow, const uint32_t* __restrict__ page_list,
    const uint32_t* __restrict__ page_count, const uint32_t* __restrict__ pos_row) {
  extern __shared__ __align__(16) float s_tab[];
  __shared__ uint32_t s_stage_row[kLbThreads / 32][kStage];
  __shared__ float s_stage_lb[kLbThreads / 32][kStage];
  for (int e = threadIdx.x; e < card * 16; e += blockDim.x) {
    float v = table[e];
    int c = e >> 4, i = e & 15;
    s_tab[c * 64 + i] = v;
    s_tab[c * 64 + 16 + i] = v;
  }
  __syncthreads();
  const float thr = thr_ptr ? __uint_as_float(*thr_ptr) : thr_value;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* st_row = s_stage_row[wib];
  float* st_lb = s_stage_lb[wib];
  int fill = 0;  // warp-uniform number of staged pairs
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t offp[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    uint32_t o0 = 4u * (16u * (lane >> 4) + ((2 * m + lane) & 15));
    uint32_t o1 = 4u * (16u * (lane >> 4) + ((2 * m + 1 + lane) & 15));
    offp[m] = o0 | (o1 << 16);
  }
  const uint32_t tab = (uint32_t)__cvta_generic_to_shared(s_tab);
  constexpr int kGpp = kPageRows / 32;  // 32-row groups per page
  const int64_t groups = page_list ? (int64_t)(*page_count) * kGpp : (n + 31) >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t it = gw * kLbUnroll; it < groups; it += W * kLbUnroll) {
    uint4 word[kLbUnroll];
    int64_t pos[kLbUnroll];
#pragma unroll
    for (int u = 0; u < kLbUnroll; ++u) {
      const int64_t v = it + u;
      const int64_t g = page_list ? (v < groups ? (int64_t)page_list[v / kGpp] * kGpp + v % kGpp : n) : v;
      pos[u] = v < groups ? g * 32 + lane : n;
      word[u] = (pos[u] < n) ? __ldcs(sax + pos[u]) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kLbUnroll; ++u) {
      const uint32_t wv[4] = {word[u].x, word[u].y, word[u].z, word[u].w};
      float lb = 0.f;
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const uint32_t sel = (4u + 2u * (kk & 1)) | ((uint32_t)(kk & 3) << 4) | (5u << 8) | (5u << 12);
        uint32_t addr = tab + __byte_perm(wv[kk >> 2], offp[kk >> 1], sel);
        float v;
        asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
        lb += v;
      }
      const bool keep = pos[u] < n && lb * kKeepScale <= thr;
      const uint32_t mk = __ballot_sync(PARIS_FULL_MASK, keep);
      if (mk) {
        if (keep) {
          int p = fill + __popc(mk & lt_mask);
          st_row[p] = pos_row ? pos_row[pos[u]] : (uint32_t)pos[u];
          st_lb[p] = lb;
        }
        fill += __popc(mk);
        __syncwarp();
        if (fill >= 32) {
          // an overflowed list is only a signal (the caller falls back); stop scanning early
          if (!flush_stage(st_row, st_lb, 32, lane, count, out_rows, out_lb, cap, status) && stop_on_overflow) return;
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
  if (fill > 0) flush_stage(st_row, st_lb, fill, lane, count, out_rows, out_lb, cap, status);
}

// --------------------------------------------------------------------- refinement (Alg. 9)
// Per-query candidate segments are padded to multiples of 32 in the flat work space so that a
// 32-candidate step of a warp never spans two queries.
__global__ void __launch_bounds__(1024) chunk_prefix_kernel(const uint32_t* __restrict__ count, int qc, int64_t cap,
                                                             uint32_t* __restrict__ prefix,
                                                             unsigned long long* __restrict__ counters) {
  uint64_t raw = 0;
  const uint64_t total = block_prefix(
      qc,
      [&](int j) {
        const uint64_t c = count[j];
        raw += c;
        const uint64_t m = c < (uint64_t)cap ? c : (uint64_t)cap;
        return (m + 31) & ~(uint64_t)31;
      },
      [&](int j, uint64_t excl, uint64_t) { prefix[j] = (uint32_t)excl; });
  if (threadIdx.x == 0) prefix[qc] = (uint32_t)total;
  for (int o = 16; o > 0; o >>= 1) raw += __shfl_xor_sync(PARIS_FULL_MASK, raw, o);
  if ((threadIdx.x & 31) == 0 && raw) atomicAdd(&counters[0], (unsigned long long)raw);
}

// Each warp step takes 32 candidates of one query (one per lane), re-tests their lower bounds
// against the query's current threshold (Alg. 9: minDist < BSF), then computes, one row at a
// time with the whole warp, the early-abandoning distance of the survivors. A completed
// distance lowers the query's BSF (k = 1: packed atomicMin; k <= 32: through a warp-private
// top-k whose k-th value bounds the query's k-th best). Steps are interleaved across warps, so
// all warps move through the lower-bound-ordered lists together.
template <int ITERS>
__global__ void __launch_bounds__(kRefineThreads) refine_kernel(
    const float* __restrict__ series, int len, int vec, const float* __restrict__ queries, int64_t q0,
    int qc, int64_t cap, const uint32_t* __restrict__ prefix, const uint32_t* __restrict__ count,
    const uint32_t* __restrict__ rows, const float* __restrict__ lbs, float* __restrict__ Fout,
    uint32_t* __restrict__ thr, unsigned long long* __restrict__ bsf, int k, float cg,
    unsigned long long* __restrict__ counters, int private_bsf) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t total = prefix[qc];
  int cur = -1;
  int64_t next_bound = 0, m_cur = 0;
  QVec<ITERS> qv;
  const float* qp = nullptr;
  float best = CUDART_INF_F;  // lane j < have: j-th best completed F of this warp and query
  int have = 0;
  unsigned long long touched = 0, updates = 0;
  // private best-so-far (nb-ParIS+ ablation): the warp's own threshold and best (F, row) for the
  // current query, published to the query's shared ones only when the warp leaves the query
  float tp = CUDART_INF_F;
  unsigned long long pbest = ~0ull;
  uint32_t pthr = 0xffffffffu;
  auto publish = [&](int64_t qi) {
    if (!private_bsf || lane != 0) return;
    if (pbest != ~0ull) atomicMin(bsf + qi, pbest);
    if (pthr != 0xffffffffu && atomicMin(thr + qi, pthr) > pthr) ++updates;
  };
  for (int64_t item0 = gw * 32; item0 < total; item0 += W * 32) {
    if (cur < 0 || item0 >= next_bound) {
      if (cur >= 0) publish(q0 + cur);
      if (cur < 0) {
        int lo = 0, hi = qc;  // last j with prefix[j] <= item0
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if ((int64_t)prefix[mid] <= item0) lo = mid; else hi = mid;
        }
        cur = lo;
      } else {
        while ((int64_t)prefix[cur + 1] <= item0) ++cur;
      }
      next_bound = prefix[cur + 1];
      m_cur = count[cur];
      if (m_cur > cap) m_cur = cap;
      qp = queries + (q0 + cur) * (int64_t)len;
      if (vec) qv.load(qp, len, lane);
      best = CUDART_INF_F;
      have = 0;
      tp = __uint_as_float(ld_volatile_u32(thr + q0 + cur));  // the seed threshold
      pbest = ~0ull;
      pthr = 0xffffffffu;
    }
    const int64_t qi = q0 + cur;
    const int64_t i = item0 - prefix[cur] + lane;
    const bool valid = i < m_cur;
    const int64_t slot = (int64_t)cur * cap + i;
    const uint32_t row = valid ? rows[slot] : 0u;
    const float lbv = valid ? lbs[slot] : CUDART_INF_F;
    float t = private_bsf ? tp : __uint_as_float(ld_volatile_u32(thr + qi));
    uint32_t todo = __ballot_sync(PARIS_FULL_MASK, valid && lbv * kKeepScale <= t);
    float myF = CUDART_INF_F;
    while (todo) {
      const int b = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t r = __shfl_sync(PARIS_FULL_MASK, row, b);
      const float lb_b = __shfl_sync(PARIS_FULL_MASK, lbv, b);
      if (!private_bsf) t = fminf(t, __uint_as_float(ld_volatile_u32(thr + qi)));
      if (lb_b * kKeepScale > t) continue;
      ++touched;
      const float* xr = series + (int64_t)r * len;
      const float F = vec ? warp_sq_dist_vec<ITERS>(xr, qv, len, lane, t) : warp_sq_dist_scalar(xr, qp, len, lane, t);
      if (lane == b) myF = F;
      if (F <= t) {
        if (k == 1) {
          const uint32_t nb = up_scaled_bits(F, cg);
          const unsigned long long packed = ((unsigned long long)__float_as_uint(F) << 32) | r;
          if (private_bsf) {
            pbest = min(pbest, packed);
            pthr = min(pthr, nb);
          } else if (lane == 0) {
            atomicMin(bsf + qi, packed);
            if (atomicMin(thr + qi, nb) > nb) ++updates;
          }
          t = fminf(t, __uint_as_float(nb));
        } else if (k <= 32) {
          uint32_t le = __ballot_sync(PARIS_FULL_MASK, lane < have && best <= F);
          int p = __popc(le);
          if (p < k) {
            float prev = __shfl_up_sync(PARIS_FULL_MASK, best, 1);
            if (lane == p) best = F;
            else if (lane > p && lane < k) best = prev;
            have = min(have + 1, k);
            if (have == k) {
              float kth = __shfl_sync(PARIS_FULL_MASK, best, k - 1);
              uint32_t nb = up_scaled_bits(kth, cg);
              if (private_bsf) {
                pthr = min(pthr, nb);
              } else if (lane == 0 && nb < __float_as_uint(t)) {
                if (atomicMin(thr + qi, nb) > nb) ++updates;
              }
              t = fminf(t, __uint_as_float(nb));
            }
          }
        }
      }
    }
    if (valid) Fout[slot] = myF;
    if (private_bsf) tp = t;
  }
  if (cur >= 0) publish(q0 + cur);
  if (lane == 0 && touched) atomicAdd(&counters[1], touched);
  if (lane == 0 && updates) atomicAdd(&counters[7], updates);
}

// Candidate order for refinement: 32 buckets of LB / (seed threshold), lowest first, so that
// the rows most likely to hold the answer tighten the best-so-far before the others are read.
constexpr int kBuckets = 32;

__device__ __forceinline__ int lb_bucket(float lb, float thr0) {
  if (!(thr0 > 0.f)) return 0;
  int b = (int)(lb * ((float)kBuckets / thr0));
  return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

__global__ void bucket_hist_kernel(const float* __restrict__ lbs, const uint32_t* __restrict__ count, int64_t cap,
                                   const uint32_t* __restrict__ thr, int64_t q0, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kBuckets];
  const int j = blockIdx.y;
  if (threadIdx.x < kBuckets) h[threadIdx.x] = 0u;
  __syncthreads();
  int64_t m = count[j];
  if (m > cap) m = cap;
  const float thr0 = __uint_as_float(thr[q0 + j]);
  const float* lb = lbs + (int64_t)j * cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[lb_bucket(lb[i], thr0)], 1u);
  __syncthreads();
  if (threadIdx.x < kBuckets && h[threadIdx.x]) atomicAdd(&hist[j * kBuckets + threadIdx.x], h[threadIdx.x]);
}

__global__ void bucket_offsets_kernel(uint32_t* __restrict__ hist, int qc) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= qc) return;
  uint32_t acc = 0;
  for (int b = 0; b < kBuckets; ++b) {
    uint32_t c = hist[j * kBuckets + b];
    hist[j * kBuckets + b] = acc;  // becomes the running cursor of bucket b
    acc += c;
  }
}

__global__ void bucket_scatter_kernel(const uint32_t* __restrict__ rows, const float* __restrict__ lbs,
                                      const uint32_t* __restrict__ count, int64_t cap,
                                      const uint32_t* __restrict__ thr, int64_t q0, uint32_t* __restrict__ cursor,
                                      uint32_t* __restrict__ rows2, float* __restrict__ lbs2) {
  const int j = blockIdx.y;
  int64_t m = count[j];
  if (m > cap) m = cap;
  const float thr0 = __uint_as_float(thr[q0 + j]);
  const int64_t base = (int64_t)j * cap;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < m; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const bool valid = i < m;
    float lb = valid ? lbs[base + i] : 0.f;
    uint32_t r = valid ? rows[base + i] : 0u;
    int b = valid ? lb_bucket(lb, thr0) : kBuckets;
    uint32_t peers = __match_any_sync(PARIS_FULL_MASK, b);
    uint32_t pos = 0;
    if (valid && lane == __ffs(peers) - 1) pos = atomicAdd(&cursor[j * kBuckets + b], (uint32_t)__popc(peers));
    pos = __shfl_sync(PARIS_FULL_MASK, pos, __ffs(peers) - 1) + __popc(peers & ((1u << lane) - 1u));
    if (valid) {
      rows2[base + pos] = r;
      lbs2[base + pos] = lb;
    }
  }
}

// ------------------------------------------------------------- k-th selection and re-rank
// Radix selection of the k-th smallest F (as fp32 bits, all non-negative) per query.
__global__ void select_init_kernel(uint32_t* sel_state, uint32_t* hist, int qc, int k) {
  int j = blockIdx.x;
  if (threadIdx.x == 0) {
    sel_state[2 * j] = 0u;
    sel_state[2 * j + 1] = (uint32_t)k;
  }
  for (int b = threadIdx.x; b < 2048; b += blockDim.x) hist[(int64_t)j * 2048 + b] = 0u;
}

__global__ void select_hist_kernel(const float* __restrict__ F, const uint32_t* __restrict__ count,
                                   int64_t cap, const uint32_t* __restrict__ sel_state,
                                   uint32_t* __restrict__ hist, int round) {
  __shared__ uint32_t h[2048];
  const int j = blockIdx.y;
  for (int b = threadIdx.x; b < 2048; b += blockDim.x) h[b] = 0u;
  __syncthreads();
  const int shift = round == 0 ? 21 : (round == 1 ? 10 : 0);
  const int width = round == 2 ? 10 : 11;
  const uint32_t prefix = sel_state[2 * j];
  const int hs = shift + width;  // bits at and above hs are decided
  int64_t m = count[j];
  if (m > cap) m = cap;
  const float* f = F + (int64_t)j * cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = __float_as_uint(f[i]);
    if (hs >= 32 || (b >> hs) == (prefix >> hs)) atomicAdd(&h[(b >> shift) & ((1u << width) - 1u)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 2048; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[(int64_t)j * 2048 + b], h[b]);
}

__global__ void select_pick_kernel(uint32_t* __restrict__ hist, uint32_t* __restrict__ sel_state,
                                   uint32_t* __restrict__ kth, int round) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_found[2];
  const int j = blockIdx.x;
  const int shift = round == 0 ? 21 : (round == 1 ? 10 : 0);
  uint32_t* h = hist + (int64_t)j * 2048;
  if (threadIdx.x == 0) {
    s_found[0] = 0u;
    s_found[1] = 0u;
  }
  // each of 256 threads owns 8 consecutive bins
  uint32_t v[8], tot = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    v[b] = h[threadIdx.x * 8 + b];
    tot += v[b];
  }
  // inclusive prefix over threads
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(PARIS_FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t before = 0;
  for (int w2 = 0; w2 < warp; ++w2) before += s_warp[w2];
  uint32_t excl = before + x - tot;
  const uint32_t rank = sel_state[2 * j + 1];  // 1-based rank still to find
  if (excl < rank && rank <= excl + tot) {
    uint32_t c = excl;
    for (int b = 0; b < 8; ++b) {
      if (c + v[b] >= rank) {
        s_found[0] = (uint32_t)(threadIdx.x * 8 + b);
        s_found[1] = c;
        break;
      }
      c += v[b];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t d = s_found[0];
    sel_state[2 * j] |= d << shift;
    sel_state[2 * j + 1] = rank - s_found[1];
    if (round == 2) kth[j] = sel_state[2 * j];
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 2048; b += blockDim.x) h[b] = 0u;
}

__global__ void kth_from_bsf_kernel(const unsigned long long* __restrict__ bsf, int64_t q0, int qc,
                                    uint32_t* __restrict__ kth) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < qc) kth[j] = (uint32_t)(bsf[q0 + j] >> 32);
}

// Rows whose fp32 distance cannot be separated from the k-th best by the fp32 error bound. An
// overflowed list holds an arbitrary subset of its candidates (possibly fewer than k finite
// distances): its query is screened and selected again, so it names no contenders here.
__global__ void contenders_kernel(const float* __restrict__ F, const uint32_t* __restrict__ rows,
                                  const uint32_t* __restrict__ count, int64_t cap,
                                  const uint32_t* __restrict__ kth, float cg, uint32_t* __restrict__ cont_count,
                                  uint32_t* __restrict__ cont_rows, uint32_t* __restrict__ status) {
  const int j = blockIdx.y;
  const int64_t m = count[j];
  if (m > cap) return;
  const float Tc = __fmul_ru(__uint_as_float(kth[j]), cg);
  const float* f = F + (int64_t)j * cap;
  const uint32_t* r = rows + (int64_t)j * cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (f[i] <= Tc) {
      uint32_t p = atomicAdd(&cont_count[j], 1u);
      if (p < (uint32_t)kContCap) cont_rows[(int64_t)j * kContCap + p] = r[i];
      else atomicOr(status, DEV_CONT_OVERFLOW);
    }
  }
}

// Adds (hi:lo) * 2^off into a little-endian limb array.
__device__ __forceinline__ void limbs_add_u128(uint32_t* acc, uint64_t lo, uint64_t hi, int off) {
  const int li = off >> 5, sh = off & 31;
  uint32_t p[4] = {(uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32)};
  uint32_t s[5];
  if (sh == 0) {
    s[0] = p[0]; s[1] = p[1]; s[2] = p[2]; s[3] = p[3]; s[4] = 0u;
  } else {
    s[0] = p[0] << sh;
#pragma unroll
    for (int m = 1; m < 4; ++m) s[m] = (p[m] << sh) | (p[m - 1] >> (32 - sh));
    s[4] = p[3] >> (32 - sh);
  }
  uint64_t carry = 0;
  for (int m = li; m < kLimbs; ++m) {
    uint64_t add = (m - li < 5) ? s[m - li] : 0u;
    uint64_t tsum = (uint64_t)acc[m] + add + carry;
    acc[m] = (uint32_t)tsum;
    carry = tsum >> 32;
    if (m - li >= 4 && carry == 0) break;
  }
}

// acc += (a - b)^2 exactly; acc's least significant bit is 2^-298.
__device__ void add_exact_sq_diff(uint32_t* acc, float a, float b) {
  uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
  uint32_t ea = (ua >> 23) & 0xffu, eb = (ub >> 23) & 0xffu;
  uint64_t ma = (ua & 0x7fffffu) | (ea ? 0x800000u : 0u);
  uint64_t mb = (ub & 0x7fffffu) | (eb ? 0x800000u : 0u);
  if (ma == 0 && mb == 0) return;
  int oa = (ea ? (int)ea : 1) - 1, ob = (eb ? (int)eb : 1) - 1;  // unit offsets above 2^-149
  int o = ma == 0 ? ob : (mb == 0 ? oa : min(oa, ob));
  int da = ma ? oa - o : 0, db = mb ? ob - o : 0;
  if (da <= 38 && db <= 38) {
    int64_t A = (int64_t)(ma << da), B = (int64_t)(mb << db);
    if (ua >> 31) A = -A;
    if (ub >> 31) B = -B;
    int64_t D = A - B;
    uint64_t M = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
    limbs_add_u128(acc, M * M, __umul64hi(M, M), 2 * o);
    return;
  }
  // far-apart magnitudes: exact difference in 320-bit fixed point, then a schoolbook square
  Wide d;
  wide_zero(d);
  wide_add_f32(d, a);
  wide_add_f32(d, -b);
  if (d.limb[9] >> 31) {
    uint64_t carry = 1;
    for (int i = 0; i < 10; ++i) {
      uint64_t tt = (uint64_t)(~d.limb[i]) + carry;
      d.limb[i] = (uint32_t)tt;
      carry = tt >> 32;
    }
  }
  for (int i = 0; i < 10; ++i) {
    if (!d.limb[i]) continue;
    for (int jj = 0; jj < 10; ++jj) {
      if (!d.limb[jj]) continue;
      uint64_t pr = (uint64_t)d.limb[i] * d.limb[jj];
      limbs_add_u128(acc, pr, 0ull, 32 * (i + jj));
    }
  }
}

__device__ __forceinline__ bool limbs_less(const uint32_t* a, uint32_t ra, const uint32_t* b, uint32_t rb) {
  for (int m = kLimbs - 1; m >= 0; --m)
    if (a[m] != b[m]) return a[m] < b[m];
  return ra < rb;
}

// One CTA per query: exact squared distances of the contenders (warp per contender), then the
// k best by (exact distance, row).
__global__ void __launch_bounds__(256) rerank_kernel(
    const float* __restrict__ series, int len, const float* __restrict__ queries, int64_t q0,
    const uint32_t* __restrict__ cont_count, const uint32_t* __restrict__ cont_rows,
    uint32_t* __restrict__ limbs, int k, int64_t* __restrict__ out_idx, float* __restrict__ out_dist,
    unsigned long long* __restrict__ counters) {
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int m = (int)min(cont_count[j], (uint32_t)kContCap);
  const float* qp = queries + (q0 + j) * (int64_t)len;
  uint32_t* L = limbs + (int64_t)j * kContCap * kLimbs;
  const uint32_t* R = cont_rows + (int64_t)j * kContCap;
  for (int c = warp; c < m; c += blockDim.x >> 5) {
    uint32_t acc[kLimbs];
#pragma unroll
    for (int i = 0; i < kLimbs; ++i) acc[i] = 0u;
    const float* xr = series + (int64_t)R[c] * len;
    for (int e = lane; e < len; e += 32) add_exact_sq_diff(acc, xr[e], qp[e]);
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < kLimbs; ++i) {
      uint64_t s = acc[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(PARIS_FULL_MASK, s, o);
      s += carry;
      if (lane == 0) L[(int64_t)c * kLimbs + i] = (uint32_t)s;
      carry = s >> 32;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    const uint32_t* la = L + (int64_t)a * kLimbs;
    uint32_t ra = R[a];
    int rank = 0;
    for (int b = 0; b < m; ++b)
      if (b != a && limbs_less(L + (int64_t)b * kLimbs, R[b], la, ra)) ++rank;
    if (rank < k) {
      out_idx[(q0 + j) * (int64_t)k + rank] = (int64_t)ra;
      if (out_dist) {
        int top = kLimbs - 1;
        while (top > 0 && la[top] == 0u) --top;
        double v = 0.0;
        for (int i = top; i >= 0 && i >= top - 2; --i) v += ldexp((double)la[i], 32 * i - 298);
        out_dist[(q0 + j) * (int64_t)k + rank] = (float)sqrt(v);
      }
    }
  }
  if (threadIdx.x == 0) atomicAdd(&counters[2], (unsigned long long)m);
}

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int iters_for(int len) {
  int it = (len + 127) / 128;
  return it <= 1 ? 1 : it <= 2 ? 2 : it <= 4 ? 4 : it <= 8 ? 8 : 16;
}

}  // namespace

paris_status launch_query_prep(const paris_index* idx, const QueryState& qs, cudaStream_t st) {
  if (qs.nq <= 0) return PARIS_OK;
  RowShape sh = make_row_shape(idx->len, idx->w, qs.queries);
  int64_t blocks = ((qs.nq + 1) / 2 + 7) / 8;
  int grid = (int)std::min<int64_t>(blocks, (int64_t)sm_count() * 8);
  const int segv = sh.fast ? sh.s / 4 : 1;
#define PREP(SV)                                                                                      \
  prep_kernel<SV><<<grid, 256, 0, st>>>(qs.queries, qs.nq, sh, idx->card, idx->bits, idx->beta_keys, \
                                        idx->beta_ext, qs.qpaa, qs.qkey, qs.qtable, qs.qsym, qs.status)
  switch (segv) {
    case 1: PREP(1); break;
    case 2: PREP(2); break;
    case 4: PREP(4); break;
    case 8: PREP(8); break;
    case 16: PREP(16); break;
    default: PREP(32); break;
  }
#undef PREP
  dim3 tg((unsigned)((idx->card * 16 + 255) / 256), (unsigned)std::min<int64_t>(qs.nq, 65535));
  qtable_kernel<<<tg, 256, 0, st>>>(qs.qpaa, qs.nq, idx->card, idx->w, (float)(idx->len / idx->w), idx->beta_ext,
                                    qs.qtable);
  note_launches(2);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

static bool vec_ok(const paris_index* idx, const float* q) {
  return idx->len % 4 == 0 && idx->len <= 2048 && ((uintptr_t)idx->series % 16u) == 0u &&
         ((uintptr_t)q % 16u) == 0u;
}

paris_status launch_descent(const paris_index* idx, const QueryState& qs, cudaStream_t st, bool adaptive) {
  if (qs.nq <= 0) return PARIS_OK;
  const int64_t* leaf_in = nullptr;
  const uint32_t* rows = idx->rows_sorted;
  if (adaptive) {
    if (!idx->ad_nodes) return fail(PARIS_EINVAL, "the index has no adaptive-split leaves");
    if (qs.keys) return fail(PARIS_EINVAL, "adaptive-split leaves take the query's own key only");
    PARIS_TRY(launch_adaptive_leaf(idx, qs, st));
    leaf_in = qs.leaf;
    rows = idx->ad_rows;
  }
  const int Lp = max(idx->leaf_cap, qs.k);
  const int nk = qs.keys ? qs.nk : 1;
  int P2 = 1;
  while (P2 < nk * Lp) P2 <<= 1;
  size_t smem = (size_t)(2 * Lp + 2 + P2) * sizeof(uint64_t);
  if (smem > 220 * 1024) return fail(PARIS_EINVAL, "too many leaves per query for the approximate search");
  int vec = vec_ok(idx, qs.queries) ? 1 : 0;
  int it = vec ? iters_for(idx->len) : 1;
  const uint64_t* qk = qs.keys ? qs.keys : qs.qkey;
#define DESC(IT)                                                                                 \
  do {                                                                                           \
    PARIS_CUDA(cudaFuncSetAttribute(descent_kernel<IT>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)smem));                                                 \
    descent_kernel<IT><<<(unsigned)qs.nq, kDescentThreads, smem, st>>>(                          \
        idx->series, idx->n, idx->len, vec, idx->keys_sorted, rows, idx->leaf_cap, qs.k,          \
        qs.queries, qk, nk, qs.leaf, qs.seed, qs.thr, qs.bsf, qs.cg, qs.counters, leaf_in);      \
  } while (0)
  switch (it) {
    case 1: DESC(1); break;
    case 2: DESC(2); break;
    case 4: DESC(4); break;
    case 8: DESC(8); break;
    default: DESC(16); break;
  }
#undef DESC
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

static paris_status lbscan_common(const paris_index* idx, const float* table, const uint32_t* thr_ptr,
                                  float thr_value, uint32_t* count, uint32_t* rows, float* lb,
                                  int64_t cap, uint32_t* status, int stop_on_overflow, cudaStream_t st) {
  size_t smem = (size_t)idx->card * 64 * sizeof(float);
  // set on every launch: the attribute is per device, and a cached flag would not be thread-safe
  PARIS_CUDA(cudaFuncSetAttribute(lbscan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t groups = (idx->n + 31) / 32;
  int64_t need_blocks = (groups + (kLbThreads / 32) * kLbUnroll - 1) / ((kLbThreads / 32) * kLbUnroll);
  int grid = (int)std::min<int64_t>(need_blocks, (int64_t)sm_count() * 2);
  if (grid < 1) grid = 1;
  lbscan_kernel<<<grid, kLbThreads, smem, st>>>(reinterpret_cast<const uint4*>(idx->sax), idx->n, table,
                                                idx->card, thr_ptr, thr_value, count, rows, lb, cap, status,
                                                stop_on_overflow, nullptr, nullptr, nullptr);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status launch_lbscan_pages(const paris_index* idx, const QueryState& qs, int64_t q, const uint32_t* page_list,
                                 const uint32_t* page_count, uint32_t* count, uint32_t* rows, float* lb, int64_t cap,
                                 uint32_t* status, int stop_on_overflow, cudaStream_t st) {
  size_t smem = (size_t)idx->card * 64 * sizeof(float);
  PARIS_CUDA(cudaFuncSetAttribute(lbscan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the kept page count is on the device: a grid for the full pass, whose warps leave early
  int64_t groups = (idx->n + 31) / 32;
  int64_t need_blocks = (groups + (kLbThreads / 32) * kLbUnroll - 1) / ((kLbThreads / 32) * kLbUnroll);
  int grid = (int)std::min<int64_t>(need_blocks, (int64_t)sm_count() * 2);
  if (grid < 1) grid = 1;
  lbscan_kernel<<<grid, kLbThreads, smem, st>>>(reinterpret_cast<const uint4*>(idx->sax_sorted), idx->n,
                                                qs.qtable + q * (int64_t)idx->card * 16, idx->card, qs.thr + q, 0.f,
                                                count, rows, lb, cap, status, stop_on_overflow, page_list,
                                                page_count, idx->rows_sorted);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status launch_lbscan(const paris_index* idx, const QueryState& qs, int64_t q, uint32_t* count,
                           uint32_t* rows, float* lb, int64_t cap, uint32_t* status, int stop_on_overflow,
                           cudaStream_t st) {
  return lbscan_common(idx, qs.qtable + q * (int64_t)idx->card * 16, qs.thr + q, 0.f, count, rows, lb, cap,
                       status, stop_on_overflow, st);
}

paris_status launch_lbscan_threshold(const paris_index* idx, const float* table, float thr,
                                     uint32_t* count, uint32_t* rows, float* lb, int64_t cap,
                                     uint32_t* status, cudaStream_t st) {
  return lbscan_common(idx, table, nullptr, thr, count, rows, lb, cap, status, 0, st);
}

paris_status launch_refine(const paris_index* idx, const QueryState& qs, const ChunkState& cs,
                           cudaStream_t st) {
  chunk_prefix_kernel<<<1, 1024, 0, st>>>(cs.count, cs.qc, cs.cap, cs.prefix, qs.counters);
  PARIS_CUDA(cudaMemsetAsync(cs.bucket, 0, (size_t)cs.qc * kBuckets * sizeof(uint32_t), st));
  {
    int64_t blocks_x = std::min<int64_t>((cs.cap + 255) / 256, 128);
    dim3 g((unsigned)std::max<int64_t>(blocks_x, 1), (unsigned)cs.qc);
    bucket_hist_kernel<<<g, 256, 0, st>>>(cs.lb, cs.count, cs.cap, qs.thr, cs.q0, cs.bucket);
    bucket_offsets_kernel<<<(cs.qc + 127) / 128, 128, 0, st>>>(cs.bucket, cs.qc);
    bucket_scatter_kernel<<<g, 256, 0, st>>>(cs.rows, cs.lb, cs.count, cs.cap, qs.thr, cs.q0, cs.bucket, cs.rows2,
                                             cs.lb2);
  }
  PARIS_CUDA(cudaGetLastError());
  int vec = vec_ok(idx, qs.queries) ? 1 : 0;
  int it = vec ? iters_for(idx->len) : 1;
  int grid = sm_count() * 8;
#define REF(IT)                                                                                   \
  refine_kernel<IT><<<grid, kRefineThreads, 0, st>>>(idx->series, idx->len, vec, qs.queries, cs.q0, cs.qc, \
                                                     cs.cap, cs.prefix, cs.count, cs.rows2, cs.lb2, cs.F, qs.thr, \
                                                     qs.bsf, qs.k, qs.cg, qs.counters, qs.private_bsf)
  switch (it) {
    case 1: REF(1); break;
    case 2: REF(2); break;
    case 4: REF(4); break;
    case 8: REF(8); break;
    default: REF(16); break;
  }
#undef REF
  note_launches(5);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status launch_select(const paris_index* idx, const QueryState& qs, const ChunkState& cs,
                           int64_t* out_idx, float* out_dist, cudaStream_t st) {
  const int qc = cs.qc;
  if (qs.k == 1) {
    kth_from_bsf_kernel<<<(qc + 127) / 128, 128, 0, st>>>(qs.bsf, cs.q0, qc, cs.kth);
    note_launches(1);
  } else {
    select_init_kernel<<<qc, 256, 0, st>>>(cs.sel_state, cs.sel_hist, qc, qs.k);
    int64_t blocks_x = std::min<int64_t>((cs.cap + 255) / 256, 64);
    dim3 g((unsigned)std::max<int64_t>(blocks_x, 1), (unsigned)qc);
    for (int r = 0; r < 3; ++r) {
      select_hist_kernel<<<g, 256, 0, st>>>(cs.F, cs.count, cs.cap, cs.sel_state, cs.sel_hist, r);
      select_pick_kernel<<<qc, 256, 0, st>>>(cs.sel_hist, cs.sel_state, cs.kth, r);
    }
    note_launches(7);
  }
  PARIS_CUDA(cudaGetLastError());
  PARIS_CUDA(cudaMemsetAsync(cs.cont_count, 0, (size_t)qc * sizeof(uint32_t), st));
  {
    int64_t blocks_x = std::min<int64_t>((cs.cap + 255) / 256, 64);
    dim3 g((unsigned)std::max<int64_t>(blocks_x, 1), (unsigned)qc);
    contenders_kernel<<<g, 256, 0, st>>>(cs.F, cs.rows2, cs.count, cs.cap, cs.kth, qs.cg, cs.cont_count,
                                         cs.cont_rows, qs.status);
  }
  rerank_kernel<<<qc, 256, 0, st>>>(idx->series, idx->len, qs.queries, cs.q0, cs.cont_count, cs.cont_rows,
                                    cs.cont_limbs, qs.k, out_idx, out_dist, qs.counters);
  note_launches(2);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

}  // namespace paris
