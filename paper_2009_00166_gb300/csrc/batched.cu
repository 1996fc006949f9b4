// Batched lower-bound scan (the batched form of Alg. 8): one persistent launch scans the
// summary array for a whole chunk of queries, a tile of QT queries at a time, so each pass over
// the 16-byte summaries serves QT queries.
//
// Each CTA keeps the tile's lower-bound tables in shared memory as FP16 pairs: one 32-bit word
// holds the entries of two queries for the same (symbol, segment), so one conflict-free lookup
// (same rotated layout as the single-query scan) feeds two queries and HADD2 sums both.
// Entries are rounded down to FP16 (and capped at 4000) so each stays below the exact
// contribution; the 16-term FP16 sum has relative error below 16 * 2^-11, so a row is kept when
// (sum * (1 - 2^-6)) <= threshold, and that scaled value is what is stored as its lower bound.
#include <cuda_fp16.h>

#include <algorithm>

#include "query.cuh"

namespace paris {

namespace {

constexpr int kBThreads = 768;
constexpr int kBUnroll = 4;
constexpr float kHalfKeep = 1.0f - 1.0f / 64.0f;
constexpr float kHalfCap = 4000.0f;

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

// FP16 pair tables of a chunk, packed once: word (pair p, entry e) = {T[2p][e], T[2p+1][e]}.
__global__ void pack_pairs_kernel(const float* __restrict__ qtable, int qc, int64_t entries, uint32_t* __restrict__ out) {
  const int64_t npairs = (qc + 1) / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npairs * entries;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / entries, e = i - p * entries;
    const int64_t qa = 2 * p, qb = qa + 1;
    const float va = qtable[qa * entries + e];
    const float vb = qb < qc ? qtable[qb * entries + e] : 0.f;
    out[i] = pack_half2_rd(va, vb);
  }
}

template <int NP>
__global__ void __launch_bounds__(kBThreads, 1) lbscan_batched_kernel(
    const uint4* __restrict__ sax, int64_t n, int card, const uint32_t* __restrict__ packed,
    const uint32_t* __restrict__ thr, int64_t q0, int qc, int ntiles, uint32_t* __restrict__ count,
    uint32_t* __restrict__ out_rows, float* __restrict__ out_lb, int64_t cap, int stop_on_overflow,
    uint32_t* __restrict__ status) {
  constexpr int QT = 2 * NP;
  extern __shared__ __align__(16) uint32_t s_tab[];  // region r (64 KB): pairs 2r, 2r+1
  __shared__ float s_thr[QT];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t offp[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    uint32_t o0 = 4u * (16u * (lane >> 4) + ((2 * m + lane) & 15));
    uint32_t o1 = 4u * (16u * (lane >> 4) + ((2 * m + 1 + lane) & 15));
    offp[m] = o0 | (o1 << 16);
  }
  const uint32_t tab = (uint32_t)__cvta_generic_to_shared(s_tab);
  const int64_t groups = (n + 31) >> 5;
  const int64_t per = (groups + gridDim.x - 1) / gridDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * per, g1 = min(groups, g0 + per);
  const int64_t entries = (int64_t)card * 16;
  for (int tile = 0; tile < ntiles; ++tile) {
    const int qb = tile * QT;
    __syncthreads();  // the previous tile's tables are no longer read
    const int npairs_chunk = (qc + 1) / 2;
    for (int64_t e4 = threadIdx.x; e4 < entries * NP / 4; e4 += blockDim.x) {  // 4 entries per thread step
      const int64_t e = 4 * e4;
      const int p = (int)(e / entries);
      const int64_t rem = e - (int64_t)p * entries;
      const int c = (int)(rem >> 4), i = (int)(rem & 15);
      const int pg = qb / 2 + p;  // pair index within the chunk
      const uint4 word = pg < npairs_chunk ? *reinterpret_cast<const uint4*>(packed + (int64_t)pg * entries + rem)
                                           : make_uint4(0u, 0u, 0u, 0u);
      const int w0 = (p >> 1) * 16384 + c * 64 + (p & 1) * 32 + i;
      *reinterpret_cast<uint4*>(&s_tab[w0]) = word;
      *reinterpret_cast<uint4*>(&s_tab[w0 + 16]) = word;
    }
    if (threadIdx.x < QT) {
      const int q = qb + threadIdx.x;
      s_thr[threadIdx.x] = q < qc ? __uint_as_float(thr[q0 + q]) : -1.0f;  // -1: nothing kept
    }
    __syncthreads();
    // FP16 thresholds per pair: keep iff sum <= thr / (1 - 2^-6), the bound rounded up so the
    // kept set is a superset of the FP32 test's
    __half2 thh[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float ta = s_thr[2 * p], tb = s_thr[2 * p + 1];
      thh[p] = __halves2half2(ta < 0.f ? __float2half(-65504.f) : __float2half_ru(fminf(ta / kHalfKeep, 65504.f)),
                              tb < 0.f ? __float2half(-65504.f) : __float2half_ru(fminf(tb / kHalfKeep, 65504.f)));
      if (ta >= 65504.f * kHalfKeep) thh[p] = __halves2half2(__float2half(65504.f), __high2half(thh[p]));
      if (tb >= 65504.f * kHalfKeep) thh[p] = __halves2half2(__low2half(thh[p]), __float2half(65504.f));
    }
    bool ovf[QT];
#pragma unroll
    for (int q = 0; q < QT; ++q) ovf[q] = false;
    for (int64_t it = g0 + (int64_t)wib * kBUnroll; it < g1; it += (int64_t)nw * kBUnroll) {
      uint4 word[kBUnroll];
#pragma unroll
      for (int u = 0; u < kBUnroll; ++u) {
        const int64_t row = (it + u) * 32 + lane;
        word[u] = (it + u < g1 && row < n) ? __ldcs(sax + row) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < kBUnroll; ++u) {
        const int64_t row = (it + u) * 32 + lane;
        const bool rv = it + u < g1 && row < n;
        const uint32_t wv[4] = {word[u].x, word[u].y, word[u].z, word[u].w};
        uint32_t addr[16];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          const uint32_t sel = (4u + 2u * (kk & 1)) | ((uint32_t)(kk & 3) << 4) | (5u << 8) | (5u << 12);
          addr[kk] = tab + __byte_perm(wv[kk >> 2], offp[kk >> 1], sel);
        }
        __half2 sum[NP];
        uint32_t keepmask = 0u;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const uint32_t off = (uint32_t)((p >> 1) * 65536 + (p & 1) * 128);
          __half2 acc0 = __floats2half2_rn(0.f, 0.f), acc1 = acc0;  // two chains: shorter latency
#pragma unroll
          for (int kk = 0; kk < 16; kk += 2) {
            uint32_t v0, v1;
            asm("ld.shared.b32 %0, [%1];" : "=r"(v0) : "r"(addr[kk] + off));
            asm("ld.shared.b32 %0, [%1];" : "=r"(v1) : "r"(addr[kk + 1] + off));
            acc0 = __hadd2(acc0, *reinterpret_cast<__half2*>(&v0));
            acc1 = __hadd2(acc1, *reinterpret_cast<__half2*>(&v1));
          }
          sum[p] = __hadd2(acc0, acc1);
          const uint32_t m = __hle2_mask(sum[p], thh[p]);
          keepmask |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * p);
        }
        keepmask = rv ? keepmask : 0u;
        const uint32_t any = __reduce_or_sync(PARIS_FULL_MASK, keepmask);
        if (any) {  // rare: some lane keeps this row for some query of the tile
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            if (!((any >> (2 * p)) & 3u)) continue;
            const int qa = qb + 2 * p;
            const float la = __low2float(sum[p]) * kHalfKeep, lbq = __high2float(sum[p]) * kHalfKeep;
            append_kept(((keepmask >> (2 * p)) & 1u) != 0u, row, la, lane, count + qa, out_rows + (int64_t)qa * cap,
                        out_lb + (int64_t)qa * cap, cap, ovf[2 * p], status);
            append_kept(((keepmask >> (2 * p)) & 2u) != 0u, row, lbq, lane, count + qa + 1,
                        out_rows + (int64_t)(qa + 1) * cap, out_lb + (int64_t)(qa + 1) * cap, cap, ovf[2 * p + 1],
                        status);
          }
        }
      }
      if (stop_on_overflow) {
        bool all = true;
#pragma unroll
        for (int q = 0; q < QT; ++q) all = all && (ovf[q] || s_thr[q] < 0.f);
        if (all) break;
      }
    }
  }
}

size_t batched_smem(int np, int card) {
  const int regions = (np + 1) / 2;
  // region r spans 64 KB of 256-byte symbol rows; the last region only needs card rows
  return (size_t)(regions - 1) * 65536 + (size_t)card * 256;
}

int sm_count_b() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

template <int NP>
paris_status launch_np(const paris_index* idx, const QueryState& qs, const ChunkState& cs, int stop, uint32_t* status,
                       cudaStream_t st) {
  const size_t smem = batched_smem(NP, idx->card);
  static int configured = 0;
  if ((int)smem > configured) {
    PARIS_CUDA(cudaFuncSetAttribute(lbscan_batched_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = (int)smem;
  }
  const int ntiles = (cs.qc + 2 * NP - 1) / (2 * NP);
  const int64_t groups = (idx->n + 31) / 32;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count_b(), (groups + 63) / 64));
  const int64_t entries = (int64_t)idx->card * 16;
  pack_pairs_kernel<<<(unsigned)std::min<int64_t>(((cs.qc + 1) / 2 * entries + 255) / 256, 4096), 256, 0, st>>>(
      qs.qtable + cs.q0 * entries, cs.qc, entries, cs.packed);
  lbscan_batched_kernel<NP><<<grid, kBThreads, smem, st>>>(reinterpret_cast<const uint4*>(idx->sax), idx->n,
                                                            idx->card, cs.packed, qs.thr, cs.q0, cs.qc, ntiles,
                                                            cs.count, cs.rows, cs.lb, cs.cap, stop, status);
  note_launches(2);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

}  // namespace

const int kQueryTiles[kNumQueryTiles] = {2, 4, 8, 12};

bool query_tile_fits(int qt, int card) { return batched_smem(qt / 2, card) <= 200 * 1024; }

paris_status launch_lbscan_batched(const paris_index* idx, const QueryState& qs, const ChunkState& cs, int qt,
                                   int stop_on_overflow, uint32_t* status, cudaStream_t st) {
  switch (qt) {
    case 2: return launch_np<1>(idx, qs, cs, stop_on_overflow, status, st);
    case 4: return launch_np<2>(idx, qs, cs, stop_on_overflow, status, st);
    case 8: return launch_np<4>(idx, qs, cs, stop_on_overflow, status, st);
    case 12: return launch_np<6>(idx, qs, cs, stop_on_overflow, status, st);
    default: return fail(PARIS_EINVAL, "query_tile must be one of 2, 4, 8, 12 (got %d)", qt);
  }
}

}  // namespace paris
