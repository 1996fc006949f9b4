// Mixed-precision screening for queries whose lower bounds keep many rows.
//
// For a query q and a row x the kernel forms d~ = |q|^2 + |x|^2 - 2 (q~ . x~) with q~, x~ the
// BF16 roundings of q and x, the dot product taken on the 5th-generation tensor cores
// (tcgen05.mma, FP32 accumulation in tensor memory) and |q|^2, |x|^2 taken in fp32 from the
// fp32 values. A proven bound M(q, x) on |d~ - |q - x|^2| then gives, per pair, the interval
// [d~ - M, d~ + M] that holds the exact squared distance:
//   pass 1 keeps, per query, the k smallest upper ends d~ + M and lowers the query's
//          best-so-far threshold with the k-th (k distinct rows bound the k-th best distance);
//   pass 2 emits every row whose lower end d~ - M does not exceed that threshold as a
//          candidate (with d~ - M as its lower bound) for the exact fp32 re-check (Alg. 9).
// Rows are only discarded when provably farther than the k-th neighbour, so answers stay exact.
//
// Per pair the epilogue first applies a cheaper test with the row tile's norm range (smallest
// and largest |x|^2, largest |x|): pass 2 drops a pair when rd(xn_min - 2 q~.x~) exceeds
// ru(thr + M_max - |q|^2) (applied as a per-query threshold on the dot product, see emit_kernel),
// which implies d~ - M > thr for the pair's own norms; only the pairs that survive get the exact
// interval above. Pass 1 ranks the looser upper ends ru(ru(xn_max - 2 q~.x~) + |q|^2 + M_max),
// which still bound the distance from above.
//
// Kernel shapes (one persistent CTA per SM; warp 0 streams the row tiles of the BF16 shadow of
// the series, 128 rows x 64 K elements per stage, into a TMA ring; warp 1 issues the tensor-core
// MMAs from one thread; warps 2-17 read the TMEM accumulators back with tcgen05.ld and run the
// epilogue; every wait between roles is bounded):
//   emit_kernel<2> (pass 2) and emit_kernel<1> (pass 1 for k = 1): rows on the MMA M side, a
//     group of up to 256 queries (fewer for series longer than 256 values, so that the group
//     fits 128 KB of shared memory) on N: one 128 x N x 16 MMA per K step, both operands in
//     shared memory, double-buffered 128 x N fp32 accumulators; a thread of the epilogue owns a
//     row and 64 of the group's queries. Up to 8 groups per launch split the CTAs and visit the
//     row tiles in the same order, so each row tile read from HBM serves every group.
//   bound_kernel (pass 1 for k > 1, series of at most 256 values): two tiles of 128 queries on M
//     against each 128-row tile on N (128 x 128 x 16 MMAs), one query per epilogue thread, which
//     keeps its k smallest upper ends in registers.
// The epilogues read each 64-row norm range from global memory ahead of use, and a row's own
// norms only for the pairs that pass the range test.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "query.cuh"

namespace paris {

namespace {

constexpr int BM = 128;             // queries per tile (MMA M)
constexpr int BN = 128;             // series rows per tile (MMA N)
constexpr int RT = 64;              // rows per norm-range tile (xtile) and per norm block
constexpr int BKE = 64;             // K elements per TMA box: 128 bytes of BF16
constexpr int QTILES = 2;           // query tiles sharing each row tile (one query group)
constexpr int GROUPS = 8;           // query groups per launch, each on its own share of the CTAs
constexpr int STAGES = 6;           // shared-memory ring depth: one (row tile, K block) per stage
constexpr int DENSE_THREADS = 576;  // warp 0: TMA, warp 1: MMA + TMEM owner, warps 2-17: epilogue
constexpr int EPI_WARPS = 16;       // per TMEM lane quadrant: one per (query tile, 64-row half)
constexpr int SAMPLE = 16;          // pass 1 visits one row tile in SAMPLE
constexpr int KMAX = 16;            // largest k the screening supports
constexpr uint32_t TMEM_COLS = 512;  // accumulators: 2 buffers x 2 query tiles x 128 columns
constexpr int MAX_KB = 4;           // len <= 256

constexpr size_t KBLK_BYTES = (size_t)BN * 128;      // one K block of a row tile (= of a query tile)
constexpr size_t A_BYTES = (size_t)QTILES * MAX_KB * BM * 128;
constexpr size_t DENSE_SMEM = 1024 + A_BYTES + STAGES * KBLK_BYTES + 256;
static_assert(BM * 128 == KBLK_BYTES, "query and row tiles share the K-block shape");
static_assert(DENSE_SMEM <= 232448, "dynamic shared memory of one CTA");
// emit_kernel: a query group of up to QG queries is the MMA N side; its BF16 rows fill at most
// Q_BYTES of shared memory, so a group holds qg = min(QG, 65536 / len) queries (rounded down to
// a multiple of 32): 256 up to len 256, 128 at len 512, 64 at len 1024
constexpr int QG = QTILES * BM;                          // largest group
constexpr int E_MAX_LEN = 1024;                          // longest series the emit kernels take
constexpr int E_STAGES = 5;                              // its ring depth
constexpr size_t Q_BYTES = (size_t)MAX_KB * QG * 128;   // the group's K blocks (128 KB)
constexpr size_t EMIT_SMEM = 1024 + Q_BYTES + E_STAGES * KBLK_BYTES + EPI_WARPS * 64 * 4 + QG * 16 + 256;
static_assert(EMIT_SMEM <= 232448, "dynamic shared memory of one CTA");
static_assert(2 * QG <= (int)TMEM_COLS, "two accumulators of QG columns");
constexpr unsigned long long kDrainNs = 100000000ull;  // extra bound of the drain waits after an abort

struct DenseParams {
  uint64_t wait_ns;  // bound of every wait of a role on another role (paris_set_wait_limit)
  int64_t n;
  int len, nkb;
  int group0, nd;        // first query group of the launch; nd < 0: read from nd_dev
  int qg;                // queries per group of emit_kernel (a multiple of 32, at most QG)
  const int* nd_dev;
  const float2* xnorm;  // [n]: (|x|^2, |x|)
  const uint32_t* qbf;  // BF16 query rows, [rows][len] (pairs of elements per word)
  const float4* xtile;  // [row tiles]: (min |x|^2, max |x|^2, max |x|, 0) of the tile's rows
  const float2* qnorm;  // [nd_pad]
  const int* qslot;     // [nd]: chunk-local slot of dense query d
  int64_t q0;           // thresholds of slot j live at thr[q0 + j]
  uint32_t* thr;
  int k;
  float cg, c1, c2;
  uint32_t* count;
  uint32_t* rows;
  float* lb;
  int64_t cap;
  uint32_t* status;    // device errors (timeouts)
  uint32_t* overflow;  // set when a list passed its capacity (the per-query count says which)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity; gives up (returning false) at the deadline or when
// another role has already given up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t deadline) {
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (globaltimer() > deadline) return false;
  }
  return true;
}
// Drain wait of a role's own asynchronous work (its TMA copies or MMAs) before the CTA releases
// shared and tensor memory: it ignores the abort flag and only stops at its own deadline.
__device__ __forceinline__ bool mbar_wait_drain(uint32_t bar, uint32_t parity, uint64_t deadline) {
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() > deadline) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle layout written by
// TMA (8-row x 128-byte atoms, 1024 bytes apart).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// BF16 MMA with FP32 accumulation into tensor memory: A (a query tile) and B (a row tile), both
// K-major in shared memory, through their descriptors.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Pass 1: the k smallest upper ends per query over every SAMPLE-th row tile (queries on the MMA
// M side, 128 x 128 x 16 MMAs: one thread per query in the epilogue keeps its own top k).
__global__ void __launch_bounds__(DENSE_THREADS, 1)
    bound_kernel(const __grid_constant__ CUtensorMap tmB, DenseParams P) {
  extern __shared__ uint8_t dsm_raw[];
  // The launch's query groups (QTILES query tiles each) split the CTAs; the CTAs of every group
  // visit the row tiles in the same order at about the same time, so a row tile read from HBM by
  // one group is served from L2 to the others. Uniform per CTA: a CTA without a group returns.
  const int nd = P.nd >= 0 ? P.nd : *P.nd_dev;
  const int groups = (nd + QTILES * BM - 1) / (QTILES * BM) - P.group0;
  if (groups <= 0) return;
  const int G = groups < GROUPS ? groups : GROUPS;
  const int cpg = (int)gridDim.x / G;  // CTAs per group (the grid holds at least GROUPS CTAs)
  const int grp = (int)blockIdx.x % G, rank = (int)blockIdx.x / G;
  if (rank >= cpg) return;
  const int qtile = (P.group0 + grp) * QTILES;
  const int nq_tiles = (qtile + 1) * BM < nd ? 2 : 1;  // query tiles of this group that hold queries
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* smA = base;            // [QTILES][MAX_KB] query K blocks, 128-byte swizzle
  uint8_t* smB = base + A_BYTES;  // [STAGES] row-tile K blocks, 128-byte swizzle (written by TMA)
  uint64_t* bars = (uint64_t*)(smB + STAGES * KBLK_BYTES);
  // bars: full[STAGES] | empty[STAGES] | acc_full[2] | acc_empty[2]
  uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 4);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + STAGES), b_accf = smem_u32(bars + 2 * STAGES),
                 b_acce = smem_u32(bars + 2 * STAGES + 2);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(b_full + 8 * s, 1);
      mbar_init(b_empty + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(b_accf + 8 * a, 1);
      mbar_init(b_acce + 8 * a, EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the query tiles go to shared memory once, in the layout the 128-byte-swizzle descriptors read:
  // K block kb of tile c holds row r's 16-byte chunk j (elements 64 kb + 8 j ...) at
  // r * 128 + 16 * (j ^ (r mod 8))
  {
    const int nkb = P.nkb;
    const int chunks = nq_tiles * nkb * BM * 8;
    for (int e = threadIdx.x; e < chunks; e += blockDim.x) {
      const int j = e & 7, r = (e >> 3) & (BM - 1), kb = (e >> 10) % nkb, c = (e >> 10) / nkb;
      const int64_t grow = (int64_t)(qtile + c) * BM + r;
      const uint4 v = *reinterpret_cast<const uint4*>(P.qbf + grow * (P.len / 2) + kb * (BKE / 2) + j * 4);
      *reinterpret_cast<uint4*>(smA + ((size_t)(c * MAX_KB + kb) * KBLK_BYTES) + r * 128 + ((j ^ (r & 7)) << 4)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const int64_t ntiles = (P.n + BN - 1) / BN;
  const int64_t nranges = (P.n + RT - 1) / RT;
  // the upper ends of any k rows bound the k-th distance: every SAMPLE-th tile is enough
  const int64_t tstep = SAMPLE;
  const int64_t tfirst = (int64_t)rank * tstep, tstride = (int64_t)cpg * tstep;
  const uint64_t deadline = globaltimer() + P.wait_ns;
  const int nkb = P.nkb;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer: one stage per (row tile, K block)
      int i = 0;
      for (int64_t t = tfirst; t < ntiles && !*abort_flag; t += tstride) {
        for (int kb = 0; kb < nkb; ++kb, ++i) {
          const int s = i % STAGES;
          const uint32_t ph = (uint32_t)((i / STAGES) & 1);
          if (!mbar_wait(b_empty + 8 * s, ph ^ 1u, abort_flag, deadline)) {
            *abort_flag = 1;
            break;
          }
          mbar_expect_tx(b_full + 8 * s, (uint32_t)KBLK_BYTES);
          tma_load_2d(smem_u32(smB + (size_t)s * KBLK_BYTES), &tmB, kb * BKE, (int)(t * BN), b_full + 8 * s);
        }
      }
      // drain: the last loads must land before the CTA may exit
      const int issued = i;
      for (int j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
        if (!mbar_wait_drain(b_full + 8 * (j % STAGES), (uint32_t)((j / STAGES) & 1), deadline + kDrainNs))
          *abort_flag = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      bool ok = true;
      int i = 0, j = 0;  // stages consumed, row tiles finished
      for (int64_t t = tfirst; ok && t < ntiles; t += tstride, ++j) {
        const int ab = j & 1;
        const uint32_t aph = (uint32_t)((j >> 1) & 1);
        if (!mbar_wait(b_acce + 8 * ab, aph ^ 1u, abort_flag, deadline)) {
          ok = false;
          break;
        }
        for (int kb = 0; kb < nkb; ++kb, ++i) {
          const int s = i % STAGES;
          const uint32_t ph = (uint32_t)((i / STAGES) & 1);
          if (!mbar_wait(b_full + 8 * s, ph, abort_flag, deadline)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t b0 = smem_u32(smB + (size_t)s * KBLK_BYTES);
          for (int qt = 0; qt < nq_tiles; ++qt) {
            const uint32_t d_tmem = tmem_base + (uint32_t)((ab * QTILES + qt) * BN);
            const uint32_t a0 = smem_u32(smA + (size_t)(qt * MAX_KB + kb) * KBLK_BYTES);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)  // 16 BF16 per MMA step along K: 32 bytes of each row
              umma_bf16(d_tmem, smem_desc_sw128(a0 + 32 * ks), smem_desc_sw128(b0 + 32 * ks), idesc,
                        (kb | ks) ? 1u : 0u);
          }
          umma_commit(b_empty + 8 * s);
        }
        if (!ok) break;
        umma_commit(b_accf + 8 * ab);
      }
      if (!ok) *abort_flag = 1;
      // drain: wait for the last MMAs before the TMEM is released (the commit of the last stage
      // covers every MMA this thread issued before it)
      if (i > 0 && !mbar_wait_drain(b_empty + 8 * ((i - 1) % STAGES), (uint32_t)(((i - 1) / STAGES) & 1),
                                    deadline + kDrainNs))
        *abort_flag = 1;
    }
  } else {  // ---- epilogue: warps 2..17, TMEM lane quadrant = warp % 4
    const int qd = warp & 3;
    const int c = ((warp - 2) >> 2) & 1;  // query tile
    const int h = (warp - 2) >> 3;        // 64-row half of each row tile
    const bool tile_on = c < nq_tiles;  // warp-uniform: this warp's query tile holds queries
    const int m = qd * 32 + lane;
    const int d = (qtile + c) * BM + m;
    const bool valid = d < nd;
    float qn = 0.f, qrt = 0.f;
    uint32_t* thr_ptr = nullptr;
    if (valid) {
      const float2 qq = P.qnorm[d];
      qn = qq.x;
      qrt = qq.y;
      thr_ptr = P.thr + P.q0 + P.qslot[d];
    }
    const float c1q = __fmul_ru(P.c1, qrt);
    float best[KMAX];
#pragma unroll
    for (int jj = 0; jj < KMAX; ++jj) best[jj] = CUDART_INF_F;
    float kth = CUDART_INF_F;
    // norm range of this warp's 64 rows of a row tile, loaded two tiles ahead (one address per warp)
    auto load_range = [&](int64_t t) {
      const int64_t r = 2 * t + h;
      return (t < ntiles && r < nranges) ? P.xtile[r] : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    float4 rng1 = load_range(tfirst), rng2 = load_range(tfirst + tstride);
    int j = 0;
    for (int64_t t = tfirst; t < ntiles; t += tstride, ++j) {
      const float4 rng = rng1;
      rng1 = rng2;
      rng2 = load_range(t + 2 * tstride);
      const int ab = j & 1;
      const uint32_t aph = (uint32_t)((j >> 1) & 1);
      if (!mbar_wait(b_accf + 8 * ab, aph, abort_flag, deadline)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (tile_on) {
        // largest margin over the rows of the range, rounded up
        const float Mmax = __fmaf_ru(c1q, rng.z, __fmul_ru(P.c2, __fadd_ru(qn, rng.y)));
#pragma unroll 1
        for (int ch = 0; ch < 2; ++ch) {
          uint32_t v[32];
          tmem_ld32(tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)((ab * QTILES + c) * BN + h * 64 + ch * 32), v);
          const int64_t row0 = t * BN + h * 64 + ch * 32;
          const int64_t left = P.n - row0;
          const int nrow = left <= 0 ? 0 : (left < 32 ? (int)left : 32);  // rows of this chunk inside the series
          const uint32_t row_mask = nrow >= 32 ? 0xffffffffu : (nrow <= 0 ? 0u : ((1u << nrow) - 1u));
          uint32_t hit = 0u;
          // the tests below are monotone in the dot product (round-toward functions of -2 dot
          // plus a constant), so the largest of the 32 dots decides whether any row can pass
          float dmax = __uint_as_float(v[0]);
#pragma unroll
          for (int jj = 1; jj < 32; ++jj) dmax = fmaxf(dmax, __uint_as_float(v[jj]));
          {
            // upper ends from the range's norms: ru(ru(xn_max - 2 dot) + ru(|q|^2 + M_max))
            const float Cq = __fadd_ru(qn, Mmax);
            if (valid && __fadd_ru(__fmaf_ru(-2.0f, dmax, rng.y), Cq) < kth) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                hit |= (__fadd_ru(__fmaf_ru(-2.0f, __uint_as_float(v[jj]), rng.y), Cq) < kth ? 1u : 0u) << jj;
            }
            hit = valid ? (hit & row_mask) : 0u;
            while (hit) {  // rare: insert into the top-k
              const int jj = __ffs(hit) - 1;
              hit &= hit - 1u;
              uint32_t dv = 0u;
#pragma unroll
              for (int q2 = 0; q2 < 32; ++q2) dv = (q2 == jj) ? v[q2] : dv;
              float x = __fadd_ru(__fmaf_ru(-2.0f, __uint_as_float(dv), rng.y), Cq);
              if (x < kth) {
#pragma unroll
                for (int q2 = 0; q2 < KMAX; ++q2) {
                  if (q2 < P.k) {
                    const float lo = fminf(best[q2], x);
                    x = fmaxf(best[q2], x);
                    best[q2] = lo;
                  }
                }
#pragma unroll
                for (int q2 = 0; q2 < KMAX; ++q2)
                  if (q2 == P.k - 1) kth = best[q2];
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_acce + 8 * ab);
    }
    if (valid && kth < CUDART_INF_F) atomicMin(thr_ptr, __float_as_uint(__fmul_ru(kth, P.cg)));
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(P.status, DEV_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// R+ of a float: the next float above it (the test rd(y) <= R holds exactly when y < R+).
__device__ __forceinline__ float next_up(float r) {
  if (r == 0.f) return __uint_as_float(1u);
  if (isinf(r) && r > 0.f) return r;
  const uint32_t b = __float_as_uint(r);
  return __uint_as_float(r > 0.f ? b + 1u : b - 1u);
}

// Pass 2: every row whose interval's lower end does not exceed the query's threshold becomes a
// candidate. Rows on the MMA M side and up to 256 queries on the N side: one 128 x N x 16 MMA
// per K step reads a row tile once for every query of the group (the tensor cores run at their
// full rate with N = 256; 128 x 128 shapes with both operands in shared memory run at about
// half of it). The accumulator of a row tile is 128 lanes (rows) x N columns (queries).
//
// Epilogue: a thread owns one row and 64 queries (two chunks of 32 columns). Per chunk and query
// the range test rd(xn_min - 2 dot) <= R, R = ru(ru(thr + M_max) - |q|^2), is applied in the
// equivalent-or-looser form dot >= L with L = rd(rd(xn_min - R+) / 2): rd(xn_min - 2 dot) <= R
// means xn_min - 2 dot < R+, that is dot > (xn_min - R+) / 2 >= L. L depends on the query and
// the row's 64-row norm range only, so each warp writes its 64 values per tile to shared memory
// and every lane reads them back (one address per warp). A pair that passes gets the row's own
// interval and is emitted when d~ - M <= thr.
//
// PASS 1 (k = 1 only) is the threshold pass in the same shape, over every SAMPLE-th row tile: a
// lane's 32 dots of a chunk go through a butterfly of shuffles that leaves lane l with the
// largest dot of query column l over the warp's 32 rows; the upper end
// ru(ru(xn_max - 2 dot) + ru(|q|^2 + M_max)) falls as the dot grows, so that dot gives the smallest
// upper end of the 32 rows, and the lane keeps its query's smallest over the visited tiles.
template <int PASS>
__global__ void __launch_bounds__(DENSE_THREADS, 1)
    emit_kernel(const __grid_constant__ CUtensorMap tmX, DenseParams P) {
  extern __shared__ uint8_t dsm_raw[];
  const int nd = P.nd >= 0 ? P.nd : *P.nd_dev;
  const int qg = P.qg;
  const int groups = (nd + qg - 1) / qg - P.group0;
  if (groups <= 0) return;
  const int G = groups < GROUPS ? groups : GROUPS;
  const int cpg = (int)gridDim.x / G;
  const int grp = (int)blockIdx.x % G, rank = (int)blockIdx.x / G;
  if (rank >= cpg) return;
  const int gq0 = (P.group0 + grp) * qg;        // first screened query of the group
  const int nq = min(qg, nd - gq0);              // its queries
  const int ncols = (nq + 31) & ~31;             // MMA N (a multiple of 16, at most 256)
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* smQ = base;                                   // [nkb][qg rows] query K blocks
  uint8_t* smX = base + Q_BYTES;                         // [E_STAGES] row-tile K blocks (TMA)
  float* smL = (float*)(smX + E_STAGES * KBLK_BYTES);    // [EPI_WARPS][64] range thresholds L
  float4* smC = (float4*)(smL + EPI_WARPS * 64);         // [QG]: |q|^2, ru(c1 |q|), thr, slot
  uint64_t* bars = (uint64_t*)(smC + QG);
  uint32_t* tmem_holder = (uint32_t*)(bars + 2 * E_STAGES + 4);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + E_STAGES),
                 b_accf = smem_u32(bars + 2 * E_STAGES), b_acce = smem_u32(bars + 2 * E_STAGES + 2);
  if (threadIdx.x == 0) {
    for (int s = 0; s < E_STAGES; ++s) {
      mbar_init(b_full + 8 * s, 1);
      mbar_init(b_empty + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(b_accf + 8 * a, 1);
      mbar_init(b_acce + 8 * a, EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the group's queries, K block kb holding query r's 16-byte chunk j at
  // kb * qg * 128 + r * 128 + 16 * (j ^ (r mod 8)) (the 128-byte swizzle of the descriptors)
  {
    const int nkb = P.nkb;
    for (int e = threadIdx.x; e < nkb * qg * 8; e += blockDim.x) {
      const int j = e & 7, r = (e >> 3) % qg, kb = (e >> 3) / qg;
      if (r >= ncols) continue;
      const uint4 v = *reinterpret_cast<const uint4*>(P.qbf + (int64_t)(gq0 + r) * (P.len / 2) + kb * (BKE / 2) + j * 4);
      *reinterpret_cast<uint4*>(smQ + (size_t)kb * qg * 128 + r * 128 + ((j ^ (r & 7)) << 4)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
    for (int q = threadIdx.x; q < QG; q += blockDim.x) {
      float4 c = make_float4(0.f, 0.f, -1.f, 0.f);  // no row passes thr = -1
      if (q < nq) {
        const float2 qq = P.qnorm[gq0 + q];
        const int slot = P.qslot[gq0 + q];
        c = make_float4(qq.x, __fmul_ru(P.c1, qq.y), __uint_as_float(*(volatile uint32_t*)(P.thr + P.q0 + slot)),
                        __int_as_float(slot));
      }
      smC[q] = c;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const int64_t ntiles = (P.n + BN - 1) / BN;
  const int64_t nranges = (P.n + RT - 1) / RT;
  const int64_t tstep = PASS == 1 ? SAMPLE : 1;
  const int64_t tfirst = rank * tstep, tstride = (int64_t)cpg * tstep;
  const uint64_t deadline = globaltimer() + P.wait_ns;
  const int nkb = P.nkb;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer: one stage per (row tile, K block)
      int i = 0;
      for (int64_t t = tfirst; t < ntiles && !*abort_flag; t += tstride) {
        for (int kb = 0; kb < nkb; ++kb, ++i) {
          const int s = i % E_STAGES;
          const uint32_t ph = (uint32_t)((i / E_STAGES) & 1);
          if (!mbar_wait(b_empty + 8 * s, ph ^ 1u, abort_flag, deadline)) {
            *abort_flag = 1;
            break;
          }
          mbar_expect_tx(b_full + 8 * s, (uint32_t)KBLK_BYTES);
          tma_load_2d(smem_u32(smX + (size_t)s * KBLK_BYTES), &tmX, kb * BKE, (int)(t * BN), b_full + 8 * s);
        }
      }
      const int issued = i;
      for (int j = (issued > E_STAGES ? issued - E_STAGES : 0); j < issued; ++j)
        if (!mbar_wait_drain(b_full + 8 * (j % E_STAGES), (uint32_t)((j / E_STAGES) & 1), deadline + kDrainNs))
          *abort_flag = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer: per stage, 4 MMAs of 128 rows x ncols queries x 16
      const uint32_t idesc = idesc_bf16(BN, ncols);
      bool ok = true;
      int i = 0, j = 0;
      for (int64_t t = tfirst; ok && t < ntiles; t += tstride, ++j) {
        const int ab = j & 1;
        const uint32_t aph = (uint32_t)((j >> 1) & 1);
        if (!mbar_wait(b_acce + 8 * ab, aph ^ 1u, abort_flag, deadline)) {
          ok = false;
          break;
        }
        const uint32_t d_tmem = tmem_base + (uint32_t)(ab * QG);
        for (int kb = 0; kb < nkb; ++kb, ++i) {
          const int s = i % E_STAGES;
          const uint32_t ph = (uint32_t)((i / E_STAGES) & 1);
          if (!mbar_wait(b_full + 8 * s, ph, abort_flag, deadline)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smX + (size_t)s * KBLK_BYTES);
          const uint32_t b0 = smem_u32(smQ + (size_t)kb * qg * 128);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            umma_bf16(d_tmem, smem_desc_sw128(a0 + 32 * ks), smem_desc_sw128(b0 + 32 * ks), idesc,
                      (kb | ks) ? 1u : 0u);
          umma_commit(b_empty + 8 * s);
        }
        if (!ok) break;
        umma_commit(b_accf + 8 * ab);
      }
      if (!ok) *abort_flag = 1;
      if (i > 0 && !mbar_wait_drain(b_empty + 8 * ((i - 1) % E_STAGES), (uint32_t)(((i - 1) / E_STAGES) & 1),
                                    deadline + kDrainNs))
        *abort_flag = 1;
    }
  } else if (PASS == 1) {  // ---- threshold epilogue (k = 1)
    const int qd = warp & 3;
    const int cq = (warp - 2) >> 2;
    const bool on = cq * 64 < ncols;
    float ubest[2] = {CUDART_INF_F, CUDART_INF_F};  // this lane's two query columns
    int j = 0;
    for (int64_t t = tfirst; t < ntiles; t += tstride, ++j) {
      const int64_t r = 2 * t + (qd >> 1);
      const float4 rng = r < nranges ? P.xtile[r] : make_float4(0.f, 0.f, 0.f, 0.f);
      const bool row_ok = t * BN + qd * 32 + lane < P.n;
      const int ab = j & 1;
      const uint32_t aph = (uint32_t)((j >> 1) & 1);
      if (!mbar_wait(b_accf + 8 * ab, aph, abort_flag, deadline)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (on) {
#pragma unroll 1
        for (int ch = 0; ch < 2; ++ch) {
          const int col0 = cq * 64 + ch * 32;
          if (col0 >= ncols) break;
          uint32_t v[32];
          tmem_ld32(tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)(ab * QG + col0), v);
          float a[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) a[c] = row_ok ? __uint_as_float(v[c]) : -CUDART_INF_F;
          // butterfly: after the step of width o, a[0 .. o) hold columns (lane's bits above o) + c
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int c = 0; c < o; ++c) {
              const float send = up ? a[c] : a[c + o];
              const float keep = up ? a[c + o] : a[c];
              a[c] = fmaxf(keep, __shfl_xor_sync(PARIS_FULL_MASK, send, o));
            }
          }
          const float4 qc = smC[col0 + lane];  // lane l now holds column col0 + l
          const float Mmax = __fmaf_ru(qc.y, rng.z, __fmul_ru(P.c2, __fadd_ru(qc.x, rng.y)));
          const float U = __fadd_ru(__fmaf_ru(-2.0f, a[0], rng.y), __fadd_ru(qc.x, Mmax));
          if (a[0] > -CUDART_INF_F) ubest[ch] = fminf(ubest[ch], U);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_acce + 8 * ab);
    }
    if (on)
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const int q = cq * 64 + ch * 32 + lane;
        if (q < nq && ubest[ch] < CUDART_INF_F)
          atomicMin(P.thr + P.q0 + P.qslot[gq0 + q], __float_as_uint(__fmul_ru(ubest[ch], P.cg)));
      }
  } else {  // ---- epilogue: warps 2..17; TMEM lane quadrant warp % 4, query quarter (warp - 2) / 4
    const int qd = warp & 3;
    const int we = warp - 2;
    const int cq = we >> 2;
    const bool on = cq * 64 < ncols;  // warp-uniform: this quarter holds queries
    float* Lw = smL + we * 64;
    // this lane's two queries for the range thresholds
    const float4 ca = smC[cq * 64 + lane], cb = smC[cq * 64 + 32 + lane];
    const bool va = cq * 64 + lane < nq, vb = cq * 64 + 32 + lane < nq;
    auto range_l = [&](const float4& c, const float4& rng) {
      const float Mmax = __fmaf_ru(c.y, rng.z, __fmul_ru(P.c2, __fadd_ru(c.x, rng.y)));
      const float R = __fsub_ru(__fadd_ru(c.z, Mmax), c.x);
      return __fmul_rd(__fsub_rd(rng.x, next_up(R)), 0.5f);
    };
    auto load_range = [&](int64_t t) {
      const int64_t r = 2 * t + (qd >> 1);
      return (t < ntiles && r < nranges) ? P.xtile[r] : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto load_norm = [&](int64_t t) {
      const int64_t row = t * BN + qd * 32 + lane;
      return (t < ntiles && row < P.n) ? P.xnorm[row] : make_float2(0.f, 0.f);
    };
    float4 rng1 = load_range(tfirst), rng2 = load_range(tfirst + tstride);
    float2 xn1 = load_norm(tfirst);
    int j = 0;
    for (int64_t t = tfirst; t < ntiles; t += tstride, ++j) {
      const float4 rng = rng1;
      rng1 = rng2;
      rng2 = load_range(t + 2 * tstride);
      const float2 xx = xn1;
      xn1 = load_norm(t + tstride);
      const int64_t row = t * BN + qd * 32 + lane;
      const bool row_ok = row < P.n;
      if (on) {
        __syncwarp();
        Lw[lane] = va ? range_l(ca, rng) : CUDART_INF_F;
        Lw[32 + lane] = vb ? range_l(cb, rng) : CUDART_INF_F;
        __syncwarp();
      }
      const int ab = j & 1;
      const uint32_t aph = (uint32_t)((j >> 1) & 1);
      if (!mbar_wait(b_accf + 8 * ab, aph, abort_flag, deadline)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (on) {
#pragma unroll 1
        for (int ch = 0; ch < 2; ++ch) {
          const int col0 = cq * 64 + ch * 32;
          if (col0 >= ncols) break;
          uint32_t v[32];
          tmem_ld32(tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)(ab * QG + col0), v);
          const float4* L4 = reinterpret_cast<const float4*>(Lw + ch * 32);
          bool any = false;
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4) {
            const float4 l = L4[c4];
            any |= (__uint_as_float(v[4 * c4]) >= l.x) | (__uint_as_float(v[4 * c4 + 1]) >= l.y) |
                   (__uint_as_float(v[4 * c4 + 2]) >= l.z) | (__uint_as_float(v[4 * c4 + 3]) >= l.w);
          }
          if (any && row_ok) {  // rare: the pairs that pass, each with the row's own interval
            uint32_t hit = 0u;
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4) {
              const float4 l = L4[c4];
              hit |= (__uint_as_float(v[4 * c4]) >= l.x ? 1u : 0u) << (4 * c4);
              hit |= (__uint_as_float(v[4 * c4 + 1]) >= l.y ? 1u : 0u) << (4 * c4 + 1);
              hit |= (__uint_as_float(v[4 * c4 + 2]) >= l.z ? 1u : 0u) << (4 * c4 + 2);
              hit |= (__uint_as_float(v[4 * c4 + 3]) >= l.w ? 1u : 0u) << (4 * c4 + 3);
            }
            while (hit) {
              const int jj = __ffs(hit) - 1;
              hit &= hit - 1u;
              uint32_t dv = 0u;
#pragma unroll
              for (int q2 = 0; q2 < 32; ++q2) dv = (q2 == jj) ? v[q2] : dv;
              const float4 qc = smC[col0 + jj];
              const float d2 = fmaf(-2.0f, __uint_as_float(dv), qc.x + xx.x);
              const float M = __fmaf_ru(qc.y, xx.y, __fmul_ru(P.c2, __fadd_ru(qc.x, xx.x)));
              const float x = fmaxf(__fsub_rd(d2, M), 0.f);  // lower end
              if (x <= qc.z) {
                const int slot = __float_as_int(qc.w);
                const uint32_t p = atomicAdd(P.count + slot, 1u);
                if ((int64_t)p < P.cap) {
                  P.rows[(int64_t)slot * P.cap + p] = (uint32_t)row;
                  P.lb[(int64_t)slot * P.cap + p] = x;
                } else {
                  atomicOr(P.overflow, DEV_CAND_OVERFLOW);
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_acce + 8 * ab);
    }
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(P.status, DEV_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// BF16 shadow of the series and fp32 (|x|^2, |x|) per row; one warp per row.
__global__ void shadow_kernel(const float* __restrict__ x, int64_t n, int len, __nv_bfloat16* __restrict__ out,
                              float2* __restrict__ norms, const int* __restrict__ gather, int64_t q0, int64_t rows_pad,
                              const int* __restrict__ n_dev = nullptr) {
  const int lane = threadIdx.x & 31;
  if (n_dev) n = *n_dev;  // rows to convert counted on the device (the rest of rows_pad is zero)
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows_pad; r += warps) {
    const bool real = r < n;
    const int64_t src = real ? (gather ? q0 + gather[r] : r) : 0;
    const float* xr = x + src * (int64_t)len;
    __nv_bfloat16* o = out + r * (int64_t)len;
    float acc = 0.f;
    for (int j = 2 * lane; j < len; j += 64) {
      float a = real ? xr[j] : 0.f, b = real ? xr[j + 1] : 0.f;
      acc = fmaf(a, a, acc);
      acc = fmaf(b, b, acc);
      *reinterpret_cast<__nv_bfloat162*>(o + j) = __floats2bfloat162_rn(a, b);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(PARIS_FULL_MASK, acc, s);
    if (lane == 0) norms[r] = make_float2(acc, __fsqrt_ru(acc));
  }
}

// The slots whose candidate list overflowed (or was routed here), in slot order.
__global__ void __launch_bounds__(1024) dense_select_kernel(const uint32_t* __restrict__ count, int qc, int64_t cap,
                                                            int* __restrict__ slots, int* __restrict__ nd) {
  const uint64_t total = block_prefix(
      qc, [&](int j) { return (int64_t)count[j] > cap ? 1ull : 0ull; },
      [&](int j, uint64_t excl, uint64_t v) {
        if (v) slots[excl] = j;
      });
  if (threadIdx.x == 0) *nd = (int)total;
}

__global__ void dense_reset_kernel(uint32_t* __restrict__ count, const int* __restrict__ slots, const int* nd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *nd) count[slots[i]] = 0u;
}

// A query whose screened list overflowed keeps the k-th best exact candidate it did store: that
// distance, rounded up by the fp32 error factor, bounds the true k-th distance, so the query's
// threshold drops to it before the screening is repeated. Counts such queries in *nover.
__global__ void tighten_kernel(const uint32_t* __restrict__ count, int qc, int64_t cap, const uint32_t* __restrict__ kth,
                               float cg, uint32_t* __restrict__ thr, int64_t q0, int* __restrict__ nover) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= qc || (int64_t)count[j] <= cap) return;
  const float t = __fmul_ru(__uint_as_float(kth[j]), cg);
  atomicMin(thr + q0 + j, __float_as_uint(t));  // non-negative floats order like their bits
  atomicAdd(nover, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

paris_status make_bf16_map(CUtensorMap* map, const void* base, int64_t rows, int len, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(PARIS_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)len, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)len * 2};
  cuuint32_t box[2] = {(cuuint32_t)BKE, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PARIS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return PARIS_OK;
}

std::mutex g_shadow_mutex;

int sm_count_dense() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

bool dense_supported(const paris_index* idx, int k) {
  return k <= KMAX && idx->len % BKE == 0 && idx->len <= E_MAX_LEN;
}

void dense_margins(int len, float* c1, float* c2) {
  // |d~ - |q-x|^2| <= c1 |q||x| + c2 (|q|^2 + |x|^2):
  //  BF16 rounding of q and x (unit roundoff 2^-8) perturbs each product by (2^-7 + 2^-16)|q_j x_j|;
  //  the tensor-core FP32 accumulation of `len` products is bounded as if every addition could
  //  lose 2^-23 (truncation): gamma' = len 2^-23 / (1 - len 2^-23), on sum |q~_j x~_j|;
  //  |q|^2, |x|^2 in fp32 (gamma_len, u = 2^-24) and the two final fp32 operations (2u);
  //  sum |q_j x_j| <= |q||x| (Cauchy-Schwarz). Everything is inflated by 2^-10 for the
  //  rounding of the margin itself.
  const double ub = std::ldexp(1.0, -8), u = std::ldexp(1.0, -24);
  const double gp = len * std::ldexp(1.0, -23) / (1.0 - len * std::ldexp(1.0, -23));
  const double gl = len * u / (1.0 - len * u);
  const double prod = 2.0 * ub + ub * ub;
  double a = 2.0 * (prod + gp * (1.0 + prod)) + 2.0 * u * (1.0 + prod) * (1.0 + gp);
  double b = gl + 2.0 * u;
  *c1 = std::nextafter((float)(a * (1.0 + std::ldexp(1.0, -10))), INFINITY);
  *c2 = std::nextafter((float)(b * (1.0 + std::ldexp(1.0, -10))), INFINITY);
}

// Norm range of each 64-row tile over its rows inside the series; one warp per tile.
__global__ void tile_range_kernel(const float2* __restrict__ nm, int64_t n, float4* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t tiles = (n + RT - 1) / RT;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tiles; t += warps) {
    float lo = CUDART_INF_F, hi = -CUDART_INF_F, rt = -CUDART_INF_F;
    for (int j = lane; j < RT; j += 32) {
      const int64_t r = t * RT + j;
      if (r < n) {
        const float2 v = nm[r];
        lo = fminf(lo, v.x);
        hi = fmaxf(hi, v.x);
        rt = fmaxf(rt, v.y);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(PARIS_FULL_MASK, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(PARIS_FULL_MASK, hi, o));
      rt = fmaxf(rt, __shfl_xor_sync(PARIS_FULL_MASK, rt, o));
    }
    if (lane == 0) out[t] = make_float4(lo, hi, rt, 0.f);
  }
}

// Row norms are stored for whole row tiles, so a tile's norms are one bulk copy.
size_t norm_bytes(int64_t n) { return (size_t)((n + RT - 1) / RT * RT) * sizeof(float2); }
size_t range_bytes(int64_t n) { return (size_t)((n + RT - 1) / RT) * sizeof(float4); }

bool dense_shape_ok(int len) { return len % BKE == 0 && len <= E_MAX_LEN; }

paris_status alloc_shadow(const paris_index* idx, ShadowBufs* out, cudaStream_t st) {
  *out = ShadowBufs{};
  const size_t bytes = (size_t)idx->n * idx->len * 2;
  out->shadow = dev_alloc(bytes, st);
  out->xnorm = (float2*)dev_alloc(norm_bytes(idx->n), st);
  out->xtile = (float4*)dev_alloc(range_bytes(idx->n), st);
  if (!out->shadow || !out->xnorm || !out->xtile) {
    free_shadow_bufs(idx, out, st);
    return fail(PARIS_ENOMEM, "BF16 shadow of the series (%zu bytes)", bytes);
  }
  return PARIS_OK;
}

void free_shadow_bufs(const paris_index* idx, ShadowBufs* b, cudaStream_t st) {
  dev_free(b->shadow, (size_t)idx->n * idx->len * 2, st);
  dev_free(b->xnorm, norm_bytes(idx->n), st);
  dev_free(b->xtile, range_bytes(idx->n), st);
  *b = ShadowBufs{};
}

// Once the shadow rows and norms are written: zero norms past the series, tile norm ranges,
// the TMA descriptor; the index takes ownership.
paris_status finish_shadow(paris_index* idx, ShadowBufs* b, cudaStream_t st) {
  PARIS_CUDA(cudaMemsetAsync(b->xnorm + idx->n, 0, norm_bytes(idx->n) - (size_t)idx->n * sizeof(float2), st));
  tile_range_kernel<<<sm_count_dense() * 8, 256, 0, st>>>(b->xnorm, idx->n, b->xtile);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  CUtensorMap* map = new CUtensorMap;
  paris_status s = make_bf16_map(map, b->shadow, idx->n, idx->len, BN);
  if (s != PARIS_OK) {
    delete map;
    free_shadow_bufs(idx, b, st);
    return s;
  }
  idx->shadow = b->shadow;
  idx->xnorm = b->xnorm;
  idx->xtile = b->xtile;
  idx->shadow_map = map;
  *b = ShadowBufs{};
  return PARIS_OK;
}

paris_status ensure_shadow(paris_index* idx, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_shadow_mutex);
  if (idx->shadow) return PARIS_OK;
  ShadowBufs b;
  PARIS_TRY(alloc_shadow(idx, &b, st));
  shadow_kernel<<<sm_count_dense() * 8, 256, 0, st>>>(idx->series, idx->n, idx->len, (__nv_bfloat16*)b.shadow,
                                                       b.xnorm, nullptr, 0, idx->n);
  note_launches(1);
  return finish_shadow(idx, &b, st);
}

paris_status launch_tighten(const QueryState& qs, const ChunkState& cs, cudaStream_t st) {
  tighten_kernel<<<(cs.qc + 255) / 256, 256, 0, st>>>(cs.count, cs.qc, cs.cap, cs.kth, qs.cg, qs.thr, cs.q0,
                                                      cs.nover);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status tighten_overflowed(const QueryState& qs, const ChunkState& cs, int* nover, cudaStream_t st) {
  *nover = 0;
  PARIS_CUDA(cudaMemsetAsync(cs.nover, 0, 4, st));
  PARIS_TRY(launch_tighten(qs, cs, st));
  PARIS_CUDA(cudaMemcpyAsync(nover, cs.nover, 4, cudaMemcpyDeviceToHost, st));
  PARIS_CUDA(cudaStreamSynchronize(st));
  return PARIS_OK;
}

void release_shadow(paris_index* idx) {
  if (idx->shadow) dev_free(idx->shadow, (size_t)idx->n * idx->len * 2, nullptr);
  if (idx->xnorm) dev_free(idx->xnorm, norm_bytes(idx->n), nullptr);
  if (idx->xtile) dev_free(idx->xtile, range_bytes(idx->n), nullptr);
  idx->xtile = nullptr;
  delete (CUtensorMap*)idx->shadow_map;
  idx->shadow = nullptr;
  idx->xnorm = nullptr;
  idx->shadow_map = nullptr;
}

// Screens the chunk's queries whose candidate lists overflowed `cap`: their lists are rebuilt
// from the BF16 pass. Eager form: the number of such queries is read back (*nd_out) and exactly
// that many query tiles are launched. Graph form (nd_out == NULL): nothing is read back; one
// launch per possible query tile, each leaving at once when its tile is past the count.
paris_status launch_dense(paris_index* idx, const QueryState& qs, const ChunkState& cs, uint32_t* overflow, int* nd_out,
                          cudaStream_t st) {
  if (nd_out) *nd_out = 0;
  int* slots = cs.dslots;
  int* ndev = cs.dnd;
  dense_select_kernel<<<1, 1024, 0, st>>>(cs.count, cs.qc, cs.cap, slots, ndev);
  note_launches(1);
  int nd = -1;
  int64_t tiles = ((int64_t)cs.qc + BM - 1) / BM;
  if (nd_out) {
    PARIS_CUDA(cudaMemcpyAsync(&nd, ndev, 4, cudaMemcpyDeviceToHost, st));
    PARIS_CUDA(cudaStreamSynchronize(st));
    *nd_out = nd;
    if (nd == 0) return PARIS_OK;
    tiles = ((int64_t)nd + BM - 1) / BM;
  }
  if (!idx->shadow) {
    if (!nd_out) return fail(PARIS_EINTERNAL, "BF16 shadow must exist before a captured screening");
    PARIS_TRY(ensure_shadow(idx, st));
  }
  const int64_t rows_pad = tiles * BM;
  shadow_kernel<<<(unsigned)std::max<int64_t>(1, (rows_pad + 7) / 8), 256, 0, st>>>(
      qs.queries, nd, idx->len, (__nv_bfloat16*)cs.dqbf, cs.dqnm, slots, cs.q0, rows_pad, nd_out ? nullptr : ndev);
  dense_reset_kernel<<<(cs.qc + 255) / 256, 256, 0, st>>>(cs.count, slots, ndev);
  note_launches(2);
  PARIS_CUDA(cudaGetLastError());
  // set on every launch: the attribute is per device, and a cached flag would not be thread-safe
  PARIS_CUDA(cudaFuncSetAttribute(bound_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DENSE_SMEM));
  PARIS_CUDA(cudaFuncSetAttribute(emit_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EMIT_SMEM));
  PARIS_CUDA(cudaFuncSetAttribute(emit_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EMIT_SMEM));
  DenseParams P;
  P.wait_ns = wait_limit_ns();
  P.n = idx->n;
  P.len = idx->len;
  P.nkb = idx->len / BKE;
  P.nd = nd;
  P.nd_dev = ndev;
  P.xnorm = idx->xnorm;
  P.qbf = (const uint32_t*)cs.dqbf;
  P.xtile = (const float4*)idx->xtile;
  P.qnorm = cs.dqnm;
  P.qslot = slots;
  P.q0 = cs.q0;
  P.thr = qs.thr;
  P.k = qs.k;
  P.cg = qs.cg;
  dense_margins(idx->len, &P.c1, &P.c2);
  P.count = cs.count;
  P.rows = cs.rows;
  P.lb = cs.lb;
  P.cap = cs.cap;
  P.status = qs.status;
  P.overflow = overflow;
  const int64_t ntiles = (idx->n + BN - 1) / BN;
  const int grid = (int)std::max<int64_t>(std::min<int64_t>(ntiles, sm_count_dense()), GROUPS);
  const CUtensorMap* mapB = (const CUtensorMap*)idx->shadow_map;
  P.qg = std::min(QG, (65536 / idx->len) & ~31);
  const int64_t rows_max = tiles * BM;  // screened queries at most (nd, or the chunk when nd is on the device)
  for (int phase = 1; phase <= 2; ++phase) {
    // the threshold pass: k = 1 in the rows-on-M shape; k > 1 with queries on M (two tiles of
    // 128 queries of up to 256 values in shared memory); longer series with k > 1 skip it (it only
    // tightens the thresholds: the emission pass is exact from any valid threshold)
    const bool qm = phase == 1 && qs.k > 1;
    if (qm && idx->len > MAX_KB * BKE) continue;
    const int64_t gsize = qm ? (int64_t)QTILES * BM : P.qg;
    const int groups = (int)((rows_max + gsize - 1) / gsize);
    for (int g0 = 0; g0 < groups; g0 += GROUPS) {
      P.group0 = g0;
      if (phase == 1 && !qm)
        emit_kernel<1><<<grid, DENSE_THREADS, EMIT_SMEM, st>>>(*mapB, P);
      else if (qm)
        bound_kernel<<<grid, DENSE_THREADS, DENSE_SMEM, st>>>(*mapB, P);
      else
        emit_kernel<2><<<grid, DENSE_THREADS, EMIT_SMEM, st>>>(*mapB, P);
      note_launches(1);
      PARIS_CUDA(cudaGetLastError());
    }
  }
  return PARIS_OK;
}

size_t dense_query_rows(int64_t qc) { return (size_t)((qc + BM - 1) / BM * BM); }

}  // namespace paris
