// Index build, step 1: exact PAA -> iSAX symbols -> summary slot + interleaved key, one warp
// per series (Sec. 2.2; Alg. 2 ConvertToSAX and SAX[position] store).
#include <cuda_bf16.h>

#include "internal.h"

namespace paris {

namespace {

constexpr int kEncodeThreads = 256;

// The FP64 breakpoint whose order key is k (inverse of double_order_key).
__device__ __forceinline__ double key_to_double(uint64_t k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Two series per warp: lanes 0-15 hold the segments of series 2p, lanes 16-31 those of 2p+1.
template <int SEGV>
__global__ void __launch_bounds__(kEncodeThreads) encode_kernel(
    const float* __restrict__ series, int64_t n, RowShape sh, int card, int bits,
    const uint64_t* __restrict__ beta_keys_g, uint8_t* __restrict__ sax_rot,
    uint8_t* __restrict__ sax_plain, uint64_t* __restrict__ key64, double* __restrict__ paa_out,
    uint32_t* __restrict__ status, __nv_bfloat16* __restrict__ shadow, float2* __restrict__ xnorm) {
  __shared__ uint64_t beta_keys[255];
  __shared__ float2 beta32[255];  // each breakpoint between two fp32 values: (round down, round up)
  __shared__ uint8_t sym_tab[kSymBuckets];
  for (int i = threadIdx.x; i < card - 1; i += blockDim.x) {
    beta_keys[i] = beta_keys_g[i];
    const double v = key_to_double(beta_keys_g[i]);
    beta32[i] = make_float2(__double2float_rd(v), __double2float_ru(v));
  }
  __syncthreads();
  build_symbol_table(beta_keys, card, sym_tab);
  __syncthreads();
  const int lane = threadIdx.x & 31, half = lane >> 4, seg = lane & 15;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t pairs = (n + 1) >> 1;
  bool nonfinite = false;
  // fast path with the segment in registers: the next row pair's values are loaded while this
  // pair is summed, encoded and converted (the loads are the kernel's bound)
  constexpr bool kPre = SEGV <= 4;
  constexpr int PN = SEGV <= 4 ? SEGV : 1;
  const bool pre = kPre && sh.fast;
  auto load_pair = [&](int64_t pr, float4 (&x)[PN]) {
    const int64_t r = 2 * pr + half;
    const bool act = pr < pairs && r < n && seg < sh.w;
    const float4* p = reinterpret_cast<const float4*>(series + r * (int64_t)sh.len + (act ? seg * sh.s : 0));
#pragma unroll
    for (int v = 0; v < PN; ++v) x[v] = act ? __ldcs(p + v) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  // Symbols without the exact sum, when the PAA itself is not wanted: the fp32 sum S of the s
  // values (any order) errs by at most gamma_{s-1} * s * M (M = largest magnitude), so the exact
  // PAA p = RN64(exact sum) / s lies within E = ru(M * (s-1) * 2^-24 * (1 + 2^-15)) + 2^-148 of
  // P = S / s (the last term covers a subnormal quotient; the factor covers gamma and the FP64
  // rounding). When the fp32 brackets of the breakpoints put no breakpoint inside [P - E, P + E],
  // the symbol of every value of that interval, p included, is the symbol of P; otherwise the
  // lane takes the exact sum below. A breakpoint lies that close to a segment mean in well under
  // 0.1% of the lanes for random walks at 256 symbols.
  const bool quick = pre && paa_out == nullptr;
  const float inv_s = __uint_as_float((uint32_t)(127 - (sh.log2s > 0 ? sh.log2s : 0)) << 23);
  const float cE = __fmul_ru((float)(sh.s - 1), 0x1.0002p-24f);
  int64_t pr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float4 nxt[PN];
  if (pre) load_pair(pr, nxt);
  for (; pr < pairs; pr += warps) {
    float4 cur[PN];
#pragma unroll
    for (int v = 0; v < PN; ++v) cur[v] = nxt[v];
    if (pre) load_pair(pr + warps, nxt);
    const int64_t r0 = 2 * pr;
    const bool has1 = r0 + 1 < n;
    const float* row0 = series + r0 * (int64_t)sh.len;
    const float* row1 = has1 ? row0 + sh.len : nullptr;
    const int64_t r = r0 + half;
    const bool rv = half == 0 || has1;
    const bool act = rv && seg < sh.w;
    int sym = 0;
    bool decided = !act;
    if (quick && act) {
      uint32_t mb = 0u;
      float S = 0.f;
#pragma unroll
      for (int v = 0; v < PN; ++v) {
        const float4 x = cur[v];
        mb = max(mb, max(max(__float_as_uint(x.x) & 0x7fffffffu, __float_as_uint(x.y) & 0x7fffffffu),
                         max(__float_as_uint(x.z) & 0x7fffffffu, __float_as_uint(x.w) & 0x7fffffffu)));
        S = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(S, x.x), x.y), x.z), x.w);
      }
      if (mb < 0x7f800000u) {  // NaN and infinity take the exact path (which reports them)
        const float P = S * inv_s;
        const float E = __fadd_ru(__fmul_ru(__uint_as_float(mb), cE), 0x1p-148f);
        const float lo = __fsub_rd(P, E), hi = __fadd_ru(P, E);
        const float f = fminf(fmaxf(P, -8.0f), 7.99f);
        int b = (int)((f + 8.0f) * 256.0f);
        b = b < 0 ? 0 : (b > kSymBuckets - 1 ? kSymBuckets - 1 : b);
        int s0 = sym_tab[b];
        s0 = s0 > card - 1 ? card - 1 : s0;
        if (s0 < card - 1 && beta32[s0].x <= P) ++s0;
        decided = (s0 == 0 || beta32[s0 - 1].y <= lo) && (s0 == card - 1 || beta32[s0].x > hi);
        if (decided) sym = s0;
      }
    }
    double paa = 0.0;
    if (!decided || !quick) {
      float fest = 0.f;
      const bool fin = pre ? lane_segment_paa<SEGV, true>(row0, row1, sh, lane, paa, fest, cur)
                           : lane_segment_paa<SEGV>(row0, row1, sh, lane, paa, fest);
      if (!fin) nonfinite = true;
      if (act) sym = symbol_of(paa, fest, beta_keys, sym_tab, card);
    }
    const uint64_t key = warp_pair_key64(sym, lane, sh.w, bits);
    // rotated summary slot: slot j holds segment (j + r) mod 16 (0 when that segment >= w)
    const int src = (seg + (int)(r & 15)) & 15;
    const int b = __shfl_sync(PARIS_FULL_MASK, sym, (half << 4) | src);
    if (SEGV <= 4 && shadow) {
      // BF16 copy of the lane's segment and the row's fp32 squared norm (the mixed-precision
      // screening's inputs), from the values this warp holds (zeros for an inactive lane)
      const bool act = rv && seg < sh.w;
      float acc = 0.f;
#pragma unroll
      for (int v = 0; v < PN; ++v) {
        const float4 x = cur[v];
        acc = fmaf(x.x, x.x, acc);
        acc = fmaf(x.y, x.y, acc);
        acc = fmaf(x.z, x.z, acc);
        acc = fmaf(x.w, x.w, acc);
        if (act) {
          __nv_bfloat162 lo = __floats2bfloat162_rn(x.x, x.y), hi = __floats2bfloat162_rn(x.z, x.w);
          uint2 pk = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
          *reinterpret_cast<uint2*>(shadow + r * (int64_t)sh.len + seg * sh.s + 4 * v) = pk;
        }
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(PARIS_FULL_MASK, acc, o);  // within the half
      if (rv && seg == 0) xnorm[r] = make_float2(acc, __fsqrt_ru(acc));
    }
    if (rv) {
      sax_rot[r * PARIS_SAX_BYTES + seg] = (uint8_t)(src < sh.w ? b : 0);
      if (sax_plain && seg < sh.w) sax_plain[r * sh.w + seg] = (uint8_t)sym;
      if (paa_out && seg < sh.w) paa_out[r * sh.w + seg] = paa;
      if (seg == 0) key64[r] = key;
    }
  }
  if (nonfinite) atomicOr(status, DEV_NONFINITE);
}

__global__ void unrotate_kernel(const uint8_t* __restrict__ sax_rot, int64_t n, int w,
                                uint8_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * w) return;
  int64_t r = i / w;
  int seg = (int)(i - r * w);
  int slot = (seg - (int)(r & 15)) & 15;
  out[i] = sax_rot[r * PARIS_SAX_BYTES + slot];
}

int encode_grid(int64_t n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = ((n + 1) / 2 + (kEncodeThreads / 32) - 1) / (kEncodeThreads / 32);
  int64_t cap = (int64_t)sms * 8;  // 8 resident blocks of 256 threads per SM
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

RowShape make_row_shape(int len, int w, const void* base_ptr) {
  RowShape sh;
  sh.len = len;
  sh.w = w;
  sh.s = len / w;
  sh.log2s = ((sh.s & (sh.s - 1)) == 0) ? __builtin_ctz((unsigned)sh.s) : -1;
  bool aligned = ((uintptr_t)base_ptr % 16u) == 0u;
  sh.fast = (len % 4 == 0) && aligned && sh.log2s >= 2 && sh.s <= 128;
  return sh;
}

paris_status launch_encode(const float* series, int64_t n, const RowShape& sh, int card, int bits,
                           const uint64_t* beta_keys, uint8_t* sax_rot, uint8_t* sax_plain,
                           uint64_t* key64, double* paa, uint32_t* status, cudaStream_t st, void* shadow,
                           float2* xnorm) {
  if (n <= 0) return PARIS_OK;
  if (shadow && !(sh.fast && sh.s / 4 <= 4)) return fail(PARIS_EINVAL, "BF16 shadow during encode needs len/w <= 16");
  int grid = encode_grid(n);
  const int segv = sh.fast ? sh.s / 4 : 1;
#define ENC(SV)                                                                                     \
  encode_kernel<SV><<<grid, kEncodeThreads, 0, st>>>(series, n, sh, card, bits, beta_keys, sax_rot, \
                                                     sax_plain, key64, paa, status,                \
                                                     (__nv_bfloat16*)shadow, xnorm)
  switch (segv) {
    case 1: ENC(1); break;
    case 2: ENC(2); break;
    case 4: ENC(4); break;
    case 8: ENC(8); break;
    case 16: ENC(16); break;
    default: ENC(32); break;
  }
#undef ENC
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

paris_status launch_unrotate_sax(const uint8_t* sax_rot, int64_t n, int w, uint8_t* out,
                                 cudaStream_t st) {
  int64_t total = n * w;
  if (total <= 0) return PARIS_OK;
  unrotate_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(sax_rot, n, w, out);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

}  // namespace paris
