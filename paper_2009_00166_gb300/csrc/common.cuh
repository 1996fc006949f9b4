// Device-side building blocks shared by the build and query kernels of the GB300 ParIS+ path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PARIS_FULL_MASK 0xffffffffu
#define PARIS_SAX_BYTES 16  // one summary slot per row: up to 16 segments of 8 bits

namespace paris {

// Device status word bits (written with atomicOr, read back by the host after a call).
enum : uint32_t {
  DEV_NONFINITE = 1u,      // a NaN or infinite input value
  DEV_CAND_OVERFLOW = 2u,  // a candidate list overflowed its capacity
  DEV_CONT_OVERFLOW = 4u,  // too many exact-re-rank contenders
  DEV_TIMEOUT = 8u,        // a bounded wait expired
  DEV_BADROW = 16u,        // a row index outside the collection
};

__device__ __forceinline__ uint64_t double_order_key(double v) {
  // Monotone map of IEEE doubles to unsigned integers (-0 normalised to +0 first); integer
  // operations only.
  uint64_t u = (uint64_t)__double_as_longlong(v);
  if ((u << 1) == 0ull) u = 0ull;
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// RN64(S) * 2^e for a signed 64-bit integer S, built bit by bit (round to nearest even).
// Requires the result to be a normal double (|S| * 2^e within [2^-1022, 2^1023]).
// 2^k as a double, exact for -1022 <= k <= 1023.
__device__ __forceinline__ double exp2_int(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

__device__ __forceinline__ double fixed_to_double(int64_t S, int e) {
  if (S == 0) return 0.0;
  uint64_t sign = S < 0 ? 0x8000000000000000ull : 0ull;
  uint64_t m = S < 0 ? (uint64_t)(-S) : (uint64_t)S;
  int p = 63 - __clzll((long long)m);  // position of the leading one
  uint64_t mant;
  if (p <= 52) {
    mant = m << (52 - p);
  } else {
    int sh = p - 52;
    mant = m >> sh;
    uint64_t rem = m & ((1ull << sh) - 1ull);
    uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      mant += 1ull;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        p += 1;
      }
    }
  }
  uint64_t biased = (uint64_t)(p + e + 1023);
  return __longlong_as_double((long long)(sign | (biased << 52) | (mant & ((1ull << 52) - 1ull))));
}

// --- exact wide accumulator: 320-bit two's complement, least significant bit 2^-149 --------
// Holds any exact sum of up to 2^16 finite fp32 values (|sum| < 2^144).
struct Wide {
  uint32_t limb[10];
};

__device__ __forceinline__ void wide_zero(Wide& a) {
#pragma unroll
  for (int i = 0; i < 10; ++i) a.limb[i] = 0u;
}

__device__ __forceinline__ void wide_add_f32(Wide& a, float x) {
  uint32_t u = __float_as_uint(x);
  uint32_t be = (u >> 23) & 0xffu;
  uint32_t mant = (u & 0x7fffffu) | (be ? 0x800000u : 0u);
  if (mant == 0u) return;
  int off = (be ? (int)be : 1) - 150 + 149;  // bit offset of the mantissa's unit in the limbs
  int li = off >> 5, sh = off & 31;
  uint64_t v = (uint64_t)mant << sh;  // < 2^55
  uint32_t part[3] = {(uint32_t)v, (uint32_t)(v >> 32), 0u};
  if (!(u >> 31)) {
    uint64_t carry = 0;
    for (int i = li; i < 10; ++i) {
      uint64_t t = (uint64_t)a.limb[i] + (i - li < 3 ? part[i - li] : 0u) + carry;
      a.limb[i] = (uint32_t)t;
      carry = t >> 32;
      if (i - li >= 2 && carry == 0) break;
    }
  } else {
    uint64_t borrow = 0;
    for (int i = li; i < 10; ++i) {
      uint64_t sub = (uint64_t)(i - li < 3 ? part[i - li] : 0u) + borrow;
      uint64_t cur = a.limb[i];
      a.limb[i] = (uint32_t)(cur - sub);
      borrow = cur < sub ? 1 : 0;
      if (i - li >= 2 && borrow == 0) break;
    }
  }
}

// Correctly rounded (nearest even) FP64 value of the accumulator.
__device__ __forceinline__ double wide_to_double(const Wide& a0) {
  Wide a = a0;
  bool neg = (a.limb[9] >> 31) != 0u;
  if (neg) {  // two's complement negate
    uint64_t carry = 1;
    for (int i = 0; i < 10; ++i) {
      uint64_t t = (uint64_t)(~a.limb[i]) + carry;
      a.limb[i] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  int top = -1;
  for (int i = 9; i >= 0; --i)
    if (a.limb[i]) {
      top = i;
      break;
    }
  if (top < 0) return 0.0;
  int p = top * 32 + (31 - __clz(a.limb[top]));  // leading one position
  // gather bits [p-63, p] into a 64-bit window and a sticky flag for the rest
  auto bit_window = [&](int lo) -> uint64_t {  // 64 bits starting at bit `lo` (may be < 0)
    uint64_t r = 0;
    for (int b = 0; b < 64; b += 32) {
      int pos = lo + b;  // fetch 32 bits at pos
      uint32_t w32;
      if (pos >= 0) {
        int li = pos >> 5, sh = pos & 31;
        uint32_t lo32 = li < 10 ? a.limb[li] : 0u;
        uint32_t hi32 = li + 1 < 10 ? a.limb[li + 1] : 0u;
        w32 = sh ? (lo32 >> sh) | (hi32 << (32 - sh)) : lo32;
      } else if (pos > -32) {
        w32 = a.limb[0] << (-pos);
      } else {
        w32 = 0u;
      }
      r |= (uint64_t)w32 << b;
    }
    return r;
  };
  int lo = p - 63;
  uint64_t win = bit_window(lo);  // bit 63 of win is the leading one
  bool sticky = false;
  if (lo > 0) {
    for (int i = 0; i < 10 && !sticky; ++i) {
      int b0 = i * 32;
      if (b0 >= lo) break;
      uint32_t m = a.limb[i];
      if (b0 + 32 > lo) m &= (1u << (lo - b0)) - 1u;
      sticky = m != 0u;
    }
  }
  uint64_t mant = win >> 11;  // 53 bits
  uint64_t rest = win & 0x7ffull;
  // round to nearest, ties to even: above half, or exactly half with an odd last bit
  bool up = (rest > 0x400ull) || (rest == 0x400ull && (sticky || (mant & 1ull)));
  if (up) {
    mant += 1ull;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      p += 1;
    }
  }
  int e = p - 149;  // value = 1.mant * 2^(p-149)
  uint64_t biased = (uint64_t)(e + 1023);
  return __longlong_as_double(
      (long long)((neg ? 0x8000000000000000ull : 0ull) | (biased << 52) | (mant & ((1ull << 52) - 1ull))));
}

// --- fixed-point conversion for the fast exact path ------------------------------------------
// x as an integer multiple of 2^lambda; sets `inexact` if x has bits below 2^lambda.
__device__ __forceinline__ int64_t to_fixed(float x, int lambda, bool& inexact) {
  uint32_t u = __float_as_uint(x);
  uint32_t be = (u >> 23) & 0xffu;
  uint32_t mant = (u & 0x7fffffu) | (be ? 0x800000u : 0u);
  int e_lsb = (be ? (int)be : 1) - 150;
  int sh = e_lsb - lambda;
  if (mant == 0u) return 0;
  if (sh < 0) {
    inexact = true;
    return 0;
  }
  int64_t v = (int64_t)((uint64_t)mant << sh);
  return (u >> 31) ? -v : v;
}

__device__ __forceinline__ int64_t shfl_xor_i64(int64_t v, int off) {
  return (int64_t)__shfl_xor_sync(PARIS_FULL_MASK, (long long)v, off);
}
__device__ __forceinline__ int64_t shfl_i64(int64_t v, int src) {
  return (int64_t)__shfl_sync(PARIS_FULL_MASK, (long long)v, src);
}

// Starting points of the symbol search: bucket b of [-8, 8) (width 1/256, narrower than any gap
// between consecutive breakpoints of up to 256 symbols) holds the number of breakpoints <= the
// bucket's lower end; the symbol of a value in the bucket is that count or one more.
constexpr int kSymBuckets = 4096;
__device__ __forceinline__ int symbol_search(uint64_t key, const uint64_t* beta_keys, int card);
// Fills the bucket table (shared memory) from the order keys of the breakpoints (shared memory);
// the caller synchronises before use.
__device__ __forceinline__ void build_symbol_table(const uint64_t* beta_keys, int card, uint8_t* tab) {
  for (int b = threadIdx.x; b < kSymBuckets; b += blockDim.x)
    tab[b] = (uint8_t)symbol_search(double_order_key(-8.0 + (double)b * (1.0 / 256.0)), beta_keys, card);
}

// Number of breakpoints <= v (upper region on ties): the bucket table's estimate, moved to the
// exact answer by comparing order keys of the FP64 values (one step at most, up to 8 tried); the
// binary search below is the fallback.
__device__ __forceinline__ int symbol_of(double v, float fest, const uint64_t* beta_keys, const uint8_t* tab,
                                         int card) {
  const uint64_t key = double_order_key(v);
  const float f = fminf(fmaxf(fest, -8.0f), 7.99f);
  int b = (int)((f + 8.0f) * 256.0f);
  b = b < 0 ? 0 : (b > kSymBuckets - 1 ? kSymBuckets - 1 : b);
  int sym = tab[b];
  sym = sym > card - 1 ? card - 1 : sym;
  // answer: beta_keys[sym-1] <= key < beta_keys[sym] (missing ends are -inf / +inf)
  for (int it = 0; it < 8; ++it) {
    if (sym > 0 && beta_keys[sym - 1] > key) {
      --sym;
    } else if (sym < card - 1 && beta_keys[sym] <= key) {
      ++sym;
    } else {
      return sym;
    }
  }
  return symbol_search(key, beta_keys, card);
}

__device__ __forceinline__ int symbol_search(uint64_t key, const uint64_t* beta_keys, int card) {
  int lo = 0, cnt = card - 1;  // upper_bound over beta_keys[0, card-1)
  while (cnt > 0) {
    int half = cnt >> 1;
    if (beta_keys[lo + half] <= key) {
      lo += half + 1;
      cnt -= half + 1;
    } else {
      cnt = half;
    }
  }
  return lo;
}

struct RowShape {
  int len, w, s, log2s;  // log2s = -1 when s is not a power of two
  int fast;              // 1: vectorised fixed-point path applies (s = 4 * SEGV, aligned rows)
};

// Exact PAA (Sec. 2.2) of one (row, segment) per lane. A warp holds two rows: lanes 0-15 the
// segments of `row0`, lanes 16-31 those of `row1` (NULL past the end). Lane l returns, when its
// segment i = l & 15 is < w, PAA_i = RN64(exact sum of the s values of segment i) / s.
// Fast path: the segment's values are integer multiples of 2^lambda, lambda picked from the
// segment's largest exponent so that the sum fits in 63 bits; they are summed exactly in int64
// and rounded once. Segments holding values finer than 2^lambda (or subnormals) take the
// 320-bit exact accumulator instead. Returns false if the lane's segment holds a NaN or infinity.
// With PRE (fast path, SEGV <= 4 only), `pre` already holds the lane's segment values (zeros
// for an inactive lane), so a caller can load the next rows while this one is summed. `fest`
// receives an fp32 estimate of PAA_i (for the symbol search's starting point).
template <int SEGV, bool PRE = false>
__device__ __forceinline__ bool lane_segment_paa(const float* __restrict__ row0, const float* __restrict__ row1,
                                                 const RowShape& sh, int lane, double& paa_out, float& fest,
                                                 const float4 (&pre)[SEGV <= 4 ? SEGV : 1]) {
  const int seg = lane & 15;
  const float* row = (lane >> 4) ? row1 : row0;
  const bool active = row != nullptr && seg < sh.w;
  const int s = sh.s;
  paa_out = 0.0;
  fest = 0.f;
  bool finite = true;
  bool done = false;
  if (sh.fast) {
    const float4* p = reinterpret_cast<const float4*>(row + (active ? (int64_t)seg * s : 0));
    constexpr bool kCache = SEGV <= 4;
    float4 cache[kCache ? SEGV : 1];
    // pass 1: the largest magnitude as bits (NaN and infinity sort above every finite value) and
    // the smallest nonzero one (as bits - 1, so that zeros drop out of the minimum)
    uint32_t mb = 0u, mn = 0xffffffffu;
#pragma unroll
    for (int v = 0; v < SEGV; ++v) {
      float4 x = (PRE && kCache) ? pre[kCache ? v : 0] : (active ? p[v] : make_float4(0.f, 0.f, 0.f, 0.f));
      if (kCache) cache[kCache ? v : 0] = x;
      const uint32_t u0 = __float_as_uint(x.x) & 0x7fffffffu, u1 = __float_as_uint(x.y) & 0x7fffffffu;
      const uint32_t u2 = __float_as_uint(x.z) & 0x7fffffffu, u3 = __float_as_uint(x.w) & 0x7fffffffu;
      mb = max(mb, max(max(u0, u1), max(u2, u3)));
      mn = min(mn, min(min(u0 - 1u, u1 - 1u), min(u2 - 1u, u3 - 1u)));
    }
    if (mb >= 0x7f800000u) {
      finite = false;
      done = true;
    } else if (mb == 0u) {
      paa_out = 0.0;
      done = true;
    } else if ((mb >> 23) != 0u && (int)((mn + 1u) >> 23) >= 25 && (int)(mb >> 23) <= 253 - sh.log2s &&
               (int)(mb >> 23) - (int)((mn + 1u) >> 23) <= 24 - 2 * sh.log2s) {
      // common case: an fp32 pair (hi, lo) with error-free TwoSum steps holds the sum exactly.
      // With s = 2^L values whose nonzero biased exponents lie in [emin, emax]:
      //  * every value, partial sum and TwoSum error is a multiple of mu = 2^(emin-150) (the ulp
      //    of the smallest value), and any multiple of mu of magnitude <= 2^24 mu is an fp32 value;
      //  * |hi| < 2^(emax-126+L), so each error is at most 2^(emax-150+L) and the s-1 nonzero
      //    errors sum to less than 2^(emax-150+2L) <= 2^24 mu when emax - emin <= 24 - 2L: every
      //    lo update is then exact (span <= 16 binades at s = 16, 12 at s = 64, 10 at s = 128);
      //  * emax <= 253 - L keeps every partial sum below the fp32 overflow threshold, and
      //    emin >= 25 keeps mu and every error above the subnormal range.
      // One FP64 addition of the exact pair then rounds the sum once, as the integer path does.
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int v = 0; v < SEGV; ++v) {
        float4 x = kCache ? cache[kCache ? v : 0] : (active ? p[v] : make_float4(0.f, 0.f, 0.f, 0.f));
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float sum = __fadd_rn(hi, xs[c]);
          const float bb = __fsub_rn(sum, hi);
          const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(xs[c], bb));
          hi = sum;
          lo = __fadd_rn(lo, err);
        }
      }
      // divide by s = 2^L by the exponent field (the sum, if nonzero, is a normal FP64 value far
      // above 2^(L-1022): it is a multiple of a normal fp32 value's ulp)
      const double S = __dadd_rn((double)hi, (double)lo);
      const uint64_t sb = (uint64_t)__double_as_longlong(S);
      paa_out = (sb << 1) == 0ull ? 0.0 : __longlong_as_double((long long)(sb - ((uint64_t)sh.log2s << 52)));
      fest = hi * __uint_as_float((uint32_t)(127 - sh.log2s) << 23);
      done = true;
    } else if ((mb >> 23) != 0u) {
      // values are integer multiples of 2^lambda when no nonzero magnitude is below 2^(lambda+23);
      // the sum of s values below 2^(emax-126) then stays below 2^63 * 2^lambda
      const int emax = (int)(mb >> 23);
      const int lambda = emax - 126 + sh.log2s - 63;
      const int te = lambda + 23 + 127;                      // biased exponent of 2^(lambda+23)
      const uint32_t tbits = te >= 1 ? (uint32_t)te << 23 : 0u;  // 0: every fp32 value qualifies
      const bool tiny = tbits != 0u && mn < tbits - 1u;      // a nonzero magnitude below 2^(lambda+23)
      if (!tiny) {
        // each value is (24-bit significand) * 2^(e - 150): in units of 2^lambda that is the
        // significand shifted left by e - 150 - lambda (0..39), added exactly in int64 with
        // integer operations only (no 64-bit conversion instructions)
        int64_t S = 0;
#pragma unroll
        for (int v = 0; v < SEGV; ++v) {
          float4 x = kCache ? cache[kCache ? v : 0] : (active ? p[v] : make_float4(0.f, 0.f, 0.f, 0.f));
          const uint32_t xb[4] = {__float_as_uint(x.x), __float_as_uint(x.y), __float_as_uint(x.z),
                                  __float_as_uint(x.w)};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint32_t ub = xb[c] & 0x7fffffffu;
            const int e = (int)(ub >> 23);
            // normal: implicit leading bit, exponent e; subnormal and zero: none, exponent 1
            const uint32_t m = e ? ((ub & 0x7fffffu) | 0x800000u) : (ub & 0x7fffffu);
            const int shl = max((e ? e : 1) - 150 - lambda, 0);  // >= 0 for every nonzero value here
            const int64_t mag = (int64_t)((uint64_t)m << shl);
            S += (xb[c] >> 31) ? -mag : mag;
          }
        }
        paa_out = fixed_to_double(S, lambda - sh.log2s);  // s is a power of two on this path
        done = true;
      }
    }
  }
  if (!done && active) {
    Wide acc;
    wide_zero(acc);
    const float* p = row + (int64_t)seg * s;
    for (int j = 0; j < s; ++j) {
      float x = p[j];
      if (((__float_as_uint(x) >> 23) & 0xffu) == 0xffu) finite = false;
      wide_add_f32(acc, x);
    }
    double S = wide_to_double(acc);
    paa_out = sh.log2s >= 0 ? S * (1.0 / (double)(1 << sh.log2s)) : __ddiv_rn(S, (double)s);
  }
  if (done && fest == 0.f && paa_out != 0.0) fest = __double2float_rn(paa_out);
  if (!done) fest = __double2float_rn(paa_out);
  return finite;
}

template <int SEGV>
__device__ __forceinline__ bool lane_segment_paa(const float* __restrict__ row0, const float* __restrict__ row1,
                                                 const RowShape& sh, int lane, double& paa_out, float& fest) {
  const float4 none[SEGV <= 4 ? SEGV : 1] = {};
  return lane_segment_paa<SEGV, false>(row0, row1, sh, lane, paa_out, fest, none);
}

// Top 64 bits of the bit-plane interleaved key of both rows of a warp (lanes 0-15: row 0,
// lanes 16-31: row 1; lane i of a half passes the symbol of segment i, 0 when i >= w).
// Plane j holds bit (bits-1-j) of segments 0..w-1, segment 0 first.
__device__ __forceinline__ uint64_t warp_pair_key64(int sym, int lane, int w, int bits) {
  uint64_t hi = 0, lo = 0;
  int filled = 0;
  // only the planes that reach the top 64 bits: ceil(64 / w) of them (4 at w = 16)
  const int planes = min(bits, (64 + w - 1) / w);
  for (int j = 0; j < planes; ++j) {
    const int b = bits - 1 - j;
    const uint32_t m = __brev(__ballot_sync(PARIS_FULL_MASK, (sym >> b) & 1));
    // row 0's lanes 0..15 are now bits 31..16, row 1's lanes 16..31 are bits 15..0
    const uint32_t half = (lane >> 4) ? (m & 0xffffu) : (m >> 16);
    const uint64_t plane = (uint64_t)(half >> (16 - w));
    hi = (hi << w) | (lo >> (64 - w));
    lo = (lo << w) | plane;
    filled += w;
  }
  const int sh = 128 - filled;
  if (sh >= 64) return lo << (sh - 64);
  if (sh > 0) return (hi << sh) | (lo >> (64 - sh));
  return hi;
}

// Exclusive prefix over m values in one block (blockDim.x a multiple of 32, at most 1024): value(j)
// gives the j-th value, write(j, excl, v) receives its exclusive prefix; returns the total. Every
// thread of the block must call it.
template <typename Value, typename Write>
__device__ uint64_t block_prefix(int m, Value value, Write write) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < m; base += blockDim.x) {
    const int j = base + threadIdx.x;
    const uint64_t v = j < m ? (uint64_t)value(j) : 0ull;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(PARIS_FULL_MASK, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t y = lane < nw ? s_w[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t z = __shfl_up_sync(PARIS_FULL_MASK, y, o);
        if (lane >= o) y += z;
      }
      if (lane < nw) s_w[lane] = y;
    }
    __syncthreads();
    if (j < m) write(j, s_carry + (warp ? s_w[warp - 1] : 0ull) + x - v, v);
    __syncthreads();
    if (threadIdx.x == 0) s_carry += s_w[nw - 1];
    __syncthreads();
  }
  return s_carry;
}

}  // namespace paris
