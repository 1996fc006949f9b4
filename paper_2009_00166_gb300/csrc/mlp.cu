// Learned best-so-far proposal: a 16 -> 256 -> 256 -> 4096 MLP over the query PAA that ranks
// 12-bit key-prefix buckets (first bit of segments 0..11). Training (softmax cross-entropy,
// AdamW on FP32 master weights) and inference run in this file's kernels: BF16 GEMMs on the
// 5th-generation tensor cores (tcgen05.mma, operands in shared memory, FP32 accumulation in
// tensor memory) with fused bias + exact-erf GELU epilogues.
#include <cuda_bf16.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "query.cuh"
#include "tcgen05.cuh"

struct paris_seed_model {
  static constexpr int IN = 16, HID = 256, OUT = 4096;
  float* w[6] = {};           // FP32 master: W1 [256][16], b1, W2 [256][256], b2, W3 [4096][256], b3
  __nv_bfloat16* wb[3] = {};  // BF16 copies of W1, W2, W3 used by the GEMMs
  float* m[6] = {};           // AdamW first moments
  float* v[6] = {};           // AdamW second moments
  size_t count[6] = {};
  int64_t step = 0;
};

namespace paris {

namespace {

constexpr int EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2;

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// GEMM tiles: 128 rows of C (the MMA M side, one TMEM lane each) x 128 columns (N), K in blocks
// of 64 BF16 values (one 128-byte row of the swizzled layout).
constexpr int T_BM = 128, T_BN = 128, T_BK = 64, T_THREADS = 128;
constexpr size_t T_TILE = (size_t)T_BM * 128;  // one operand's K block: 128 rows x 128 bytes
// 56 KB of shared memory per CTA: at most four CTAs per SM, whose 128 TMEM columns each fit the
// SM's 512 (an allocation then never waits for another CTA)
constexpr size_t T_SMEM = 56 * 1024;
static_assert(1024 + 2 * T_TILE + 64 <= T_SMEM, "tiles and barrier fit");
constexpr uint32_t T_TMEM_COLS = 128;

__device__ uint32_t g_gemm_status;  // set when a GEMM's wait for its MMAs ran out

// C[M][N] = sum_k A(m,k) B(k,n) with A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn];
// operands rounded to BF16 when staged in shared memory, FP32 accumulation in tensor memory.
// Per K block all threads stage both operands (16-byte chunks, 128-byte swizzle, K-major), one
// thread issues four 128 x 128 x 16 MMAs and commits them to an mbarrier that every thread waits
// on (bounded) before the next staging. Epilogues: store, + bias[n], or + bias[n] then GELU
// (C receives the pre-activation, H the activation).
template <typename TA, typename TB, int EPI>
__global__ void __launch_bounds__(T_THREADS) gemm_tc_kernel(int M, int N, int K, const TA* __restrict__ A,
                                                            int64_t sam, int64_t sak, const TB* __restrict__ B,
                                                            int64_t sbk, int64_t sbn, float* __restrict__ C,
                                                            int64_t ldc, const float* __restrict__ bias,
                                                            float* __restrict__ H, uint64_t wait_ns) {
  extern __shared__ uint8_t g_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)g_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + T_TILE;
  uint64_t* bar = (uint64_t*)(sB + T_TILE);
  uint32_t* holder = (uint32_t*)(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * T_BM, n0 = blockIdx.x * T_BN;
  const uint32_t b_mma = tc::smem_u32(bar);
  if (tid == 0) tc::mbar_init(b_mma, 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(holder), T_TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *holder;
  const uint64_t deadline = tc::globaltimer() + wait_ns;
  constexpr uint32_t idesc = tc::idesc_bf16(T_BM, T_BN);
  bool ok = true;
  uint32_t phase = 0;
  const int nkb = (K + T_BK - 1) / T_BK;
  for (int kb = 0; kb < nkb && ok; ++kb) {
    const int k0 = kb * T_BK;
    // row r's 16-byte chunk j (elements k0 + 8j .. k0 + 8j + 7) at r * 128 + 16 * (j ^ (r mod 8))
    for (int e = tid; e < T_BM * 8; e += T_THREADS) {
      const int r = e >> 3, j = e & 7;
      float va[8], vb[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + 8 * j + i;
        va[i] = (m0 + r < M && k < K) ? to_f(A[(int64_t)(m0 + r) * sam + (int64_t)k * sak]) : 0.f;
        vb[i] = (n0 + r < N && k < K) ? to_f(B[(int64_t)k * sbk + (int64_t)(n0 + r) * sbn]) : 0.f;
      }
      uint4 pa, pb;
      __nv_bfloat162 t;
#define PACK(dst, src)                                   \
  t = __floats2bfloat162_rn(src[0], src[1]);             \
  dst.x = *reinterpret_cast<uint32_t*>(&t);              \
  t = __floats2bfloat162_rn(src[2], src[3]);             \
  dst.y = *reinterpret_cast<uint32_t*>(&t);              \
  t = __floats2bfloat162_rn(src[4], src[5]);             \
  dst.z = *reinterpret_cast<uint32_t*>(&t);              \
  t = __floats2bfloat162_rn(src[6], src[7]);             \
  dst.w = *reinterpret_cast<uint32_t*>(&t);
      PACK(pa, va)
      PACK(pb, vb)
#undef PACK
      const int off = r * 128 + ((j ^ (r & 7)) << 4);
      *reinterpret_cast<uint4*>(sA + off) = pa;
      *reinterpret_cast<uint4*>(sB + off) = pb;
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < T_BK / 16; ++ks)
        tc::mma_bf16(tmem, tc::desc_sw128(tc::smem_u32(sA) + 32 * ks), tc::desc_sw128(tc::smem_u32(sB) + 32 * ks),
                     idesc, (kb | ks) ? 1u : 0u);
      tc::commit(b_mma);
    }
    // the MMAs read shared memory until they complete: every thread waits before restaging
    ok = tc::mbar_wait_until(b_mma, phase, deadline);
    phase ^= 1u;
    tc::fence_after();
    ok = __syncthreads_and(ok);
  }
  if (ok) {
    const int row = m0 + warp * 32 + lane;  // TMEM lane = row of the tile
#pragma unroll 1
    for (int c0 = 0; c0 < T_BN; c0 += 32) {
      if (n0 + c0 >= N) break;
      uint32_t v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int col = n0 + c0 + jj;
          if (col < N) {
            float val = __uint_as_float(v[jj]);
            if (EPI != EPI_STORE) val += bias[col];
            C[(int64_t)row * ldc + col] = val;
            if (EPI == EPI_BIAS_GELU) H[(int64_t)row * ldc + col] = gelu_f(val);
          }
        }
      }
    }
  } else {
    // the MMAs were not seen to finish: wait (at most 0.1 s more) before the tensor memory they
    // write is released, and report the timeout
    if (tid == 0) atomicOr(&g_gemm_status, 1u);
    tc::mbar_wait_until(b_mma, phase ^ 1u, tc::globaltimer() + 100000000ull);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_free(tmem, T_TMEM_COLS);
  }
}

template <typename TA, typename TB, int EPI>
void gemm(int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk, int64_t sbn, float* C,
          int64_t ldc, const float* bias, float* H, cudaStream_t st) {
  cudaFuncSetAttribute(gemm_tc_kernel<TA, TB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T_SMEM);
  dim3 grid((N + T_BN - 1) / T_BN, (M + T_BM - 1) / T_BM);
  gemm_tc_kernel<TA, TB, EPI><<<grid, T_THREADS, T_SMEM, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, H,
                                                               wait_limit_ns());
  note_launches(1);
}

// PARIS_ETIMEOUT when a GEMM since the last check gave up waiting for its MMAs (then cleared).
paris_status check_gemm_status(cudaStream_t st) {
  uint32_t s = 0;
  PARIS_CUDA(cudaMemcpyFromSymbolAsync(&s, g_gemm_status, 4, 0, cudaMemcpyDeviceToHost, st));
  PARIS_CUDA(cudaStreamSynchronize(st));
  if (s) {
    const uint32_t zero = 0;
    PARIS_CUDA(cudaMemcpyToSymbolAsync(g_gemm_status, &zero, 4, 0, cudaMemcpyHostToDevice, st));
    PARIS_CUDA(cudaStreamSynchronize(st));
    return fail(PARIS_ETIMEOUT, "a seed-model GEMM's wait for its tensor-core operations expired");
  }
  return PARIS_OK;
}

// Mean softmax cross-entropy: per row, D <- (softmax(L) - onehot(y)) / B; loss += CE / B.
__global__ void softmax_ce_kernel(float* __restrict__ L, int N, const int* __restrict__ y, int B,
                                  float* __restrict__ loss) {
  const int row = blockIdx.x;
  float* l = L + (int64_t)row * N;
  __shared__ float red[32];
  float mx = -CUDART_INF_F;
  for (int i = threadIdx.x; i < N; i += blockDim.x) mx = fmaxf(mx, l[i]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(PARIS_FULL_MASK, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = -CUDART_INF_F;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
  __syncthreads();
  float s = 0.f;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += expf(l[i] - mx);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(PARIS_FULL_MASK, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  s = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  const int label = y[row];
  const float ly = l[label];
  __syncthreads();
  const float inv = 1.0f / s, invB = 1.0f / (float)B;
  for (int i = threadIdx.x; i < N; i += blockDim.x) l[i] = (expf(l[i] - mx) * inv - (i == label ? 1.f : 0.f)) * invB;
  if (threadIdx.x == 0 && loss) atomicAdd(loss, (logf(s) + mx - ly) * invB);
}

__global__ void gelu_backward_kernel(float* __restrict__ dh, const float* __restrict__ z, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dh[i] *= gelu_grad_f(z[i]);
}

__global__ void colsum_kernel(const float* __restrict__ D, int B, int N, float* __restrict__ out) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += D[(int64_t)b * N + n];
  out[n] = s;
}

__global__ void adamw_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps, float wd,
                             float c1, float c2, __nv_bfloat16* __restrict__ wb) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  const float wi = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) wb[i] = __float2bfloat16_rn(w[i]);
}

// Batch gather: rows a*i + c (mod m), a coprime with m: a fixed pseudo-random visiting order.
__global__ void gather_batch_kernel(const double* __restrict__ x, const int* __restrict__ y, int64_t m, int64_t start,
                                    int B, uint64_t a, uint64_t c, float* __restrict__ xb, int* __restrict__ yb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * 16) return;
  const int b = i >> 4, f = i & 15;
  const uint64_t src = (a * (uint64_t)(start + b) + c) % (uint64_t)m;
  xb[i] = (float)x[src * 16 + f];
  if (f == 0) yb[b] = y[src];
}

// The r best buckets of each row (r <= 8), ties to the lower bucket; one warp per row.
__global__ void topr_kernel(const float* __restrict__ L, int rows, int N, int r, int* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= rows) return;
  const float* l = L + (int64_t)row * N;
  float bv[8];
  int bi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    bv[j] = -CUDART_INF_F;
    bi[j] = 0x7fffffff;
  }
  for (int i = lane; i < N; i += 32) {  // per-lane sorted top-r (value desc, index asc)
    float x = l[i];
    int xi = i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j < r) {
        const bool better = x > bv[j] || (x == bv[j] && xi < bi[j]);
        const float tv = better ? bv[j] : x;
        const int ti = better ? bi[j] : xi;
        if (better) {
          bv[j] = x;
          bi[j] = xi;
        }
        x = tv;
        xi = ti;
      }
    }
  }
  for (int j = 0; j < r; ++j) {  // r rounds of a warp-wide argmax over the lanes' heads
    float v = bv[0];
    int vi = bi[0];
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(PARIS_FULL_MASK, v, o);
      const int oi = __shfl_xor_sync(PARIS_FULL_MASK, vi, o);
      if (ov > v || (ov == v && oi < vi)) {
        v = ov;
        vi = oi;
      }
    }
    if (lane == 0) out[row * r + j] = vi;
    if (bi[0] == vi) {  // the owner pops its head
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        bv[q] = bv[q + 1];
        bi[q] = bi[q + 1];
      }
      bv[7] = -CUDART_INF_F;
      bi[7] = 0x7fffffff;
    }
  }
}

__global__ void paa_to_f32_kernel(const double* __restrict__ qpaa, int64_t nq, float* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nq * 16) out[i] = (float)qpaa[i];
}

// Keys for the learned leaves: the query key with its top 12 bits replaced by each bucket.
__global__ void bucket_keys_kernel(const uint64_t* __restrict__ qkey, const int* __restrict__ buckets, int64_t nq,
                                   int r, uint64_t* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const uint64_t k0 = qkey[i];
  keys[i * (r + 1)] = k0;
  for (int j = 0; j < r; ++j)
    keys[i * (r + 1) + 1 + j] = (k0 & ((1ull << 52) - 1ull)) | ((uint64_t)buckets[i * r + j] << 52);
}

struct Workspace {
  DevBuf buf;
  float *xb, *z1, *h1, *z2, *h2, *lg, *g, *loss;
  int* yb;
  paris_status alloc(int B, cudaStream_t st) {
    using Mdl = paris_seed_model;
    size_t nparams = (size_t)Mdl::HID * Mdl::IN + Mdl::HID + (size_t)Mdl::HID * Mdl::HID + Mdl::HID +
                     (size_t)Mdl::OUT * Mdl::HID + Mdl::OUT;
    size_t f = (size_t)B * 16 + 4 * (size_t)B * Mdl::HID + (size_t)B * Mdl::OUT + nparams + 64;
    if (!buf.alloc(f * 4 + (size_t)B * 4 + 1024, st)) return fail(PARIS_ENOMEM, "MLP workspace");
    float* p = buf.as<float>();
    xb = p; p += (size_t)B * 16;
    z1 = p; p += (size_t)B * Mdl::HID;
    h1 = p; p += (size_t)B * Mdl::HID;
    z2 = p; p += (size_t)B * Mdl::HID;
    h2 = p; p += (size_t)B * Mdl::HID;
    lg = p; p += (size_t)B * Mdl::OUT;
    g = p; p += nparams;
    loss = p; p += 64;
    yb = reinterpret_cast<int*>(p);
    return PARIS_OK;
  }
};

size_t offset_of(const paris_seed_model* md, int t) {
  size_t o = 0;
  for (int i = 0; i < t; ++i) o += md->count[i];
  return o;
}

// Forward over a batch x [B][16] (device fp32); leaves logits in ws.lg.
void forward(const paris_seed_model* md, const float* x, int B, Workspace& ws, cudaStream_t st) {
  using Mdl = paris_seed_model;
  gemm<float, __nv_bfloat16, EPI_BIAS_GELU>(B, Mdl::HID, Mdl::IN, x, Mdl::IN, 1, md->wb[0], 1, Mdl::IN, ws.z1, Mdl::HID,
                                            md->w[1], ws.h1, st);
  gemm<float, __nv_bfloat16, EPI_BIAS_GELU>(B, Mdl::HID, Mdl::HID, ws.h1, Mdl::HID, 1, md->wb[1], 1, Mdl::HID, ws.z2,
                                            Mdl::HID, md->w[3], ws.h2, st);
  gemm<float, __nv_bfloat16, EPI_BIAS>(B, Mdl::OUT, Mdl::HID, ws.h2, Mdl::HID, 1, md->wb[2], 1, Mdl::HID, ws.lg,
                                       Mdl::OUT, md->w[5], nullptr, st);
}

// Loss and gradients (into ws.g, in W1 b1 W2 b2 W3 b3 order) of a batch (x, y) of size B.
void backward(const paris_seed_model* md, const float* x, const int* y, int B, Workspace& ws, cudaStream_t st) {
  using Mdl = paris_seed_model;
  forward(md, x, B, ws, st);
  softmax_ce_kernel<<<B, 256, 0, st>>>(ws.lg, Mdl::OUT, y, B, ws.loss);
  float* gW1 = ws.g + offset_of(md, 0);
  float* gb1 = ws.g + offset_of(md, 1);
  float* gW2 = ws.g + offset_of(md, 2);
  float* gb2 = ws.g + offset_of(md, 3);
  float* gW3 = ws.g + offset_of(md, 4);
  float* gb3 = ws.g + offset_of(md, 5);
  const float* D3 = ws.lg;
  // dW3[o][j] = sum_b D3[b][o] h2[b][j]
  gemm<float, float, EPI_STORE>(Mdl::OUT, Mdl::HID, B, D3, 1, Mdl::OUT, ws.h2, Mdl::HID, 1, gW3, Mdl::HID, nullptr,
                                nullptr, st);
  colsum_kernel<<<(Mdl::OUT + 255) / 256, 256, 0, st>>>(D3, B, Mdl::OUT, gb3);
  // dh2 = D3 W3 (reuses h1's buffer order: dh2 -> z-sized buffer ws.h2 after its last use)
  float* dh2 = ws.h2;
  gemm<float, __nv_bfloat16, EPI_STORE>(B, Mdl::HID, Mdl::OUT, D3, Mdl::OUT, 1, md->wb[2], Mdl::HID, 1, dh2, Mdl::HID,
                                        nullptr, nullptr, st);
  gelu_backward_kernel<<<(unsigned)(((int64_t)B * Mdl::HID + 255) / 256), 256, 0, st>>>(dh2, ws.z2,
                                                                                       (int64_t)B * Mdl::HID);
  // dW2[i][j] = sum_b dz2[b][i] h1[b][j]
  gemm<float, float, EPI_STORE>(Mdl::HID, Mdl::HID, B, dh2, 1, Mdl::HID, ws.h1, Mdl::HID, 1, gW2, Mdl::HID, nullptr,
                                nullptr, st);
  colsum_kernel<<<(Mdl::HID + 255) / 256, 256, 0, st>>>(dh2, B, Mdl::HID, gb2);
  float* dh1 = ws.h1;  // h1 is no longer needed
  gemm<float, __nv_bfloat16, EPI_STORE>(B, Mdl::HID, Mdl::HID, dh2, Mdl::HID, 1, md->wb[1], Mdl::HID, 1, dh1, Mdl::HID,
                                        nullptr, nullptr, st);
  gelu_backward_kernel<<<(unsigned)(((int64_t)B * Mdl::HID + 255) / 256), 256, 0, st>>>(dh1, ws.z1,
                                                                                       (int64_t)B * Mdl::HID);
  gemm<float, float, EPI_STORE>(Mdl::HID, Mdl::IN, B, dh1, 1, Mdl::HID, x, Mdl::IN, 1, gW1, Mdl::IN, nullptr, nullptr,
                                st);
  colsum_kernel<<<(Mdl::HID + 255) / 256, 256, 0, st>>>(dh1, B, Mdl::HID, gb1);
  note_launches(6);
}

void refresh_bf16(paris_seed_model* md, cudaStream_t st) {
  const int idx[3] = {0, 2, 4};
  for (int i = 0; i < 3; ++i) {
    to_bf16_kernel<<<(unsigned)((md->count[idx[i]] + 255) / 256), 256, 0, st>>>(md->w[idx[i]], md->wb[i],
                                                                               (int64_t)md->count[idx[i]]);
    note_launches(1);
  }
}

void free_model(paris_seed_model* md) {
  if (!md) return;
  for (int i = 0; i < 6; ++i) {
    dev_free(md->w[i], md->count[i] * 4, nullptr);
    dev_free(md->m[i], md->count[i] * 4, nullptr);
    dev_free(md->v[i], md->count[i] * 4, nullptr);
  }
  for (int i = 0; i < 3; ++i) dev_free(md->wb[i], md->count[2 * i] * 2, nullptr);
  delete md;
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void row_buckets_kernel(const uint8_t* __restrict__ sax_rot, int64_t n, int w, int bits,
                                   const int64_t* __restrict__ rows, int64_t m, int32_t* __restrict__ out,
                                   uint32_t* __restrict__ status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t r = rows[i];
  if (r < 0 || r >= n) {
    atomicOr(status, DEV_BADROW);
    out[i] = -1;
    return;
  }
  // first 12 bits of the interleaved key: plane j holds bit (bits-1-j) of segments 0..w-1
  int got = 0, bucket = 0;
  for (int j = 0; j < bits && got < 12; ++j)
    for (int seg = 0; seg < w && got < 12; ++seg) {
      const int sym = sax_rot[r * PARIS_SAX_BYTES + ((seg - (int)(r & 15)) & 15)];
      bucket = (bucket << 1) | ((sym >> (bits - 1 - j)) & 1);
      ++got;
    }
  out[i] = bucket << (12 - got);
}

}  // namespace

paris_status launch_row_buckets(const paris_index* idx, const int64_t* rows, int64_t m, int32_t* out,
                                uint32_t* status, cudaStream_t st) {
  if (m <= 0) return PARIS_OK;
  row_buckets_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(idx->sax, idx->n, idx->w, idx->bits, rows, m, out,
                                                                  status);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return PARIS_OK;
}

// Learned leaves for the approximate search: keys [nq][r+1] (own key first) from the model.
paris_status learned_keys(const paris_index* idx, const paris_seed_model* md, int r, const QueryState& qs,
                          uint64_t* keys, cudaStream_t st) {
  (void)idx;
  Workspace ws;
  const int64_t nq = qs.nq;
  const int B = 1024;
  PARIS_TRY(ws.alloc(B, st));
  DevBuf xb, bk;
  if (!xb.alloc((size_t)nq * 16 * 4, st) || !bk.alloc((size_t)nq * r * 4, st)) return fail(PARIS_ENOMEM, "seed inputs");
  paa_to_f32_kernel<<<(unsigned)((nq * 16 + 255) / 256), 256, 0, st>>>(qs.qpaa, nq, xb.as<float>());
  note_launches(1);
  for (int64_t b0 = 0; b0 < nq; b0 += B) {
    const int nb = (int)std::min<int64_t>(B, nq - b0);
    forward(md, xb.as<float>() + b0 * 16, nb, ws, st);
    topr_kernel<<<(nb + 7) / 8, 256, 0, st>>>(ws.lg, nb, paris_seed_model::OUT, r, bk.as<int>() + b0 * r);
    note_launches(1);
  }
  bucket_keys_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(qs.qkey, bk.as<int>(), nq, r, keys);
  note_launches(1);
  PARIS_CUDA(cudaGetLastError());
  return check_gemm_status(st);
}

}  // namespace paris

using namespace paris;

extern "C" {

paris_status paris_seed_model_create(uint64_t init_seed, void* stream, paris_seed_model** out) {
  clear_error();
  if (!out) return fail(PARIS_EINVAL, "out is NULL");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  paris_seed_model* md = new (std::nothrow) paris_seed_model();
  if (!md) return fail(PARIS_ENOMEM, "model object");
  using Mdl = paris_seed_model;
  const size_t cnt[6] = {(size_t)Mdl::HID * Mdl::IN, Mdl::HID, (size_t)Mdl::HID * Mdl::HID, Mdl::HID,
                         (size_t)Mdl::OUT * Mdl::HID, Mdl::OUT};
  for (int i = 0; i < 6; ++i) {
    md->count[i] = cnt[i];
    md->w[i] = (float*)dev_alloc(cnt[i] * 4, st);
    md->m[i] = (float*)dev_alloc(cnt[i] * 4, st);
    md->v[i] = (float*)dev_alloc(cnt[i] * 4, st);
    if (!md->w[i] || !md->m[i] || !md->v[i]) {
      free_model(md);
      return fail(PARIS_ENOMEM, "model parameters");
    }
    cudaMemsetAsync(md->m[i], 0, cnt[i] * 4, st);
    cudaMemsetAsync(md->v[i], 0, cnt[i] * 4, st);
  }
  for (int i = 0; i < 3; ++i) {
    md->wb[i] = (__nv_bfloat16*)dev_alloc(cnt[2 * i] * 2, st);
    if (!md->wb[i]) {
      free_model(md);
      return fail(PARIS_ENOMEM, "model parameters");
    }
  }
  // Xavier-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)), zero biases; the uniform
  // draws come from splitmix64 seeded with init_seed.
  uint64_t s = init_seed;
  const int fan[3][2] = {{Mdl::IN, Mdl::HID}, {Mdl::HID, Mdl::HID}, {Mdl::HID, Mdl::OUT}};
  for (int l = 0; l < 3; ++l) {
    std::vector<float> w(cnt[2 * l]);
    const double a = std::sqrt(6.0 / (fan[l][0] + fan[l][1]));
    for (auto& x : w) x = (float)(a * (2.0 * ((splitmix64(s) >> 11) * 0x1.0p-53) - 1.0));
    std::vector<float> b(cnt[2 * l + 1], 0.f);
    if (cudaMemcpyAsync(md->w[2 * l], w.data(), w.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(md->w[2 * l + 1], b.data(), b.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      free_model(md);
      return fail(PARIS_ECUDA, "uploading initial weights");
    }
    cudaStreamSynchronize(st);
  }
  refresh_bf16(md, st);
  PARIS_CUDA(cudaStreamSynchronize(st));
  *out = md;
  return PARIS_OK;
}

void paris_seed_model_free(paris_seed_model* md) {
  if (!md) return;
  cudaDeviceSynchronize();
  free_model(md);
}

paris_status paris_seed_model_set_weights(paris_seed_model* md, const float* params_host, void* stream) {
  clear_error();
  if (!md || !params_host) return fail(PARIS_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  size_t o = 0;
  for (int i = 0; i < 6; ++i) {
    PARIS_CUDA(cudaMemcpyAsync(md->w[i], params_host + o, md->count[i] * 4, cudaMemcpyHostToDevice, st));
    PARIS_CUDA(cudaMemsetAsync(md->m[i], 0, md->count[i] * 4, st));
    PARIS_CUDA(cudaMemsetAsync(md->v[i], 0, md->count[i] * 4, st));
    o += md->count[i];
  }
  md->step = 0;
  refresh_bf16(md, st);
  PARIS_CUDA(cudaStreamSynchronize(st));
  return PARIS_OK;
}

paris_status paris_seed_model_get_weights(const paris_seed_model* md, float* params_host, void* stream) {
  clear_error();
  if (!md || !params_host) return fail(PARIS_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  size_t o = 0;
  for (int i = 0; i < 6; ++i) {
    PARIS_CUDA(cudaMemcpyAsync(params_host + o, md->w[i], md->count[i] * 4, cudaMemcpyDeviceToHost, st));
    o += md->count[i];
  }
  PARIS_CUDA(cudaStreamSynchronize(st));
  return PARIS_OK;
}

paris_status paris_seed_model_forward(const paris_seed_model* md, const double* paa, int64_t m, float* logits,
                                      void* stream) {
  clear_error();
  if (!md || (m > 0 && (!paa || !logits))) return fail(PARIS_EINVAL, "NULL argument");
  if (m > 0 && (!is_device_ptr(paa) || !is_device_ptr(logits)))
    return fail(PARIS_EINVAL, "paa and logits must be device memory");
  if (m == 0) return PARIS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  const int B = 1024;
  PARIS_TRY(ws.alloc(B, st));
  DevBuf xf;
  if (!xf.alloc((size_t)m * 16 * 4, st)) return fail(PARIS_ENOMEM, "inputs");
  paa_to_f32_kernel<<<(unsigned)((m * 16 + 255) / 256), 256, 0, st>>>(paa, m, xf.as<float>());
  note_launches(1);
  for (int64_t b0 = 0; b0 < m; b0 += B) {
    const int nb = (int)std::min<int64_t>(B, m - b0);
    forward(md, xf.as<float>() + b0 * 16, nb, ws, st);
    PARIS_CUDA(cudaMemcpyAsync(logits + b0 * paris_seed_model::OUT, ws.lg, (size_t)nb * paris_seed_model::OUT * 4,
                               cudaMemcpyDeviceToDevice, st));
  }
  PARIS_CUDA(cudaGetLastError());
  PARIS_CUDA(cudaStreamSynchronize(st));
  PARIS_TRY(check_gemm_status(st));
  return PARIS_OK;
}

paris_status paris_seed_model_topr(const paris_seed_model* md, const double* paa, int64_t m, int32_t r,
                                   int32_t* out_buckets, void* stream) {
  clear_error();
  if (!md || (m > 0 && (!paa || !out_buckets))) return fail(PARIS_EINVAL, "NULL argument");
  if (r < 1 || r > 8) return fail(PARIS_EINVAL, "top_r must be in [1, 8]");
  if (m < 0) return fail(PARIS_EINVAL, "m < 0");
  if (m == 0) return PARIS_OK;
  if (!is_device_ptr(paa) || !is_device_ptr(out_buckets))
    return fail(PARIS_EINVAL, "paa and out_buckets must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  const int B = 1024;
  PARIS_TRY(ws.alloc(B, st));
  DevBuf xf;
  if (!xf.alloc((size_t)m * 16 * 4, st)) return fail(PARIS_ENOMEM, "inputs");
  paa_to_f32_kernel<<<(unsigned)((m * 16 + 255) / 256), 256, 0, st>>>(paa, m, xf.as<float>());
  note_launches(1);
  for (int64_t b0 = 0; b0 < m; b0 += B) {
    const int nb = (int)std::min<int64_t>(B, m - b0);
    forward(md, xf.as<float>() + b0 * 16, nb, ws, st);
    topr_kernel<<<(nb + 7) / 8, 256, 0, st>>>(ws.lg, nb, paris_seed_model::OUT, r, out_buckets + b0 * r);
    note_launches(1);
  }
  PARIS_CUDA(cudaGetLastError());
  PARIS_CUDA(cudaStreamSynchronize(st));
  PARIS_TRY(check_gemm_status(st));
  return PARIS_OK;
}

paris_status paris_seed_model_gradients(const paris_seed_model* md, const double* paa, const int32_t* labels, int32_t m,
                                        float* grads, float* loss_host, void* stream) {
  clear_error();
  if (!md || !paa || !labels || !grads || m < 1) return fail(PARIS_EINVAL, "bad arguments");
  if (!is_device_ptr(paa) || !is_device_ptr(labels) || !is_device_ptr(grads))
    return fail(PARIS_EINVAL, "paa, labels and grads must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  PARIS_TRY(ws.alloc(m, st));
  DevBuf xf;
  if (!xf.alloc((size_t)m * 16 * 4, st)) return fail(PARIS_ENOMEM, "inputs");
  paa_to_f32_kernel<<<(unsigned)(((int64_t)m * 16 + 255) / 256), 256, 0, st>>>(paa, m, xf.as<float>());
  note_launches(1);
  PARIS_CUDA(cudaMemsetAsync(ws.loss, 0, 4, st));
  backward(md, xf.as<float>(), labels, m, ws, st);
  const size_t total = offset_of(md, 6);
  PARIS_CUDA(cudaMemcpyAsync(grads, ws.g, total * 4, cudaMemcpyDeviceToDevice, st));
  float l = 0.f;
  PARIS_CUDA(cudaMemcpyAsync(&l, ws.loss, 4, cudaMemcpyDeviceToHost, st));
  PARIS_CUDA(cudaStreamSynchronize(st));
  PARIS_TRY(check_gemm_status(st));
  if (loss_host) *loss_host = l;
  return PARIS_OK;
}

paris_status paris_seed_model_train(paris_seed_model* md, const double* paa, const int32_t* labels, int64_t m,
                                    int32_t batch, int32_t epochs, float lr, float weight_decay, uint64_t order_seed,
                                    float* loss_per_epoch, void* stream) {
  clear_error();
  if (!md || !paa || !labels || m < 1 || batch < 1 || epochs < 0) return fail(PARIS_EINVAL, "bad arguments");
  if (!is_device_ptr(paa) || !is_device_ptr(labels)) return fail(PARIS_EINVAL, "paa and labels must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  PARIS_TRY(ws.alloc(batch, st));
  DevBuf xb;
  if (!xb.alloc((size_t)batch * 16 * 4, st)) return fail(PARIS_ENOMEM, "batch buffer");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  uint64_t s = order_seed;
  for (int e = 0; e < epochs; ++e) {
    // visiting order a*i + c mod m with a coprime to m
    uint64_t a = (splitmix64(s) % (uint64_t)m) | 1ull;
    while (std::gcd<uint64_t>(a, (uint64_t)m) != 1) a += 2;
    const uint64_t c = splitmix64(s) % (uint64_t)m;
    PARIS_CUDA(cudaMemsetAsync(ws.loss, 0, 4, st));
    int nb = 0;
    for (int64_t b0 = 0; b0 + batch <= m || (b0 == 0 && m < batch); b0 += batch) {
      const int B = (int)std::min<int64_t>(batch, m - b0);
      gather_batch_kernel<<<(B * 16 + 255) / 256, 256, 0, st>>>(paa, labels, m, b0, B, a, c, xb.as<float>(), ws.yb);
      note_launches(1);
      backward(md, xb.as<float>(), ws.yb, B, ws, st);
      md->step += 1;
      const float c1 = 1.f - std::pow(b1, (float)md->step), c2 = 1.f - std::pow(b2, (float)md->step);
      size_t o = 0;
      for (int i = 0; i < 6; ++i) {
        adamw_kernel<<<(unsigned)((md->count[i] + 255) / 256), 256, 0, st>>>(
            md->w[i], ws.g + o, md->m[i], md->v[i], (int64_t)md->count[i], lr, b1, b2, eps, weight_decay, c1, c2,
            (i % 2 == 0) ? md->wb[i / 2] : nullptr);
        o += md->count[i];
      }
      note_launches(6);
      ++nb;
    }
    float l = 0.f;
    PARIS_CUDA(cudaMemcpyAsync(&l, ws.loss, 4, cudaMemcpyDeviceToHost, st));
    PARIS_CUDA(cudaStreamSynchronize(st));
    if (loss_per_epoch) loss_per_epoch[e] = nb ? l / (float)nb : 0.f;
  }
  PARIS_CUDA(cudaGetLastError());
  PARIS_CUDA(cudaStreamSynchronize(st));
  PARIS_TRY(check_gemm_status(st));
  return PARIS_OK;
}

}  // extern "C"
