// Index build, step 1: exact PAA -> iSAX symbols -> summary slot + interleaved key, one warp
// per series (Sec. 2.2; Alg. 2 ConvertToSAX and SAX[position] store).
#include "internal.h"

namespace paris {

namespace {

constexpr int kEncodeThreads = 256;

template <int ITERS>
__global__ void __launch_bounds__(kEncodeThreads) encode_kernel(
    const float* __restrict__ series, int64_t n, RowShape sh, int card, int bits,
    const uint64_t* __restrict__ beta_keys_g, uint8_t* __restrict__ sax_rot,
    uint8_t* __restrict__ sax_plain, uint64_t* __restrict__ key64, double* __restrict__ paa_out,
    uint32_t* __restrict__ status) {
  __shared__ uint64_t beta_keys[255];
  for (int i = threadIdx.x; i < card - 1; i += blockDim.x) beta_keys[i] = beta_keys_g[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  bool nonfinite = false;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
    const float* row = series + r * (int64_t)sh.len;
    double paa = 0.0;
    bool ok = warp_row_paa<ITERS>(row, sh, lane, paa);
    if (!ok) nonfinite = true;
    int sym = (lane < sh.w) ? symbol_of(paa, beta_keys, card) : 0;
    uint64_t key = warp_key64(sym, lane, sh.w, bits);
    // rotated summary slot: slot j holds segment (j + r) mod 16 (0 when that segment >= w)
    int seg = (lane + (int)(r & 15)) & 15;
    int b = __shfl_sync(PARIS_FULL_MASK, sym, seg);
    if (lane < PARIS_SAX_BYTES) sax_rot[r * PARIS_SAX_BYTES + lane] = (uint8_t)(seg < sh.w ? b : 0);
    if (sax_plain && lane < sh.w) sax_plain[r * sh.w + lane] = (uint8_t)sym;
    if (paa_out && lane < sh.w) paa_out[r * sh.w + lane] = paa;
    if (lane == 0) key64[r] = key;
  }
  if (nonfinite && lane == 0) atomicOr(status, DEV_NONFINITE);
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
  int64_t want = (n + (kEncodeThreads / 32) - 1) / (kEncodeThreads / 32);
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
  sh.fast = (len % 4 == 0) && aligned && sh.log2s >= 2 && sh.s <= 128 && len <= 128 * 16;
  return sh;
}

paris_status launch_encode(const float* series, int64_t n, const RowShape& sh, int card, int bits,
                           const uint64_t* beta_keys, uint8_t* sax_rot, uint8_t* sax_plain,
                           uint64_t* key64, double* paa, uint32_t* status, cudaStream_t st) {
  if (n <= 0) return PARIS_OK;
  int grid = encode_grid(n);
  int iters = sh.fast ? (sh.len + 127) / 128 : 1;
  if (iters <= 1)
    encode_kernel<1><<<grid, kEncodeThreads, 0, st>>>(series, n, sh, card, bits, beta_keys, sax_rot, sax_plain, key64, paa, status);
  else if (iters <= 2)
    encode_kernel<2><<<grid, kEncodeThreads, 0, st>>>(series, n, sh, card, bits, beta_keys, sax_rot, sax_plain, key64, paa, status);
  else if (iters <= 4)
    encode_kernel<4><<<grid, kEncodeThreads, 0, st>>>(series, n, sh, card, bits, beta_keys, sax_rot, sax_plain, key64, paa, status);
  else if (iters <= 8)
    encode_kernel<8><<<grid, kEncodeThreads, 0, st>>>(series, n, sh, card, bits, beta_keys, sax_rot, sax_plain, key64, paa, status);
  else
    encode_kernel<16><<<grid, kEncodeThreads, 0, st>>>(series, n, sh, card, bits, beta_keys, sax_rot, sax_plain, key64, paa, status);
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
