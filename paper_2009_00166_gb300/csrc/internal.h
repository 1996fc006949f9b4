// Host-side internals of the GB300 ParIS+ library: the index object, error plumbing, memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/paris.h"
#include "common.cuh"

struct paris_index {
  int64_t n = 0;
  int32_t len = 0, w = 0, card = 0, bits = 0, leaf_cap = 2048;
  int device = 0;
  const float* series = nullptr;  // device [n][len]; borrowed unless series_owned
  void* series_owned = nullptr;
  size_t series_owned_bytes = 0;
  const void* host_registered = nullptr;  // host series registered by the build (series_on_host)
  uint8_t* sax = nullptr;           // device [n][16], slot j of row r = segment (j + r) % 16
  uint64_t* keys_sorted = nullptr;  // device [n]
  uint32_t* rows_sorted = nullptr;  // device [n]
  // index order (leaf pruning): position p's summary rotated by p mod 16, and the envelope of
  // every page of kPageRows positions (smallest then largest symbol per segment, 16 B each,
  // rotated by the page number mod 16)
  uint8_t* sax_sorted = nullptr;    // device [n][16]
  uint8_t* env = nullptr;           // device [npages][2][16]
  int64_t npages = 0;
  uint64_t* beta_keys = nullptr;    // device [card-1] order keys of the breakpoints
  double* beta_ext = nullptr;       // device [card+1]: -inf, beta_1..beta_{card-1}, +inf
  std::vector<double> beta_host;
  // BF16 shadow of the series and fp32 row norms for the mixed-precision path (made on first use)
  void* shadow = nullptr;       // device [n][len] bf16
  float2* xnorm = nullptr;      // device [n rounded up to 64]: (|x|^2, |x|) in fp32, zero past n
  void* xtile = nullptr;        // device float4 per 64-row tile: (min |x|^2, max |x|^2, max |x|, 0)
  void* shadow_map = nullptr;   // host copy of the TMA descriptor of the shadow (CUtensorMap)
  // adaptive-split leaves (paris_build_adaptive_leaves): tree nodes, root-child table, and per
  // leaf-order position the series row and the leaf holding it
  void* ad_nodes = nullptr;         // device AdNode [ad_cap]
  int64_t ad_nnodes = 0, ad_cap = 0, ad_leaves = 0;
  int32_t ad_depth = 0;
  int32_t* ad_root = nullptr;       // device [2^w]: node of each first-bit word (nearest non-empty)
  uint32_t* ad_rows = nullptr;      // device [n]
  int32_t* ad_leaf_of = nullptr;    // device [n]
  // learned approximate-search proposal (borrowed; see paris_attach_seed_model)
  const paris_seed_model* seed_model = nullptr;
  int seed_r = 0;
};

namespace paris {

paris_status fail(paris_status s, const char* fmt, ...);
void clear_error();

void* dev_alloc(size_t bytes, cudaStream_t st);
void dev_free(void* p, size_t bytes, cudaStream_t st);

// RAII device buffer drawn from the library allocator on one stream.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  bool alloc(size_t b, cudaStream_t s) {
    release();
    st = s;
    bytes = b ? b : 16;
    p = dev_alloc(bytes, s);
    return p != nullptr;
  }
  void release() {
    if (p) dev_free(p, bytes, st);
    p = nullptr;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

#define PARIS_CUDA(expr)                                                                     \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess)                                                                   \
      return ::paris::fail(PARIS_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(_e));     \
  } while (0)

#define PARIS_TRY(expr)                    \
  do {                                     \
    paris_status _s = (expr);              \
    if (_s != PARIS_OK) return _s;         \
  } while (0)

// Breakpoints Phi^-1(j/card), j = 1..card-1 (AS241).
std::vector<double> normal_breakpoints(int card);
void breakpoint_tables(const std::vector<double>& beta, std::vector<uint64_t>& keys,
                       std::vector<double>& ext);

// Row geometry for the encode kernels.
RowShape make_row_shape(int len, int w, const void* base_ptr);

// Kernel launchers (return PARIS_OK or a launch failure).
paris_status launch_encode(const float* series, int64_t n, const RowShape& sh, int card, int bits,
                           const uint64_t* beta_keys, uint8_t* sax_rot, uint8_t* sax_plain,
                           uint64_t* key64, double* paa, uint32_t* status, cudaStream_t st,
                           void* shadow = nullptr, float2* xnorm = nullptr);
paris_status launch_unrotate_sax(const uint8_t* sax_rot, int64_t n, int w, uint8_t* out,
                                 cudaStream_t st);
paris_status radix_sort_index(uint64_t* keys, uint32_t* rows, int64_t n, cudaStream_t st);
// In-place exclusive prefix sum of m 32-bit counts (sums must fit in 32 bits).
paris_status exclusive_scan(uint32_t* a, int64_t m, cudaStream_t st);
// Frees the adaptive-split leaves of an index (NULL-safe fields).
void release_adaptive(paris_index* idx);

// Bound of the device-side waits of the pipelined kernels (paris_set_wait_limit), in ns.
uint64_t wait_limit_ns();

// Number of kernels this library has launched since it was loaded (all threads).
void note_launches(int count);
uint64_t launch_count();

// Pointer classification: true if p is device (or managed) memory on the current device.
bool is_device_ptr(const void* p);

}  // namespace paris
