// Lower-bound scan for callers that cannot allocate device memory.
//
// Some callers cannot let a library call cudaMalloc (or any allocating routine) while they run:
// services that reserve their whole device memory up front and forbid allocation on the request
// path (an allocation there can fail under memory pressure or stall behind other work), and
// hosts that hand a library nothing but pre-existing buffers. paris_lb_scan_noalloc serves them:
// it runs the same query-preparation and lower-bound-scan kernels as paris_lb_scan, but keeps
// its scratch -- each query's PAA, key and lower-bound table, the candidate counters and a status
// word -- in one fixed array in device memory that this library declares statically. Every GPU
// that loads the library holds that array until the process exits.
#include <mutex>

#include "query.cuh"

namespace paris {

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)PARIS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The shared scratch. Host code must not use this name as an address (it is a host-side
// stand-in); it uses the device address obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
paris_status scratch_address(void** out) {
  int dev = 0;
  PARIS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PARIS_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(PARIS_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PARIS_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

}  // namespace paris

using namespace paris;

extern "C" paris_status paris_lb_scan_noalloc(const paris_index* idx, const float* queries, int64_t nq,
                                              const float* thresholds_sq, uint32_t* out_rows, float* out_lb,
                                              int64_t capacity, int64_t* out_counts, void* stream) {
  clear_error();
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  if (nq < 0) return fail(PARIS_EINVAL, "nq must be >= 0");
  if (nq == 0) return PARIS_OK;
  if (!queries || !thresholds_sq || !out_counts) return fail(PARIS_EINVAL, "NULL argument");
  if (capacity < 0 || (capacity > 0 && (!out_rows || !out_lb)))
    return fail(PARIS_EINVAL, "bad output buffers");
  if (!is_device_ptr(queries)) return fail(PARIS_EINVAL, "queries must be device memory");
  if (capacity > 0 && (!is_device_ptr(out_rows) || !is_device_ptr(out_lb)))
    return fail(PARIS_EINVAL, "out_rows/out_lb must be device memory");
  // scratch layout: status | counters[nq] | qkey[nq] | qpaa[nq][16] | qtable[nq][card][16]
  const size_t need = align256(4) + align256((size_t)nq * 4) + align256((size_t)nq * 8) +
                      align256((size_t)nq * 16 * 8) + align256((size_t)nq * idx->card * 16 * 4);
  if (need > kNoallocScratchBytes)
    return fail(PARIS_EINVAL,
                "paris_lb_scan_noalloc: %lld queries at %d symbols need %zu bytes of scratch, more than the "
                "%zu-byte static scratch; pass fewer queries per call",
                (long long)nq, idx->card, need, kNoallocScratchBytes);
  void* base = nullptr;
  PARIS_TRY(scratch_address(&base));
  cudaStream_t st = (cudaStream_t)stream;
  char* b = (char*)base;
  size_t off = 0;
  uint32_t* status = (uint32_t*)(b + off);
  off += align256(4);
  uint32_t* counts = (uint32_t*)(b + off);
  off += align256((size_t)nq * 4);
  QueryState qs;
  qs.nq = nq;
  qs.k = 1;
  qs.queries = queries;
  qs.status = status;
  qs.qkey = (uint64_t*)(b + off);
  off += align256((size_t)nq * 8);
  qs.qpaa = (double*)(b + off);
  off += align256((size_t)nq * 16 * 8);
  qs.qtable = (float*)(b + off);
  // the array keeps the previous call's contents: zero what must start at zero
  PARIS_CUDA(cudaMemsetAsync(b, 0, align256(4) + align256((size_t)nq * 4), st));
  PARIS_TRY(launch_query_prep(idx, qs, st));
  for (int64_t q = 0; q < nq; ++q)
    PARIS_TRY(launch_lbscan_threshold(idx, qs.qtable + q * (int64_t)idx->card * 16, thresholds_sq[q], counts + q,
                                      capacity ? out_rows + q * capacity : nullptr,
                                      capacity ? out_lb + q * capacity : nullptr, capacity, status, st));
  uint32_t host_status = 0;
  PARIS_CUDA(cudaMemcpyAsync(&host_status, status, 4, cudaMemcpyDeviceToHost, st));
  uint32_t tmp[64];  // counts come back through a stack buffer: no host allocation either
  for (int64_t q0 = 0; q0 < nq; q0 += 64) {
    const int m = (int)(nq - q0 < 64 ? nq - q0 : 64);
    PARIS_CUDA(cudaMemcpyAsync(tmp, counts + q0, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
    PARIS_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < m; ++j) out_counts[q0 + j] = tmp[j];
  }
  if (host_status & DEV_NONFINITE) return fail(PARIS_EINVAL, "paris_lb_scan_noalloc: query holds a NaN or infinity");
  return PARIS_OK;  // counts above capacity report an overflow of the caller's buffers
}
