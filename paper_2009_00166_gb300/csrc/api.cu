// C ABI of the GB300 ParIS+ library: argument checking, memory, staging and orchestration of
// the build (encode -> sort) and query (prep -> approximate search -> LB scan -> refine ->
// select/re-rank) kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <utility>
#include <vector>
#include <new>
#include <string>

#include "query.cuh"

namespace paris {

namespace {
thread_local std::string g_err;
paris_alloc_fn g_alloc = nullptr;
constexpr uint64_t kDefaultWaitNs = 4000000000ull;  // 4 s
std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};
paris_free_fn g_free = nullptr;
void* g_ctx = nullptr;
}  // namespace

uint64_t wait_limit_ns() { return g_wait_ns.load(); }

paris_status fail(paris_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

void clear_error() { g_err.clear(); }

namespace {
std::atomic<uint64_t> g_launches{0};
}
void note_launches(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {
// The library's own stream-ordered pool per device: freed blocks stay cached for the next call
// (release threshold = unlimited) instead of going back to the driver at every synchronisation.
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[64] = {};

cudaMemPool_t library_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t threshold = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}
}  // namespace

void* dev_alloc(size_t bytes, cudaStream_t st) {
  if (g_alloc) return g_alloc(bytes, st, g_ctx);
  void* p = nullptr;
  cudaMemPool_t pool = library_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t st) {
  if (!p) return;
  if (g_free) {
    g_free(p, bytes, st, g_ctx);
    return;
  }
  cudaFreeAsync(p, st);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace paris

using namespace paris;

namespace {

float gamma_scale(int len) {
  // (1 + gamma) / (1 - gamma) with gamma = gamma_{len+2} = m u / (1 - m u), u = 2^-24, rounded up
  double m = (double)len + 2.0, u = std::ldexp(1.0, -24);
  double g = m * u / (1.0 - m * u);
  double cg = (1.0 + g) / (1.0 - g) * (1.0 + std::ldexp(1.0, -20));
  return std::nextafter((float)cg, INFINITY);
}

paris_status check_status_word(const uint32_t* dev_status, cudaStream_t st, const char* what) {
  uint32_t s = 0;
  PARIS_CUDA(cudaMemcpyAsync(&s, dev_status, sizeof s, cudaMemcpyDeviceToHost, st));
  PARIS_CUDA(cudaStreamSynchronize(st));
  // an expired wait leaves the later phases without their inputs: it is the error to report
  if (s & DEV_TIMEOUT) return fail(PARIS_ETIMEOUT, "%s: a device-side wait expired", what);
  if (s & DEV_NONFINITE) return fail(PARIS_EINVAL, "%s: input holds a NaN or infinite value", what);
  if (s & DEV_CONT_OVERFLOW)
    return fail(PARIS_EINTERNAL, "%s: more than %d rows tie with the k-th neighbour within the fp32 bound",
                what, kContCap);
  if (s & DEV_CAND_OVERFLOW) return fail(PARIS_EINTERNAL, "%s: candidate list overflow", what);
  return PARIS_OK;
}

bool valid_card(int card) { return card >= 2 && card <= 256 && (card & (card - 1)) == 0; }

paris_status upload_breakpoints(paris_index* idx, cudaStream_t st) {
  idx->beta_host = normal_breakpoints(idx->card);
  std::vector<uint64_t> keys;
  std::vector<double> ext;
  breakpoint_tables(idx->beta_host, keys, ext);
  idx->beta_keys = (uint64_t*)dev_alloc(keys.size() * 8, st);
  idx->beta_ext = (double*)dev_alloc(ext.size() * 8, st);
  if (!idx->beta_keys || !idx->beta_ext) return fail(PARIS_ENOMEM, "breakpoint tables");
  PARIS_CUDA(cudaMemcpyAsync(idx->beta_keys, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice, st));
  PARIS_CUDA(cudaMemcpyAsync(idx->beta_ext, ext.data(), ext.size() * 8, cudaMemcpyHostToDevice, st));
  PARIS_CUDA(cudaStreamSynchronize(st));  // host vectors die with this scope
  return PARIS_OK;
}

void release_index(paris_index* idx) {
  if (!idx) return;
  cudaStream_t st = nullptr;
  dev_free(idx->series_owned, idx->series_owned_bytes, st);
  if (idx->host_registered) cudaHostUnregister(const_cast<void*>(idx->host_registered));
  dev_free(idx->sax, (size_t)idx->n * PARIS_SAX_BYTES, st);
  dev_free(idx->keys_sorted, (size_t)idx->n * 8, st);
  dev_free(idx->rows_sorted, (size_t)idx->n * 4, st);
  dev_free(idx->sax_sorted, (size_t)idx->n * PARIS_SAX_BYTES, st);
  dev_free(idx->env, (size_t)(idx->npages + (idx->npages + 15) / 16) * 32, st);
  dev_free(idx->beta_keys, (size_t)(idx->card - 1) * 8, st);
  dev_free(idx->beta_ext, (size_t)(idx->card + 1) * 8, st);
  release_shadow(idx);
  release_adaptive(idx);
  delete idx;
}

// A device view of a caller buffer that may live on the host (staged through device memory).
struct Staged {
  DevBuf buf;
  void* dev = nullptr;
  void* host = nullptr;
  size_t bytes = 0;
  paris_status in(const void* p, size_t b, cudaStream_t st) {
    bytes = b;
    if (is_device_ptr(p)) {
      dev = const_cast<void*>(p);
      return PARIS_OK;
    }
    if (!buf.alloc(b, st)) return fail(PARIS_ENOMEM, "staging %zu bytes", b);
    dev = buf.p;
    PARIS_CUDA(cudaMemcpyAsync(dev, p, b, cudaMemcpyHostToDevice, st));
    return PARIS_OK;
  }
  paris_status out(void* p, size_t b, cudaStream_t st) {
    bytes = b;
    if (!p) return PARIS_OK;
    if (is_device_ptr(p)) {
      dev = p;
      return PARIS_OK;
    }
    if (!buf.alloc(b, st)) return fail(PARIS_ENOMEM, "staging %zu bytes", b);
    dev = buf.p;
    host = p;
    return PARIS_OK;
  }
  paris_status finish(cudaStream_t st) {
    if (host) PARIS_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st));
    return PARIS_OK;
  }
};

// Per-phase device time: events recorded on the call's stream, summed once the call is done,
// so that timing adds no host synchronisation inside the call.
struct PhaseTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[6];
  explicit PhaseTimer(bool enable, cudaStream_t s) : on(enable), st(s) {}
  void begin(int phase) {
    if (!on) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    ev[phase].push_back({a, b});
  }
  void end(int phase) {
    if (on) cudaEventRecord(ev[phase].back().second, st);
  }
  void collect(double* out6) {
    for (int p = 0; p < 6; ++p) {
      for (auto& e : ev[p]) {
        float ms = 0.f;
        cudaEventSynchronize(e.second);
        cudaEventElapsedTime(&ms, e.first, e.second);
        if (out6) out6[p] += ms;
      }
    }
  }
  ~PhaseTimer() {
    for (auto& v : ev)
      for (auto& e : v) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
  }
};

// Query tile of the batched scan for a (len, card) shape: the fastest of the candidate tiles per
// query, timed once per shape on the first chunk that needs it, then remembered.
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int>, int> g_tuned;

paris_status tuned_query_tile(const paris_index* idx, const QueryState& qs, const ChunkState& cs, bool prune,
                              cudaStream_t st, int* out) {
  // one choice per device, shape, collection size (binary order of magnitude) and pruning mode
  int lg = 0;
  while (lg < 62 && (int64_t(1) << (lg + 1)) <= idx->n) ++lg;
  const auto key = std::make_tuple(idx->device, idx->len, idx->card, lg, prune ? 1 : 0);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      *out = it->second;
      return PARIS_OK;
    }
  }
  // Trial launches on up to three spread samples of 24 queries (start, middle and end of the
  // chunk; 24 fills the largest tile), so the choice sees the chunk's mix of tight and loose
  // thresholds.
  int offs[3] = {0, 0, 0}, nsub = 1, m = (int)std::min<int64_t>(cs.qc, 24);
  if (cs.qc >= 72) {
    m = 24;
    nsub = 3;
    offs[1] = cs.qc / 2 - 12;
    offs[2] = cs.qc - 24;
  }
  auto sub_of = [&](int j) {
    ChunkState sub = cs;
    sub.q0 = cs.q0 + offs[j];
    sub.qc = m;
    sub.count = cs.count + offs[j];
    sub.rows = cs.rows + (int64_t)offs[j] * cs.cap;
    sub.lb = cs.lb + (int64_t)offs[j] * cs.cap;
    if (cs.pagebits) {
      sub.pagebits = cs.pagebits + (int64_t)offs[j] * page_words(idx->n);
      sub.page_count = cs.page_count + offs[j];
      sub.page_list = cs.page_list + (int64_t)offs[j] * page_list_cap(idx->n);
    }
    return sub;
  };
  DevBuf scratch_status;
  if (!scratch_status.alloc(4, st)) return fail(PARIS_ENOMEM, "tuning scratch");
  struct Events {  // destroyed on every return path
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  PARIS_CUDA(cudaEventCreate(&ev.a));
  PARIS_CUDA(cudaEventCreate(&ev.b));
  const cudaEvent_t e0 = ev.a, e1 = ev.b;
  int best = 2;
  float best_t = 1e30f;
  for (int i = 0; i < kNumQueryTiles; ++i) {
    const int qt = kQueryTiles[i];
    if (!query_tile_fits(qt, idx->card)) continue;
    float total = 0.f;
    for (int j = 0; j < nsub; ++j) {
      const ChunkState sub = sub_of(j);
      PARIS_CUDA(cudaMemsetAsync(sub.count, 0, (size_t)sub.qc * 4, st));
      cudaEventRecord(e0, st);
      paris_status s = launch_lbscan_batched(idx, qs, sub, qt, 1, scratch_status.as<uint32_t>(), st);
      cudaEventRecord(e1, st);
      if (s != PARIS_OK) return s;
      PARIS_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      total += ms;
    }
    const float per_query = total / (float)(m * nsub);
    // tiles are tried from small to large; a larger tile within 3% of the best so far wins
    // (fewer passes over the summaries, and a stable choice when trial timings are this close)
    if (per_query < best_t * 1.03f) {
      best_t = per_query;
      best = qt;
    }
  }
  for (int j = 0; j < nsub; ++j) PARIS_CUDA(cudaMemsetAsync(cs.count + offs[j], 0, (size_t)m * 4, st));
  // the trial scans' lookups are not the call's (tuning runs before any chunk is scanned)
  PARIS_CUDA(cudaMemsetAsync(qs.counters + 4, 0, 8, st));
  PARIS_CUDA(cudaMemsetAsync(qs.counters + 6, 0, 8, st));
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned[key] = best;
  *out = best;
  return PARIS_OK;
}

}  // namespace

extern "C" {

const char* paris_last_error(void) { return g_err.c_str(); }

uint64_t paris_kernel_launches(void) { return launch_count(); }

paris_status paris_set_wait_limit(uint64_t ns) {
  clear_error();
  if (ns > 60000000000ull) return fail(PARIS_EINVAL, "wait limit above 60 s");
  g_wait_ns.store(ns ? ns : kDefaultWaitNs);
  return PARIS_OK;
}

paris_status paris_trim_memory(void) {
  clear_error();
  int dev = 0;
  PARIS_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool = library_pool();
  if (pool) {
    PARIS_CUDA(cudaDeviceSynchronize());
    PARIS_CUDA(cudaMemPoolTrimTo(pool, 0));
  }
  return PARIS_OK;
}

paris_status paris_set_allocator(paris_alloc_fn alloc, paris_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(PARIS_EINVAL, "paris_set_allocator: give both functions or neither");
  g_alloc = alloc;
  g_free = free_fn;
  g_ctx = ctx;
  return PARIS_OK;
}

paris_status paris_breakpoints(int32_t card, double* out_host) {
  clear_error();
  if (!valid_card(card)) return fail(PARIS_EINVAL, "card must be a power of two in [2, 256], got %d", card);
  if (!out_host) return fail(PARIS_EINVAL, "out_host is NULL");
  std::vector<double> b = normal_breakpoints(card);
  std::memcpy(out_host, b.data(), b.size() * sizeof(double));
  return PARIS_OK;
}

static paris_status check_shape(int64_t n, int32_t len, int32_t w, int32_t card) {
  if (n < 1 || n > 0xffffffffll) return fail(PARIS_EINVAL, "n must be in [1, 2^32), got %lld", (long long)n);
  if (len < 1) return fail(PARIS_EINVAL, "len must be >= 1, got %d", len);
  if (w < 1 || w > 16) return fail(PARIS_EINVAL, "w must be in [1, 16], got %d", w);
  if (len % w) return fail(PARIS_EINVAL, "len (%d) must be a multiple of w (%d)", len, w);
  if (!valid_card(card)) return fail(PARIS_EINVAL, "card must be a power of two in [2, 256], got %d", card);
  if ((int64_t)len / w > 65536) return fail(PARIS_EINVAL, "segments longer than 65536 points are not supported");
  return PARIS_OK;
}

namespace {
// Library copy streams of a device (two DMA engines copy concurrently).
std::mutex g_copy_mutex;
cudaStream_t g_copy_streams[64][2] = {};

paris_status copy_streams(cudaStream_t* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(PARIS_ECUDA, "current device");
  std::lock_guard<std::mutex> lock(g_copy_mutex);
  for (int i = 0; i < 2; ++i) {
    if (!g_copy_streams[dev][i] && cudaStreamCreateWithFlags(&g_copy_streams[dev][i], cudaStreamNonBlocking) != cudaSuccess)
      return fail(PARIS_ECUDA, "copy stream");
    out[i] = g_copy_streams[dev][i];
  }
  return PARIS_OK;
}
}  // namespace

// A host series is copied to the device in chunks on two copy streams while the encode pass
// works through the chunks already copied. Chunks start at multiples of 16 rows (the rotation
// of the summary slots follows the row number).
// With `staging` (two buffers of `rows` rows each; the series stays on the host), chunk j is copied
// into staging[j % 2] once the encode of chunk j - 2 has read that buffer.
static paris_status copy_and_encode(paris_index* idx, const float* host, const RowShape& sh, ShadowBufs& shb,
                                    uint32_t* status, cudaStream_t st, float* const* staging = nullptr,
                                    int64_t staging_rows = 0) {
  const int64_t n = idx->n, len = idx->len;
  const size_t row_bytes = (size_t)len * sizeof(float);
  int64_t rows = staging ? staging_rows : (int64_t)((size_t)(512u << 20) / row_bytes);  // about 512 MB per chunk
  rows = std::max<int64_t>(16, rows / 16 * 16);
  cudaStream_t cs[2];
  PARIS_TRY(copy_streams(cs));
  cudaEvent_t ready;
  PARIS_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  PARIS_CUDA(cudaEventRecord(ready, st));  // the device copy's memory is allocated on st
  for (int i = 0; i < 2; ++i) PARIS_CUDA(cudaStreamWaitEvent(cs[i], ready, 0));
  cudaEventDestroy(ready);
  float* dst = (float*)idx->series_owned;
  paris_status s = PARIS_OK;
  int j = 0;
  for (int64_t r0 = 0; r0 < n && s == PARIS_OK; r0 += rows, ++j) {
    const int64_t m = std::min(rows, n - r0);
    float* chunk = staging ? staging[j & 1] : dst + r0 * len;
    cudaEvent_t done = nullptr, freed = nullptr;
    bool ok = cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess;
    if (ok && staging && j >= 2) {  // the buffer's previous chunk must have been encoded
      ok = cudaEventCreateWithFlags(&freed, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventRecord(freed, st) == cudaSuccess && cudaStreamWaitEvent(cs[j & 1], freed, 0) == cudaSuccess;
    }
    ok = ok &&
         cudaMemcpyAsync(chunk, host + r0 * len, (size_t)m * row_bytes, cudaMemcpyHostToDevice, cs[j & 1]) ==
             cudaSuccess &&
         cudaEventRecord(done, cs[j & 1]) == cudaSuccess && cudaStreamWaitEvent(st, done, 0) == cudaSuccess;
    if (done) cudaEventDestroy(done);
    if (freed) cudaEventDestroy(freed);
    if (!ok) {
      cudaGetLastError();
      s = fail(PARIS_ECUDA, "copying the series to the device");
      break;
    }
    s = launch_encode(chunk, m, sh, idx->card, idx->bits, idx->beta_keys, idx->sax + r0 * PARIS_SAX_BYTES,
                      nullptr, idx->keys_sorted + r0, nullptr, status, st,
                      shb.shadow ? (void*)((uint16_t*)shb.shadow + r0 * len) : nullptr,
                      shb.xnorm ? shb.xnorm + r0 : nullptr);
  }
  // on failure the caller frees the device copy: no copy may still be writing into it
  if (s != PARIS_OK)
    for (int i = 0; i < 2; ++i) cudaStreamSynchronize(cs[i]);
  return s;
}

paris_status paris_build_ex(const float* series, int64_t n, int32_t len, int32_t w, int32_t card,
                            const paris_build_opts* opts, void* stream, paris_index** out) {
  clear_error();
  if (!out) return fail(PARIS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!series) return fail(PARIS_EINVAL, "series is NULL");
  PARIS_TRY(check_shape(n, len, w, card));
  int leaf = opts && opts->leaf_capacity ? opts->leaf_capacity : 2048;
  if (leaf < 1 || leaf > kMaxLeaf) return fail(PARIS_EINVAL, "leaf_capacity must be in [1, %d]", kMaxLeaf);
  if (opts) {
    for (int i = 0; i < 5; ++i)
      if (opts->reserved[i]) return fail(PARIS_EINVAL, "paris_build_opts.reserved must be zero");
    if (opts->bf16_shadow != 0 && opts->bf16_shadow != 1) return fail(PARIS_EINVAL, "bf16_shadow must be 0 or 1");
    if (opts->series_on_host != 0 && opts->series_on_host != 1)
      return fail(PARIS_EINVAL, "series_on_host must be 0 or 1");
  }
  const bool on_host = opts && opts->series_on_host;
  cudaStream_t st = (cudaStream_t)stream;
  paris_index* idx = new (std::nothrow) paris_index();
  if (!idx) return fail(PARIS_ENOMEM, "index object");
  idx->n = n;
  idx->len = len;
  idx->w = w;
  idx->card = card;
  idx->bits = __builtin_ctz((unsigned)card);
  idx->leaf_cap = leaf;
  cudaGetDevice(&idx->device);
  auto bail = [&](paris_status s) {
    cudaStreamSynchronize(st);
    release_index(idx);
    return s;
  };
  const size_t series_bytes = (size_t)n * len * sizeof(float);
  const float* host_src = nullptr;  // a host series, copied in while the encode pass runs
  DevBuf stage[2];
  float* staging[2] = {nullptr, nullptr};
  int64_t staging_rows = 0;
  if (is_device_ptr(series)) {
    idx->series = series;
  } else if (on_host) {
    // the series stays where it is: the kernels read it through its device mapping
    cudaPointerAttributes a;
    void* mapped = nullptr;
    if (cudaPointerGetAttributes(&a, series) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer) {
      mapped = a.devicePointer;
    } else {
      cudaGetLastError();
      if (cudaHostRegister(const_cast<float*>(series), series_bytes, cudaHostRegisterMapped) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PARIS_ECUDA, "registering the host series (%zu bytes)", series_bytes));
      }
      idx->host_registered = series;
      if (cudaHostGetDevicePointer(&mapped, const_cast<float*>(series), 0) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(PARIS_ECUDA, "device mapping of the host series"));
      }
    }
    idx->series = (const float*)mapped;
    staging_rows = std::max<int64_t>(16, (int64_t)((size_t)(512u << 20) / ((size_t)len * 4)) / 16 * 16);
    staging_rows = std::min<int64_t>(staging_rows, (n + 15) / 16 * 16);
    for (int i = 0; i < 2; ++i) {
      if (!stage[i].alloc((size_t)staging_rows * len * 4, st)) return bail(fail(PARIS_ENOMEM, "staging buffers"));
      staging[i] = stage[i].as<float>();
    }
    host_src = series;
  } else {
    idx->series_owned = dev_alloc(series_bytes, st);
    if (!idx->series_owned) return bail(fail(PARIS_ENOMEM, "device copy of the series (%zu bytes)", series_bytes));
    idx->series_owned_bytes = series_bytes;
    idx->series = (const float*)idx->series_owned;
    host_src = series;
  }
  paris_status s = upload_breakpoints(idx, st);
  if (s != PARIS_OK) return bail(s);
  idx->sax = (uint8_t*)dev_alloc((size_t)n * PARIS_SAX_BYTES, st);
  idx->keys_sorted = (uint64_t*)dev_alloc((size_t)n * 8, st);
  idx->rows_sorted = (uint32_t*)dev_alloc((size_t)n * 4, st);
  DevBuf status;
  if (!idx->sax || !idx->keys_sorted || !idx->rows_sorted || !status.alloc(4, st))
    return bail(fail(PARIS_ENOMEM, "index arrays for %lld series", (long long)n));
  if (cudaMemsetAsync(status.p, 0, 4, st) != cudaSuccess) return bail(fail(PARIS_ECUDA, "memset"));
  RowShape sh = make_row_shape(len, w, idx->series);
  // the mixed-precision screening's inputs, written by the same pass when asked for
  ShadowBufs shb;
  const bool fused = opts && opts->bf16_shadow && dense_shape_ok(len) && sh.fast && sh.s <= 16;
  if (fused) {
    s = alloc_shadow(idx, &shb, st);
    if (s != PARIS_OK) return bail(s);
  }
  s = host_src ? copy_and_encode(idx, host_src, sh, shb, status.as<uint32_t>(), st, on_host ? staging : nullptr,
                                 staging_rows)
               : launch_encode(idx->series, n, sh, card, idx->bits, idx->beta_keys, idx->sax, nullptr,
                               idx->keys_sorted, nullptr, status.as<uint32_t>(), st, shb.shadow, shb.xnorm);
  if (s == PARIS_OK && fused) s = finish_shadow(idx, &shb, st);
  if (s != PARIS_OK) {
    free_shadow_bufs(idx, &shb, st);
    return bail(s);
  }
  s = radix_sort_index(idx->keys_sorted, idx->rows_sorted, n, st);
  if (s != PARIS_OK) return bail(s);
  s = build_leaf_envelopes(idx, st);
  if (s != PARIS_OK) return bail(s);
  s = check_status_word(status.as<uint32_t>(), st, "paris_build");
  if (s != PARIS_OK) return bail(s);
  *out = idx;
  return PARIS_OK;
}

paris_status paris_build(const float* series, int64_t n, int32_t len, int32_t w, int32_t card, void* stream,
                         paris_index** out) {
  return paris_build_ex(series, n, len, w, card, nullptr, stream, out);
}

void paris_free(paris_index* idx) {
  if (!idx) return;
  cudaDeviceSynchronize();
  release_index(idx);
  cudaDeviceSynchronize();
}

paris_status paris_index_describe(const paris_index* idx, paris_index_view* out) {
  clear_error();
  if (!idx || !out) return fail(PARIS_EINVAL, "NULL argument");
  out->n = idx->n;
  out->len = idx->len;
  out->w = idx->w;
  out->card = idx->card;
  out->leaf_capacity = idx->leaf_cap;
  out->series = idx->series;
  out->keys_sorted = idx->keys_sorted;
  out->rows_sorted = idx->rows_sorted;
  return PARIS_OK;
}

paris_status paris_export_sax(const paris_index* idx, uint8_t* out_sax, void* stream) {
  clear_error();
  if (!idx || !out_sax) return fail(PARIS_EINVAL, "NULL argument");
  if (!is_device_ptr(out_sax)) return fail(PARIS_EINVAL, "out_sax must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  PARIS_TRY(launch_unrotate_sax(idx->sax, idx->n, idx->w, out_sax, st));
  PARIS_CUDA(cudaStreamSynchronize(st));
  return PARIS_OK;
}

paris_status paris_export_order(const paris_index* idx, uint64_t* out_keys, uint32_t* out_rows, void* stream) {
  clear_error();
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (out_keys) PARIS_CUDA(cudaMemcpyAsync(out_keys, idx->keys_sorted, (size_t)idx->n * 8, cudaMemcpyDefault, st));
  if (out_rows) PARIS_CUDA(cudaMemcpyAsync(out_rows, idx->rows_sorted, (size_t)idx->n * 4, cudaMemcpyDefault, st));
  PARIS_CUDA(cudaStreamSynchronize(st));
  return PARIS_OK;
}

paris_status paris_encode(const float* series, int64_t n, int32_t len, int32_t w, int32_t card, uint8_t* out_sax,
                          uint64_t* out_key64, double* out_paa, void* stream) {
  clear_error();
  if (!series || !out_sax || !out_key64) return fail(PARIS_EINVAL, "NULL argument");
  PARIS_TRY(check_shape(n, len, w, card));
  if (!is_device_ptr(series) || !is_device_ptr(out_sax) || !is_device_ptr(out_key64) ||
      (out_paa && !is_device_ptr(out_paa)))
    return fail(PARIS_EINVAL, "paris_encode takes device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> beta = normal_breakpoints(card);
  std::vector<uint64_t> keys;
  std::vector<double> ext;
  breakpoint_tables(beta, keys, ext);
  DevBuf bk, rot, status;
  if (!bk.alloc(keys.size() * 8 + 8, st) || !rot.alloc((size_t)n * PARIS_SAX_BYTES, st) || !status.alloc(4, st))
    return fail(PARIS_ENOMEM, "encode scratch");
  PARIS_CUDA(cudaMemcpyAsync(bk.p, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice, st));
  PARIS_CUDA(cudaMemsetAsync(status.p, 0, 4, st));
  RowShape sh = make_row_shape(len, w, series);
  PARIS_TRY(launch_encode(series, n, sh, card, __builtin_ctz((unsigned)card), bk.as<uint64_t>(), rot.as<uint8_t>(),
                          out_sax, out_key64, out_paa, status.as<uint32_t>(), st));
  return check_status_word(status.as<uint32_t>(), st, "paris_encode");
}

// Allocates the per-call query state for nq queries.
static paris_status alloc_query_state(const paris_index* idx, int64_t nq, int k, const float* dq, QueryState& qs,
                                      DevBuf& block, cudaStream_t st) {
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) & ~(size_t)255;
    return o;
  };
  size_t o_paa = take((size_t)nq * 16 * 8), o_key = take((size_t)nq * 8),
         o_tab = take((size_t)nq * idx->card * 16 * 4), o_thr = take((size_t)nq * 4), o_bsf = take((size_t)nq * 8),
         o_leaf = take((size_t)nq * 16), o_seed = take((size_t)nq * 4), o_stat = take(4), o_cnt = take(8 * 8),
         o_sym = take((size_t)nq * 16);
  if (!block.alloc(off, st)) return fail(PARIS_ENOMEM, "query state (%zu bytes)", off);
  char* b = block.as<char>();
  qs.nq = nq;
  qs.k = k;
  qs.queries = dq;
  qs.qpaa = (double*)(b + o_paa);
  qs.qkey = (uint64_t*)(b + o_key);
  qs.qtable = (float*)(b + o_tab);
  qs.thr = (uint32_t*)(b + o_thr);
  qs.bsf = (unsigned long long*)(b + o_bsf);
  qs.leaf = (int64_t*)(b + o_leaf);
  qs.seed = (float*)(b + o_seed);
  qs.status = (uint32_t*)(b + o_stat);
  qs.counters = (unsigned long long*)(b + o_cnt);
  qs.qsym = (uint8_t*)(b + o_sym);
  qs.cg = gamma_scale(idx->len);
  PARIS_CUDA(cudaMemsetAsync(qs.status, 0, 4, st));
  PARIS_CUDA(cudaMemsetAsync(qs.counters, 0, 64, st));
  return PARIS_OK;
}

static paris_status check_query_args(const paris_index* idx, const float* queries, int64_t nq, int32_t k) {
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  if (nq < 0) return fail(PARIS_EINVAL, "nq must be >= 0");
  if (nq > 0 && !queries) return fail(PARIS_EINVAL, "queries is NULL");
  if (k < 1 || k > 1024 || (int64_t)k > idx->n)
    return fail(PARIS_EINVAL, "k must be in [1, min(n, 1024)], got %d (n = %lld)", k, (long long)idx->n);
  return PARIS_OK;
}

static paris_status check_query_opts(const paris_index* idx, const paris_query_opts& o) {
  if (o.reserved[0]) return fail(PARIS_EINVAL, "paris_query_opts.reserved must be zero");
  if (o.private_bsf != 0 && o.private_bsf != 1) return fail(PARIS_EINVAL, "private_bsf must be 0 or 1");
  if (o.no_leaf_pruning != 0 && o.no_leaf_pruning != 1) return fail(PARIS_EINVAL, "no_leaf_pruning must be 0 or 1");
  if (o.seed != PARIS_SEED_DESCENT && o.seed != PARIS_SEED_LEARNED && o.seed != PARIS_SEED_ADAPTIVE)
    return fail(PARIS_EINVAL, "unknown seed mode");
  if (o.seed == PARIS_SEED_ADAPTIVE && !idx->ad_nodes)
    return fail(PARIS_EINVAL, "PARIS_SEED_ADAPTIVE needs paris_build_adaptive_leaves first");
  if (o.seed == PARIS_SEED_LEARNED && !idx->seed_model)
    return fail(PARIS_EINVAL, "PARIS_SEED_LEARNED needs a model attached with paris_attach_seed_model");
  if (o.precision != PARIS_REFINE_FP32 && o.precision != PARIS_REFINE_MIXED)
    return fail(PARIS_EINVAL, "unknown precision %d", o.precision);
  if (o.mode != PARIS_MODE_PLAIN && o.mode != PARIS_MODE_BATCHED)
    return fail(PARIS_EINVAL, "unknown mode %d", o.mode);
  if (o.mode == PARIS_MODE_BATCHED && o.query_tile) {
    bool known = false;
    for (int i = 0; i < kNumQueryTiles; ++i) known = known || kQueryTiles[i] == o.query_tile;
    if (!known || !query_tile_fits(o.query_tile, idx->card))
      return fail(PARIS_EINVAL, "query_tile %d is not one of 2, 4, 8, 12, 16, 24 or does not fit", o.query_tile);
  }
  return PARIS_OK;
}

namespace {

// One collection's exact k-NN call: staged queries and outputs, query state, the candidate
// lists of the current chunk of queries and the per-phase timers. The phases are split so that
// several collections can share one batched lower-bound scan launch per chunk round.
struct KnnJob {
  const paris_index* idx = nullptr;
  int64_t nq = 0;
  int k = 1;
  paris_query_opts o{};
  paris_query_stats* stats = nullptr;
  cudaStream_t st = nullptr;
  Staged sq, si, sd;
  QueryState qs;
  DevBuf qblock, lkeys, lbstatus, cblock;
  ChunkState cs;
  PhaseTimer timer{false, nullptr};
  bool mixed = false;
  uint32_t* lb_status = nullptr;  // MIXED: overflow is the signal, not an error
  int64_t qc = 0;
  int qt = 0;
  int64_t dense_total = 0;
  int rescreens = 0;
  bool prune = true;          // leaf pruning: page lower bounds before the row scans
  int64_t paged_chunk = -1;   // chunk whose page bits are ready (BATCHED)
  int64_t pages_examined = 0;

  int64_t chunks() const { return qc > 0 ? (nq + qc - 1) / qc : 0; }

  // Staging, query preparation, approximate search and the candidate-list buffers.
  paris_status setup(const paris_index* index, const float* queries, int64_t n_q, int32_t kk, int64_t* out_idx,
                     float* out_dist, const paris_query_opts& opts, paris_query_stats* st_out, cudaStream_t stream,
                     double budget_share) {
    idx = index;
    nq = n_q;
    k = kk;
    o = opts;
    stats = st_out;
    st = stream;
    timer.on = stats != nullptr;
    timer.st = st;
    if (stats) std::memset(stats, 0, sizeof *stats);
    if (nq == 0) return PARIS_OK;
    const size_t qbytes = (size_t)nq * idx->len * sizeof(float);
    PARIS_TRY(sq.in(queries, qbytes, st));
    PARIS_TRY(si.out(out_idx, (size_t)nq * k * sizeof(int64_t), st));
    PARIS_TRY(sd.out(out_dist, (size_t)nq * k * sizeof(float), st));
    PARIS_TRY(alloc_query_state(idx, nq, k, (const float*)sq.dev, qs, qblock, st));
    qs.private_bsf = o.private_bsf;
    if (o.seed == PARIS_SEED_LEARNED) {
      if (!lkeys.alloc((size_t)nq * (idx->seed_r + 1) * 8, st)) return fail(PARIS_ENOMEM, "learned keys");
      qs.keys = lkeys.as<uint64_t>();
      qs.nk = idx->seed_r + 1;
    }
    // chunks of queries whose candidate lists are resident together; in MIXED precision the lists
    // are short and a query whose list overflows is screened by the BF16 tensor-core pass instead
    mixed = o.precision == PARIS_REFINE_MIXED && dense_supported(idx, k);
    const int64_t cap = mixed ? std::min<int64_t>(idx->n, std::max<int64_t>(idx->n / 128, 8192)) : idx->n;
    if (!lbstatus.alloc(4, st)) return fail(PARIS_ENOMEM, "status word");
    lb_status = mixed ? lbstatus.as<uint32_t>() : qs.status;
    qc = o.chunk;
    if (qc <= 0) {
      size_t freeb = 0, totalb = 0;
      cudaMemGetInfo(&freeb, &totalb);
      double budget = std::min((double)freeb * 0.3, 24.0e9) * budget_share;
      qc = (int64_t)(budget / ((double)cap * 20.0 + (double)kContCap * (4 * kLimbs + 4) + 16384.0 +
                               (double)page_list_cap(idx->n) * 4.0 + (double)page_words(idx->n) * 4.0 +
                               (double)idx->card * 32.0));
      qc = std::max<int64_t>(1, std::min<int64_t>(qc, 4096));
    }
    qc = std::min<int64_t>(std::min(qc, nq), 65535);  // per-query grids of a chunk use the y extent
    size_t off = 0;
    auto take = [&](size_t b) {
      size_t o2 = off;
      off += (b + 255) & ~(size_t)255;
      return o2;
    };
    size_t o_count = take((size_t)qc * 4), o_rows = take((size_t)qc * cap * 4), o_lb = take((size_t)qc * cap * 4),
           o_F = take((size_t)qc * cap * 4), o_pre = take((size_t)(qc + 1) * 4), o_kth = take((size_t)qc * 4),
           o_hist = take((size_t)qc * 2048 * 4), o_sel = take((size_t)qc * 8), o_cc = take((size_t)qc * 4),
           o_cr = take((size_t)qc * kContCap * 4), o_cl = take((size_t)qc * kContCap * kLimbs * 4),
           o_r2 = take((size_t)qc * cap * 4), o_l2 = take((size_t)qc * cap * 4), o_bk = take((size_t)qc * 32 * 4),
           o_pk = take((size_t)((qc + 1) / 2 + 1) * idx->card * 16 * 4), o_pl = take((size_t)qc * 8), o_pm = take((size_t)qc * 4),
           o_ds = take((size_t)qc * 4), o_dn = take(8), o_no = take(8),
           o_dq = take(dense_query_rows(qc) * idx->len * 2), o_dm = take(dense_query_rows(qc) * 8),
           o_pb = take((size_t)qc * page_words(idx->n) * 4),
           o_pls = take((size_t)std::max<int64_t>(qc * page_list_cap(idx->n), page_count(idx->n)) * 4),
           o_pc = take((size_t)qc * 4), o_ip = take((size_t)(qc + 1) * 4);
    if (!cblock.alloc(off, st)) return fail(PARIS_ENOMEM, "candidate lists (%zu bytes)", off);
    char* b = cblock.as<char>();
    cs.cap = cap;
    cs.count = (uint32_t*)(b + o_count);
    cs.rows = (uint32_t*)(b + o_rows);
    cs.lb = (float*)(b + o_lb);
    cs.F = (float*)(b + o_F);
    cs.prefix = (uint32_t*)(b + o_pre);
    cs.kth = (uint32_t*)(b + o_kth);
    cs.sel_hist = (uint32_t*)(b + o_hist);
    cs.sel_state = (uint32_t*)(b + o_sel);
    cs.cont_count = (uint32_t*)(b + o_cc);
    cs.cont_rows = (uint32_t*)(b + o_cr);
    cs.cont_limbs = (uint32_t*)(b + o_cl);
    cs.rows2 = (uint32_t*)(b + o_r2);
    cs.lb2 = (float*)(b + o_l2);
    cs.bucket = (uint32_t*)(b + o_bk);
    cs.packed = (uint32_t*)(b + o_pk);
    cs.pilot = (uint32_t*)(b + o_pl);
    cs.perm = (int*)(b + o_pm);
    cs.dslots = (int*)(b + o_ds);
    cs.dnd = (int*)(b + o_dn);
    cs.nover = (int*)(b + o_no);
    cs.dqbf = (void*)(b + o_dq);
    cs.dqnm = (float2*)(b + o_dm);
    cs.dq_rows = (int64_t)dense_query_rows(qc);
    prune = o.no_leaf_pruning == 0;
    cs.pagebits = prune ? (uint32_t*)(b + o_pb) : nullptr;
    cs.page_list = (uint32_t*)(b + o_pls);
    cs.page_count = (uint32_t*)(b + o_pc);
    cs.item_prefix = (uint32_t*)(b + o_ip);
    paged_chunk = -1;
    pages_examined = 0;
    qt = o.mode == PARIS_MODE_BATCHED ? o.query_tile : 0;
    return PARIS_OK;
  }

  // Page bits of the current chunk's queries (BATCHED leaf pruning).
  paris_status page_pass(int64_t c) {
    if (!prune || o.mode != PARIS_MODE_BATCHED || paged_chunk == c) return PARIS_OK;
    timer.begin(2);
    // in MIXED refinement a query over its list is screened on the tensor cores: its page bits
    // and exact page count are not needed (no tile scan runs then)
    PARIS_TRY(launch_page_lb(idx, qs, cs.q0, cs.qc, cs.pagebits, cs.page_list, cs.page_count,
                             page_list_cap(idx->n), st, mixed && cs.cap < idx->n));
    timer.end(2);
    pages_examined += idx->npages * (int64_t)cs.qc;
    paged_chunk = c;
    return PARIS_OK;
  }

  // Query preparation and approximate search (the seeds of every query).
  paris_status front() {
    if (nq == 0) return PARIS_OK;
    timer.begin(0);
    PARIS_TRY(launch_query_prep(idx, qs, st));
    timer.end(0);
    timer.begin(1);
    if (o.seed == PARIS_SEED_LEARNED)
      PARIS_TRY(learned_keys(idx, idx->seed_model, idx->seed_r, qs, lkeys.as<uint64_t>(), st));
    PARIS_TRY(launch_descent(idx, qs, st, o.seed == PARIS_SEED_ADAPTIVE));
    timer.end(1);
    return PARIS_OK;
  }

  // The whole call as one stream of launches with no host synchronisation (for graph capture):
  // the query tile must be known; screened lists that overflow are only counted (cs.nover).
  paris_status record_all() {
    if (nq == 0) return PARIS_OK;
    if (o.mode == PARIS_MODE_BATCHED && qt == 0) return fail(PARIS_EINTERNAL, "query tile unknown at capture");
    PARIS_CUDA(cudaMemsetAsync(qs.status, 0, 4, st));
    PARIS_CUDA(cudaMemsetAsync(qs.counters, 0, 64, st));
    PARIS_CUDA(cudaMemsetAsync(cs.nover, 0, 4, st));
    PARIS_TRY(front());
    paged_chunk = -1;
    pages_examined = 0;
    for (int64_t c = 0; c < chunks(); ++c) {
      cs.q0 = c * qc;
      cs.qc = (int)std::min<int64_t>(qc, nq - cs.q0);
      PARIS_CUDA(cudaMemsetAsync(cs.count, 0, (size_t)cs.qc * 4, st));
      PARIS_TRY(page_pass(c));
      PARIS_TRY(scan_chunk());
      if (mixed) PARIS_TRY(launch_dense(const_cast<paris_index*>(idx), qs, cs, lb_status, nullptr, st));
      PARIS_TRY(launch_refine(idx, qs, cs, st));
      PARIS_TRY(launch_select(idx, qs, cs, (int64_t*)si.dev, (float*)sd.dev, st));
      if (mixed) PARIS_TRY(launch_tighten(qs, cs, st));
    }
    return PARIS_OK;
  }

  // The whole call with host decisions (tuning, screening tile counts, repeated screenings).
  paris_status run_eager(const char* what) {
    if (nq == 0) return PARIS_OK;
    PARIS_CUDA(cudaMemsetAsync(qs.status, 0, 4, st));
    PARIS_CUDA(cudaMemsetAsync(qs.counters, 0, 64, st));
    dense_total = 0;
    rescreens = 0;
    paged_chunk = -1;
    pages_examined = 0;
    PARIS_TRY(front());
    for (int64_t c = 0; c < chunks(); ++c) {
      PARIS_TRY(begin_chunk(c));
      PARIS_TRY(scan_chunk());
      PARIS_TRY(finish_chunk());
    }
    return finish(what);
  }

  // Selects chunk `c` and clears its candidate counts; tunes the query tile on first use.
  paris_status begin_chunk(int64_t c) {
    cs.q0 = c * qc;
    cs.qc = (int)std::min<int64_t>(qc, nq - cs.q0);
    PARIS_CUDA(cudaMemsetAsync(cs.count, 0, (size_t)cs.qc * 4, st));
    PARIS_TRY(page_pass(c));  // before tuning: the trial scans visit the kept pages only
    if (o.mode == PARIS_MODE_BATCHED && qt == 0) PARIS_TRY(tuned_query_tile(idx, qs, cs, prune, st, &qt));
    return PARIS_OK;
  }

  // This collection's own lower-bound scan of the current chunk.
  paris_status scan_chunk() {
    timer.begin(2);
    if (o.mode == PARIS_MODE_BATCHED) {
      PARIS_TRY(launch_lbscan_batched(idx, qs, cs, qt, mixed ? 1 : 0, lb_status, st));
    } else if (prune) {
      // the paper's one-query pass, over the pages whose envelope may hold a kept row
      for (int j = 0; j < cs.qc; ++j) {
        PARIS_TRY(launch_page_lb(idx, qs, cs.q0 + j, 1, nullptr, cs.page_list, cs.page_count, idx->npages, st));
        PARIS_TRY(launch_lbscan_pages(idx, qs, cs.q0 + j, cs.page_list, cs.page_count, cs.count + j,
                                      cs.rows + (int64_t)j * cs.cap, cs.lb + (int64_t)j * cs.cap, cs.cap, lb_status,
                                      mixed ? 1 : 0, st));
      }
      pages_examined += idx->npages * (int64_t)cs.qc;
    } else {
      for (int j = 0; j < cs.qc; ++j)
        PARIS_TRY(launch_lbscan(idx, qs, cs.q0 + j, cs.count + j, cs.rows + (int64_t)j * cs.cap,
                                cs.lb + (int64_t)j * cs.cap, cs.cap, lb_status, mixed ? 1 : 0, st));
    }
    timer.end(2);
    return PARIS_OK;
  }

  // Tensor-core screening (MIXED), refinement and selection of the current chunk.
  paris_status finish_chunk() {
    if (mixed) {
      int nd = 0;
      timer.begin(5);
      PARIS_TRY(launch_dense(const_cast<paris_index*>(idx), qs, cs, lb_status, &nd, st));
      timer.end(5);
      dense_total += nd;
    }
    timer.begin(3);
    PARIS_TRY(launch_refine(idx, qs, cs, st));
    timer.end(3);
    timer.begin(4);
    PARIS_TRY(launch_select(idx, qs, cs, (int64_t*)si.dev, (float*)sd.dev, st));
    timer.end(4);
    // a screened list that overflowed: lower the query's threshold to the k-th best candidate it
    // stored and screen it again (rare; the other queries' lists are unchanged by the repeat)
    for (int retry = 0; mixed; ++retry) {
      int nover = 0;
      PARIS_TRY(tighten_overflowed(qs, cs, &nover, st));
      if (nover == 0) break;
      if (retry == kDenseRetries) return fail(PARIS_EINTERNAL, "paris_exact_knn: candidate list overflow");
      rescreens += nover;
      int nd = 0;
      timer.begin(5);
      PARIS_TRY(launch_dense(const_cast<paris_index*>(idx), qs, cs, lb_status, &nd, st));
      timer.end(5);
      timer.begin(3);
      PARIS_TRY(launch_refine(idx, qs, cs, st));
      timer.end(3);
      timer.begin(4);
      PARIS_TRY(launch_select(idx, qs, cs, (int64_t*)si.dev, (float*)sd.dev, st));
      timer.end(4);
    }
    return PARIS_OK;
  }

  // Outputs back to host buffers, device status and statistics.
  paris_status finish(const char* what) {
    if (nq == 0) return PARIS_OK;
    PARIS_TRY(si.finish(st));
    PARIS_TRY(sd.finish(st));
    PARIS_TRY(check_status_word(qs.status, st, what));
    if (stats) {
      double ms[6] = {0, 0, 0, 0, 0, 0};
      timer.collect(ms);
      stats->ms_dense = ms[5];
      stats->query_tile = qt;
      stats->rescreens = rescreens;
      stats->dense_queries = dense_total;
      stats->ms_prep = ms[0];
      stats->ms_descent = ms[1];
      stats->ms_lbscan = ms[2];
      stats->ms_refine = ms[3];
      stats->ms_select = ms[4];
      unsigned long long c[8];
      PARIS_CUDA(cudaMemcpyAsync(c, qs.counters, sizeof c, cudaMemcpyDeviceToHost, st));
      PARIS_CUDA(cudaStreamSynchronize(st));
      stats->candidates = (int64_t)c[0];
      stats->refined = (int64_t)c[1];
      stats->contenders = (int64_t)c[2];
      stats->leaf_rows = (int64_t)c[3];
      stats->lb_lookups = (int64_t)c[4];
      stats->pages_kept = (int64_t)c[5];
      stats->pages_examined = pages_examined;
      stats->list_rows = (int64_t)c[6];
      stats->bsf_updates = (int64_t)c[7];
    }
    return PARIS_OK;
  }
};

}  // namespace

paris_status paris_exact_knn_ex(const paris_index* idx, const float* queries, int64_t nq, int32_t k,
                                int64_t* out_idx, float* out_dist, const paris_query_opts* opts,
                                paris_query_stats* stats, void* stream) {
  clear_error();
  PARIS_TRY(check_query_args(idx, queries, nq, k));
  if (nq > 0 && !out_idx) return fail(PARIS_EINVAL, "out_idx is NULL");
  paris_query_opts o{};
  if (opts) o = *opts;
  PARIS_TRY(check_query_opts(idx, o));
  KnnJob job;
  PARIS_TRY(job.setup(idx, queries, nq, k, out_idx, out_dist, o, stats, (cudaStream_t)stream, 1.0));
  return job.run_eager("paris_exact_knn");
}

namespace {

// The query tile of a multi-collection scan launch: the tuned tile of the collection with the
// most work (rows x chunk queries) in this round.
int multi_round_tile(KnnJob* jobs, int nidx, int64_t r) {
  int qt = 0;
  double most = -1.0;
  for (int c = 0; c < nidx; ++c) {
    if (r >= jobs[c].chunks()) continue;
    const double work = (double)jobs[c].idx->n * jobs[c].cs.qc;
    if (work > most) {
      most = work;
      qt = jobs[c].qt;
    }
  }
  return qt;
}

// Several collections with host decisions (tuning, screening tile counts, repeated screenings):
// per chunk round, one batched scan launch over every collection's chunk.
paris_status multi_run_eager(KnnJob* jobs, int nidx, const char* what) {
  const paris_query_opts& o = jobs[0].o;
  int64_t rounds = 0;
  for (int c = 0; c < nidx; ++c) {
    if (jobs[c].nq > 0) {
      PARIS_CUDA(cudaMemsetAsync(jobs[c].qs.status, 0, 4, jobs[c].st));
      PARIS_CUDA(cudaMemsetAsync(jobs[c].qs.counters, 0, 64, jobs[c].st));
    }
    jobs[c].dense_total = 0;
    jobs[c].rescreens = 0;
    jobs[c].paged_chunk = -1;
    jobs[c].pages_examined = 0;
    PARIS_TRY(jobs[c].front());
    rounds = std::max(rounds, jobs[c].chunks());
  }
  for (int64_t r = 0; r < rounds; ++r) {
    ScanJob sj[kMaxScanJobs];
    int m = 0;
    for (int c = 0; c < nidx; ++c) {
      if (r >= jobs[c].chunks()) continue;
      PARIS_TRY(jobs[c].begin_chunk(r));
      if (o.mode == PARIS_MODE_BATCHED)
        sj[m++] = ScanJob{jobs[c].idx, &jobs[c].qs, &jobs[c].cs, jobs[c].mixed ? 1 : 0, jobs[c].lb_status};
      else
        PARIS_TRY(jobs[c].scan_chunk());
    }
    if (m > 0) {
      // one launch scans every collection's chunk; its time is charged to each collection
      for (int c = 0; c < nidx; ++c)
        if (r < jobs[c].chunks()) jobs[c].timer.begin(2);
      PARIS_TRY(launch_lbscan_batched_multi(sj, m, multi_round_tile(jobs, nidx, r), jobs[0].st));
      for (int c = 0; c < nidx; ++c)
        if (r < jobs[c].chunks()) jobs[c].timer.end(2);
    }
    for (int c = 0; c < nidx; ++c)
      if (r < jobs[c].chunks()) PARIS_TRY(jobs[c].finish_chunk());
  }
  for (int c = 0; c < nidx; ++c) PARIS_TRY(jobs[c].finish(what));
  return PARIS_OK;
}

// The same call as one stream of launches without host synchronisation (for graph capture):
// every collection's query tile must be known; overflowed screened lists are only counted.
paris_status multi_record(KnnJob* jobs, int nidx) {
  const paris_query_opts& o = jobs[0].o;
  int64_t rounds = 0;
  for (int c = 0; c < nidx; ++c) {
    KnnJob& J = jobs[c];
    if (J.nq == 0) continue;
    if (o.mode == PARIS_MODE_BATCHED && J.qt == 0) return fail(PARIS_EINTERNAL, "query tile unknown at capture");
    PARIS_CUDA(cudaMemsetAsync(J.qs.status, 0, 4, J.st));
    PARIS_CUDA(cudaMemsetAsync(J.qs.counters, 0, 64, J.st));
    PARIS_CUDA(cudaMemsetAsync(J.cs.nover, 0, 4, J.st));
    J.paged_chunk = -1;
    J.pages_examined = 0;
    PARIS_TRY(J.front());
    rounds = std::max(rounds, J.chunks());
  }
  for (int64_t r = 0; r < rounds; ++r) {
    ScanJob sj[kMaxScanJobs];
    int m = 0;
    for (int c = 0; c < nidx; ++c) {
      KnnJob& J = jobs[c];
      if (r >= J.chunks()) continue;
      J.cs.q0 = r * J.qc;
      J.cs.qc = (int)std::min<int64_t>(J.qc, J.nq - J.cs.q0);
      PARIS_CUDA(cudaMemsetAsync(J.cs.count, 0, (size_t)J.cs.qc * 4, J.st));
      PARIS_TRY(J.page_pass(r));
      if (o.mode == PARIS_MODE_BATCHED)
        sj[m++] = ScanJob{J.idx, &J.qs, &J.cs, J.mixed ? 1 : 0, J.lb_status};
      else
        PARIS_TRY(J.scan_chunk());
    }
    if (m > 0) PARIS_TRY(launch_lbscan_batched_multi(sj, m, multi_round_tile(jobs, nidx, r), jobs[0].st));
    for (int c = 0; c < nidx; ++c) {
      KnnJob& J = jobs[c];
      if (r >= J.chunks()) continue;
      if (J.mixed) PARIS_TRY(launch_dense(const_cast<paris_index*>(J.idx), J.qs, J.cs, J.lb_status, nullptr, J.st));
      PARIS_TRY(launch_refine(J.idx, J.qs, J.cs, J.st));
      PARIS_TRY(launch_select(J.idx, J.qs, J.cs, (int64_t*)J.si.dev, (float*)J.sd.dev, J.st));
      if (J.mixed) PARIS_TRY(launch_tighten(J.qs, J.cs, J.st));
    }
  }
  return PARIS_OK;
}

}  // namespace

// A captured query pipeline: the plan owns the query and output buffers of each of its
// collections (one, or up to kMaxScanJobs for a multi-collection batch) and one KnnJob per
// collection; the first run executes eagerly (choosing the query tiles) and then records the
// whole call as one CUDA graph that later runs replay.
struct paris_knn_plan {
  int nj = 0;
  const paris_index* idx[kMaxScanJobs] = {};
  int64_t nq[kMaxScanJobs] = {};
  int k = 1;
  paris_query_opts o{};
  cudaStream_t pst = nullptr;
  cudaEvent_t ev = nullptr;
  DevBuf qbuf[kMaxScanJobs], obi[kMaxScanJobs], obd[kMaxScanJobs];
  KnnJob* job = nullptr;  // [nj]
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0, replays = 0, eager_runs = 0;
  bool capture_failed = false;
};

namespace {
paris_status plan_create(const paris_index* const* idx, int nidx, const int64_t* nq, int32_t k,
                         const paris_query_opts* opts, paris_knn_plan** out) {
  if (!out) return fail(PARIS_EINVAL, "out is NULL");
  *out = nullptr;
  if (nidx < 1 || nidx > kMaxScanJobs) return fail(PARIS_EINVAL, "between 1 and %d collections per plan", kMaxScanJobs);
  paris_query_opts o{};
  if (opts) o = *opts;
  int64_t total_q = 0;
  for (int c = 0; c < nidx; ++c) {
    if (nq[c] < 0) return fail(PARIS_EINVAL, "nq must be >= 0");
    total_q += nq[c];
    PARIS_TRY(check_query_args(idx[c], (const float*)1, std::max<int64_t>(nq[c], 1), k));
    PARIS_TRY(check_query_opts(idx[c], o));
    if (idx[c]->card != idx[0]->card) return fail(PARIS_EINVAL, "the collections must share the cardinality");
  }
  if (total_q < 1) return fail(PARIS_EINVAL, "a plan needs nq >= 1");
  if (o.seed == PARIS_SEED_LEARNED) return fail(PARIS_EINVAL, "captured plans use the descent seed only");
  auto* pl = new (std::nothrow) paris_knn_plan;
  if (!pl) return fail(PARIS_ENOMEM, "plan");
  pl->nj = nidx;
  pl->k = k;
  pl->o = o;
  auto bail = [&](paris_status s) {
    paris_knn_plan_free(pl);
    return s;
  };
  if (cudaStreamCreateWithFlags(&pl->pst, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(PARIS_ECUDA, "plan stream"));
  }
  pl->job = new (std::nothrow) KnnJob[nidx];
  if (!pl->job) return bail(fail(PARIS_ENOMEM, "plan"));
  double rows = 0.0;
  for (int c = 0; c < nidx; ++c) rows += (double)idx[c]->n;
  for (int c = 0; c < nidx; ++c) {
    pl->idx[c] = idx[c];
    pl->nq[c] = nq[c];
    const int64_t m = std::max<int64_t>(nq[c], 1);
    if (!pl->qbuf[c].alloc((size_t)m * idx[c]->len * 4, pl->pst) || !pl->obi[c].alloc((size_t)m * k * 8, pl->pst) ||
        !pl->obd[c].alloc((size_t)m * k * 4, pl->pst))
      return bail(fail(PARIS_ENOMEM, "plan buffers"));
    paris_status st = pl->job[c].setup(idx[c], pl->qbuf[c].as<float>(), nq[c], k, pl->obi[c].as<int64_t>(),
                                       pl->obd[c].as<float>(), o, nullptr, pl->pst, (double)idx[c]->n / rows);
    if (st != PARIS_OK) return bail(st);
    if (pl->job[c].mixed) {
      st = ensure_shadow(const_cast<paris_index*>(idx[c]), pl->pst);
      if (st != PARIS_OK) return bail(st);
    }
  }
  if (cudaStreamSynchronize(pl->pst) != cudaSuccess) return bail(fail(PARIS_ECUDA, "plan setup"));
  *out = pl;
  return PARIS_OK;
}

paris_status plan_capture(paris_knn_plan* pl) {
  const uint64_t before = launch_count();
  if (cudaStreamBeginCapture(pl->pst, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return fail(PARIS_ECUDA, "stream capture could not start");
  }
  paris_status s = pl->nj == 1 ? pl->job[0].record_all() : multi_record(pl->job, pl->nj);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(pl->pst, &g);
  if (s != PARIS_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return s != PARIS_OK ? s : fail(PARIS_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
  }
  if (cudaGraphInstantiate(&pl->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(PARIS_ECUDA, "graph instantiation failed");
  }
  pl->graph = g;
  pl->kernels = (int64_t)(launch_count() - before);
  // the recording counted kernels it did not run; replays count them when they run
  note_launches(-(int)pl->kernels);
  return PARIS_OK;
}

paris_status plan_run(paris_knn_plan* pl, const float* const* queries, int64_t* const* out_idx,
                      float* const* out_dist, void* stream) {
  for (int c = 0; c < pl->nj; ++c)
    if (pl->nq[c] > 0 && (!queries[c] || !out_idx[c])) return fail(PARIS_EINVAL, "NULL argument");
  cudaStream_t cst = (cudaStream_t)stream;
  PARIS_CUDA(cudaEventRecord(pl->ev, cst));
  PARIS_CUDA(cudaStreamWaitEvent(pl->pst, pl->ev, 0));
  for (int c = 0; c < pl->nj; ++c)
    if (pl->nq[c] > 0)
      PARIS_CUDA(cudaMemcpyAsync(pl->qbuf[c].p, queries[c], (size_t)pl->nq[c] * pl->idx[c]->len * 4,
                                 cudaMemcpyDefault, pl->pst));
  bool eager = true;
  if (pl->exec) {
    PARIS_CUDA(cudaGraphLaunch(pl->exec, pl->pst));
    note_launches((int)pl->kernels);
    ++pl->replays;
    uint32_t nover[kMaxScanJobs] = {};
    for (int c = 0; c < pl->nj; ++c)
      if (pl->nq[c] > 0)
        PARIS_CUDA(cudaMemcpyAsync(&nover[c], pl->job[c].cs.nover, 4, cudaMemcpyDeviceToHost, pl->pst));
    PARIS_CUDA(cudaStreamSynchronize(pl->pst));
    // a screened list that overflowed needs the host-driven repeats: run the batch eagerly
    eager = false;
    for (int c = 0; c < pl->nj; ++c) eager = eager || nover[c] != 0u;
    if (!eager)
      for (int c = 0; c < pl->nj; ++c)
        if (pl->nq[c] > 0) PARIS_TRY(check_status_word(pl->job[c].qs.status, pl->pst, "paris_knn_plan_run"));
  }
  if (eager) {
    if (pl->nj == 1)
      PARIS_TRY(pl->job[0].run_eager("paris_knn_plan_run"));
    else
      PARIS_TRY(multi_run_eager(pl->job, pl->nj, "paris_knn_plan_run_multi"));
    ++pl->eager_runs;
    if (!pl->exec && !pl->capture_failed) {
      // the query tiles are settled now; later runs replay the recorded call
      if (plan_capture(pl) != PARIS_OK) {
        pl->capture_failed = true;  // keep running eagerly
        clear_error();
      }
    }
  }
  for (int c = 0; c < pl->nj; ++c) {
    if (pl->nq[c] == 0) continue;
    PARIS_CUDA(cudaMemcpyAsync(out_idx[c], pl->obi[c].p, (size_t)pl->nq[c] * pl->k * 8, cudaMemcpyDefault, pl->pst));
    if (out_dist && out_dist[c])
      PARIS_CUDA(cudaMemcpyAsync(out_dist[c], pl->obd[c].p, (size_t)pl->nq[c] * pl->k * 4, cudaMemcpyDefault,
                                 pl->pst));
  }
  PARIS_CUDA(cudaEventRecord(pl->ev, pl->pst));
  PARIS_CUDA(cudaStreamWaitEvent(cst, pl->ev, 0));
  PARIS_CUDA(cudaStreamSynchronize(pl->pst));
  return PARIS_OK;
}
}  // namespace

paris_status paris_knn_plan_create(const paris_index* idx, int64_t nq, int32_t k, const paris_query_opts* opts,
                                   paris_knn_plan** out) {
  clear_error();
  if (out) *out = nullptr;
  if (nq < 1) return fail(PARIS_EINVAL, "a plan needs nq >= 1");
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  return plan_create(&idx, 1, &nq, k, opts, out);
}

paris_status paris_knn_plan_create_multi(const paris_index* const* idx, int32_t nidx, const int64_t* nq, int32_t k,
                                         const paris_query_opts* opts, paris_knn_plan** out) {
  clear_error();
  if (out) *out = nullptr;
  if (!idx || !nq) return fail(PARIS_EINVAL, "NULL argument array");
  for (int c = 0; c < nidx && c < kMaxScanJobs; ++c)
    if (!idx[c]) return fail(PARIS_EINVAL, "index %d is NULL", c);
  paris_query_opts o{};
  if (opts) o = *opts;
  if (o.mode != PARIS_MODE_BATCHED) return fail(PARIS_EINVAL, "multi-collection plans use BATCHED mode");
  return plan_create(idx, nidx, nq, k, &o, out);
}

void paris_knn_plan_free(paris_knn_plan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  delete[] pl->job;
  for (int c = 0; c < kMaxScanJobs; ++c) {
    pl->qbuf[c].release();
    pl->obi[c].release();
    pl->obd[c].release();
  }
  if (pl->pst) {
    cudaStreamSynchronize(pl->pst);
    cudaStreamDestroy(pl->pst);
  }
  if (pl->ev) cudaEventDestroy(pl->ev);
  delete pl;
}

paris_status paris_knn_plan_run(paris_knn_plan* pl, const float* queries, int64_t* out_idx, float* out_dist,
                                void* stream) {
  clear_error();
  if (!pl || !queries || !out_idx) return fail(PARIS_EINVAL, "NULL argument");
  if (pl->nj != 1) return fail(PARIS_EINVAL, "a multi-collection plan runs with paris_knn_plan_run_multi");
  float* const od[1] = {out_dist};
  return plan_run(pl, &queries, &out_idx, out_dist ? od : nullptr, stream);
}

paris_status paris_knn_plan_run_multi(paris_knn_plan* pl, const float* const* queries, int64_t* const* out_idx,
                                      float* const* out_dist, void* stream) {
  clear_error();
  if (!pl || !queries || !out_idx) return fail(PARIS_EINVAL, "NULL argument");
  return plan_run(pl, queries, out_idx, out_dist, stream);
}

paris_status paris_knn_plan_info(const paris_knn_plan* pl, paris_knn_plan_stats* out) {
  clear_error();
  if (!pl || !out) return fail(PARIS_EINVAL, "NULL argument");
  std::memset(out, 0, sizeof *out);
  out->graph_kernels = pl->kernels;
  out->replays = pl->replays;
  out->eager_runs = pl->eager_runs;
  out->captured = pl->exec != nullptr;
  out->query_tile = pl->job ? pl->job[0].qt : 0;
  return PARIS_OK;
}

paris_status paris_exact_knn_multi(const paris_index* const* idx, int32_t nidx, const float* const* queries,
                                   const int64_t* nq, int32_t k, int64_t* const* out_idx, float* const* out_dist,
                                   const paris_query_opts* opts, paris_query_stats* stats, void* stream) {
  clear_error();
  if (nidx < 1 || nidx > kMaxScanJobs) return fail(PARIS_EINVAL, "nidx must be in [1, %d]", kMaxScanJobs);
  if (!idx || !queries || !nq || !out_idx) return fail(PARIS_EINVAL, "NULL argument array");
  paris_query_opts o{};
  if (opts) o = *opts;
  for (int c = 0; c < nidx; ++c) {
    PARIS_TRY(check_query_args(idx[c], queries[c], nq[c], k));
    if (nq[c] > 0 && !out_idx[c]) return fail(PARIS_EINVAL, "out_idx[%d] is NULL", c);
    PARIS_TRY(check_query_opts(idx[c], o));
    if (idx[c]->card != idx[0]->card) return fail(PARIS_EINVAL, "the collections must share the cardinality");
    for (int d = 0; d < c; ++d)
      if (out_idx[d] && out_idx[d] == out_idx[c]) return fail(PARIS_EINVAL, "out_idx[%d] aliases out_idx[%d]", c, d);
  }
  cudaStream_t st = (cudaStream_t)stream;
  KnnJob jobs[kMaxScanJobs];
  double total = 0.0;
  for (int c = 0; c < nidx; ++c) total += (double)idx[c]->n;
  for (int c = 0; c < nidx; ++c) {
    // candidate-list memory is shared in proportion to collection size
    PARIS_TRY(jobs[c].setup(idx[c], queries[c], nq[c], k, out_idx[c], out_dist ? out_dist[c] : nullptr, o,
                            stats ? &stats[c] : nullptr, st, (double)idx[c]->n / total));
  }
  return multi_run_eager(jobs, nidx, "paris_exact_knn_multi");
}

paris_status paris_exact_knn(const paris_index* idx, const float* queries, int64_t nq, int32_t k,
                             int64_t* out_idx, float* out_dist, void* stream) {
  return paris_exact_knn_ex(idx, queries, nq, k, out_idx, out_dist, nullptr, nullptr, stream);
}

paris_status paris_approx_search(const paris_index* idx, const float* queries, int64_t nq, int32_t k,
                                 int64_t* out_leaf, float* out_seed_sq, void* stream) {
  return paris_approx_search_ex(idx, queries, nq, k, PARIS_SEED_DESCENT, out_leaf, out_seed_sq, stream);
}

paris_status paris_attach_seed_model(paris_index* idx, const paris_seed_model* model, int32_t top_r) {
  clear_error();
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  if (model && (top_r < 1 || top_r > 8)) return fail(PARIS_EINVAL, "top_r must be in [1, 8]");
  if (model && (int64_t)(top_r + 1) * std::max(idx->leaf_cap, 16) > 16384)
    return fail(PARIS_EINVAL, "top_r + 1 leaves of %d rows exceed the approximate search's buffer", idx->leaf_cap);
  idx->seed_model = model;
  idx->seed_r = model ? top_r : 0;
  return PARIS_OK;
}

paris_status paris_row_buckets(const paris_index* idx, const int64_t* rows, int64_t m, int32_t* out_buckets,
                               void* stream) {
  clear_error();
  if (!idx || (m > 0 && (!rows || !out_buckets))) return fail(PARIS_EINVAL, "NULL argument");
  if (m <= 0) return PARIS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Staged sr, so;
  PARIS_TRY(sr.in(rows, (size_t)m * 8, st));
  PARIS_TRY(so.out(out_buckets, (size_t)m * 4, st));
  DevBuf status;
  if (!status.alloc(4, st)) return fail(PARIS_ENOMEM, "status");
  PARIS_CUDA(cudaMemsetAsync(status.p, 0, 4, st));
  PARIS_TRY(launch_row_buckets(idx, (const int64_t*)sr.dev, m, (int32_t*)so.dev, status.as<uint32_t>(), st));
  PARIS_TRY(so.finish(st));
  uint32_t s = 0;
  PARIS_CUDA(cudaMemcpyAsync(&s, status.p, 4, cudaMemcpyDeviceToHost, st));
  PARIS_CUDA(cudaStreamSynchronize(st));
  if (s & DEV_BADROW) return fail(PARIS_EINVAL, "paris_row_buckets: row index outside [0, n)");
  return PARIS_OK;
}

paris_status paris_approx_search_ex(const paris_index* idx, const float* queries, int64_t nq, int32_t k,
                                    int32_t seed_mode, int64_t* out_leaf, float* out_seed_sq, void* stream) {
  clear_error();
  PARIS_TRY(check_query_args(idx, queries, nq, k));
  if (seed_mode != PARIS_SEED_DESCENT && seed_mode != PARIS_SEED_LEARNED && seed_mode != PARIS_SEED_ADAPTIVE)
    return fail(PARIS_EINVAL, "unknown seed mode");
  if (seed_mode == PARIS_SEED_LEARNED && !idx->seed_model) return fail(PARIS_EINVAL, "no seed model attached");
  if (seed_mode == PARIS_SEED_ADAPTIVE && !idx->ad_nodes) return fail(PARIS_EINVAL, "no adaptive-split leaves built");
  if (nq == 0) return PARIS_OK;
  if (!out_leaf) return fail(PARIS_EINVAL, "out_leaf is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  Staged sq, sl, ss;
  PARIS_TRY(sq.in(queries, (size_t)nq * idx->len * 4, st));
  PARIS_TRY(sl.out(out_leaf, (size_t)nq * 16, st));
  PARIS_TRY(ss.out(out_seed_sq, (size_t)nq * 4, st));
  QueryState qs;
  DevBuf qblock;
  PARIS_TRY(alloc_query_state(idx, nq, k, (const float*)sq.dev, qs, qblock, st));
  PARIS_TRY(launch_query_prep(idx, qs, st));
  DevBuf lkeys;
  if (seed_mode == PARIS_SEED_LEARNED) {
    if (!lkeys.alloc((size_t)nq * (idx->seed_r + 1) * 8, st)) return fail(PARIS_ENOMEM, "learned keys");
    PARIS_TRY(learned_keys(idx, idx->seed_model, idx->seed_r, qs, lkeys.as<uint64_t>(), st));
    qs.keys = lkeys.as<uint64_t>();
    qs.nk = idx->seed_r + 1;
  }
  PARIS_TRY(launch_descent(idx, qs, st, seed_mode == PARIS_SEED_ADAPTIVE));
  PARIS_CUDA(cudaMemcpyAsync(sl.dev, qs.leaf, (size_t)nq * 16, cudaMemcpyDeviceToDevice, st));
  if (out_seed_sq) PARIS_CUDA(cudaMemcpyAsync(ss.dev, qs.seed, (size_t)nq * 4, cudaMemcpyDeviceToDevice, st));
  PARIS_TRY(sl.finish(st));
  PARIS_TRY(ss.finish(st));
  return check_status_word(qs.status, st, "paris_approx_search");
}

paris_status paris_build_adaptive_leaves(paris_index* idx, void* stream) {
  clear_error();
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  return build_adaptive(idx, (cudaStream_t)stream);
}

paris_status paris_adaptive_leaves_info(const paris_index* idx, int64_t* n_nodes, int64_t* n_leaves, int32_t* depth) {
  clear_error();
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  if (!idx->ad_nodes) return fail(PARIS_EINVAL, "no adaptive-split leaves built");
  if (n_nodes) *n_nodes = idx->ad_nnodes;
  if (n_leaves) *n_leaves = idx->ad_leaves;
  if (depth) *depth = idx->ad_depth;
  return PARIS_OK;
}

paris_status paris_adaptive_leaves_export(const paris_index* idx, uint32_t* rows_host, int64_t* nodes_host,
                                          void* stream) {
  clear_error();
  if (!idx) return fail(PARIS_EINVAL, "index is NULL");
  if (!idx->ad_nodes) return fail(PARIS_EINVAL, "no adaptive-split leaves built");
  return export_adaptive(idx, rows_host, nodes_host, (cudaStream_t)stream);
}

paris_status paris_leaf_scan(const paris_index* idx, const float* query, float threshold_sq, uint32_t* out_bits,
                             int64_t* out_kept, void* stream) {
  clear_error();
  PARIS_TRY(check_query_args(idx, query, 1, 1));
  if (!out_bits || !out_kept) return fail(PARIS_EINVAL, "NULL output");
  if (!is_device_ptr(out_bits)) return fail(PARIS_EINVAL, "out_bits must be device memory");
  if (!(threshold_sq >= 0.f)) return fail(PARIS_EINVAL, "threshold_sq must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  Staged sq;
  PARIS_TRY(sq.in(query, (size_t)idx->len * 4, st));
  QueryState qs;
  DevBuf qblock;
  PARIS_TRY(alloc_query_state(idx, 1, 1, (const float*)sq.dev, qs, qblock, st));
  PARIS_TRY(launch_query_prep(idx, qs, st));
  uint32_t tb = 0;
  std::memcpy(&tb, &threshold_sq, 4);
  PARIS_CUDA(cudaMemcpyAsync(qs.thr, &tb, 4, cudaMemcpyHostToDevice, st));
  DevBuf cnt;
  if (!cnt.alloc(4, st)) return fail(PARIS_ENOMEM, "counter");
  PARIS_TRY(launch_page_lb(idx, qs, 0, 1, out_bits, nullptr, cnt.as<uint32_t>(), 0, st));
  unsigned long long kept = 0;
  PARIS_CUDA(cudaMemcpyAsync(&kept, qs.counters + 5, 8, cudaMemcpyDeviceToHost, st));
  PARIS_TRY(check_status_word(qs.status, st, "paris_leaf_scan"));
  *out_kept = (int64_t)kept;
  return PARIS_OK;
}

paris_status paris_lb_scan(const paris_index* idx, const float* query, float threshold_sq, uint32_t* out_rows,
                           float* out_lb, int64_t capacity, int64_t* out_count, void* stream) {
  clear_error();
  PARIS_TRY(check_query_args(idx, query, 1, 1));
  if (!out_count || capacity < 0 || (capacity > 0 && (!out_rows || !out_lb)))
    return fail(PARIS_EINVAL, "bad output arguments");
  if (capacity > 0 && (!is_device_ptr(out_rows) || !is_device_ptr(out_lb)))
    return fail(PARIS_EINVAL, "out_rows/out_lb must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  Staged sq;
  PARIS_TRY(sq.in(query, (size_t)idx->len * 4, st));
  QueryState qs;
  DevBuf qblock, cnt;
  PARIS_TRY(alloc_query_state(idx, 1, 1, (const float*)sq.dev, qs, qblock, st));
  if (!cnt.alloc(4, st)) return fail(PARIS_ENOMEM, "counter");
  PARIS_CUDA(cudaMemsetAsync(cnt.p, 0, 4, st));
  PARIS_TRY(launch_query_prep(idx, qs, st));
  PARIS_TRY(launch_lbscan_threshold(idx, qs.qtable, threshold_sq, cnt.as<uint32_t>(), out_rows, out_lb, capacity,
                                    qs.status, st));
  uint32_t c = 0;
  PARIS_CUDA(cudaMemcpyAsync(&c, cnt.p, 4, cudaMemcpyDeviceToHost, st));
  paris_status s = check_status_word(qs.status, st, "paris_lb_scan");
  *out_count = c;
  if (s == PARIS_EINTERNAL) return PARIS_OK;  // overflow of the caller's capacity is reported by the count
  return s;
}

}  // extern "C"
