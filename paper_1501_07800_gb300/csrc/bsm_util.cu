// Host utilities: stream-ordered allocation, pinned scratch, CUB scans/sorts.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <array>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "bsm_internal.cuh"

bsm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BSM_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return BSM_ERR_OOM;
  }
  return BSM_ERR_CUDA;
}

// Allocations of at least kBulkBytes (a product's C values, large staging
// buffers) come from a second pool of the library's own, the rest from the
// device's default pool.  With one pool, the short-lived buffers of the next
// product (its symbolic arrays, a download's staging) were carved out of the
// block a destroyed C had left, and the next C's allocation then waited
// 16-30 ms on the host while the driver assembled a fresh range from the
// pieces; kept apart, a bulk block is reused whole.
constexpr size_t kBulkBytes = (size_t)1 << 30;
static cudaMemPool_t g_bulk[64] = {};

static void pool_attributes(cudaMemPool_t pool) {
  // keep freed memory in this process's pool instead of returning it to the
  // driver at every synchronisation
  uint64_t thr = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  // memory freed on one stream is never handed to an allocation on another
  // stream by making that stream wait: work on different streams (batched
  // products' workers, a download beside the next product) stays
  // independent, at the price of a larger pool
  int no = 0;
  cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
}

static void configure_pool_once(int dev) {
  static std::mutex mu;
  static bool done[64] = {};
  std::lock_guard<std::mutex> g(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) pool_attributes(pool);
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t bulk = nullptr;
  if (cudaMemPoolCreate(&bulk, &props) == cudaSuccess) {
    pool_attributes(bulk);
    g_bulk[dev] = bulk;
  } else {
    cudaGetLastError();  // every allocation then uses the default pool
  }
  done[dev] = true;
}

// Bytes in use by live allocations in both pools of a device.
static bsm_status pools_in_use(int dev, uint64_t *used) {
  configure_pool_once(dev);
  cudaMemPool_t pool;
  uint64_t a = 0, b = 0;
  BSM_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  BSM_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &a));
  if (dev >= 0 && dev < 64 && g_bulk[dev])
    BSM_CUDA(cudaMemPoolGetAttribute(g_bulk[dev], cudaMemPoolAttrUsedMemCurrent, &b));
  *used = a + b;
  return BSM_OK;
}

// Cap on the pool's in-use bytes (bsm_set_memory_limit); 0 = none.
static std::atomic<uint64_t> g_mem_limit{0};

bsm_status dev_alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  int dev = 0;
  cudaGetDevice(&dev);
  configure_pool_once(dev);
  if (const uint64_t cap = g_mem_limit.load(std::memory_order_relaxed)) {
    uint64_t used = 0;
    if (pools_in_use(dev, &used) != BSM_OK) {
      cudaGetLastError();
      return BSM_ERR_CUDA;
    }
    if (used + bytes > cap) return BSM_ERR_OOM;
  }
  cudaMemPool_t bulk = bytes >= kBulkBytes && dev >= 0 && dev < 64 ? g_bulk[dev] : nullptr;
  cudaError_t e = bulk ? cudaMallocFromPoolAsync(p, bytes, bulk, s) : cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BSM_ERR_OOM : BSM_ERR_CUDA;
  }
  return BSM_OK;
}

void dev_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

void *HostScratch::get(size_t bytes) {
  if (bytes <= n) return p;
  if (p) cudaFreeHost(p);
  p = nullptr;
  n = 0;
  size_t want = bytes < 4096 ? 4096 : bytes;
  if (cudaMallocHost(&p, want) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return nullptr;
  }
  n = want;
  return p;
}
HostScratch::~HostScratch() {
  // process teardown may have destroyed the context already; ignore errors
  if (p) cudaFreeHost(p);
}
HostScratch &host_scratch() {
  static thread_local HostScratch h;
  return h;
}

// One block copies `n` 32-bit words from device memory to the device-mapped
// address of page-locked host memory.
__global__ void k_readback(uint32_t *__restrict__ dst, const uint32_t *__restrict__ src,
                           int64_t n) {
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

bsm_status readback(void *host, const void *dev, size_t bytes, cudaStream_t s) {
  void *hd = nullptr;
  if (bytes % 4 == 0 && (uintptr_t)host % 4 == 0 && (uintptr_t)dev % 4 == 0 &&
      cudaHostGetDevicePointer(&hd, host, 0) == cudaSuccess && hd) {
    if (bytes == 0) return BSM_OK;
    count_launch();
    k_readback<<<1, 256, 0, s>>>(static_cast<uint32_t *>(hd), static_cast<const uint32_t *>(dev),
                                 (int64_t)(bytes / 4));
    return cuda_status(cudaGetLastError());
  }
  cudaGetLastError();
  return cuda_status(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
}

LastStats &last_stats() {
  static thread_local LastStats st;
  return st;
}

int64_t &launch_counter() {
  static thread_local int64_t n = 0;
  return n;
}

static thread_local int t_timing = -1;  // -1: follow the environment
bool timing_enabled() {
  if (t_timing < 0) {
    const char *e = getenv("BSM_TIMING");
    t_timing = (e && e[0] == '1') ? 1 : 0;
  }
  return t_timing == 1;
}

extern "C" bsm_status bsm_set_timing(int on) {
  if (on != 0 && on != 1) return BSM_ERR_INVALID_ARG;
  t_timing = on;
  return BSM_OK;
}

extern "C" bsm_status bsm_release_memory(void) {
  int dev = 0;
  BSM_CUDA(cudaGetDevice(&dev));
  BSM_CUDA(cudaDeviceSynchronize());
  configure_pool_once(dev);
  cudaMemPool_t pool;
  BSM_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  BSM_CUDA(cudaMemPoolTrimTo(pool, 0));
  if (dev >= 0 && dev < 64 && g_bulk[dev]) BSM_CUDA(cudaMemPoolTrimTo(g_bulk[dev], 0));
  return BSM_OK;
}

extern "C" bsm_status bsm_set_memory_limit(uint64_t bytes) {
  g_mem_limit.store(bytes, std::memory_order_relaxed);
  return BSM_OK;
}

extern "C" bsm_status bsm_memory_in_use(uint64_t *bytes) {
  if (!bytes) return BSM_ERR_INVALID_ARG;
  int dev = 0;
  BSM_CUDA(cudaGetDevice(&dev));
  BSM_CUDA(cudaDeviceSynchronize());
  if (dev < 0 || dev >= 64) return BSM_ERR_UNSUPPORTED;
  uint64_t used = 0;
  BSM_TRY(pools_in_use(dev, &used));
  *bytes = used;
  return BSM_OK;
}

namespace {
struct PendingTiming {
  std::vector<cudaEvent_t> ev;
  std::vector<std::array<int, 3>> spans;  // (phase, first event, last event)
  int rest[3] = {-1, -1, -1};             // (phase, first event, last event)
  void clear() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    spans.clear();
    rest[0] = -1;
  }
};
thread_local PendingTiming t_pending;

// Waits for the last recorded event and turns the spans into phase times.
void timing_resolve(LastStats &ls) {
  PendingTiming &p = t_pending;
  if (p.ev.empty()) return;
  if (cudaEventSynchronize(p.ev.back()) == cudaSuccess) {
    double ms[3] = {0, 0, 0};
    auto el = [&](int a, int b) {
      float t = 0;
      if (a >= 0 && b >= 0) cudaEventElapsedTime(&t, p.ev[a], p.ev[b]);
      return (double)t;
    };
    for (auto &sp : p.spans) ms[sp[0]] += el(sp[1], sp[2]);
    if (p.rest[0] >= 0) {
      double other = 0;
      for (int i = 0; i < 3; i++)
        if (i != p.rest[0]) other += ms[i];
      ms[p.rest[0]] = el(p.rest[1], p.rest[2]) - other;
    }
    for (int i = 0; i < 3; i++) ls.phase_ms[i] = ms[i];
  }
  p.clear();
}
}  // namespace

void timing_begin() { t_pending.clear(); }

int timing_mark(cudaStream_t s) {
  if (!timing_enabled()) return -1;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return -1;
  cudaEventRecord(e, s);
  t_pending.ev.push_back(e);
  return (int)t_pending.ev.size() - 1;
}

void timing_span(int phase, int e0, int e1) {
  if (e0 >= 0 && e1 >= 0) t_pending.spans.push_back({phase, e0, e1});
}

void timing_rest(int phase, int e0, int e1) {
  if (e0 < 0 || e1 < 0) return;
  t_pending.rest[0] = phase;
  t_pending.rest[1] = e0;
  t_pending.rest[2] = e1;
}

extern "C" bsm_status bsm_last_phase_ms(double *ms, int cap, int *nphase, int64_t *launches) {
  LastStats &ls = last_stats();
  timing_resolve(ls);
  if (nphase) *nphase = 3;
  if (launches) *launches = ls.launches;
  if (ms) {
    if (cap < 3) return BSM_ERR_BUFFER_TOO_SMALL;
    for (int i = 0; i < 3; i++) ms[i] = ls.phase_ms[i];
  }
  return BSM_OK;
}



template <typename F>
static bsm_status run_cub(F f, cudaStream_t s) {
  size_t tmp = 0;
  BSM_CUDA(f(nullptr, tmp));
  void *t = nullptr;
  BSM_TRY(dev_alloc(&t, tmp, s));
  cudaError_t e = f(t, tmp);
  dev_free(t, s);
  return cuda_status(e);
}

bsm_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return BSM_OK;
  count_launch(2);  // scan init + scan
  return run_cub([&](void *t, size_t &b) {
    return cub::DeviceScan::ExclusiveSum(t, b, in, out, n, s);
  }, s);
}

bsm_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return BSM_OK;
  count_launch(2);
  return run_cub([&](void *t, size_t &b) {
    return cub::DeviceScan::ExclusiveSum(t, b, in, out, n, s);
  }, s);
}

bsm_status scan_exclusive_u64(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return BSM_OK;
  count_launch(2);
  return run_cub([&](void *t, size_t &b) {
    return cub::DeviceScan::ExclusiveSum(t, b, in, out, n, s);
  }, s);
}

struct SatAddU64 {
  __host__ __device__ uint64_t operator()(uint64_t a, uint64_t b) const {
    const uint64_t c = a + b;
    return c < a ? ~0ull : c;
  }
};

bsm_status scan_inclusive_u64_sat(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return BSM_OK;
  count_launch(2);
  return run_cub([&](void *t, size_t &b) {
    return cub::DeviceScan::InclusiveScan(t, b, in, out, SatAddU64(), n, s);
  }, s);
}

bsm_status sort_keys_u64(const uint64_t *kin, uint64_t *kout, const int32_t *vin, int32_t *vout,
                         int64_t n, int end_bit, cudaStream_t s) {
  if (n <= 0) return BSM_OK;
  if (end_bit < 1) end_bit = 1;
  count_launch(2 + (end_bit + 7) / 8);  // histogram, offsets, one pass per 8-bit digit
  return run_cub([&](void *t, size_t &b) {
    return cub::DeviceRadixSort::SortPairs(t, b, kin, kout, vin, vout, n, 0, end_bit, s);
  }, s);
}

bsm_status sort_pairs_u32_u64(const uint32_t *kin, uint32_t *kout, const uint64_t *vin,
                              uint64_t *vout, int64_t n, cudaStream_t s) {
  if (n <= 0) return BSM_OK;
  count_launch(2 + 4);
  return run_cub([&](void *t, size_t &b) {
    return cub::DeviceRadixSort::SortPairs(t, b, kin, kout, vin, vout, n, 0, 32, s);
  }, s);
}

extern "C" const char *bsm_status_string(bsm_status s) {
  switch (s) {
    case BSM_OK: return "ok";
    case BSM_ERR_INVALID_ARG: return "invalid argument";
    case BSM_ERR_DIM_MISMATCH: return "dimension mismatch (A.ncols != B.nrows)";
    case BSM_ERR_BLOCKSIZE: return "unsupported or mismatched block size";
    case BSM_ERR_OUT_OF_RANGE: return "block coordinate out of range";
    case BSM_ERR_DUPLICATE: return "duplicate block coordinate";
    case BSM_ERR_OOM: return "out of device memory";
    case BSM_ERR_CUDA: return "CUDA runtime error";
    case BSM_ERR_TIMEOUT: return "bounded device wait timed out";
    case BSM_ERR_BUFFER_TOO_SMALL: return "output buffer too small";
    case BSM_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}
