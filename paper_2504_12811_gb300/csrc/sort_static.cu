// aaag_radix_sort_static: the radix sort of sort.cu for callers that cannot
// allocate device memory.  All scratch lives in one file-scope device array of
// fixed size, so the call needs nothing from the caller but the arrays to sort.
//
// Capacity: kStaticSortMax keys.  Every GPU that loads this library holds the
// array (about 9 MB) until the process exits.
#include <cstring>
#include <mutex>

#include "aaag_internal.cuh"

namespace aaag {
namespace {

constexpr int64_t kStaticSortMax = 1 << 20;
constexpr int64_t kStaticTiles = sort_max_tiles(kStaticSortMax);

// Layout (bytes):
//   [0, 4096)              histograms, 4 passes x 256 x uint32
//   [4096, 4112)           per-pass tile counters
//   [4160, 4168)           look-back epoch (uint64); [4168, 4176) timeout flag
//   [4176, 4180)           key count (uint32)
//   [4352, +kStaticTiles*2048)  look-back words
//   then keys_alt, vals_alt (kStaticSortMax uint32 each)
constexpr size_t kOffHist = 0;
constexpr size_t kOffCounters = 4096;
constexpr size_t kOffEpoch = 4160;
constexpr size_t kOffTimeout = 4168;
constexpr size_t kOffCount = 4176;
constexpr size_t kOffLookback = 4352;
constexpr size_t kOffKeysAlt = kOffLookback + (size_t)kStaticTiles * 256 * 8;
constexpr size_t kOffValsAlt = kOffKeysAlt + (size_t)kStaticSortMax * 4;
constexpr size_t kStaticBytes = kOffValsAlt + (size_t)kStaticSortMax * 4;

// Zero at module load: the epoch starts at 0 and no look-back word can match a
// later epoch.  Host code must not use this name as an address.
static __device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

__global__ void store_count_kernel(uint32_t* p, uint32_t v) { *p = v; }

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (resolved once per
// device, with that device current).
aaag_status scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("aaag_radix_sort_static: no usable current device");
    return AAAG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p) {
      set_error("aaag_radix_sort_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return AAAG_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return AAAG_OK;
}

}  // namespace

// The bounded look-back wait of the radix sort, run out on purpose against the
// fixed array's own words and timeout flag (failure detection test).
aaag_status static_sort_wait_selftest(cudaStream_t st) {
  unsigned char* base = nullptr;
  const aaag_status e = scratch_address(&base);
  if (e != AAAG_OK) return e;
  unsigned long long* timeout = reinterpret_cast<unsigned long long*>(base + kOffTimeout);
  if (cudaMemsetAsync(timeout, 0, 8, st) != cudaSuccess) return check_launch("static sort self-test memset");
  return launch_sort_wait_selftest(reinterpret_cast<unsigned long long*>(base + kOffLookback), timeout, st);
}

}  // namespace aaag

using namespace aaag;

extern "C" aaag_status aaag_radix_sort_static_status(void) {
  unsigned char* base = nullptr;
  const aaag_status e = scratch_address(&base);
  if (e != AAAG_OK) return e;
  unsigned long long flag = 0;
  if (cudaMemcpy(&flag, base + kOffTimeout, sizeof(flag), cudaMemcpyDeviceToHost) != cudaSuccess)
    return check_launch("aaag_radix_sort_static_status");
  if (flag) {
    set_error("aaag_radix_sort_static: a bounded look-back wait gave up; the output is unspecified");
    return AAAG_ERR_TIMEOUT;
  }
  return AAAG_OK;
}

extern "C" int64_t aaag_radix_sort_static_capacity(void) { return kStaticSortMax; }

extern "C" aaag_status aaag_radix_sort_static(uint32_t* keys, uint32_t* vals, int64_t n, int32_t key_bits,
                                              cudaStream_t stream) {
  if (n < 0 || key_bits < 1 || key_bits > 32) {
    set_error("aaag_radix_sort_static: invalid n or key_bits");
    return AAAG_ERR_INVALID_ARG;
  }
  if (n > kStaticSortMax) {
    set_error("aaag_radix_sort_static: %lld keys exceed the fixed capacity of %lld", (long long)n,
              (long long)kStaticSortMax);
    return AAAG_ERR_CAPACITY;
  }
  if (n > 0 && (!keys || !vals)) {
    set_error("aaag_radix_sort_static: null pointer");
    return AAAG_ERR_INVALID_ARG;
  }
  if (n == 0) return AAAG_OK;
  unsigned char* base = nullptr;
  aaag_status e = scratch_address(&base);
  if (e != AAAG_OK) return e;
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
  uint32_t* counters = reinterpret_cast<uint32_t*>(base + kOffCounters);
  unsigned long long* epoch = reinterpret_cast<unsigned long long*>(base + kOffEpoch);
  unsigned long long* timeout = reinterpret_cast<unsigned long long*>(base + kOffTimeout);
  uint32_t* n_dev = reinterpret_cast<uint32_t*>(base + kOffCount);
  unsigned long long* lookback = reinterpret_cast<unsigned long long*>(base + kOffLookback);
  uint32_t* keys_alt = reinterpret_cast<uint32_t*>(base + kOffKeysAlt);
  uint32_t* vals_alt = reinterpret_cast<uint32_t*>(base + kOffValsAlt);
  // the timeout flag and the histograms start from zero on every call (the
  // histograms are cleared inside the sort)
  if (cudaMemsetAsync(timeout, 0, 8, stream) != cudaSuccess) return check_launch("radix_sort_static memset");
  store_count_kernel<<<1, 1, 0, stream>>>(n_dev, (uint32_t)n);
  e = check_launch("radix_sort_static count");
  if (e != AAAG_OK) return e;
  int alt = 0;
  e = radix_sort_device_n(keys, vals, keys_alt, vals_alt, n_dev, n, key_bits, hist, counters, lookback,
                          kStaticTiles * 256, epoch, timeout, &alt, stream);
  if (e != AAAG_OK) return e;
  if (alt) {   // an odd number of passes left the result in the scratch buffers
    if (cudaMemcpyAsync(keys, keys_alt, (size_t)n * 4, cudaMemcpyDeviceToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(vals, vals_alt, (size_t)n * 4, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
      return check_launch("radix_sort_static copy back");
  }
  return AAAG_OK;
}
