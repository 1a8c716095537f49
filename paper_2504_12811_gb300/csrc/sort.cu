// K3 + K4: stable LSD radix sort of the (key, Gaussian index) pairs and the
// per-tile ranges (paper Sec. 3.1 'Blending Sort Order': tile-major, depth
// minor).
//
// Onesweep structure: one histogram kernel reads every key once and counts
// all digit positions; then one kernel per 8-bit digit ranks a 1024- to 4096-key
// tile per block (warp-level multisplit with __match_any_sync, preserving
// input order), publishes its per-digit counts, resolves the exclusive prefix
// of earlier tiles by decoupled look-back, and scatters through shared memory.
// Tiles are taken in launch order from an atomic counter, so every tile a
// block waits on belongs to a block that is already running.
//
// Look-back words are 64-bit: (epoch << 32) | (flag << 30) | count.  The epoch
// (a device counter bumped by every sort, times 8 plus the pass, 32 bits) marks
// a word as written by the current pass, so the look-back buffer needs no
// clearing between sorts; only when the counter starts a new cycle of 2^29
// sorts does the histogram kernel clear every word, so that a word written
// 2^29 sorts earlier cannot pass for one of this sort.  Every wait is bounded
// in time; on expiry the block sets a timeout flag, proceeds with what it has
// and the frame is reported invalid.
#include <algorithm>
#include <utility>

#include "aaag_internal.cuh"

namespace aaag {
namespace {

constexpr int kRadix = 256;
constexpr unsigned long long kFlagAggregate = 1ull << 30;
constexpr unsigned long long kFlagPrefix = 2ull << 30;
constexpr unsigned long long kCountMask = (1ull << 30) - 1ull;
constexpr long long kWaitCycles = 2000000000ll;   // ~1 s at 2 GHz
constexpr int kLookWindow = 4;                    // look-back words loaded per round trip

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__global__ void sort_init_kernel(uint32_t* hist, uint32_t* counters, unsigned long long* epoch) {
  pdl_begin();
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x < 4) counters[threadIdx.x] = 0;
  if (threadIdx.x == 0) *epoch += 1ull;
}

__global__ void __launch_bounds__(256)
sort_histogram_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                      int64_t n_max, int passes, uint32_t* __restrict__ hist,
                      unsigned long long* __restrict__ lookback, int64_t lb_words,
                      const unsigned long long* __restrict__ epoch) {
  pdl_begin();
  __shared__ uint32_t sh[4][kRadix];
  // a new cycle of look-back tags: clear every word (the passes come later)
  if ((*epoch & ((1ull << 29) - 1ull)) == 0ull)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lb_words;
         i += (int64_t)gridDim.x * blockDim.x)
      lookback[i] = 0ull;
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = min((int64_t)*n_dev, n_max);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(k >> (8 * p)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&hist[i], v);
  }
}

// exclusive scan of 256 values held one per thread (blockDim == 256)
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t* tmp8) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp8[warp] = x;
  __syncthreads();
  uint32_t pre = 0;
  for (int w = 0; w < warp; ++w) pre += tmp8[w];
  __syncthreads();
  return pre + x - v;
}

template <int TILE>
struct SortSmem {
  uint32_t keys[TILE];
  uint32_t vals[TILE];
  uint32_t warp[kSortThreads / 32][kRadix];   // per-warp digit counts -> prefixes
  uint32_t digit_start[kRadix];               // block-local digit starts
  uint32_t global[kRadix];                    // global start of this block's digits
  uint32_t tmp[8];
  int tile;
};

// Decoupled look-back of one digit (thread tid = digit) for tile `tile` > 0:
// kLookWindow predecessor words per round trip, loaded together and consumed
// nearest first until an inclusive prefix, or a word not yet published (then
// the window is reloaded from there).  Returns the exclusive prefix.  The
// wait is bounded: after kWaitCycles without progress the timeout flag is
// raised and the prefix found so far returned.
__device__ __forceinline__ uint32_t digit_lookback(const volatile unsigned long long* lb, int64_t tile, int tid,
                                                   unsigned long long tag, unsigned long long* timeout_flag) {
  uint32_t prefix = 0;
  int64_t t = tile - 1;   // nearest predecessor not yet consumed
  const long long t0 = clock64();
  for (;;) {
    unsigned long long w[kLookWindow];
#pragma unroll
    for (int j = 0; j < kLookWindow; ++j)
      w[j] = t - j >= 0 ? lb[(t - j) * kRadix + tid] : (tag | kFlagPrefix);   // tile 0 ends it first
    int used = 0;
    bool stop = false, stall = false;
#pragma unroll
    for (int j = 0; j < kLookWindow; ++j) {
      if (!stop && !stall) {
        const unsigned long long x = w[j];
        if ((x & 0xffffffff00000000ull) != tag || (x & (3ull << 30)) == 0) {
          stall = true;
        } else {
          prefix += (uint32_t)(x & kCountMask);
          ++used;
          stop = (x & kFlagPrefix) != 0;
        }
      }
    }
    if (stop) return prefix;
    t -= used;
    if (used == 0) {
      if (clock64() - t0 > kWaitCycles) {
        atomicExch(timeout_flag, 1ull);
        return prefix;
      }
      __nanosleep(20);
    }
  }
}

// Tiles of ITEMS keys per thread, taken in order from the pass counter.
template <int ITEMS, int TILE>
__device__ __forceinline__ void sort_pass_tiles(SortSmem<TILE>& sm, const uint32_t* __restrict__ keys_in,
                                                const uint32_t* __restrict__ vals_in,
                                                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                int64_t n, int shift, uint32_t gofs, uint32_t* __restrict__ counter,
                                                unsigned long long* __restrict__ lookback, unsigned long long tag,
                                                unsigned long long* __restrict__ timeout_flag) {
  constexpr int kTileKeys = ITEMS * kSortThreads;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n_tiles = (n + kTileKeys - 1) / kTileKeys;
  uint32_t* s_keys = sm.keys;
  uint32_t* s_vals = sm.vals;
  uint32_t (*s_warp)[kRadix] = sm.warp;
  uint32_t* s_digit_start = sm.digit_start;
  uint32_t* s_global = sm.global;
  uint32_t* s_tmp = sm.tmp;
  int& s_tile = sm.tile;

  for (;;) {
    if (tid == 0) s_tile = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= n_tiles) break;

    // ---- load the keys (warp-striped: coalesced) and rank within each warp;
    // the values are read only at the scatter, so that they hold no
    // registers while the keys are ranked
    uint32_t k[ITEMS], r[ITEMS];
    const uint32_t n32 = (uint32_t)n;
    const uint32_t base = (uint32_t)tile * kTileKeys + (uint32_t)warp * (32 * ITEMS) + (uint32_t)lane;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t idx = base + j * 32;
      const bool ok = idx < n32;
      k[j] = ok ? keys_in[idx] : 0xffffffffu;
    }
    for (int i = lane; i < kRadix; i += 32) s_warp[warp][i] = 0;
    __syncwarp();
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t d = (k[j] >> shift) & 0xffu;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      // the lowest lane of each digit group claims the group's ranks
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (lane == leader) before = atomicAdd(&s_warp[warp][d], (uint32_t)__popc(peers));
      before = __shfl_sync(0xffffffffu, before, leader);
      r[j] = before + __popc(peers & lt);
    }
    __syncthreads();

    // ---- per digit (thread tid = digit): warp prefixes and block count
    uint32_t count = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
      const uint32_t c = s_warp[w][tid];
      s_warp[w][tid] = count;
      count += c;
    }
    volatile unsigned long long* lb = lookback;
    if (tile == 0) {
      lb[tid] = tag | kFlagPrefix | count;
    } else {
      lb[tile * kRadix + tid] = tag | kFlagAggregate | count;
    }
    const uint32_t local_start = block_exclusive_scan_256(count, s_tmp);
    s_digit_start[tid] = local_start;
    __syncthreads();

    // ---- scatter into shared memory in digit order (needs only this tile's
    // counts, so it runs before the look-back: the predecessors get that
    // much longer to publish their prefixes), then to global memory
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t d = (k[j] >> shift) & 0xffu;
      const uint32_t pos = s_digit_start[d] + s_warp[warp][d] + r[j];
      const uint32_t idx = base + j * 32;
      s_keys[pos] = k[j];
      s_vals[pos] = idx < n32 ? vals_in[idx] : 0u;
    }

    uint32_t prefix = 0;
    if (tile > 0) {
      prefix = digit_lookback(lb, tile, tid, tag, timeout_flag);
      lb[tile * kRadix + tid] = tag | kFlagPrefix | (unsigned long long)(prefix + count);
    }
    s_global[tid] = gofs + prefix;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int q = tid + i * kSortThreads;
      const uint32_t key = s_keys[q];
      const uint32_t d = (key >> shift) & 0xffu;
      const uint32_t g = s_global[d] + ((uint32_t)q - s_digit_start[d]);
      if (g < n32) {
        keys_out[g] = key;
        vals_out[g] = s_vals[q];
      }
    }
    __syncthreads();
  }
}

// Self-test of the bounded wait: digit tid of tile 1 waits on tile 0, whose
// words carry a tag no pass uses (lb[0 .. kRadix) cleared first), so every
// thread gives up after kWaitCycles and raises the flag.
__global__ void sort_wait_selftest_kernel(unsigned long long* lb, unsigned long long* timeout_flag) {
  lb[threadIdx.x] = 0ull;
  __syncthreads();
  const unsigned long long tag = 0xfffffffeull << 32;
  digit_lookback(lb, 1, (int)threadIdx.x, tag, timeout_flag);
}

// Keys per thread by problem size: small sorts use small tiles so that every
// SM has work and the look-back chains stay short in time.
__device__ __forceinline__ int sort_items_for(int64_t n) {
  return n >= kSortWideKeys / 2 ? 8 : 4;
}

// Sorts whose size is known on the host take larger tiles: 12 keys per
// thread (3072) from kSortWideMin keys, 16 (4096) from kSortXWideMin.  Each
// size is a kernel of its own, so that each gets its own register budget
// (the 16-key one capped for three blocks per SM).
constexpr int kWideItems = 12;
constexpr int kXWideItems = 16;
constexpr int64_t kSortWideMin = 4 << 20;
constexpr int64_t kSortXWideMin = 32 << 20;

// One pass; ITEMS = 0 picks 4 or 8 keys per thread from the device count.
template <int ITEMS>
__device__ __forceinline__ void sort_pass(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                                          uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                          const uint32_t* __restrict__ n_dev, int64_t n_max, int pass,
                                          const uint32_t* __restrict__ hist, uint32_t* __restrict__ counter,
                                          unsigned long long* __restrict__ lookback,
                                          const unsigned long long* __restrict__ epoch_dev,
                                          unsigned long long* __restrict__ timeout_flag) {
  pdl_begin();
  __shared__ SortSmem<(ITEMS ? ITEMS : kSortItems) * kSortThreads> sm;
  const int64_t n = min((int64_t)*n_dev, n_max);
  const unsigned long long epoch = ((*epoch_dev) * 8ull + (unsigned long long)pass) & 0xffffffffull;
  const unsigned long long tag = epoch << 32;
  // global exclusive offset of digit `threadIdx.x` for this pass
  const uint32_t gofs = block_exclusive_scan_256(hist[pass * kRadix + threadIdx.x], sm.tmp);
  if constexpr (ITEMS != 0) {
    sort_pass_tiles<ITEMS>(sm, keys_in, vals_in, keys_out, vals_out, n, 8 * pass, gofs, counter, lookback, tag,
                           timeout_flag);
  } else {
    if (sort_items_for(n) == 8)
      sort_pass_tiles<8>(sm, keys_in, vals_in, keys_out, vals_out, n, 8 * pass, gofs, counter, lookback, tag,
                         timeout_flag);
    else
      sort_pass_tiles<4>(sm, keys_in, vals_in, keys_out, vals_out, n, 8 * pass, gofs, counter, lookback, tag,
                         timeout_flag);
  }
}

// the parameter list shared by the pass kernels below (those of sort_pass)
#define AAAG_SORT_PASS_ARGS                                                                              \
  const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out, \
      uint32_t *__restrict__ vals_out, const uint32_t *__restrict__ n_dev, int64_t n_max, int pass,          \
      const uint32_t *__restrict__ hist, uint32_t *__restrict__ counter, unsigned long long *__restrict__ lookback, \
      const unsigned long long *__restrict__ epoch_dev, unsigned long long *__restrict__ timeout_flag

template <bool WIDE>
__global__ void __launch_bounds__(kSortThreads) sort_pass_kernel(AAAG_SORT_PASS_ARGS) {
  sort_pass<WIDE ? kWideItems : 0>(keys_in, vals_in, keys_out, vals_out, n_dev, n_max, pass, hist, counter, lookback,
                                   epoch_dev, timeout_flag);
}

__global__ void __launch_bounds__(kSortThreads, 3) sort_pass_kernel_x16(AAAG_SORT_PASS_ARGS) {
  sort_pass<kXWideItems>(keys_in, vals_in, keys_out, vals_out, n_dev, n_max, pass, hist, counter, lookback, epoch_dev,
                         timeout_flag);
}
#undef AAAG_SORT_PASS_ARGS

__global__ void ranges_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_dev,
                              int64_t n_max, int depth_bits, uint2* __restrict__ ranges) {
  pdl_begin();
  const int64_t n = min((int64_t)*n_dev, n_max);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = keys[i] >> depth_bits;
    if (i == 0 || (keys[i - 1] >> depth_bits) != t) ranges[t].x = (uint32_t)i;
    if (i == n - 1 || (keys[i + 1] >> depth_bits) != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

}  // namespace

void configure_sort(LaunchConfig& c) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_pass_kernel<false>, kSortThreads, 0);
  c.sort_pass_per_sm = std::max(1, per_sm);
  per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_pass_kernel<true>, kSortThreads, 0);
  c.sort_wide_per_sm = std::max(1, per_sm);
  per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_pass_kernel_x16, kSortThreads, 0);
  c.sort_xwide_per_sm = std::max(1, per_sm);
}

size_t radix_sort_scratch(int64_t n_max) {
  const int64_t tiles = sort_max_tiles(n_max);
  // hist [4][256] u32, counters [4] u32 (padded), lookback [tiles][256] u64, epoch u64, n u32
  return 4 * kRadix * 4 + 256 + (size_t)(tiles > 0 ? tiles : 1) * kRadix * 8 + 256;
}

aaag_status radix_sort_device_n(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                                uint32_t* vals_alt, const uint32_t* n_dev, int64_t n_max,
                                int key_bits, uint32_t* hist, uint32_t* counters,
                                unsigned long long* lookback, int64_t lookback_words,
                                unsigned long long* epoch, unsigned long long* timeout_flag,
                                int* result_in_alt, cudaStream_t st, bool prepared, bool n_exact) {
  const int passes = (key_bits + 7) / 8;
  *result_in_alt = passes & 1;
  if (n_max <= 0 || passes == 0) {
    *result_in_alt = 0;
    return AAAG_OK;
  }
  const LaunchConfig& lc = launch_config();
  if (!prepared) launch_chained(sort_init_kernel, 1, 256, 0, st, hist, counters, epoch);
  const int64_t hblocks = std::min<int64_t>((n_max + 4095) / 4096, (int64_t)lc.sms * 4);
  launch_chained(sort_histogram_kernel, (unsigned)hblocks, 256, 0, st, keys, n_dev, n_max, passes, hist, lookback,
                                                           lookback_words, epoch);
  aaag_status e = check_launch("sort_histogram");
  if (e != AAAG_OK) return e;
  // wider tiles when the count is known to be large (n_max is the count
  // itself, not a capacity)
  const int items = !n_exact ? 0 : n_max >= kSortXWideMin ? kXWideItems : n_max >= kSortWideMin ? kWideItems : 0;
  const int64_t tiles = items ? (n_max + items * kSortThreads - 1) / (items * kSortThreads) : sort_max_tiles(n_max);
  const int per_sm = items == kXWideItems ? lc.sort_xwide_per_sm
                     : items == kWideItems ? lc.sort_wide_per_sm
                                           : lc.sort_pass_per_sm;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)lc.sms * per_sm);
  auto pass_kernel = items == kXWideItems ? sort_pass_kernel_x16
                     : items == kWideItems ? sort_pass_kernel<true>
                                           : sort_pass_kernel<false>;
  uint32_t* kin = keys;
  uint32_t* vin = vals;
  uint32_t* kout = keys_alt;
  uint32_t* vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    launch_chained(pass_kernel, (unsigned)grid, kSortThreads, 0, st, kin, vin, kout, vout, n_dev, n_max, p, hist,
                                                               counters + p, lookback, epoch, timeout_flag);
    e = check_launch("sort_pass");
    if (e != AAAG_OK) return e;
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  return AAAG_OK;
}

aaag_status launch_sort_wait_selftest(unsigned long long* lookback, unsigned long long* timeout_flag,
                                      cudaStream_t st) {
  sort_wait_selftest_kernel<<<1, kRadix, 0, st>>>(lookback, timeout_flag);
  return check_launch("sort wait self-test");
}

aaag_status launch_sort_pairs(aaag_workspace* ws, cudaStream_t st) {
  // device-side pair count, clipped to the capacity by the pair scan of K2
  const uint32_t* n_dev = reinterpret_cast<const uint32_t*>(ws->stats + kStatPairsClipped);
  int alt = 0;
  // zeroed digit histograms and pass counters and a fresh epoch come from K2
  const int key_bits = ws->fc.tile_bits + ws->fc.depth_bits;
  aaag_status e = radix_sort_device_n(ws->keys[0], ws->vals[0], ws->keys[1], ws->vals[1], n_dev, ws->capacity, key_bits,
                          ws->sort_hist, ws->sort_counters, ws->sort_lookback,
                          (ws->n_sort_tiles + 1) * kRadix, ws->stats + kStatSortEpoch, ws->stats + kStatTimeout, &alt, st, true);
  if (e != AAAG_OK) return e;
  ws->sorted_in_alt = alt;
  // (the tile ranges were zeroed by K2's chunk_offsets_kernel)
  const int64_t rblocks = std::min<int64_t>((ws->capacity + 255) / 256, (int64_t)launch_config().sms * 8);
  launch_chained(ranges_kernel, (unsigned)std::max<int64_t>(rblocks, 1), 256, 0, st,
                 ws->keys[alt], n_dev, ws->capacity, ws->fc.depth_bits, ws->ranges);
  return check_launch("ranges");
}

}  // namespace aaag
