// K2: 3D frustum tile culling and pair emission (paper Sec. 3.4, Eq. 18; the
// near-plane tile rule of Sec. 3.3).
//
// Work is balanced in chunks of 32 candidate tiles: the rectangle of a visible
// Gaussian (from K1) is cut into ceil(tiles / 32) chunks, so a Gaussian that
// covers the whole screen becomes hundreds of independent warps instead of one
// long serial loop.
//   1. exclusive scan of the per-Gaussian chunk counts (written by K1)
//   2. expand: each Gaussian writes its index into its chunks' owner slots
//   3. test: one warp per chunk, one lane per tile; the warp ballot of kept
//      tiles is stored (32-bit mask per chunk)
//   4. exclusive scan of the mask popcounts -> pair offset of each chunk
//   5. emit: one warp per chunk writes its pairs contiguously
// Pairs therefore land at deterministic positions: Gaussian order, then
// rectangle row-major tile order.  Chunk and pair counts stay on the device;
// the kernels loop over them with grid-stride warps.
#include <algorithm>

#include "aaag_internal.cuh"
#include "geometry.cuh"

namespace aaag {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t device_count(const uint32_t* n_dev, int64_t n_max) {
  return n_dev ? min((int64_t)*n_dev, n_max) : n_max;
}

template <bool POPC>
__device__ __forceinline__ uint32_t scan_input(const uint32_t* in, int64_t i) {
  const uint32_t v = in[i];
  return POPC ? (uint32_t)__popc(v) : v;
}

// ---- exclusive scan over a device-sized array: block sums, scan of the
// block sums (one block), downsweep.  Blocks loop over 4096-element pieces.

template <bool POPC>
__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const uint32_t* __restrict__ in, const uint32_t* __restrict__ n_dev, int64_t n_max,
                   unsigned long long* __restrict__ partials) {
  const int64_t n = device_count(n_dev, n_max);
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  __shared__ unsigned long long ws[kScanThreads / 32];
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t base = b * kScanChunk;
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const int64_t i = base + j * kScanThreads + threadIdx.x;
      if (i < n) s += scan_input<POPC>(in, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
      partials[b] = t;
    }
    __syncthreads();
  }
}

// single block: exclusive scan of the block partials; the total goes to
// stats[total_slot]; the total clipped to `cap` goes to *clipped (uint32), and
// exceeding `cap` raises the overflow flag.
__global__ void __launch_bounds__(1024)
scan_partials_kernel(unsigned long long* __restrict__ partials, const uint32_t* __restrict__ n_dev,
                     int64_t n_max, int64_t cap, unsigned long long* __restrict__ stats, int total_slot,
                     uint32_t* __restrict__ clipped) {
  const int64_t n = device_count(n_dev, n_max);
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    const int64_t b = b0 + threadIdx.x;
    const unsigned long long v = b < nb ? partials[b] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const unsigned long long incl = x + (warp > 0 ? wsum[warp - 1] : 0ull) + carry;
    if (b < nb) partials[b] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[total_slot] = carry;
    if (carry > (unsigned long long)cap) stats[kStatOverflow] = 1ull;
    *clipped = (uint32_t)(carry < (unsigned long long)cap ? carry : (unsigned long long)cap);
  }
}

template <bool POPC>
__global__ void __launch_bounds__(kScanThreads)
scan_down_kernel(const uint32_t* __restrict__ in, const uint32_t* __restrict__ n_dev, int64_t n_max,
                 const unsigned long long* __restrict__ partials, uint32_t* __restrict__ out) {
  const int64_t n = device_count(n_dev, n_max);
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  __shared__ unsigned long long wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    // each thread owns kScanItems consecutive elements
    const int64_t base = b * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      c[j] = base + j < n ? scan_input<POPC>(in, base + j) : 0u;
      s += c[j];
    }
    unsigned long long x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    unsigned long long pre = partials[b] + x - s;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      if (base + j < n) out[base + j] = pre > 0xffffffffull ? 0xffffffffu : (uint32_t)pre;
      pre += c[j];
    }
    __syncthreads();
  }
}

// ---- chunk ownership

__global__ void __launch_bounds__(kThreads)
expand_chunks_kernel(const uint32_t* __restrict__ chunk_counts, const uint32_t* __restrict__ chunk_offsets,
                     int64_t n, int64_t chunk_cap, uint32_t* __restrict__ owner) {
  for (int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x; g < n; g += (int64_t)gridDim.x * kThreads) {
    const uint32_t c = chunk_counts[g];
    const uint64_t off = chunk_offsets[g];
    for (uint32_t j = 0; j < c && off + j < (uint64_t)chunk_cap; ++j) owner[off + j] = (uint32_t)g;
  }
}

struct ChunkGeom {
  int64_t g;
  uint4 a;
  int tx0, ty0, nx, total, local;   // local: chunk index inside the Gaussian
};

__device__ __forceinline__ ChunkGeom chunk_geom(int64_t c, const uint32_t* owner, const uint32_t* chunk_offsets,
                                                const uint4* aux) {
  ChunkGeom q;
  q.g = owner[c];
  q.a = aux[q.g];
  int tx1, ty1;
  unpack_rect(q.a, q.tx0, q.ty0, tx1, ty1);
  q.nx = tx1 - q.tx0 + 1;
  q.total = q.nx * (ty1 - q.ty0 + 1);
  q.local = (int)(c - (int64_t)chunk_offsets[q.g]);
  return q;
}

__global__ void __launch_bounds__(kThreads)
cull_test_kernel(const Record* __restrict__ rec, const uint4* __restrict__ aux, const FrameConst* __restrict__ fcp,
                 const uint32_t* __restrict__ owner, const uint32_t* __restrict__ chunk_offsets,
                 const uint32_t* __restrict__ n_chunks_dev, int64_t chunk_cap, uint32_t* __restrict__ masks,
                 unsigned long long* __restrict__ stats) {
  const FrameConst fc = *fcp;
  const int64_t nch = min((int64_t)*n_chunks_dev, chunk_cap);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const bool cull = !(fc.flags & AAAG_FLAG_NO_CULL);
  unsigned long long tested = 0;
  for (int64_t c = warp0; c < nch; c += nwarps) {
    const ChunkGeom q = chunk_geom(c, owner, chunk_offsets, aux);
    const int j = q.local * 32 + lane;
    bool keep = false;
    if (j < q.total) {
      const int tx = q.tx0 + j % q.nx, ty = q.ty0 + j / q.nx;
      if (!cull) {
        keep = true;
      } else {
        const float4* r = reinterpret_cast<const float4*>(rec + q.g);
        const float4 t1 = __ldg(r + 0), t2 = __ldg(r + 1), t3 = __ldg(r + 2);
        const float tau_signed = __uint_as_float(q.a.z);
        const float tau = inflate_tau(fabsf(tau_signed));
        const float xlo = (float)(tx * kTile), ylo = (float)(ty * kTile);
        const float xhi = xlo + kTile, yhi = ylo + kTile;
        if (tau_signed < 0.0f) {
          // the front of the ellipsoid reaches z_near: frustum truncated there
          keep = frustum_hit<true>(t1, t2, t3, fc.fx, fc.fy, fc.cx, fc.cy, fc.znear, xlo, xhi, ylo, yhi, tau);
        } else {
          ConicTester ct;
          ct.init(t1, t2, t3, fc.fx, fc.fy, fc.cx, fc.cy, tau);
          keep = ct.hit(xlo, ylo, xhi, yhi);
        }
      }
      ++tested;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) masks[c] = ball;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tested += __shfl_xor_sync(0xffffffffu, tested, o);
  if (lane == 0 && tested) atomicAdd(&stats[kStatTilesTested], tested);
}

__global__ void __launch_bounds__(kThreads)
cull_emit_kernel(const uint4* __restrict__ aux, const FrameConst* __restrict__ fcp, const uint32_t* __restrict__ owner,
                 const uint32_t* __restrict__ chunk_offsets, const uint32_t* __restrict__ n_chunks_dev,
                 int64_t chunk_cap, const uint32_t* __restrict__ masks, const uint32_t* __restrict__ pair_offsets,
                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int64_t capacity) {
  const FrameConst fc = *fcp;
  const int64_t nch = min((int64_t)*n_chunks_dev, chunk_cap);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t c = warp0; c < nch; c += nwarps) {
    const uint32_t m = masks[c];
    if (!(m >> lane & 1u)) continue;
    const ChunkGeom q = chunk_geom(c, owner, chunk_offsets, aux);
    const int j = q.local * 32 + lane;
    const int tx = q.tx0 + j % q.nx, ty = q.ty0 + j / q.nx;
    const uint64_t p = (uint64_t)pair_offsets[c] + __popc(m & lt);
    if (p < (uint64_t)capacity) {
      const uint32_t tile = (uint32_t)(ty * fc.tiles_x + tx);
      keys[p] = (tile << fc.depth_bits) | q.a.w;
      vals[p] = (uint32_t)q.g;
    }
  }
}

int g_sms = 0;
int sm_count() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms < 1) g_sms = 1;
  }
  return g_sms;
}

template <bool POPC>
aaag_status scan(const uint32_t* in, const uint32_t* n_dev, int64_t n_max, int64_t cap, uint32_t* out,
                 unsigned long long* partials, unsigned long long* stats, int total_slot, uint32_t* clipped,
                 cudaStream_t st) {
  const int64_t nb = std::max<int64_t>((n_max + kScanChunk - 1) / kScanChunk, 1);
  const unsigned grid = (unsigned)std::min<int64_t>(nb, (int64_t)sm_count() * 8);
  scan_reduce_kernel<POPC><<<grid, kScanThreads, 0, st>>>(in, n_dev, n_max, partials);
  scan_partials_kernel<<<1, 1024, 0, st>>>(partials, n_dev, n_max, cap, stats, total_slot, clipped);
  scan_down_kernel<POPC><<<grid, kScanThreads, 0, st>>>(in, n_dev, n_max, partials, out);
  return check_launch("scan");
}

}  // namespace

aaag_status launch_cull(aaag_workspace* ws, cudaStream_t st) {
  const int64_t n = ws->n;
  uint32_t* n_chunks = reinterpret_cast<uint32_t*>(ws->stats + kStatChunksClipped);
  uint32_t* n_pairs = reinterpret_cast<uint32_t*>(ws->stats + kStatPairsClipped);
  // 1. chunk offsets per Gaussian
  aaag_status e = scan<false>(ws->counts, nullptr, n, ws->chunk_capacity, ws->offsets, ws->scan_partials,
                              ws->stats, kStatChunks, n_chunks, st);
  if (e != AAAG_OK) return e;
  // 2. owners
  const unsigned gblocks = (unsigned)std::max<int64_t>(std::min<int64_t>((n + kThreads - 1) / kThreads,
                                                                        (int64_t)sm_count() * 16), 1);
  expand_chunks_kernel<<<gblocks, kThreads, 0, st>>>(ws->counts, ws->offsets, n, ws->chunk_capacity,
                                                     ws->chunk_owner);
  e = check_launch("expand_chunks");
  if (e != AAAG_OK) return e;
  // 3. test
  const unsigned cblocks = (unsigned)std::max<int64_t>(
      std::min<int64_t>((ws->chunk_capacity + kWarps - 1) / kWarps, (int64_t)sm_count() * 16), 1);
  cull_test_kernel<<<cblocks, kThreads, 0, st>>>(ws->records, ws->aux, ws->fc_dev, ws->chunk_owner, ws->offsets,
                                                 n_chunks, ws->chunk_capacity, ws->chunk_mask, ws->stats);
  e = check_launch("cull_test");
  if (e != AAAG_OK) return e;
  // 4. pair offsets per chunk
  e = scan<true>(ws->chunk_mask, n_chunks, ws->chunk_capacity, ws->capacity, ws->chunk_pair_offsets,
                 ws->scan_partials, ws->stats, kStatPairs, n_pairs, st);
  if (e != AAAG_OK) return e;
  // 5. emit
  cull_emit_kernel<<<cblocks, kThreads, 0, st>>>(ws->aux, ws->fc_dev, ws->chunk_owner, ws->offsets, n_chunks,
                                                 ws->chunk_capacity, ws->chunk_mask, ws->chunk_pair_offsets,
                                                 ws->keys[0], ws->vals[0], ws->capacity);
  return check_launch("cull_emit");
}

}  // namespace aaag
