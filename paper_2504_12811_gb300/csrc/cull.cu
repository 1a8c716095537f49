// K2: 3D frustum tile culling and pair emission (paper Sec. 3.4, Eq. 18; the
// near-plane tile rule of Sec. 3.3).
//
// Work is balanced in chunks of 32 candidate tiles: the rectangle of a visible
// Gaussian (from K1) is cut into ceil(tiles / 32) chunks, so a Gaussian that
// covers the whole screen becomes hundreds of independent warps instead of one
// long serial loop.  Three kernels; A and C are single passes with decoupled
// look-back over tiles taken in order from an atomic counter:
//   A. chunk_offsets_kernel: tiles of 2048 Gaussians; exclusive scan of the
//      per-Gaussian chunk counts (written by K1) -> each Gaussian's first
//      chunk, and each Gaussian writes its index into its chunks' owner slots
//      (it also prepares K3's counters and empties K4's tile ranges).
//   B. cull_test_kernel: windows of 16 chunks per warp (grid-stride), one
//      lane per tile, several small chunks packed into one round of 32 lanes;
//      the mask of the needed tiles is stored per chunk.
//   C. cull_emit_kernel: tiles of 256 chunks; the tile's pair count is
//      resolved into its global pair offset by look-back, and each lane
//      writes its own chunk's pairs.
// Pairs therefore land at deterministic positions: Gaussian order, then
// rectangle row-major tile order.  Chunk and pair counts stay on the device.
//
// Look-back words are 64-bit: (frame epoch, 24 bits) << 40 | flag << 38 |
// value (38 bits); the epoch is bumped once per frame by the kernel that
// writes the frame constants, so the words never need clearing.  Every wait is
// bounded in time; on expiry the timeout flag is raised and the frame is
// reported invalid.
#include <algorithm>

#include "aaag_internal.cuh"
#include "geometry.cuh"

namespace aaag {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kOffItems = 8;                        // Gaussians per thread in kernel A
constexpr int kOffTile = kThreads * kOffItems;      // 2048
constexpr int kChunkTile = kWarps * 32;             // 256 chunks per tile of kernel C
constexpr int kTestWindow = 16;                     // chunks per warp window of kernel B

constexpr unsigned long long kLbAggregate = 1ull << 38;
constexpr unsigned long long kLbInclusive = 2ull << 38;
constexpr unsigned long long kLbValue = (1ull << 38) - 1ull;
constexpr long long kWaitCycles = 2000000000ll;     // ~1 s at 2 GHz

__device__ __forceinline__ unsigned long long lb_tag(unsigned long long epoch) {
  return (epoch & 0xffffffull) << 40;
}

// Warp-parallel decoupled look-back for tile `tile` (> 0), run by one full
// warp: lanes read the words of 32 predecessors at once and consume them
// nearest first, up to the first inclusive prefix; a word not yet published
// stops the window there and is polled again.  Returns the exclusive prefix.
__device__ __forceinline__ unsigned long long warp_lookback(const volatile unsigned long long* lb, int64_t tile,
                                                            unsigned long long tag,
                                                            unsigned long long* timeout_flag) {
  const int lane = threadIdx.x & 31;
  unsigned long long prefix = 0;
  int64_t next = tile - 1;   // nearest predecessor not yet consumed
  const long long t0 = clock64();
  for (;;) {
    const int64_t idx = next - lane;
    const unsigned long long w = idx >= 0 ? lb[idx] : (tag | kLbInclusive);
    const bool ready = (w & ~((1ull << 40) - 1ull)) == tag && (w & (3ull << 38)) != 0;
    const bool incl = ready && (w & kLbInclusive);
    const unsigned ready_m = __ballot_sync(0xffffffffu, ready);
    const unsigned incl_m = __ballot_sync(0xffffffffu, incl);
    const int first_wait = ready_m == 0xffffffffu ? 32 : __ffs(~ready_m) - 1;
    const int first_incl = incl_m ? __ffs(incl_m) - 1 : 32;
    const bool done = first_incl < first_wait;
    const int take = done ? first_incl + 1 : first_wait;
    unsigned long long v = lane < take ? (w & kLbValue) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    prefix += v;
    if (done) return prefix;
    next -= take;
    if (take == 0) {
      if (clock64() - t0 > kWaitCycles) {
        if (lane == 0) atomicExch(timeout_flag, 1ull);
        return prefix;
      }
      __nanosleep(32);
    }
  }
}

// Self-test of the bounded wait: tile 1 waits on tile 0, whose word carries a
// tag no frame uses (cleared first), so the warp gives up after kWaitCycles and
// raises the flag.
__global__ void cull_wait_selftest_kernel(unsigned long long* lb, unsigned long long* timeout_flag) {
  if (threadIdx.x == 0) lb[0] = 0ull;
  __syncwarp();
  warp_lookback(lb, 1, lb_tag(0xfffffeull), timeout_flag);
}

// exclusive scan of one value per thread over the block; returns the block
// total in *total (all threads)
__device__ __forceinline__ unsigned long long block_scan(unsigned long long v, unsigned long long* wsum,
                                                         unsigned long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  unsigned long long pre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const unsigned long long s = wsum[w];
    pre += w < warp ? s : 0ull;
    tot += s;
  }
  __syncthreads();
  *total = tot;
  return pre + x - v;
}

// ---- A: chunk offsets and owners
__global__ void __launch_bounds__(kThreads)
chunk_offsets_kernel(const uint32_t* __restrict__ counts, int64_t n, int64_t chunk_cap,
                     uint32_t* __restrict__ offsets, uint32_t* __restrict__ owner,
                     unsigned long long* __restrict__ lookback, unsigned long long* __restrict__ stats,
                     uint32_t* __restrict__ n_chunks_clipped, uint32_t* __restrict__ sort_hist,
                     uint32_t* __restrict__ sort_counters, uint2* __restrict__ ranges, int n_ranges) {
  pdl_begin();
  // empty tile ranges for K4, which writes only the tiles that hold pairs
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_ranges; i += gridDim.x * blockDim.x)
    ranges[i] = make_uint2(0u, 0u);
  __shared__ unsigned long long s_wsum[kWarps];
  __shared__ unsigned long long s_prefix;
  __shared__ int64_t s_tile;
  if (blockIdx.x == 0) {
    // prepare K3 for this frame's pairs: zeroed digit histograms and pass
    // counters, and a fresh epoch for its look-back words
    for (int i = threadIdx.x; i < 4 * 256; i += kThreads) sort_hist[i] = 0u;
    if (threadIdx.x < 4) sort_counters[threadIdx.x] = 0u;
    if (threadIdx.x == 0) stats[kStatSortEpoch] += 1ull;
  }
  const unsigned long long tag = lb_tag(stats[kStatFrameEpoch]);
  uint32_t* counter = reinterpret_cast<uint32_t*>(stats + kStatCullTileA);
  const int64_t n_tiles = (n + kOffTile - 1) / kOffTile;
  volatile unsigned long long* lb = lookback;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= n_tiles) break;
    const int64_t base = tile * kOffTile + (int64_t)threadIdx.x * kOffItems;
    uint32_t c[kOffItems];
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < kOffItems; ++j) {
      c[j] = base + j < n ? counts[base + j] : 0u;
      s += c[j];
    }
    unsigned long long total;
    const unsigned long long pre = block_scan(s, s_wsum, &total);
    if (threadIdx.x < 32) {
      unsigned long long p = 0;
      if (tile == 0) {
        if (threadIdx.x == 0) lb[0] = tag | kLbInclusive | (total & kLbValue);
      } else {
        if (threadIdx.x == 0) lb[tile] = tag | kLbAggregate | (total & kLbValue);
        p = warp_lookback(lb, tile, tag, stats + kStatTimeout);
        if (threadIdx.x == 0) lb[tile] = tag | kLbInclusive | ((p + total) & kLbValue);
      }
      if (threadIdx.x == 0) {
        s_prefix = p;
        if (tile == n_tiles - 1) {
          const unsigned long long all = p + total;
          stats[kStatChunks] = all;
          if (all > (unsigned long long)chunk_cap) stats[kStatOverflow] = 1ull;
          *n_chunks_clipped = (uint32_t)(all < (unsigned long long)chunk_cap ? all : (unsigned long long)chunk_cap);
        }
      }
    }
    __syncthreads();
    unsigned long long off = s_prefix + pre;
#pragma unroll
    for (int j = 0; j < kOffItems; ++j) {
      const int64_t g = base + j;
      if (g < n) {
        offsets[g] = off > 0xffffffffull ? 0xffffffffu : (uint32_t)off;
        for (uint32_t k = 0; k < c[j] && off + k < (unsigned long long)chunk_cap; ++k) owner[off + k] = (uint32_t)g;
      }
      off += c[j];
    }
    __syncthreads();
  }
}

// ---- B: tile tests, pair offsets and emission

// Is tile (tx, ty) needed by the Gaussian with rows t1..t3 and signed tau
// (min rho^2 over the tile frustum below tau, Eq. 18; with the near-plane
// rule of Sec. 3.3 when tau is negative)?
__device__ __forceinline__ bool tile_needed(float4 t1, float4 t2, float4 t3, float tau_signed,
                                            const FrameConst& fc, int tx, int ty) {
  const float tau = inflate_tau(fabsf(tau_signed));
  const float xlo = (float)(tx * kTile), ylo = (float)(ty * kTile);
  const float xhi = xlo + kTile, yhi = ylo + kTile;
  if (tau_signed < 0.0f) {
    // the front of the ellipsoid reaches z_near
    NearTester nt;
    nt.init(t1, t2, t3, fc.fx, fc.fy, fc.cx, fc.cy, fc.znear, tau);
    return nt.hit(xlo, ylo, xhi, yhi);
  }
  ConicTester ct;
  ct.init(t1, t2, t3, fc.fx, fc.fy, fc.cx, fc.cy, tau);
  return ct.hit(xlo, ylo, xhi, yhi);
}

// Depth key of a (Gaussian, tile) pair: the ray maximum of a pixel lies at
// t* = G.d / |d|^2 (render_core.cuh), with d affine in the pixel centre and
// G the Gaussian's constant vector.  Over the rectangle of the tile's pixel
// centres (tile-relative x, y in [0.5, 15.5]) the smallest t* is found at a
// corner: when every corner has G.d > 0, let m be the smallest corner value
// of t*; then h = G.d - m |d|^2 is concave (affine minus a convex quadratic
// with m > 0) and non-negative at the corners, so non-negative on the whole
// rectangle, i.e. t* >= m at every pixel of the tile, and m is attained.  The
// bound is lowered by the float32 rounding of either side (the render's t*
// and this one): 1e-5 of sum |G_i d_i| / |d|^2, which is at least 1e-5 t* and
// grows where G.d cancels, plus 1e-6; quantised like the Gaussian's own key
// and rounded down; 0 (the smallest key) when no bound results.  The pair key
// is the larger of this and the Gaussian's key: both are lower bounds, and a
// tighter one lets more contributors blend at once instead of waiting in the
// per-pixel queue.
struct KeyGeom {
  float3 A1, A2, T3;   // rows of T_view without their last column
  float3 G;            // fx fy adj(A) mu_v: t* = G.d / |d|^2
};

__device__ __forceinline__ KeyGeom key_geom(float4 t1, float4 t2, float4 t3, const FrameConst& fc) {
  KeyGeom k;
  k.A1 = f3(t1.x, t1.y, t1.z);
  k.A2 = f3(t2.x, t2.y, t2.z);
  k.T3 = f3(t3.x, t3.y, t3.z);
  k.G = (fc.fx * fc.fy) * (t1.w * cross3(k.A2, k.T3) + t2.w * cross3(k.T3, k.A1) + t3.w * cross3(k.A1, k.A2));
  return k;
}

__device__ __forceinline__ uint32_t tile_depth_key(const KeyGeom& kg, const FrameConst& fc, int tx, int ty) {
  const float cxm = fc.cx - (float)(tx * kTile), cym = fc.cy - (float)(ty * kTile);
  const float3 T3 = kg.T3, G = kg.G;
  const float3 Uv = fc.fx * kg.A1 + cxm * T3;
  const float3 Wv = fc.fy * kg.A2 + cym * T3;
  const float3 D0 = cross3(Uv, Wv), Dx = cross3(Wv, T3), Dy = cross3(T3, Uv);
  float z = 3.0e38f;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float x = (k & 1) ? 15.5f : 0.5f, y = (k & 2) ? 15.5f : 0.5f;
    const float3 d = D0 + x * Dx + y * Dy;
    const float gd = dot3(G, d), dd = dot3(d, d);
    const float mag = fabsf(G.x * d.x) + fabsf(G.y * d.y) + fabsf(G.z * d.z);
    ok = ok && gd > 0.0f && dd > 0.0f;
    z = fminf(z, (gd - 1e-5f * mag) / dd - 1e-6f);
  }
  if (!ok || !(z > fc.znear)) return 0u;
  const uint32_t dmax = (fc.depth_bits >= 32) ? 0xffffffffu : ((1u << fc.depth_bits) - 1u);
  return min((__float_as_uint(z) - fc.znear_bits) >> fc.depth_shift, dmax);
}

// Windows of kTestWindow chunks per warp (grid-stride), one lane per tile: the
// mask of each chunk's needed tiles is stored.
__global__ void __launch_bounds__(kThreads, 3)
cull_test_kernel(const Record* __restrict__ rec, const uint4* __restrict__ aux, const FrameConst* __restrict__ fcp,
                 const uint32_t* __restrict__ owner, const uint32_t* __restrict__ chunk_offsets,
                 const uint32_t* __restrict__ n_chunks_dev, int64_t chunk_cap, uint32_t* __restrict__ masks,
                 unsigned long long* __restrict__ stats) {
  pdl_begin();
  const FrameConst fc = *fcp;
  const int64_t nch = min((int64_t)*n_chunks_dev, chunk_cap);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const bool cull = !(fc.flags & AAAG_FLAG_NO_CULL);
  unsigned long long tested = 0;
  // A warp takes a window of kTestWindow consecutive chunks (lane i < kTestWindow
  // holds chunk w0 + i) and tests their tiles in rounds: each round packs as
  // many of the next chunks as fit in 32 lanes, one lane per tile, so the
  // chunks of small Gaussians (a few tiles each) share a round instead of
  // leaving most lanes idle.
  for (int64_t w0 = warp0 * kTestWindow; w0 < nch; w0 += nwarps * kTestWindow) {
    const int64_t c = w0 + lane;
    const bool valid = lane < kTestWindow && c < nch;
    uint32_t g = 0u, cnt = 0u;
    uint4 a = make_uint4(0u, 0u, 0u, 0u);
    int local = 0;
    if (valid) {
      g = owner[c];
      a = aux[g];
      local = (int)(c - (int64_t)chunk_offsets[g]);
      int tx0, ty0, tx1, ty1;
      unpack_rect(a, tx0, ty0, tx1, ty1);
      const int total = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
      cnt = (uint32_t)min(32, total - 32 * local);
    }
    uint32_t mine = 0u;   // the mask of this lane's chunk
    int next = 0;         // first chunk of the window not yet tested (warp-uniform)
    while (__any_sync(0xffffffffu, valid && lane >= next)) {
      // inclusive scan of the tile counts of the untested chunks
      const uint32_t v = (valid && lane >= next) ? cnt : 0u;
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t excl = incl - v;
      const bool in_round = v > 0u && incl <= 32u;   // always true for the chunk `next`
      const unsigned starts = __reduce_or_sync(0xffffffffu, in_round ? 1u << excl : 0u);
      const int n_round = __popc(__ballot_sync(0xffffffffu, in_round));
      const uint32_t used = __reduce_max_sync(0xffffffffu, in_round ? incl : 0u);
      // this lane's tile: chunk `slot` of the window, tile t of that chunk
      const int slot = next + __popc(starts & ((2u << lane) - 1u)) - 1;
      const uint32_t gs = __shfl_sync(0xffffffffu, g, slot);
      const uint32_t ax = __shfl_sync(0xffffffffu, a.x, slot), ay = __shfl_sync(0xffffffffu, a.y, slot);
      const uint32_t az = __shfl_sync(0xffffffffu, a.z, slot);
      const int ls = __shfl_sync(0xffffffffu, local, slot);
      const uint32_t es = __shfl_sync(0xffffffffu, excl, slot);
      bool keep = false;
      if ((uint32_t)lane < used) {
        int tx0, ty0, tx1, ty1;
        unpack_rect(make_uint4(ax, ay, 0u, 0u), tx0, ty0, tx1, ty1);
        const int nx = tx1 - tx0 + 1;
        const int j = ls * 32 + (lane - (int)es);
        if (cull) {
          const float4* r = reinterpret_cast<const float4*>(rec + gs);
          keep = tile_needed(__ldg(r + 0), __ldg(r + 1), __ldg(r + 2), __uint_as_float(az), fc, tx0 + j % nx,
                             ty0 + j / nx);
        } else {
          keep = true;
        }
        ++tested;
      }
      const unsigned ball = __ballot_sync(0xffffffffu, keep);
      if (in_round) mine = (ball >> excl) & (cnt == 32u ? 0xffffffffu : ((1u << cnt) - 1u));
      next += n_round;
    }
    if (valid) masks[c] = mine;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tested += __shfl_xor_sync(0xffffffffu, tested, o);
  if (lane == 0 && tested) atomicAdd(&stats[kStatTilesTested], tested);
}

// Tiles of 256 chunks (8 warps x 32): the tile's pair count is resolved into
// its global pair offset by look-back, then lane i of each warp writes the
// pairs of the warp's chunk i at their scanned positions.
__global__ void __launch_bounds__(kThreads)
cull_emit_kernel(const Record* __restrict__ rec, const uint4* __restrict__ aux, const FrameConst* __restrict__ fcp,
                 const uint32_t* __restrict__ owner, const uint32_t* __restrict__ chunk_offsets,
                 const uint32_t* __restrict__ n_chunks_dev, int64_t chunk_cap, const uint32_t* __restrict__ masks,
                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int64_t capacity,
                 unsigned long long* __restrict__ lookback, unsigned long long* __restrict__ stats,
                 uint32_t* __restrict__ n_pairs_clipped) {
  pdl_begin();
  __shared__ uint32_t s_wcount[kWarps];
  __shared__ unsigned long long s_prefix;
  __shared__ int64_t s_tile;
  const FrameConst fc = *fcp;
  const unsigned long long tag = lb_tag(stats[kStatFrameEpoch]);
  uint32_t* counter = reinterpret_cast<uint32_t*>(stats + kStatCullTileB);
  const int64_t nch = min((int64_t)*n_chunks_dev, chunk_cap);
  const int64_t n_tiles = (nch + kChunkTile - 1) / kChunkTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  volatile unsigned long long* lb = lookback;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= n_tiles) break;
    // lane `lane` of warp `warp` owns chunk c0 + lane
    const int64_t c0 = tile * kChunkTile + warp * 32;
    const int64_t c = c0 + lane;
    uint32_t m = 0u, g = 0u;
    uint4 a = make_uint4(0u, 0u, 0u, 0u);
    int local = 0;
    if (c < nch) {
      m = masks[c];
      if (m) {
        g = owner[c];
        a = aux[g];
        local = (int)(c - (int64_t)chunk_offsets[g]);
      }
    }
    const uint32_t cnt = (uint32_t)__popc(m);
    // inclusive scan of the chunk counts inside the warp
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wcount[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t wc = lane < kWarps ? s_wcount[lane] : 0u;
      unsigned long long total = wc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
      unsigned long long p = 0;
      if (tile == 0) {
        if (lane == 0) lb[0] = tag | kLbInclusive | (total & kLbValue);
      } else {
        if (lane == 0) lb[tile] = tag | kLbAggregate | (total & kLbValue);
        p = warp_lookback(lb, tile, tag, stats + kStatTimeout);
        if (lane == 0) lb[tile] = tag | kLbInclusive | ((p + total) & kLbValue);
      }
      if (lane == 0) {
        s_prefix = p;
        if (tile == n_tiles - 1) {
          const unsigned long long all = p + total;
          stats[kStatPairs] = all;
          if (all > (unsigned long long)capacity) stats[kStatOverflow] = 1ull;
          *n_pairs_clipped = (uint32_t)(all < (unsigned long long)capacity ? all : (unsigned long long)capacity);
        }
      }
    }
    __syncthreads();
    unsigned long long wbase = s_prefix;
    for (int w = 0; w < warp; ++w) wbase += s_wcount[w];
    // every lane writes the pairs of its own chunk, in tile order: the warp
    // takes as many rounds as the largest chunk has tiles (a warp of small
    // Gaussians' chunks finishes in a few), and each lane loads its
    // Gaussian's rows and the parts of its key bound that do not depend on
    // the tile once
    if (m != 0u) {
      int tx0, ty0, tx1, ty1;
      unpack_rect(a, tx0, ty0, tx1, ty1);
      const int nx = tx1 - tx0 + 1;
      const bool tile_keys = !(fc.flags & kMeanDepthKeyFlags);
      KeyGeom kg;
      if (tile_keys) {
        const float4* r = reinterpret_cast<const float4*>(rec + g);
        kg = key_geom(__ldg(r + 0), __ldg(r + 1), __ldg(r + 2), fc);
      }
      uint64_t at = wbase + (incl - cnt);
      for (uint32_t mm = m; mm != 0u; mm &= mm - 1u, ++at) {
        if (at >= (uint64_t)capacity) break;
        const int j = local * 32 + (__ffs(mm) - 1);
        const int txi = tx0 + j % nx, tyi = ty0 + j / nx;
        const uint32_t t = (uint32_t)(tyi * fc.tiles_x + txi);
        uint32_t dk = a.w;
        if (tile_keys) dk = max(dk, tile_depth_key(kg, fc, txi, tyi));
        keys[at] = (t << fc.depth_bits) | dk;
        vals[at] = g;
      }
    }
    __syncthreads();
  }
}

}  // namespace

void configure_cull(LaunchConfig& c) {
  int a = 1, b = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, chunk_offsets_kernel, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cull_emit_kernel, kThreads, 0);
  c.cull_a_per_sm = std::max(1, a);
  c.cull_b_per_sm = std::max(1, b);
}

aaag_status launch_cull_wait_selftest(aaag_workspace* ws, cudaStream_t st) {
  cull_wait_selftest_kernel<<<1, 32, 0, st>>>(ws->cull_lookback, ws->stats + kStatTimeout);
  return check_launch("cull wait self-test");
}

int64_t cull_lookback_words(int64_t n, int64_t chunk_cap) {
  return (n + kOffTile - 1) / kOffTile + (chunk_cap + kChunkTile - 1) / kChunkTile + 2;
}

aaag_status launch_cull(aaag_workspace* ws, cudaStream_t st) {
  const LaunchConfig& lc = launch_config();
  const int64_t n = ws->n;
  uint32_t* n_chunks = reinterpret_cast<uint32_t*>(ws->stats + kStatChunksClipped);
  uint32_t* n_pairs = reinterpret_cast<uint32_t*>(ws->stats + kStatPairsClipped);
  unsigned long long* look_a = ws->cull_lookback;
  unsigned long long* look_b = ws->cull_lookback + (ws->n_max + kOffTile - 1) / kOffTile + 1;
  const int64_t tiles_a = std::max<int64_t>((n + kOffTile - 1) / kOffTile, 1);
  const unsigned grid_a = (unsigned)std::min<int64_t>(tiles_a, (int64_t)lc.sms * lc.cull_a_per_sm);
  launch_chained(chunk_offsets_kernel, grid_a, kThreads, 0, st, ws->counts, n, ws->chunk_capacity, ws->offsets,
                                                    ws->chunk_owner, look_a, ws->stats, n_chunks, ws->sort_hist,
                                                    ws->sort_counters, ws->ranges, (int)ws->n_tiles);
  aaag_status e = check_launch("chunk_offsets");
  if (e != AAAG_OK) return e;
  const unsigned grid_t = (unsigned)std::max<int64_t>(
      std::min<int64_t>((ws->chunk_capacity + kWarps - 1) / kWarps, (int64_t)lc.sms * 16), 1);
  launch_chained(cull_test_kernel, grid_t, kThreads, 0, st, ws->records, ws->aux, ws->fc_dev, ws->chunk_owner, ws->offsets,
                                                n_chunks, ws->chunk_capacity, ws->chunk_mask, ws->stats);
  e = check_launch("cull_test");
  if (e != AAAG_OK) return e;
  const int64_t tiles_b = std::max<int64_t>((ws->chunk_capacity + kChunkTile - 1) / kChunkTile, 1);
  const unsigned grid_b = (unsigned)std::min<int64_t>(tiles_b, (int64_t)lc.sms * lc.cull_b_per_sm);
  launch_chained(cull_emit_kernel, grid_b, kThreads, 0, st, ws->records, ws->aux, ws->fc_dev, ws->chunk_owner, ws->offsets, n_chunks,
                                                ws->chunk_capacity, ws->chunk_mask, ws->keys[0], ws->vals[0],
                                                ws->capacity, look_b, ws->stats, n_pairs);
  return check_launch("cull_emit");
}

}  // namespace aaag
