// K5: per-pixel 3D evaluation, per-pixel re-sort and compositing (paper
// Sec. 3.1 'Evaluation in 3D', 'Blending Sort Order'; Sec. 4 implementation
// details: per-ray sorting retained from hierarchical rasterisation).
//
// One 256-thread block per 16x16 tile, one thread per pixel.  The tile's pairs
// arrive sorted by (tile, front depth).  They are staged in shared memory in
// batches of 256 as plane coefficients relative to the tile origin (see
// render_core.cuh), so one pixel x Gaussian evaluation is 12 FMA for the two
// affine 3-vectors, two dot products, one reciprocal and one exp2.
//
// Per-pixel ordering: contributors (alpha >= 1/255, t* >= znear) enter a
// queue sorted by (t*, arrival).  Pairs arrive with non-decreasing key L, a
// lower bound of the t* of every later contributor, so a queued entry with
// t* < L can never be overtaken and is blended at once.  When the queue is
// full, the farthest contributors are deferred to another pass over the tile
// (depth peeling), so the order is exact; only the bounded-buffer ablation
// releases entries early (counted as potential misorders).  Blending stops
// before the contributor that would take transmittance below 1e-4.
#include <algorithm>
#include <cstring>

#include <cuda_runtime.h>

#include "aaag_internal.cuh"
#include "render_core.cuh"

namespace aaag {
namespace {

struct ForwardBlend {
  using Queue = IndexQueue;
  const StageSmem* st;
  const Record* rec;
  float T, Cr, Cg, Cb;
  bool done;
  uint32_t nblend;
  // blend Gaussian gid with opacity a (its colour is read from its record)
  __device__ __forceinline__ void blend(float a, uint32_t gid) {
    const float Tn = T * (1.0f - a);
    if (Tn < kTStop) {
      done = true;
      return;
    }
    const float4 c = __ldg(reinterpret_cast<const float4*>(rec + gid) + 3);
    const float w = a * T;
    Cr = fmaf(c.x, w, Cr);
    Cg = fmaf(c.y, w, Cg);
    Cb = fmaf(c.z, w, Cb);
    T = Tn;
    ++nblend;
  }
  __device__ __forceinline__ uint32_t payload(int k) const { return st->gid[k]; }
  __device__ __forceinline__ void blend_new(float a, const EvalState& ev) { blend(a, st->gid[ev.k]); }
  __device__ __forceinline__ void begin_batch(uint32_t, int) {}
};

// Render one tile of one frame (all threads of the block).  EXACT: the frame
// has neither ordering ablation.
template <bool EXACT = false>
__device__ __forceinline__ void render_tile(TileSmem<IndexQueue>& s, int tile, const uint2* __restrict__ ranges,
                                           const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                           const Record* __restrict__ rec, const uint4* __restrict__ aux,
                                           const FrameConst& fc,
                                           float* __restrict__ rgb, float* __restrict__ alpha,
                                           float* __restrict__ final_T, uint32_t* __restrict__ n_blended,
                                           unsigned long long* __restrict__ stats) {
  const int tx = tile % fc.tiles_x, ty = tile / fc.tiles_x;
  int lx, ly;
  tile_pixel(threadIdx.x, lx, ly);
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool in_image = px < fc.W && py < fc.H;

  ForwardBlend bl;
  bl.st = &s.st;
  bl.rec = rec;
  bl.T = 1.0f;
  bl.Cr = bl.Cg = bl.Cb = 0.0f;
  bl.done = !in_image;
  bl.nblend = 0;
  uint32_t neval = 0;   // evaluations of this pixel (far below 2^32 per tile)
  uint32_t nmis = 0, npass = 0;
  traverse_tile<false, EXACT>(s, ranges[tile], keys, vals, rec, aux, fc, tx, ty, (float)lx + 0.5f, (float)ly + 0.5f,
                              bl, neval, nmis, npass);

  if (in_image) {
    const size_t HW = (size_t)fc.W * fc.H;
    const size_t p = (size_t)py * fc.W + px;
    rgb[p] = fmaf(bl.T, fc.bg[0], bl.Cr);
    rgb[HW + p] = fmaf(bl.T, fc.bg[1], bl.Cg);
    rgb[2 * HW + p] = fmaf(bl.T, fc.bg[2], bl.Cb);
    alpha[p] = 1.0f - bl.T;
    final_T[p] = bl.T;
    n_blended[p] = bl.nblend;
  }
  unsigned long long e = neval, b = bl.nblend, m = nmis, x = npass;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    m += __shfl_xor_sync(0xffffffffu, m, o);
    x += __shfl_xor_sync(0xffffffffu, x, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicAdd(&stats[kStatEvaluations], e);
    if (b) atomicAdd(&stats[kStatBlended], b);
    if (m) atomicAdd(&stats[kStatMisorders], m);
    if (x) atomicAdd(&stats[kStatExtraPasses], x);
  }
}

// Tile order of the persistent render: tiles in descending order of their
// pair counts (two buckets per octave), so that the longest tiles start first
// and the short ones fill in behind them.  One block; the lanes of a warp that
// fall into one bucket add to its counter with one atomic (a few buckets hold
// most tiles, and per-lane atomics on them serialise).  Also resets the work
// counter.
__global__ void __launch_bounds__(1024)
tile_order_kernel(const uint2* __restrict__ ranges, const FrameConst* __restrict__ fcp,
                  uint32_t* __restrict__ order, uint32_t* __restrict__ counter) {
  pdl_begin();
  constexpr int kBuckets = 64;
  __shared__ uint32_t base[kBuckets];
  const int n_tiles = fcp->tiles_x * fcp->tiles_y;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  auto bucket = [&](int t) {
    if (t >= n_tiles) return kBuckets;                             // past the end
    const uint2 r = ranges[t];
    const uint32_t c = r.y - r.x + 1u;
    const int lz = 32 - __clz(c);                                   // 1..32
    const int half = lz >= 2 ? (int)((c >> (lz - 2)) & 1u) : 0;
    return kBuckets - 1 - min(kBuckets - 1, 2 * lz + half);        // longest first
  };
  if (threadIdx.x < kBuckets) base[threadIdx.x] = 0;
  if (threadIdx.x == 0) *counter = 0;
  __syncthreads();
  const int rounds = (n_tiles + (int)blockDim.x - 1) / (int)blockDim.x;   // the same for every lane
  for (int r = 0; r < rounds; ++r) {
    const int b = bucket(r * (int)blockDim.x + (int)threadIdx.x);
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (b < kBuckets && lane == __ffs(peers) - 1) atomicAdd(&base[b], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < 32) {   // exclusive scan of the 64 counts, two per lane
    const uint32_t c0 = base[2 * threadIdx.x], c1 = base[2 * threadIdx.x + 1];
    uint32_t incl = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)threadIdx.x >= o) incl += v;
    }
    const uint32_t excl = incl - c0 - c1;
    base[2 * threadIdx.x] = excl;
    base[2 * threadIdx.x + 1] = excl + c0;
  }
  __syncthreads();
  for (int r = 0; r < rounds; ++r) {
    const int t = r * (int)blockDim.x + (int)threadIdx.x;
    const int b = bucket(t);
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    uint32_t first = 0;
    if (b < kBuckets && lane == leader) first = atomicAdd(&base[b], (uint32_t)__popc(peers));
    first = __shfl_sync(0xffffffffu, first, leader);
    if (b < kBuckets) order[first + (uint32_t)__popc(peers & lt)] = (uint32_t)t;
  }
}

// Persistent: blocks take tiles in the order above from a work counter.
// EXACT: compiled for frames without an ordering ablation.
template <bool EXACT>
__global__ void __launch_bounds__(kTilePixels, 3)
render_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
              const uint32_t* __restrict__ vals, const Record* __restrict__ rec, const uint4* __restrict__ aux,
              const FrameConst* __restrict__ fcp, float* __restrict__ rgb, float* __restrict__ alpha,
              float* __restrict__ final_T, uint32_t* __restrict__ n_blended, unsigned long long* __restrict__ stats,
              const uint32_t* __restrict__ order, uint32_t* __restrict__ counter) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<IndexQueue>& s = *reinterpret_cast<TileSmem<IndexQueue>*>(smem_raw);
  __shared__ uint32_t s_item;
  const FrameConst fc = *fcp;
  const uint32_t n_tiles = (uint32_t)(fc.tiles_x * fc.tiles_y);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= n_tiles) break;
    render_tile<EXACT>(s, (int)order[item], ranges, keys, vals, rec, aux, fc, rgb, alpha, final_T, n_blended, stats);
  }
}

// ---- K8: one persistent launch over the tiles of several frames.
// Blocks take (frame, tile) work items in order from one atomic counter; the
// frames' descriptors travel by value in the kernel parameters.  Nothing
// waits on anything: every item is known at launch.
struct RenderJob {
  const uint2* ranges;
  const uint32_t* keys;
  const uint32_t* vals;
  const Record* rec;
  const uint4* aux;
  const FrameConst* fc;
  float* rgb;
  float* alpha;
  float* final_T;
  uint32_t* n_blended;
  unsigned long long* stats;
  uint32_t first;   // first work item of this frame
  uint32_t tiles;
};
constexpr int kMaxBatch = 64;
struct RenderBatch {
  RenderJob job[kMaxBatch];
  int n;
  uint32_t total;
};

__global__ void __launch_bounds__(kTilePixels, 3)
serve_render_kernel(const __grid_constant__ RenderBatch b, uint32_t* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<IndexQueue>& s = *reinterpret_cast<TileSmem<IndexQueue>*>(smem_raw);
  __shared__ uint32_t s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= b.total) break;
    int j = 0;
    while (j + 1 < b.n && b.job[j + 1].first <= item) ++j;
    const RenderJob& J = b.job[j];
    const FrameConst fc = *J.fc;
    render_tile(s, (int)(item - J.first), J.ranges, J.keys, J.vals, J.rec, J.aux, fc, J.rgb, J.alpha, J.final_T,
                J.n_blended, J.stats);
  }
}

}  // namespace

void configure_render(LaunchConfig& c) {
  cudaFuncSetAttribute(render_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kForwardSmemBytes);
  cudaFuncSetAttribute(render_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kForwardSmemBytes);
  cudaFuncSetAttribute(serve_render_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kForwardSmemBytes);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_render_kernel, kTilePixels, kForwardSmemBytes);
  c.serve_per_sm = std::max(1, per_sm);
}

aaag_status launch_render_batch(aaag_workspace* const* ws, float* const* rgb, float* const* alpha, int n,
                                cudaStream_t st) {
  const LaunchConfig& lc = launch_config();
  RenderBatch b;
  std::memset(&b, 0, sizeof(b));
  uint32_t total = 0;
  for (int i = 0; i < n; ++i) {
    const aaag_workspace* w = ws[i];
    RenderJob& J = b.job[i];
    const int alt = w->sorted_in_alt;
    J.ranges = w->ranges;
    J.keys = w->keys[alt];
    J.vals = w->vals[alt];
    J.rec = w->records;
    J.aux = w->aux;
    J.fc = w->fc_dev;
    J.rgb = rgb[i];
    J.alpha = alpha[i];
    J.final_T = w->final_T;
    J.n_blended = w->n_blended;
    J.stats = w->stats;
    J.first = total;
    J.tiles = (uint32_t)w->n_tiles;
    total += J.tiles;
  }
  b.n = n;
  b.total = total;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws[0]->stats + kStatBatchCounter);
  if (cudaMemsetAsync(counter, 0, 4, st) != cudaSuccess) return check_launch("render_batch memset");
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)lc.sms * lc.serve_per_sm, total));
  serve_render_kernel<<<grid, kTilePixels, kForwardSmemBytes, st>>>(b, counter);
  return check_launch("serve_render");
}

aaag_status launch_tile_order(aaag_workspace* ws, uint32_t* counter, cudaStream_t st) {
  launch_chained(tile_order_kernel, 1, 1024, 0, st, ws->ranges, ws->fc_dev, ws->tile_order, counter);
  return check_launch("tile_order");
}

aaag_status launch_render(aaag_workspace* ws, float* rgb, float* alpha, cudaStream_t st) {
  const LaunchConfig& lc = launch_config();
  const int alt = ws->sorted_in_alt;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws->stats + kStatRenderCounter);
  aaag_status e = launch_tile_order(ws, counter, st);
  if (e != AAAG_OK) return e;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)lc.sms * lc.serve_per_sm, ws->n_tiles));
  auto kernel = (ws->fc.flags & (AAAG_FLAG_NO_RESORT | AAAG_FLAG_KBUFFER)) ? render_kernel<false> : render_kernel<true>;
  launch_chained(kernel, grid, kTilePixels, kForwardSmemBytes, st, ws->ranges, ws->keys[alt], ws->vals[alt], ws->records, ws->aux,
                                                        ws->fc_dev, rgb, alpha, ws->final_T, ws->n_blended, ws->stats,
                                                        ws->tile_order, counter);
  return check_launch("render");
}

}  // namespace aaag
