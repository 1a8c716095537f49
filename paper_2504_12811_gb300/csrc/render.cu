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
// register queue sorted by (t*, arrival).  Pairs arrive with non-decreasing
// key L, a lower bound of the t* of every later contributor, so a queued
// entry with t* < L can never be overtaken and is blended at once.  Only when
// the queue is full is an entry released early (counted as a potential
// misorder).  Blending stops before the contributor that would take
// transmittance below 1e-4.
#include <cuda_runtime.h>

#include "aaag_internal.cuh"
#include "render_core.cuh"

namespace aaag {
namespace {

struct ForwardBlend {
  const Record* rec;
  float T, Cr, Cg, Cb;
  bool done;
  uint32_t nblend;
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
};

__global__ void __launch_bounds__(kTilePixels, 3)
render_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
              const uint32_t* __restrict__ vals, const Record* __restrict__ rec, FrameConst fc,
              float* __restrict__ rgb, float* __restrict__ alpha, float* __restrict__ final_T,
              uint32_t* __restrict__ n_blended, unsigned long long* __restrict__ stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem& s = *reinterpret_cast<TileSmem*>(smem_raw);
  const int tile = blockIdx.x;
  const int tx = tile % fc.tiles_x, ty = tile / fc.tiles_x;
  const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool in_image = px < fc.W && py < fc.H;

  ForwardBlend bl;
  bl.rec = rec;
  bl.T = 1.0f;
  bl.Cr = bl.Cg = bl.Cb = 0.0f;
  bl.done = !in_image;
  bl.nblend = 0;
  unsigned long long neval = 0;
  uint32_t nmis = 0;
  traverse_tile(s, ranges[tile], keys, vals, rec, fc, tx, ty, (float)lx + 0.5f, (float)ly + 0.5f,
                        bl, neval, nmis);

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
  unsigned long long e = neval, b = bl.nblend, m = nmis;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    m += __shfl_xor_sync(0xffffffffu, m, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicAdd(&stats[kStatEvaluations], e);
    if (b) atomicAdd(&stats[kStatBlended], b);
    if (m) atomicAdd(&stats[kStatMisorders], m);
  }
}

}  // namespace

aaag_status launch_render(aaag_workspace* ws, float* rgb, float* alpha, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(render_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemBytes);
    configured = true;
  }
  const int alt = ws->sorted_in_alt;
  render_kernel<<<(unsigned)ws->n_tiles, kTilePixels, kTileSmemBytes, st>>>(ws->ranges, ws->keys[alt], ws->vals[alt],
                                                               ws->records, ws->fc, rgb, alpha, ws->final_T,
                                                               ws->n_blended, ws->stats);
  return check_launch("render");
}

}  // namespace aaag
