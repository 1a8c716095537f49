// K6 + K7: gradients of the rendered image with respect to the scene
// parameters (means, log-scales, quaternions, opacity logits, SH).
//
// K6 (render backward) replays the forward traversal of every tile with the
// same code (render_core.cuh), so it blends the same contributors in the same
// order.  Compositing is differentiated front to back: with the forward output
// F = C_final + T_final bg known, the colour behind contributor i after it is
// blended is S_i = F - C_{<=i}, so
//   dF/dc_i     = alpha_i T_i
//   dF/dalpha_i = c_i T_i - S_i / (1 - alpha_i)
//   dA/dalpha_i = T_final / (1 - alpha_i)            (A = 1 - T_final)
// No per-blend state is cached.  For a contributor blended at once (the
// staged Gaussian of the current item), rho^2 = |num|^2/|d|^2 is
// differentiated back to the staged plane coefficients: its 22 moments
// (dL/dnum and dL/dd weighted by 1, x, y; do_hat; dcolour) are reduced across
// the warp into a per-slot shared accumulator, converted once per (tile,
// Gaussian) into gradients of the rows t1, t2, t3 of T_view.  A queued
// contributor recomputes its planes (Eq. 4-5) from the record at release and
// forms its 16 row gradients.  Releases run as warp-wide rounds, so the
// lanes releasing the same Gaussian (the common case, since neighbouring
// pixels hold similar queues) issue their vector atomics together, and a
// group of at least kMinGroup lanes first adds its gradients with one
// butterfly.  (Per-lane atomics from divergent release loops took half the
// kernel's time; per-lane shared atomics into the slot accumulators
// serialise badly.)
//
// K7 (preprocess backward) is one thread per Gaussian: it recomputes the
// forward preprocessing and applies the chain rule through T_view = Rv R S'
// and mu_v, the filtered scales s' = sqrt(s^2 + k / v'^2), the amplitude
// factor of Eq. 12 (and v' = min(v_train, f / z) when the view term is the
// active branch), the opacity sigmoid, the quaternion normalisation and the SH
// colour with its viewing direction.  Discrete decisions (discards, bounds,
// culling, clamps) are held fixed.
#include <algorithm>

#include "aaag_internal.cuh"
#include "render_core.cuh"

namespace aaag {
namespace {

// Per-slot accumulators of the fast path, in shared memory after TileSmem:
// [kTilePixels][kAccStride]:  dL/dN0, dL/dNx, dL/dNy, dL/dD0, dL/dDx, dL/dDy
// (3 each, tile-relative plane coefficients of render_core.cuh), dL/do_hat,
// dL/dcolour (3).
constexpr int kMoments = 22;
constexpr size_t kStageBytes = sizeof(TileSmem<IndexQueue>);
constexpr int kAccStride = kMoments + 1;   // odd: slot-major rows fall in distinct banks
constexpr size_t kBackwardSmemBytes = kStageBytes + sizeof(float) * kAccStride * kTilePixels;
constexpr int kMinGroup = 24;   // lanes releasing one Gaussian in a round that are summed before the atomics

// One level of the halving reduce-scatter of end_item: M values per lane
// (positions 0 .. M-1) become (M + 1) / 2, exchanged with lane ^ H.
template <int H, int M>
__device__ __forceinline__ void halving_level(float* v, int lane, int& off, int& left) {
  constexpr int kHalf = (M + 1) / 2;
  const bool upper = (lane & H) != 0;
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    const float lo = v[i], hi = i + kHalf < M ? v[i + kHalf] : 0.0f;
    const float send = upper ? lo : hi;
    const float keep = upper ? hi : lo;
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, H);
  }
  if (upper) {
    off += kHalf;
    left = max(left - kHalf, 0);
  } else {
    left = min(left, kHalf);
  }
}

struct BackwardBlend {
  using Queue = IndexQueue;
  const StageSmem* st;
  const Record* rec;
  float4* grad;        // [n][4] accumulators: dt1, dt2, dt3, (dr, dg, db, do_hat)
  const FrameConst* fc;
  float* sacc;         // [kMoments][kTilePixels] shared
  const uint32_t* vals;
  float cxm, cym;      // principal point relative to the tile origin
  float T, Cr, Cg, Cb;
  bool done;
  uint32_t nblend;
  float X, Y;          // absolute pixel centre
  float x, y;          // tile-relative pixel centre
  float gr, gg, gb;    // dL/dRGB
  float ga;            // dL/dalpha (output alpha)
  float Fr, Fg, Fb;    // forward output colour (includes T_final bg)
  float Tfinal;
  float acc[kMoments];
  bool has;

  // compositing part shared by both paths: returns dL/dalpha (0 when done)
  __device__ __forceinline__ bool composite(float a, float4 c, float& dal, float& w) {
    const float Tn = T * (1.0f - a);
    if (Tn < kTStop) {
      done = true;
      return false;
    }
    w = a * T;
    Cr = fmaf(c.x, w, Cr);
    Cg = fmaf(c.y, w, Cg);
    Cb = fmaf(c.z, w, Cb);
    const float inv1ma = 1.0f / (1.0f - a);
    dal = gr * (c.x * T - (Fr - Cr) * inv1ma) + gg * (c.y * T - (Fg - Cg) * inv1ma) +
          gb * (c.z * T - (Fb - Cb) * inv1ma) + ga * Tfinal * inv1ma;
    T = Tn;
    ++nblend;
    return true;
  }

  // moments of contributor (alpha a, raw alpha o_hat G) at this pixel from its
  // num, d, 1/|d|^2 and rho^2; false when the pixel is done
  __device__ __forceinline__ bool moments(float a, float4 c, float oh, float n0, float n1, float n2, float d0,
                                          float d1, float d2, float inv, float rho2, float m[kMoments]) {
    float dal, w;
    if (!composite(a, c, dal, w)) return false;
    const float G = __expf(-0.5f * rho2);
    const float raw = oh * G;
#pragma unroll
    for (int i = 0; i < 19; ++i) m[i] = 0.0f;
    if (raw < kAlphaMax) {
      const float drho2 = -0.5f * dal * raw;
      const float sn = 2.0f * drho2 * inv;
      const float sd = -2.0f * drho2 * rho2 * inv;
      const float dn[3] = {sn * n0, sn * n1, sn * n2};
      const float ddv[3] = {sd * d0, sd * d1, sd * d2};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        m[i] = dn[i];
        m[3 + i] = x * dn[i];
        m[6 + i] = y * dn[i];
        m[9 + i] = ddv[i];
        m[12 + i] = x * ddv[i];
        m[15 + i] = y * ddv[i];
      }
      m[18] = dal * G;
    }
    m[19] = gr * w;
    m[20] = gg * w;
    m[21] = gb * w;
    return true;
  }
  __device__ __forceinline__ void begin_batch(uint32_t, int) {}
  __device__ __forceinline__ uint32_t payload(int k) const { return st->gid[k]; }
  // One warp-wide release round: lanes with w blend their popped contributor
  // gid, recompute its planes (Eq. 4-5) at this pixel from the record and form
  // its 16 row gradients; lanes releasing the same Gaussian add theirs with a
  // butterfly over the warp and share one set of atomics (neighbouring pixels
  // mostly release the same Gaussian in the same round).
  __device__ __forceinline__ void release_round(bool w, float a, uint32_t gid) {
    float g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = 0.0f;
    bool live = false;
    if (w) {
      const float4* r = reinterpret_cast<const float4*>(rec + gid);
      const float4 c = __ldg(r + 3);
      float dal, wt;
      if (composite(a, c, dal, wt)) {
        live = true;
        const float4 t1 = __ldg(r + 0), t2 = __ldg(r + 1), t3 = __ldg(r + 2);
        const float cx_ = fc->cx - X, cy_ = fc->cy - Y;
        const float3 n1 = f3(fmaf(cx_, t3.x, fc->fx * t1.x), fmaf(cx_, t3.y, fc->fx * t1.y), fmaf(cx_, t3.z, fc->fx * t1.z));
        const float h1 = fmaf(cx_, t3.w, fc->fx * t1.w);
        const float3 n2 = f3(fmaf(cy_, t3.x, fc->fy * t2.x), fmaf(cy_, t3.y, fc->fy * t2.y), fmaf(cy_, t3.z, fc->fy * t2.z));
        const float h2 = fmaf(cy_, t3.w, fc->fy * t2.w);
        const float3 num = h1 * n2 - h2 * n1;
        const float3 dv = cross3(n1, n2);
        const float inv = 1.0f / dot3(dv, dv);
        const float rho2 = dot3(num, num) * inv;
        const float G = __expf(-0.5f * rho2);
        const float raw = c.w * G;
        if (raw < kAlphaMax) {
          const float drho2 = -0.5f * dal * raw;
          const float3 dnum = (2.0f * drho2 * inv) * num;
          const float3 ddv = (-2.0f * drho2 * rho2 * inv) * dv;
          const float dh1 = dot3(n2, dnum), dh2 = -dot3(n1, dnum);
          const float3 dn1 = (-h2) * dnum + cross3(n2, ddv);
          const float3 dn2 = h1 * dnum + cross3(ddv, n1);
          g[0] = fc->fx * dn1.x;
          g[1] = fc->fx * dn1.y;
          g[2] = fc->fx * dn1.z;
          g[3] = fc->fx * dh1;
          g[4] = fc->fy * dn2.x;
          g[5] = fc->fy * dn2.y;
          g[6] = fc->fy * dn2.z;
          g[7] = fc->fy * dh2;
          g[8] = cx_ * dn1.x + cy_ * dn2.x;
          g[9] = cx_ * dn1.y + cy_ * dn2.y;
          g[10] = cx_ * dn1.z + cy_ * dn2.z;
          g[11] = cx_ * dh1 + cy_ * dh2;
          g[15] = dal * G;
        }
        g[12] = gr * wt;
        g[13] = gg * wt;
        g[14] = gb * wt;
      }
    }
    // accumulator layout per Gaussian: dt1, dt2, dt3, (dr, dg, db, do_hat).
    // Lanes in groups below kMinGroup issue their own vector atomics (in the
    // same instruction when they share a Gaussian); larger groups are summed
    // first.  Measured on the 1M-Gaussian 1080p frames: butterflies for every
    // group 3.4 ms, from 24 lanes 2.5 ms, never 3.9 ms.
    const int lane = threadIdx.x & 31;
    const unsigned live_mask = __ballot_sync(0xffffffffu, live);
    unsigned grp = 1u << lane;
    if (__popc(live_mask) >= kMinGroup) grp = __match_any_sync(0xffffffffu, live ? gid : 0xffffffffu);
    const bool alone = live && __popc(grp) < kMinGroup;
    if (alone) {
      float4* acc4 = grad + 4 * (size_t)gid;
      atomicAdd(acc4 + 0, make_float4(g[0], g[1], g[2], g[3]));
      atomicAdd(acc4 + 1, make_float4(g[4], g[5], g[6], g[7]));
      atomicAdd(acc4 + 2, make_float4(g[8], g[9], g[10], g[11]));
      atomicAdd(acc4 + 3, make_float4(g[12], g[13], g[14], g[15]));
    }
    unsigned pend = __ballot_sync(0xffffffffu, live && !alone);
    while (pend) {
      const int L = __ffs(pend) - 1;
      const unsigned m = __shfl_sync(0xffffffffu, grp, L);   // lanes releasing lane L's Gaussian
      const uint32_t lg = __shfl_sync(0xffffffffu, gid, L);
      pend &= ~m;
      const bool in = (m >> lane) & 1u;
      // halving exchanges over bits 3..0 leave lane i with value i & 15
      // summed over its half-warp; the last exchange adds the other half
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = in ? g[i] : 0.0f;
#pragma unroll
      for (int h = 8; h > 0; h >>= 1) {
        const bool upper = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
          const float send = upper ? v[i] : v[i + h];
          const float keep = upper ? v[i + h] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
      }
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
      // lanes 0, 4, 8, 12 gather values 4j .. 4j + 3 for one vector atomic each
      const float v1 = __shfl_down_sync(0xffffffffu, v[0], 1), v2 = __shfl_down_sync(0xffffffffu, v[0], 2),
                  v3 = __shfl_down_sync(0xffffffffu, v[0], 3);
      if (lane < 16 && (lane & 3) == 0) atomicAdd(grad + 4 * (size_t)lg + (lane >> 2), make_float4(v[0], v1, v2, v3));
    }
  }

  // the staged Gaussian k: moments stay in registers until the warp-level
  // reduction at the end of item k
  __device__ __forceinline__ void blend_new(float a, const EvalState& ev) {
    const float4 c = __ldg(reinterpret_cast<const float4*>(rec + st->gid[ev.k]) + 3);
    if (moments(a, c, st->a[ev.k].w, ev.n0, ev.n1, ev.n2, ev.d0, ev.d1, ev.d2, ev.inv, ev.rho2, acc)) has = true;
  }
  // Warp reduction of the 22 moments of item k by halving exchanges
  // (reduce-scatter): at each level a lane keeps one half of its values and
  // receives its partner's copy of that half, so the value count per lane
  // goes 22 -> 11 -> 6 -> 3 -> 2 -> 1 (23 shuffles; padding to 32 values
  // would take 31).  Position p of a lane's kept upper half stands for
  // position p + half before the level; a lane ends with the warp total of
  // one moment, or of nothing when its path ran past the real positions
  // (22 of the 32 lanes hold one moment each).  Those lanes add it to slot k.
  __device__ __forceinline__ void end_item(int k) {
    const unsigned any = __ballot_sync(0xffffffffu, has);
    if (!any) return;
    const int lane = threadIdx.x & 31;
    float v[kMoments];
#pragma unroll
    for (int i = 0; i < kMoments; ++i) v[i] = has ? acc[i] : 0.0f;
    int off = 0, left = kMoments;   // moment held at position 0; real positions left
    halving_level<16, kMoments>(v, lane, off, left);
    halving_level<8, (kMoments + 1) / 2>(v, lane, off, left);
    halving_level<4, (kMoments + 3) / 4>(v, lane, off, left);
    halving_level<2, (kMoments + 7) / 8>(v, lane, off, left);
    halving_level<1, (kMoments + 15) / 16>(v, lane, off, left);
    if (left > 0 && v[0] != 0.0f) atomicAdd(&sacc[k * kAccStride + off], v[0]);
#pragma unroll
    for (int i = 0; i < kMoments; ++i) acc[i] = 0.0f;
    has = false;
  }


  // block-converged: convert each staged Gaussian's moments to gradients of
  // its T_view rows, one set of vector atomics per (tile, Gaussian)
  __device__ __forceinline__ void end_batch(uint32_t, int count) {
    __syncthreads();
    const int t = threadIdx.x;
    if (t < count) {
      float m[kMoments];
      bool nz = false;
#pragma unroll
      for (int i = 0; i < kMoments; ++i) {
        m[i] = sacc[t * kAccStride + i];
        nz |= m[i] != 0.0f;
        sacc[t * kAccStride + i] = 0.0f;
      }
      if (nz) {
        const uint32_t gid = st->gid[t];
        const float4* r = reinterpret_cast<const float4*>(rec + gid);
        const float4 t1 = __ldg(r + 0), t2 = __ldg(r + 1), t3 = __ldg(r + 2);
        const float3 T3 = f3(t3.x, t3.y, t3.z);
        const float3 Uv = f3(fmaf(cxm, t3.x, fc->fx * t1.x), fmaf(cxm, t3.y, fc->fx * t1.y), fmaf(cxm, t3.z, fc->fx * t1.z));
        const float Uw = fmaf(cxm, t3.w, fc->fx * t1.w);
        const float3 Wv = f3(fmaf(cym, t3.x, fc->fy * t2.x), fmaf(cym, t3.y, fc->fy * t2.y), fmaf(cym, t3.z, fc->fy * t2.z));
        const float Ww = fmaf(cym, t3.w, fc->fy * t2.w);
        const float3 gN0 = f3(m[0], m[1], m[2]), gNx = f3(m[3], m[4], m[5]), gNy = f3(m[6], m[7], m[8]);
        const float3 gD0 = f3(m[9], m[10], m[11]), gDx = f3(m[12], m[13], m[14]), gDy = f3(m[15], m[16], m[17]);
        // N0 = Uw Wv - Ww Uv, Nx = Ww T3 - T3w Wv, Ny = T3w Uv - Uw T3,
        // D0 = Uv x Wv, Dx = Wv x T3, Dy = T3 x Uv
        const float gUw = dot3(gN0, Wv) - dot3(gNy, T3);
        const float gWw = -dot3(gN0, Uv) + dot3(gNx, T3);
        const float gTw = -dot3(gNx, Wv) + dot3(gNy, Uv);
        const float3 gUv = (-Ww) * gN0 + t3.w * gNy + cross3(Wv, gD0) + cross3(gDy, T3);
        const float3 gWv = Uw * gN0 - t3.w * gNx + cross3(gD0, Uv) + cross3(T3, gDx);
        const float3 gTv = Ww * gNx - Uw * gNy + cross3(gDx, Wv) + cross3(Uv, gDy);
        // U = fx t1 + cxm t3, W = fy t2 + cym t3
        const float4 g1 = make_float4(fc->fx * gUv.x, fc->fx * gUv.y, fc->fx * gUv.z, fc->fx * gUw);
        const float4 g2 = make_float4(fc->fy * gWv.x, fc->fy * gWv.y, fc->fy * gWv.z, fc->fy * gWw);
        const float4 g3 = make_float4(cxm * gUv.x + cym * gWv.x + gTv.x, cxm * gUv.y + cym * gWv.y + gTv.y,
                                      cxm * gUv.z + cym * gWv.z + gTv.z, cxm * gUw + cym * gWw + gTw);
        float4* acc4 = grad + 4 * (size_t)gid;
        atomicAdd(acc4 + 0, g1);
        atomicAdd(acc4 + 1, g2);
        atomicAdd(acc4 + 2, g3);
        atomicAdd(acc4 + 3, make_float4(m[19], m[20], m[21], m[18]));
      }
    }
  }
};

// The backward of one tile (all threads of the block).
__device__ __forceinline__ void backward_tile(TileSmem<IndexQueue>& s, float* sacc, int tile,
                                              const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
                                              const uint32_t* __restrict__ vals, const Record* __restrict__ rec,
                                              const uint4* __restrict__ aux, const FrameConst& fc,
                                              const float* __restrict__ rgb, const float* __restrict__ drgb,
                                              const float* __restrict__ dalpha, const float* __restrict__ final_T,
                                              const uint32_t* __restrict__ n_blended, float4* __restrict__ grad,
                                              unsigned long long* __restrict__ stats) {
  const int tx = tile % fc.tiles_x, ty = tile / fc.tiles_x;
  int lx, ly;
  tile_pixel(threadIdx.x, lx, ly);
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool in_image = px < fc.W && py < fc.H;
  const size_t HW = (size_t)fc.W * fc.H;
  const size_t p = in_image ? (size_t)py * fc.W + px : 0;
  for (int i = threadIdx.x; i < kAccStride * kTilePixels; i += kTilePixels) sacc[i] = 0.0f;

  BackwardBlend bl;
  bl.st = &s.st;
  bl.rec = rec;
  bl.grad = grad;
  bl.fc = &fc;
  bl.sacc = sacc;
  bl.vals = vals;
  bl.cxm = fc.cx - (float)(tx * kTile);
  bl.cym = fc.cy - (float)(ty * kTile);
  bl.T = 1.0f;
  bl.Cr = bl.Cg = bl.Cb = 0.0f;
  bl.nblend = 0;
  bl.X = (float)px + 0.5f;
  bl.Y = (float)py + 0.5f;
  bl.x = (float)lx + 0.5f;
  bl.y = (float)ly + 0.5f;
#pragma unroll
  for (int i = 0; i < kMoments; ++i) bl.acc[i] = 0.0f;
  bl.has = false;
  float Tf = 1.0f;
  if (in_image) {
    bl.gr = drgb[p];
    bl.gg = drgb[HW + p];
    bl.gb = drgb[2 * HW + p];
    bl.ga = dalpha ? dalpha[p] : 0.0f;
    bl.Fr = rgb[p];
    bl.Fg = rgb[HW + p];
    bl.Fb = rgb[2 * HW + p];
    Tf = final_T[p];
  } else {
    bl.gr = bl.gg = bl.gb = bl.ga = bl.Fr = bl.Fg = bl.Fb = 0.0f;
  }
  bl.Tfinal = Tf;
  bl.done = !in_image;
  uint32_t neval = 0;   // evaluations of this pixel (far below 2^32 per tile)
  uint32_t nmis = 0, npass = 0;
  __syncthreads();
  traverse_tile<true>(s, ranges[tile], keys, vals, rec, aux, fc, tx, ty, bl.x, bl.y, bl, neval, nmis, npass);
  // the replay must reproduce the forward blend count
  const bool mismatch = in_image && bl.nblend != n_blended[p];
  const unsigned ball = __ballot_sync(0xffffffffu, mismatch);
  if ((threadIdx.x & 31) == 0 && ball) atomicAdd(&stats[kStatReplayMismatch], (unsigned long long)__popc(ball));
}

// Persistent: blocks take tiles from a work counter, longest first (the order
// of tile_order_kernel, computed again from the frame's tile ranges).
__global__ void __launch_bounds__(kTilePixels, 2)
render_backward_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
                       const uint32_t* __restrict__ vals, const Record* __restrict__ rec,
                       const uint4* __restrict__ aux, const FrameConst* __restrict__ fcp,
                       const float* __restrict__ rgb,
                       const float* __restrict__ drgb, const float* __restrict__ dalpha,
                       const float* __restrict__ final_T, const uint32_t* __restrict__ n_blended,
                       float4* __restrict__ grad, unsigned long long* __restrict__ stats,
                       const uint32_t* __restrict__ order, uint32_t* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<IndexQueue>& s = *reinterpret_cast<TileSmem<IndexQueue>*>(smem_raw);
  float* sacc = reinterpret_cast<float*>(smem_raw + kStageBytes);
  __shared__ uint32_t s_item;
  const FrameConst fc = *fcp;
  const uint32_t n_tiles = (uint32_t)(fc.tiles_x * fc.tiles_y);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= n_tiles) break;
    backward_tile(s, sacc, (int)order[item], ranges, keys, vals, rec, aux, fc, rgb, drgb, dalpha, final_T,
                  n_blended, grad, stats);
  }
}

// ---------------------------------------------------------------------------
// K7
// ---------------------------------------------------------------------------

constexpr float kY00 = 0.28209479177387814f;
constexpr float kY1 = 0.4886025119029199f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.5462742152960396f;
constexpr float kY3a = 0.5900435899266435f;
constexpr float kY3b = 2.890611442640554f;
constexpr float kY3c = 0.4570457994644658f;
constexpr float kY3d = 0.3731763325901154f;
constexpr float kY3e = 1.445305721320277f;

// SH basis values Y[k] and their gradients dY[k] = dY_k/d(x,y,z) of the same
// polynomials as the forward preprocess.
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, int deg, float* Y, float3* dY) {
  Y[0] = kY00;
  dY[0] = f3(0.f, 0.f, 0.f);
  if (deg < 1) return;
  Y[1] = -kY1 * y;  dY[1] = f3(0.f, -kY1, 0.f);
  Y[2] = kY1 * z;   dY[2] = f3(0.f, 0.f, kY1);
  Y[3] = -kY1 * x;  dY[3] = f3(-kY1, 0.f, 0.f);
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;                 dY[4] = f3(kY2a * y, kY2a * x, 0.f);
  Y[5] = -kY2a * y * z;                dY[5] = f3(0.f, -kY2a * z, -kY2a * y);
  Y[6] = kY2b * (2.f * zz - xx - yy);  dY[6] = f3(-2.f * kY2b * x, -2.f * kY2b * y, 4.f * kY2b * z);
  Y[7] = -kY2a * x * z;                dY[7] = f3(-kY2a * z, 0.f, -kY2a * x);
  Y[8] = kY2c * (xx - yy);             dY[8] = f3(2.f * kY2c * x, -2.f * kY2c * y, 0.f);
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.f * xx - yy);
  dY[9] = f3(-6.f * kY3a * x * y, -kY3a * (3.f * xx - 3.f * yy), 0.f);
  Y[10] = kY3b * x * y * z;
  dY[10] = f3(kY3b * y * z, kY3b * x * z, kY3b * x * y);
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  dY[11] = f3(2.f * kY3c * x * y, -kY3c * (4.f * zz - xx - 3.f * yy), -8.f * kY3c * y * z);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  dY[12] = f3(-6.f * kY3d * x * z, -6.f * kY3d * y * z, kY3d * (6.f * zz - 3.f * xx - 3.f * yy));
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  dY[13] = f3(-kY3c * (4.f * zz - 3.f * xx - yy), 2.f * kY3c * x * y, -8.f * kY3c * x * z);
  Y[14] = kY3e * z * (xx - yy);
  dY[14] = f3(2.f * kY3e * x * z, -2.f * kY3e * y * z, kY3e * (xx - yy));
  Y[15] = -kY3a * x * (xx - 3.f * yy);
  dY[15] = f3(-kY3a * (3.f * xx - 3.f * yy), 6.f * kY3a * x * y, 0.f);
}

__global__ void __launch_bounds__(128)
preprocess_backward_kernel(SceneDev s, const FrameConst* __restrict__ fcp, const uint32_t* __restrict__ counts,
                           const float4* __restrict__ grad, float* __restrict__ g_means,
                           float* __restrict__ g_log_scales, float* __restrict__ g_quats,
                           float* __restrict__ g_opacity, float* __restrict__ g_sh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const FrameConst fc = *fcp;
  const int K = (s.sh_degree + 1) * (s.sh_degree + 1);

  float* gsh = g_sh + (size_t)i * K * 3;
  if (counts[i] == 0u) {   // not visible (no tile): zero gradient
    for (int j = 0; j < 3; ++j) g_means[3 * i + j] = g_log_scales[3 * i + j] = 0.0f;
    for (int j = 0; j < 4; ++j) g_quats[4 * i + j] = 0.0f;
    g_opacity[i] = 0.0f;
    for (int j = 0; j < K * 3; ++j) gsh[j] = 0.0f;
    return;
  }
  const float4 G1 = grad[4 * i + 0], G2 = grad[4 * i + 1], G3 = grad[4 * i + 2], G4 = grad[4 * i + 3];

  // ---- forward recomputation
  const float mu[3] = {s.means[3 * i], s.means[3 * i + 1], s.means[3 * i + 2]};
  const float ls[3] = {s.log_scales[3 * i], s.log_scales[3 * i + 1], s.log_scales[3 * i + 2]};
  const float4 q4 = reinterpret_cast<const float4*>(s.quats)[i];
  const float logit = s.opacity_logits[i];
  const float vtrain = s.vhat_train[i];
  const float vz = fc.Rv[6] * mu[0] + fc.Rv[7] * mu[1] + fc.Rv[8] * mu[2] + fc.tv[2];
  float sc[3], a2[3];
  for (int j = 0; j < 3; ++j) {
    sc[j] = expf(ls[j]);
    a2[j] = sc[j] * sc[j];
  }
  const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
  const float qinv = rsqrtf(qn2);
  const float qw = q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
  float R[9];
  R[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
  R[1] = 2.0f * (qx * qy - qw * qz);
  R[2] = 2.0f * (qx * qz + qw * qy);
  R[3] = 2.0f * (qx * qy + qw * qz);
  R[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
  R[5] = 2.0f * (qy * qz - qw * qx);
  R[6] = 2.0f * (qx * qz - qw * qy);
  R[7] = 2.0f * (qy * qz + qw * qx);
  R[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
  const float opac = 1.0f / (1.0f + expf(-logit));
  float kv = 0.0f, veff = 0.0f;
  bool view_branch = false;
  if (!(fc.flags & AAAG_FLAG_NO_FILTER)) {
    const float vhat = fc.fx / fmaxf(vz, fc.znear);
    view_branch = vhat < vtrain;
    veff = fminf(vtrain, vhat);
    kv = fc.k / (veff * veff);
  }
  float b[3], sp[3];
  for (int j = 0; j < 3; ++j) {
    b[j] = a2[j] + kv;
    sp[j] = sqrtf(b[j]);
  }
  const float df[3] = {mu[0] - fc.o[0], mu[1] - fc.o[1], mu[2] - fc.o[2]};
  const float dist = sqrtf(df[0] * df[0] + df[1] * df[1] + df[2] * df[2]);
  const float d[3] = {df[0] / dist, df[1] / dist, df[2] / dist};
  float dp[3];
  for (int j = 0; j < 3; ++j) dp[j] = R[j] * d[0] + R[3 + j] * d[1] + R[6 + j] * d[2];
  float w[3], r[3];
  for (int j = 0; j < 3; ++j) {
    w[j] = dp[j] * dp[j] / b[j];
    r[j] = a2[j] / b[j];
  }
  const float P = w[0] * r[1] * r[2] + w[1] * r[0] * r[2] + w[2] * r[0] * r[1];
  const float Q = w[0] + w[1] + w[2];
  const float phi2 = P / Q;
  const float phi = sqrtf(phi2);

  // ---- gradients
  float gmu[3] = {0.f, 0.f, 0.f}, gR[9], gb[3] = {0.f, 0.f, 0.f}, ga2[3] = {0.f, 0.f, 0.f};
  float gd[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < 9; ++j) gR[j] = 0.0f;
  // T_view rows: t_r = (A_r, mu_v,r), A = Rv R S', mu_v = Rv mu + tv
  const float gA[9] = {G1.x, G1.y, G1.z, G2.x, G2.y, G2.z, G3.x, G3.y, G3.z};
  const float gmv[3] = {G1.w, G2.w, G3.w};
  for (int j = 0; j < 3; ++j) gmu[j] += fc.Rv[j] * gmv[0] + fc.Rv[3 + j] * gmv[1] + fc.Rv[6 + j] * gmv[2];
  // dM = Rv^T dA, M = R diag(s')
  for (int k = 0; k < 3; ++k) {
    for (int j = 0; j < 3; ++j) {
      const float gM = fc.Rv[k] * gA[j] + fc.Rv[3 + k] * gA[3 + j] + fc.Rv[6 + k] * gA[6 + j];
      gR[3 * k + j] += gM * sp[j];
      gb[j] += gM * R[3 * k + j] * 0.5f / sp[j];   // s' = sqrt(b)
    }
  }
  // o_hat = o phi
  const float goh = G4.w;
  const float gopac = goh * phi;
  const float gphi2 = goh * opac * 0.5f / phi;
  const float gP = gphi2 / Q, gQ = -gphi2 * phi2 / Q;
  const float gw[3] = {gP * r[1] * r[2] + gQ, gP * r[0] * r[2] + gQ, gP * r[0] * r[1] + gQ};
  const float gr[3] = {gP * (w[1] * r[2] + w[2] * r[1]), gP * (w[0] * r[2] + w[2] * r[0]),
                       gP * (w[0] * r[1] + w[1] * r[0])};
  float gdp[3];
  for (int j = 0; j < 3; ++j) {
    gb[j] += -gw[j] * w[j] / b[j] - gr[j] * r[j] / b[j];
    ga2[j] += gr[j] / b[j];
    gdp[j] = gw[j] * 2.0f * dp[j] / b[j];
  }
  float gkv = 0.0f;
  for (int j = 0; j < 3; ++j) {
    ga2[j] += gb[j];
    gkv += gb[j];
  }
  // d' = R^T d
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) {
      gR[3 * k + j] += d[k] * gdp[j];
      gd[k] += R[3 * k + j] * gdp[j];
    }
  // colour: max(0, sum_k Y_k(d) sh_k + 0.5)
  {
    float Y[16];
    float3 dY[16];
    sh_basis_grad(d[0], d[1], d[2], s.sh_degree, Y, dY);
    const float* shp = s.sh + (size_t)i * K * 3;
    float raw[3] = {0.5f, 0.5f, 0.5f};
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < 3; ++c) raw[c] += Y[k] * shp[3 * k + c];
    const float gcol[3] = {raw[0] > 0.f ? G4.x : 0.f, raw[1] > 0.f ? G4.y : 0.f, raw[2] > 0.f ? G4.z : 0.f};
    for (int k = 0; k < K; ++k) {
      float gy = 0.0f;
      for (int c = 0; c < 3; ++c) {
        gsh[3 * k + c] = gcol[c] * Y[k];
        gy += gcol[c] * shp[3 * k + c];
      }
      gd[0] += gy * dY[k].x;
      gd[1] += gy * dY[k].y;
      gd[2] += gy * dY[k].z;
    }
  }
  // d = (mu - o) / |mu - o|
  const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
  for (int j = 0; j < 3; ++j) gmu[j] += (gd[j] - d[j] * dd) / dist;
  // kv = k / v'^2, v' = fx / z on the view branch (z > znear)
  if (view_branch && vz > fc.znear) {
    const float gveff = -2.0f * kv / veff * gkv;
    const float gvz = -veff / vz * gveff;          // d(fx/z)/dz = -(fx/z)/z
    for (int j = 0; j < 3; ++j) gmu[j] += fc.Rv[6 + j] * gvz;
  }
  // s^2 = exp(2 log s)
  for (int j = 0; j < 3; ++j) g_log_scales[3 * i + j] = 2.0f * a2[j] * ga2[j];
  for (int j = 0; j < 3; ++j) g_means[3 * i + j] = gmu[j];
  g_opacity[i] = gopac * opac * (1.0f - opac);
  // R(q_hat) -> q_hat -> q
  float gq[4];
  gq[0] = -2.f * qz * gR[1] + 2.f * qy * gR[2] + 2.f * qz * gR[3] - 2.f * qx * gR[5] - 2.f * qy * gR[6] +
          2.f * qx * gR[7];
  gq[1] = 2.f * qy * gR[1] + 2.f * qz * gR[2] + 2.f * qy * gR[3] - 4.f * qx * gR[4] - 2.f * qw * gR[5] +
          2.f * qz * gR[6] + 2.f * qw * gR[7] - 4.f * qx * gR[8];
  gq[2] = -4.f * qy * gR[0] + 2.f * qx * gR[1] + 2.f * qw * gR[2] + 2.f * qx * gR[3] + 2.f * qz * gR[5] -
          2.f * qw * gR[6] + 2.f * qz * gR[7] - 4.f * qy * gR[8];
  gq[3] = -4.f * qz * gR[0] - 2.f * qw * gR[1] + 2.f * qx * gR[2] + 2.f * qw * gR[3] - 4.f * qz * gR[4] +
          2.f * qy * gR[5] + 2.f * qx * gR[6] + 2.f * qy * gR[7];
  const float qh[4] = {qw, qx, qy, qz};
  const float proj = gq[0] * qh[0] + gq[1] * qh[1] + gq[2] * qh[2] + gq[3] * qh[3];
  for (int j = 0; j < 4; ++j) g_quats[4 * i + j] = (gq[j] - qh[j] * proj) * qinv;
}

}  // namespace

void configure_backward(LaunchConfig& c) {
  cudaFuncSetAttribute(render_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kBackwardSmemBytes);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_backward_kernel, kTilePixels, kBackwardSmemBytes);
  c.backward_per_sm = std::max(1, per_sm);
}

aaag_status launch_render_backward(const SceneDev& s, aaag_workspace* ws, const float* rgb, const float* drgb,
                                   const float* dalpha, const aaag_grads* out, cudaStream_t st) {
  if (cudaMemsetAsync(ws->grad_acc, 0, (size_t)ws->n * sizeof(float4) * 4, st) != cudaSuccess)
    return check_launch("backward memset");
  const LaunchConfig& lc = launch_config();
  const int alt = ws->sorted_in_alt;
  uint32_t* counter = reinterpret_cast<uint32_t*>(ws->stats + kStatBackwardCounter);
  aaag_status e = launch_tile_order(ws, counter, st);
  if (e != AAAG_OK) return e;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)lc.sms * lc.backward_per_sm,
                                                                          ws->n_tiles));
  render_backward_kernel<<<grid, kTilePixels, kBackwardSmemBytes, st>>>(
      ws->ranges, ws->keys[alt], ws->vals[alt], ws->records, ws->aux, ws->fc_dev, rgb, drgb, dalpha, ws->final_T,
      ws->n_blended, ws->grad_acc, ws->stats, ws->tile_order, counter);
  e = check_launch("render_backward");
  if (e != AAAG_OK || s.n == 0) return e;
  const unsigned blocks = (unsigned)((s.n + 127) / 128);
  preprocess_backward_kernel<<<blocks, 128, 0, st>>>(s, ws->fc_dev, ws->counts, ws->grad_acc, out->means,
                                                     out->log_scales, out->quats, out->opacity_logits, out->sh);
  return check_launch("preprocess_backward");
}

}  // namespace aaag
