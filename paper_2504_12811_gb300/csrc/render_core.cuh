// Per-tile traversal shared by the forward render (K5) and its backward (K6).
//
// Both kernels walk a tile's sorted pairs with identical arithmetic (explicit
// fmaf everywhere, so the two compile to the same rounding), the same
// per-pixel re-sort queue and the same release rule; they differ in what
// happens when a contributor is blended, which is a functor, and in how the
// releases of a warp's lanes are scheduled (per lane in the forward, in
// warp-wide rounds in the backward), which leaves each pixel's sequence
// unchanged.  The backward pass therefore replays exactly the blend sequence
// of the forward pass.
//
// Plane form (paper Sec. 3.1, Eq. 4-5): with t_i the rows of T_view and tile
// origin (x_t, y_t), U = fx t1 + (cx - x_t) t3 and W = fy t2 + (cy - y_t) t3.
// For the tile-relative pixel centre (x, y) the transformed planes are
// (n1, h1) = U - x t3 and (n2, h2) = W - y t3, and
//     num = h1 n2 - h2 n1 = N0 + x Nx + y Ny,     d = n1 x n2 = D0 + x Dx + y Dy
// (the xy terms cancel).  rho^2 = |num|^2 / |d|^2 is the squared distance of
// the ray to the Gaussian's centre in its normalised space.  d is parallel to
// the ray direction in Gaussian space, d = fx fy det(A) A^-1 r, so the view
// depth of the maximum is t* = G.d / |d|^2 with G = fx fy adj(A) mu_v.
//
// Per-pixel order.  Pairs arrive sorted by key; the key of pair k+1, L_{k+1},
// is a lower bound of the t* of every contributor arriving after pair k.  When
// pair k contributes with depth t:
//   1. queued entries with depth <= t and < L_{k+1} are blended (in order);
//   2. if t < L_{k+1} the new contributor is blended at once, followed by the
//      queued entries below L_{k+1}: nothing later can precede any of them;
//   3. otherwise it is inserted into the pixel's sorted queue.
// This is the exact (t*, arrival) order while the queue has room.  When it is
// full, the order stays exact by depth peeling: a pass blends only the
// contributors with lo <= t* < hi.  The queue keeps the nearest ones; the
// farther of the new entry and the queue's last entry is deferred, hi drops
// to its depth, and every queued entry at or beyond hi leaves too.  Once
// L_{k+1} >= hi nothing later can fall inside the window, so the pixel drains
// its queue and closes the pass.  A pixel that deferred anything runs another
// pass over its tile with lo = hi, starting at the first pair that inserted
// into its queue after it was last empty before the first deferral (every
// deferred contributor arrived there or later; everything before it was
// blended).  Each pass blends its window completely, in order, so the
// passes together blend exactly the plain (t*, arrival) sequence.  When the
// queue is full and its nearest entry lies at lo itself, that entry is
// released at once instead (nothing this pass can precede it), so hi > lo and
// every pass advances.  The bounded-buffer ablation (AAAG_FLAG_KBUFFER)
// keeps the approximate rule: a full queue releases its nearest entry early.
// Queue entries stay in
// fixed per-thread slots in shared memory, laid out [slot][thread] (bank-
// conflict free); their order lives in one 64-bit register holding the slot
// numbers nearest first, 4 bits each, so an insertion moves no entry (a scan
// of depths from the far end, then a register shift) and a release reads one.
// The front's depth stays in a register.  Shared memory per block is kept
// at 74 KB so that three tile blocks fit on an SM: the traversal is bound by
// latency, and resident warps are what hides it.
//
// Warp skipping.  Warp w of a tile block owns the 8x4 pixel block at
// (8 (w & 1), 4 (w >> 1)).  When a Gaussian is staged, the pixel-centre ranges
// from its view-space bounds (Eq. 14-17) give the set of warps holding a pixel
// that can see it, as an 8-bit mask; the other warps skip it without
// evaluating.  A skipped pixel could not contribute (its centre lies outside
// the bounds), so the blends and their order are unchanged.  In the per-lane
// traversal each warp first turns the staged masks into a bitmap of its own
// Gaussians (one ballot per 32) and walks only its set bits, instead of
// loading and testing every staged mask (2% of the 1080p render, 3% of a
// dense training view).
#pragma once

#include <type_traits>

#include "aaag_internal.cuh"

namespace aaag {

constexpr int kQueue = 16;   // per-pixel re-sort queue entries (power of two)

// Coefficients of the staged Gaussians (one batch of pairs of one tile).
struct StageSmem {
  float4 a[kTilePixels];    // N0.xyz, o_hat
  float4 b[kTilePixels];    // Nx.xyz, ub | wmask: an upper bound of t* over the tile whose
                            // low 8 bits are the mask of the warps holding a pixel that can see it
  float4 c[kTilePixels];    // Ny.xyz, tau+: |num|^2 > tau+ |d|^2 rules out alpha >= 1/255
  float4 d[kTilePixels];    // D0.xyz, G.x
  float4 e[kTilePixels];    // Dx.xyz, G.y
  float4 f[kTilePixels];    // Dy.xyz, G.z
  float L[kTilePixels];     // L_next: lower bound of t* for every later pair
  uint32_t gid[kTilePixels];  // Gaussian index
  // per warp, bit k % 32 of word k / 32: staged Gaussian k can be seen from a
  // pixel of the warp (the per-lane traversal visits only those)
  uint32_t wbits[kTilePixels / 32][kTilePixels / 32];
  uint32_t start;           // first pair of the next depth-peeling pass
};

// Queue store, [slot][thread], one array per field: (t*, alpha, Gaussian
// index).  The Payload type is what an entry carries besides (t*, alpha).
struct IndexQueue {
  using Payload = uint32_t;
  float t_[kQueue][kTilePixels];      // t*
  float a_[kQueue][kTilePixels];      // alpha
  uint32_t g_[kQueue][kTilePixels];   // Gaussian index
  __device__ __forceinline__ float t(int s, int tid) const { return t_[s][tid]; }
  __device__ __forceinline__ void load(int s, int tid, float& a, Payload& p) const {
    a = a_[s][tid];
    p = g_[s][tid];
  }
  __device__ __forceinline__ void put(int s, int tid, float t, float a, Payload p) {
    t_[s][tid] = t;
    a_[s][tid] = a;
    g_[s][tid] = p;
  }
};

template <class Q>
struct TileSmem {
  StageSmem st;
  Q q;
};
constexpr size_t kForwardSmemBytes = sizeof(TileSmem<IndexQueue>);
static_assert(3 * (kForwardSmemBytes + 1024) <= 228 * 1024, "three tile blocks per SM");

// Tile-relative pixel of thread tid: warp w owns the 8x4 block at
// (8 (w & 1), 4 (w >> 1)), lanes row-major inside it.
__device__ __forceinline__ void tile_pixel(int tid, int& lx, int& ly) {
  const int w = tid >> 5, lane = tid & 31;
  lx = ((w & 1) << 3) | (lane & 7);
  ly = ((w >> 1) << 2) | (lane >> 3);
}

// Warps of the tile at (ox, oy) that hold a pixel of the inclusive pixel
// rectangle [x0, x1] x [y0, y1] packed in r (16 bits each), as a bit mask.
__device__ __forceinline__ uint32_t warp_mask(uint2 r, int ox, int oy) {
  const int x0 = max((int)(r.x & 0xffffu) - ox, 0), x1 = min((int)(r.y & 0xffffu) - ox, kTile - 1);
  const int y0 = max((int)(r.x >> 16) - oy, 0), y1 = min((int)(r.y >> 16) - oy, kTile - 1);
  if (x0 > x1 || y0 > y1) return 0u;
  const uint32_t cols = (2u << (x1 >> 3)) - (1u << (x0 >> 3));   // warp columns 0..1
  uint32_t m = 0u;
#pragma unroll
  for (int wy = 0; wy < 4; ++wy)
    if (wy >= (y0 >> 2) && wy <= (y1 >> 2)) m |= cols << (2 * wy);
  return m;
}

__device__ __forceinline__ float decode_depth(uint32_t key, const FrameConst& fc) {
  const uint32_t dk = key & ((fc.depth_bits >= 32) ? 0xffffffffu : ((1u << fc.depth_bits) - 1u));
  return __uint_as_float((dk << fc.depth_shift) + fc.znear_bits);
}

__device__ __forceinline__ float3 fma3(float s, float3 a, float3 b) {   // s a + b
  return f3(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z));
}
__device__ __forceinline__ float3 crs(float3 a, float3 b) {
  return f3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}

// An upper bound of the depth t* = G.d / |d|^2 of the ray maximum over the
// rectangle of the tile's pixel centres (d = D0 + x Dx + y Dy, x and y in
// [0.5, 15.5]), used by later depth-peeling passes to skip Gaussians that lie
// entirely in front of their window.  Returned as float bits rounded up to a
// multiple of 256 (the low 8 bits then carry the warp mask and only raise
// it); kNoCap (a huge finite value) when there is no bound.
constexpr uint32_t kNoCap = 0x7f000000u;   // about 1.7e38

__device__ __forceinline__ uint32_t cap_bits(float ub) {
  if (!(ub < 1.0e37f)) return kNoCap;
  return (__float_as_uint(ub) + 0x100u) & ~0xffu;
}

// The largest G.d (affine: at a corner) over the smallest |d|^2 on the
// rectangle (convex: its unconstrained minimum when that lies inside, else the
// minimum along one of the edges), raised by 0.1%.  (The exact maximum of t*
// over the tile, found by checking M |d|^2 - G.d >= 0 at its minimisers,
// skipped 6% more evaluations in dense views but cost more than it saved.)
__device__ __forceinline__ uint32_t tile_depth_cap(float3 D0, float3 Dx, float3 Dy, float3 G) {
  const float g0 = dot3(G, D0), gx = dot3(G, Dx), gy = dot3(G, Dy);
  const float gmax = g0 + fmaxf(0.5f * gx, 15.5f * gx) + fmaxf(0.5f * gy, 15.5f * gy);
  if (!(gmax > 0.0f)) return kNoCap;
  const float a = dot3(Dx, Dx), b = dot3(Dx, Dy), c = dot3(Dy, Dy);
  const float e = dot3(D0, Dx), f = dot3(D0, Dy);
  auto q = [&](float x, float y) {
    const float3 d = fma3(y, Dy, fma3(x, Dx, D0));
    return dot3(d, d);
  };
  auto clampc = [](float v) { return fminf(fmaxf(v, 0.5f), 15.5f); };
  float qmin = 3.0e38f;
  const float det = a * c - b * b;
  if (det > 0.0f) {
    const float x = (b * f - c * e) / det, y = (b * e - a * f) / det;
    if (x >= 0.5f && x <= 15.5f && y >= 0.5f && y <= 15.5f) qmin = q(x, y);
  }
  if (c > 0.0f) {
    qmin = fminf(qmin, q(0.5f, clampc(-(f + 0.5f * b) / c)));
    qmin = fminf(qmin, q(15.5f, clampc(-(f + 15.5f * b) / c)));
  }
  if (a > 0.0f) {
    qmin = fminf(qmin, q(clampc(-(e + 0.5f * b) / a), 0.5f));
    qmin = fminf(qmin, q(clampc(-(e + 15.5f * b) / a), 15.5f));
  }
  qmin = fminf(qmin, fminf(fminf(q(0.5f, 0.5f), q(15.5f, 0.5f)), fminf(q(0.5f, 15.5f), q(15.5f, 15.5f))));
  if (!(qmin > 0.0f)) return kNoCap;
  return cap_bits(gmax / qmin * 1.001f);
}

// Coefficients of one Gaussian for the tile at (ox, oy) (cxm = cx - ox,
// cym = cy - oy); rect: its pixel-centre ranges.
__device__ __forceinline__ void stage_one(StageSmem& s, int slot, const Record* rec, uint32_t gid, uint2 rect,
                                          float Lnext, const FrameConst& fc, float cxm, float cym, int ox,
                                          int oy) {
  const float4* r = reinterpret_cast<const float4*>(rec + gid);
  const float4 t1 = __ldg(r + 0), t2 = __ldg(r + 1), t3 = __ldg(r + 2), cw = __ldg(r + 3);
  const float3 T3 = f3(t3.x, t3.y, t3.z);
  const float3 Uv = fma3(cxm, T3, fc.fx * f3(t1.x, t1.y, t1.z));
  const float Uw = fmaf(cxm, t3.w, fc.fx * t1.w);
  const float3 Wv = fma3(cym, T3, fc.fy * f3(t2.x, t2.y, t2.z));
  const float Ww = fmaf(cym, t3.w, fc.fy * t2.w);
  const float3 N0 = fma3(Uw, Wv, -Ww * Uv);
  const float3 Nx = fma3(Ww, T3, -t3.w * Wv);
  const float3 Ny = fma3(t3.w, Uv, -Uw * T3);
  const float3 D0 = crs(Uv, Wv);
  const float3 Dx = crs(Wv, T3);
  const float3 Dy = crs(T3, Uv);
  const float3 A1 = f3(t1.x, t1.y, t1.z), A2 = f3(t2.x, t2.y, t2.z);
  const float fxfy = fc.fx * fc.fy;
  const float3 G = fxfy * fma3(t1.w, crs(A2, T3), fma3(t2.w, crs(T3, A1), t3.w * crs(A1, A2)));
  s.a[slot] = make_float4(N0.x, N0.y, N0.z, cw.w);
  s.b[slot] = make_float4(Nx.x, Nx.y, Nx.z, __uint_as_float(kNoCap | warp_mask(rect, ox, oy)));
  s.L[slot] = Lnext;
  // rho^2 <= tau_rho exactly where o_hat exp(-rho^2/2) >= 1/255; the margin
  // keeps the division-free prefilter conservative under float32 rounding
  const float tau = 2.0f * logf(cw.w * 255.0f);
  s.c[slot] = make_float4(Ny.x, Ny.y, Ny.z, fmaf(tau, 1e-4f, tau) + 1e-4f);
  s.d[slot] = make_float4(D0.x, D0.y, D0.z, G.x);
  s.e[slot] = make_float4(Dx.x, Dx.y, Dx.z, G.y);
  s.f[slot] = make_float4(Dy.x, Dy.y, Dy.z, G.z);
  s.gid[slot] = gid;
}

// Per-thread sorted queue: entries in fixed slots, order in a register.
template <class Q>
struct SmemQueue {
  static_assert(kQueue == 16, "the order word holds 16 four-bit slot numbers");
  using P = typename Q::Payload;
  Q* q;
  int tid, n;
  unsigned long long order;   // nibble i: slot of the i-th nearest entry
  uint32_t used;              // bit s: slot s holds an entry
  float ft;                   // t* of the nearest entry (n > 0)
  __device__ __forceinline__ int slot_at(int i) const { return (int)((order >> (4 * i)) & 15ull); }
  // remove the nearest entry, returning its alpha and payload
  __device__ __forceinline__ void pop(float& a, P& p) {
    const int s = (int)(order & 15ull);
    q->load(s, tid, a, p);
    order >>= 4;
    used &= ~(1u << s);
    if (--n > 0) ft = q->t((int)(order & 15ull), tid);
  }
  // blend the nearest entry and remove it
  template <class Blender>
  __device__ __forceinline__ void release(Blender& bl) {
    float a;
    P p;
    pop(a, p);
    bl.blend(a, p);
  }
  // t* of the farthest entry (n > 0)
  __device__ __forceinline__ float back_t() const { return q->t(slot_at(n - 1), tid); }
  // remove every entry with t* >= h from the far end (deferred to a later pass)
  __device__ __forceinline__ void drop_from(float h) {
    while (n > 0) {
      const int s = slot_at(n - 1);
      if (q->t(s, tid) < h) break;
      used &= ~(1u << s);
      order &= ~(15ull << (4 * (n - 1)));
      --n;
    }
  }
  // sorted insert (n < kQueue), after every entry with an equal t*
  __device__ __forceinline__ void insert(float t, float a, P p) {
    int i = n;
    while (i > 0 && q->t(slot_at(i - 1), tid) > t) --i;
    const int s = __ffs(~used) - 1;   // a free slot: fewer than 16 are used
    used |= 1u << s;
    q->put(s, tid, t, a, p);
    const unsigned long long low = order & ((1ull << (4 * i)) - 1ull);   // 4 i <= 60
    order = low | ((unsigned long long)s << (4 * i)) | ((order ^ low) << 4);
    if (i == 0) ft = t;
    ++n;
  }
};

// Values of the current evaluation handed to a blend of the newly evaluated
// (staged) Gaussian: its slot and the pixel's num, d, 1/|d|^2 and rho^2.
struct EvalState {
  int k;
  float n0, n1, n2, d0, d1, d2, inv, rho2;
};

// Warp-wide release rounds (convergent traversal): while any lane of the warp
// wants to release its nearest entry, every such lane pops one and the whole
// warp calls Blender::release_round, so that lanes releasing the same
// Gaussian can be combined.  Each lane releases in the same order as with a
// per-lane loop.
template <class Q, class Blender, class Want>
__device__ __forceinline__ void release_rounds(SmemQueue<Q>& q, Blender& bl, Want want) {
  for (;;) {
    const bool w = want();
    if (!__any_sync(0xffffffffu, w)) return;
    float a = 0.0f;
    typename Q::Payload p{};
    if (w) q.pop(a, p);
    bl.release_round(w, a, p);
  }
}

// Traverse one tile for one pixel.  Blender must provide:
//   using Queue;                                     its queue store
//   bool done;                                       pixel finished
//   void blend_new(float alpha, const EvalState&);   blend the staged Gaussian k
//   Queue::Payload payload(int k);                   what a queued entry of k carries
//   void begin_batch(uint32_t b0, int cnt);          pairs b0 .. b0+cnt-1 are staged
// and, without CONVERGENT (each lane releases in its own loop),
//   void blend(float alpha, Queue::Payload);         blend a queued contributor
// With CONVERGENT, every lane runs every iteration (no early exit from the
// pair loop), every release is a warp-wide round, and the Blender provides
// instead
//   void release_round(bool w, float a, Queue::Payload);   warp-converged; lanes
//                                                    with w blend the popped entry
//   void end_item(int k);                            warp-converged, after item k
//   void end_batch(uint32_t b0, int cnt);            block-converged, after a batch
// The arithmetic, and so every blend decision, is the same either way.
// npass counts this pixel's passes beyond the first (depth peeling); nmis the
// early releases of the bounded-buffer ablation.  EXACT: the frame has neither
// ordering ablation (the flags are then known at compile time).
template <bool CONVERGENT, bool EXACT = false, class Blender>
__device__ __forceinline__ void traverse_tile(TileSmem<typename Blender::Queue>& sm, const uint2 range, const uint32_t* __restrict__ keys,
                                              const uint32_t* __restrict__ vals, const Record* __restrict__ rec,
                                              const uint4* __restrict__ aux, const FrameConst& fc, int tile_x,
                                              int tile_y, float x, float y, Blender& bl,
                                              uint32_t& neval, uint32_t& nmis, uint32_t& npass) {
  const int ox = tile_x * kTile, oy = tile_y * kTile;
  const float cxm = fc.cx - (float)ox, cym = fc.cy - (float)oy;
  const uint32_t wbit = 1u << (threadIdx.x >> 5);
  // ablations: blend in pair order (no re-sort); release only when the
  // buffer is full (no release by key)
  const bool resort = EXACT || !(fc.flags & AAAG_FLAG_NO_RESORT);
  const bool by_key = EXACT || !(fc.flags & AAAG_FLAG_KBUFFER);
  const bool peel = resort && by_key;   // exact order: defer instead of releasing early
  const float kInf = __int_as_float(0x7f800000);
  constexpr uint32_t kNone = 0xffffffffu;
  StageSmem& s = sm.st;
  SmemQueue<typename Blender::Queue> q;
  q.q = &sm.q;
  q.tid = threadIdx.x;
  q.ft = 0.0f;
  float lo = -kInf;              // this pass blends contributors with lo <= t* < hi
  uint32_t jfirst = range.x;     // earlier pairs hold nothing for this pixel's pass
  bool more = !bl.done;          // this pixel takes part in the pass
  uint32_t start = range.x;
  bool first_pass = true;        // block-wide: no pixel has a lower window bound yet
  for (;;) {
    float hi = kInf;
    bool open = more;
    uint32_t jnext = kNone;      // where the next pass can start for this pixel
    uint32_t jfill = range.x;    // pair that last inserted into an empty queue
    q.n = 0;
    q.order = 0ull;
    q.used = 0u;
    for (uint32_t b0 = start; b0 < range.y; b0 += kTilePixels) {
      // close the pass once no pair from here on can hold a contributor below hi
      if constexpr (!CONVERGENT) {
        if (open && hi < kInf && decode_depth(keys[b0], fc) >= hi) {
          while (q.n > 0 && !bl.done) q.release(bl);
          open = false;
        }
      } else {
        const bool close = open && hi < kInf && decode_depth(keys[b0], fc) >= hi;
        release_rounds(q, bl, [&] { return close && q.n > 0 && !bl.done; });
        if (close) open = false;
      }
      if (__syncthreads_count(open && !bl.done) == 0) break;
      const uint32_t j = b0 + threadIdx.x;
      if (j < range.y) {
        const float Lnext = j + 1 < range.y ? decode_depth(keys[j + 1], fc) : kInf;
        const uint32_t gid = vals[j];
        const uint4 ax = __ldg(aux + gid);
        stage_one(s, threadIdx.x, rec, gid, make_uint2(ax.x, ax.y), Lnext, fc, cxm, cym, ox, oy);
        if (!first_pass) {
          // the depth cap only matters to later passes (the first has lo = -inf);
          // computed from the staged planes of this thread's own slot
          const float4 d = s.d[threadIdx.x], e = s.e[threadIdx.x], f = s.f[threadIdx.x];
          const uint32_t cap = tile_depth_cap(f3(d.x, d.y, d.z), f3(e.x, e.y, e.z), f3(f.x, f.y, f.z),
                                              f3(d.w, e.w, f.w));
          const uint32_t mask = __float_as_uint(s.b[threadIdx.x].w) & 0xffu;
          s.b[threadIdx.x].w = __uint_as_float(cap | mask);
        }
      }
      __syncthreads();
      const int cnt = (int)min((uint32_t)kTilePixels, range.y - b0);
      bl.begin_batch(b0, cnt);
      if constexpr (!CONVERGENT) {
        // this warp's staged Gaussians as a bitmap (the same in all its lanes)
        const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
        for (int wd = 0; wd * 32 < cnt; ++wd) {
          const int kk = wd * 32 + lane;
          const bool mine = kk < cnt && (__float_as_uint(s.b[kk].w) & wbit) != 0u;
          const unsigned word = __ballot_sync(0xffffffffu, mine);
          if (lane == 0) s.wbits[wi][wd] = word;
        }
        __syncwarp();
      }
      if constexpr (CONVERGENT) {
        for (int k = 0; k < cnt; ++k) {
          const float4 bq = s.b[k];
          const uint32_t jk = b0 + (uint32_t)k;
          if (__float_as_uint(bq.w) & wbit) {   // warp-uniform
            // the same decisions as the per-lane loop below, with the releases
            // taken out of the per-lane branches into warp-wide rounds
            bool contrib = false;
            float ts = 0.0f, ca = 0.0f, Lnext = 0.0f;
            EvalState ev{k, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (open && !bl.done && jk >= jfirst && !(bq.w < lo)) {
              ++neval;
              const float4 a = s.a[k], c = s.c[k], d = s.d[k], e = s.e[k], f = s.f[k];
              const float n0 = fmaf(y, c.x, fmaf(x, bq.x, a.x));
              const float n1 = fmaf(y, c.y, fmaf(x, bq.y, a.y));
              const float n2 = fmaf(y, c.z, fmaf(x, bq.z, a.z));
              const float d0 = fmaf(y, f.x, fmaf(x, e.x, d.x));
              const float d1 = fmaf(y, f.y, fmaf(x, e.y, d.y));
              const float d2 = fmaf(y, f.z, fmaf(x, e.z, d.z));
              const float nn = fmaf(n2, n2, fmaf(n1, n1, n0 * n0));
              const float dd = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
              if (nn <= c.w * dd) {
                const float inv = __fdividef(1.0f, dd);
                const float rho2 = nn * inv;
                const float raw = a.w * __expf(-0.5f * rho2);
                const float t = fmaf(f.w, d2, fmaf(e.w, d1, d.w * d0)) * inv;
                if (raw >= kAlphaMin && t >= fc.znear && t >= lo && t < hi) {
                  contrib = true;
                  ts = t;
                  ca = fminf(raw, kAlphaMax);
                  Lnext = by_key ? s.L[k] : -kInf;
                  ev = EvalState{k, n0, n1, n2, d0, d1, d2, inv, rho2};
                }
              }
            }
            // 1. queued entries in front of the new one that nothing later can precede
            release_rounds(q, bl, [&] { return contrib && q.n > 0 && !bl.done && q.ft <= ts && q.ft < Lnext; });
            const bool live = contrib && !bl.done;
            const bool imm = live && (ts < Lnext || !resort);
            bool ins = live && !imm;
            // 2. the new contributor, then the rest below L_next; 3. queue it.
            // A full queue defers the farther of the new entry and its last
            // one to a later pass (exact), or, in the bounded-buffer ablation
            // or when its nearest entry lies at lo, releases the nearer of its
            // front and the new entry.  The lanes of 2 and 3 are disjoint, so
            // their releases share rounds.
            if (imm) bl.blend_new(ca, ev);
            bool early = false;
            if (ins && q.n == kQueue) {
              if (peel && q.ft > lo) {
                if (jnext == kNone) jnext = jfill;
                hi = fmaxf(ts, q.back_t());
                q.drop_from(hi);
                ins = ts < hi;
              } else {
                if (!peel) ++nmis;
                if (ts < q.ft) {
                  bl.blend_new(ca, ev);
                  ins = false;
                } else {
                  early = true;
                }
              }
            }
            release_rounds(q, bl, [&] {
              const bool e = early;
              early = false;
              return e || (imm && q.n > 0 && !bl.done && q.ft < Lnext);
            });
            if (ins && !bl.done) {
              if (q.n == 0) jfill = jk;
              q.insert(ts, ca, bl.payload(k));
            }
            bl.end_item(k);
          }
          // close the pass once no later pair can hold a contributor below hi
          const bool close = open && !bl.done && hi < kInf && s.L[k] >= hi;
          release_rounds(q, bl, [&] { return close && q.n > 0 && !bl.done; });
          if (close) open = false;
          if (__all_sync(0xffffffffu, !open || bl.done)) break;   // warp-uniform
        }
        bl.end_batch(b0, cnt);
      } else if (open && !bl.done) {
        // The first pass takes every pair from the tile's start with no lower
        // window bound; a later one skips the pairs before jfirst (they hold
        // nothing for this pixel's window) and tests lo.
        auto pairs = [&](auto first) {
          constexpr bool FIRST = decltype(first)::value;
          int k0 = 0;
          if constexpr (!FIRST) k0 = jfirst > b0 ? (int)min((uint32_t)cnt, jfirst - b0) : 0;
          const uint32_t* words = s.wbits[threadIdx.x >> 5];
          for (int wd = k0 >> 5; wd * 32 < cnt; ++wd) {
            unsigned m = words[wd];   // warp-uniform
            if (wd == (k0 >> 5)) m &= ~0u << (k0 & 31);
            while (m != 0u) {
              const int k = wd * 32 + __ffs(m) - 1;
              m &= m - 1u;
              const float4 bq = s.b[k];
              if constexpr (!FIRST) {
                if (bq.w < lo) continue;   // its t* lies in front of this pass's window
              }
              ++neval;
              const float4 a = s.a[k], c = s.c[k], d = s.d[k], e = s.e[k], f = s.f[k];
              const float n0 = fmaf(y, c.x, fmaf(x, bq.x, a.x));
              const float n1 = fmaf(y, c.y, fmaf(x, bq.y, a.y));
              const float n2 = fmaf(y, c.z, fmaf(x, bq.z, a.z));
              const float d0 = fmaf(y, f.x, fmaf(x, e.x, d.x));
              const float d1 = fmaf(y, f.y, fmaf(x, e.y, d.y));
              const float d2 = fmaf(y, f.z, fmaf(x, e.z, d.z));
              const float nn = fmaf(n2, n2, fmaf(n1, n1, n0 * n0));
              const float dd = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
              // rho^2 > tau+ rules out alpha >= 1/255 without a division
              if (nn <= c.w * dd) {
                const float inv = __fdividef(1.0f, dd);
                const float rho2 = nn * inv;
                const float raw = a.w * __expf(-0.5f * rho2);
                const float ts = fmaf(f.w, d2, fmaf(e.w, d1, d.w * d0)) * inv;
                if (raw >= kAlphaMin && ts >= fc.znear && (FIRST || ts >= lo) && ts < hi) {
                  const float Lnext = by_key ? s.L[k] : -kInf;
                  const float ca = fminf(raw, kAlphaMax);
                  const EvalState ev{k, n0, n1, n2, d0, d1, d2, inv, rho2};
                  // 1. queued entries in front of the new one that nothing later can precede
                  while (q.n > 0 && !bl.done && q.ft <= ts && q.ft < Lnext) q.release(bl);
                  if (!bl.done) {
                    if (ts < Lnext || !resort) {
                      // 2. the new contributor, then the rest below L_next
                      bl.blend_new(ca, ev);
                      while (q.n > 0 && !bl.done && q.ft < Lnext) q.release(bl);
                    } else {
                      // 3. queue it.  A full queue defers the farther of the new
                      // entry and its last one to a later pass; in the
                      // bounded-buffer ablation, or when its nearest entry lies
                      // at lo, it releases the nearer of its front and the new
                      // entry instead
                      bool insert = true;
                      if (q.n == kQueue) {
                        if (peel && q.ft > lo) {
                          if (jnext == kNone) jnext = jfill;
                          hi = fmaxf(ts, q.back_t());
                          q.drop_from(hi);
                          insert = ts < hi;
                        } else {
                          if (!peel) ++nmis;
                          if (ts < q.ft) {
                            bl.blend_new(ca, ev);
                            insert = false;
                          } else {
                            q.release(bl);
                          }
                        }
                      }
                      if (insert && !bl.done) {
                        if (q.n == 0) jfill = b0 + (uint32_t)k;
                        q.insert(ts, ca, bl.payload(k));
                      }
                    }
                    if constexpr (!FIRST) {
                      // close the pass once no later pair can hold a contributor below hi
                      if (Lnext >= hi) {
                        while (q.n > 0 && !bl.done) q.release(bl);
                        open = false;
                        goto pairs_done;
                      }
                    }
                  }
                  if (bl.done) goto pairs_done;   // blends are the only change of done
                }
              }
            }
          }
          pairs_done:;
        };
        if (lo == -kInf) {
          pairs(std::true_type{});
        } else {
          pairs(std::false_type{});
        }
      }
      __syncthreads();
    }
    if constexpr (CONVERGENT) {
      release_rounds(q, bl, [&] { return q.n > 0 && !bl.done; });
    } else {
      while (q.n > 0 && !bl.done) q.release(bl);
    }
    // another pass for the pixels that deferred contributors
    more = more && !bl.done && hi < kInf;
    if (threadIdx.x == 0) s.start = kNone;
    if (__syncthreads_count(more) == 0) break;
    if (more) {
      lo = hi;
      jfirst = jnext;
      ++npass;
      atomicMin(&s.start, jnext);
    }
    __syncthreads();
    start = s.start;
    first_pass = false;
  }
}

}  // namespace aaag
