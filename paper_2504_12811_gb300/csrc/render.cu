// K5: per-pixel 3D evaluation, per-pixel re-sort and compositing (paper
// Sec. 3.1 'Evaluation in 3D', 'Blending Sort Order'; Sec. 4 implementation
// details: per-ray sorting retained from hierarchical rasterisation).
//
// One 256-thread block per 16x16 tile, one thread per pixel.  The tile's pairs
// arrive sorted by (tile, front depth of the Gaussian).  They are staged in
// shared memory in batches of 256: each thread converts one Gaussian's record
// into the coefficients of the two pixel planes, relative to the tile origin.
//
// For pixel (x, y), with U = fx t1 + (cx - x_t) t3 and W = fy t2 + (cy - y_t)
// t3 (t_i rows of T_view, x_t the tile origin), the transformed planes of
// Eq. 5 are (n1, h1) = U - x t3 and (n2, h2) = W - y t3.  Both
//     num = h1 n2 - h2 n1  and  d = n1 x n2
// are affine in (x, y) (the xy terms cancel), so rho^2 = |num|^2 / |d|^2 costs
// 12 FMAs plus two dot products per pixel.  d is parallel to the ray direction
// in Gaussian space; the view depth of the maximum is t* = g.d / |d|^2 with
// g = fx fy adj(A) mu_v (A = Rv R S').
//
// Per-pixel ordering: contributors (alpha >= 1/255, t* >= znear) go into a
// small register buffer sorted by (t*, arrival).  Pairs arrive with
// non-decreasing key L (a lower bound of every later contributor's t*), so a
// buffered entry with t* < L can never be overtaken and is blended at once.
// Only when the buffer is full is its front blended early (counted as a
// potential misorder).  Blending stops before the contributor that would take
// transmittance below 1e-4.
#include <cuda_runtime.h>

#include "aaag_internal.cuh"

namespace aaag {
namespace {

constexpr int kBuf = 16;   // per-pixel re-sort buffer entries

struct Staged {
  // 24 floats per Gaussian, stored as 6 float4 planes of shared memory
  float4 a;  // N0.xyz, o_hat
  float4 b;  // Nx.xyz, L (lower bound of t* for this and later pairs)
  float4 c;  // Ny.xyz, gid (as bits)
  float4 d;  // D0.xyz, -
  float4 e;  // Dx.xyz, -
  float4 f;  // Dy.xyz, -
  float4 g;  // G.xyz, -
};

__device__ __forceinline__ float decode_depth(uint32_t key, const FrameConst& fc) {
  const uint32_t dk = key & ((fc.depth_bits >= 32) ? 0xffffffffu : ((1u << fc.depth_bits) - 1u));
  return __uint_as_float((dk << fc.depth_shift) + fc.znear_bits);
}

template <int B>
__global__ void __launch_bounds__(kTilePixels)
render_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
              const uint32_t* __restrict__ vals, const Record* __restrict__ rec, FrameConst fc,
              float* __restrict__ rgb, float* __restrict__ alpha, float* __restrict__ final_T,
              uint32_t* __restrict__ n_blended, unsigned long long* __restrict__ stats) {
  __shared__ float4 s_a[kTilePixels], s_b[kTilePixels], s_c[kTilePixels], s_d[kTilePixels],
      s_e[kTilePixels], s_f[kTilePixels], s_g[kTilePixels];

  const int tile = blockIdx.x;
  const int tx = tile % fc.tiles_x, ty = tile / fc.tiles_x;
  const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  const bool in_image = px < fc.W && py < fc.H;
  const float x = (float)lx + 0.5f, y = (float)ly + 0.5f;   // tile-relative pixel centre
  const float cxm = fc.cx - (float)(tx * kTile), cym = fc.cy - (float)(ty * kTile);
  const float fxfy = fc.fx * fc.fy;

  const uint2 range = ranges[tile];
  float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
  bool done = !in_image;
  uint32_t nblend = 0, nmis = 0;
  unsigned long long neval = 0;

  float bt[B], ba[B];
  uint32_t bg[B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    bt[i] = __int_as_float(0x7f800000);   // +inf: empty
    ba[i] = 0.0f;
    bg[i] = 0u;
  }
  int nb = 0;

  auto blend = [&](float a, uint32_t gid) {
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
  };
  auto pop_front = [&]() {
#pragma unroll
    for (int i = 0; i < B - 1; ++i) {
      bt[i] = bt[i + 1];
      ba[i] = ba[i + 1];
      bg[i] = bg[i + 1];
    }
    bt[B - 1] = __int_as_float(0x7f800000);
    --nb;
  };

  for (uint32_t b0 = range.x; b0 < range.y; b0 += kTilePixels) {
    if (__syncthreads_count(done) == kTilePixels) break;
    // ---- stage one batch of Gaussians
    const uint32_t j = b0 + threadIdx.x;
    if (j < range.y) {
      const uint32_t gid = vals[j];
      const float L = decode_depth(keys[j], fc);
      const float4* r = reinterpret_cast<const float4*>(rec + gid);
      const float4 t1 = __ldg(r + 0), t2 = __ldg(r + 1), t3 = __ldg(r + 2), cw = __ldg(r + 3);
      const float3 T3 = f3(t3.x, t3.y, t3.z);
      const float3 Uv = f3(fc.fx * t1.x + cxm * t3.x, fc.fx * t1.y + cxm * t3.y, fc.fx * t1.z + cxm * t3.z);
      const float Uw = fc.fx * t1.w + cxm * t3.w;
      const float3 Wv = f3(fc.fy * t2.x + cym * t3.x, fc.fy * t2.y + cym * t3.y, fc.fy * t2.z + cym * t3.z);
      const float Ww = fc.fy * t2.w + cym * t3.w;
      const float3 N0 = Uw * Wv - Ww * Uv;
      const float3 Nx = Ww * T3 - t3.w * Wv;
      const float3 Ny = t3.w * Uv - Uw * T3;
      const float3 D0 = cross3(Uv, Wv);
      const float3 Dx = cross3(Wv, T3);
      const float3 Dy = cross3(T3, Uv);
      const float3 A1 = f3(t1.x, t1.y, t1.z), A2 = f3(t2.x, t2.y, t2.z);
      const float3 G = fxfy * (t1.w * cross3(A2, T3) + t2.w * cross3(T3, A1) + t3.w * cross3(A1, A2));
      s_a[threadIdx.x] = make_float4(N0.x, N0.y, N0.z, cw.w);
      s_b[threadIdx.x] = make_float4(Nx.x, Nx.y, Nx.z, L);
      s_c[threadIdx.x] = make_float4(Ny.x, Ny.y, Ny.z, __uint_as_float(gid));
      s_d[threadIdx.x] = make_float4(D0.x, D0.y, D0.z, 0.0f);
      s_e[threadIdx.x] = make_float4(Dx.x, Dx.y, Dx.z, 0.0f);
      s_f[threadIdx.x] = make_float4(Dy.x, Dy.y, Dy.z, 0.0f);
      s_g[threadIdx.x] = make_float4(G.x, G.y, G.z, 0.0f);
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kTilePixels, range.y - b0);
    if (!done) {
      neval += (unsigned long long)cnt;
      for (int k = 0; k < cnt; ++k) {
        const float4 a = s_a[k], bq = s_b[k], c = s_c[k], d = s_d[k], e = s_e[k], f = s_f[k];
        const float n0 = fmaf(y, c.x, fmaf(x, bq.x, a.x));
        const float n1 = fmaf(y, c.y, fmaf(x, bq.y, a.y));
        const float n2 = fmaf(y, c.z, fmaf(x, bq.z, a.z));
        const float d0 = fmaf(y, f.x, fmaf(x, e.x, d.x));
        const float d1 = fmaf(y, f.y, fmaf(x, e.y, d.y));
        const float d2 = fmaf(y, f.z, fmaf(x, e.z, d.z));
        const float nn = fmaf(n2, n2, fmaf(n1, n1, n0 * n0));
        const float dd = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
        const float inv = __fdividef(1.0f, dd);
        const float rho2 = nn * inv;
        const float raw = a.w * __expf(-0.5f * rho2);
        if (raw >= kAlphaMin) {
          const float4 g = s_g[k];
          const float ts = fmaf(g.z, d2, fmaf(g.y, d1, g.x * d0)) * inv;
          if (ts >= fc.znear) {
            const float L = bq.w;
            // release buffered entries no later pair can precede
            while (nb > 0 && bt[0] < L && !done) {
              blend(ba[0], bg[0]);
              pop_front();
            }
            if (done) break;
            float ct = ts, ca = fminf(raw, kAlphaMax);
            uint32_t cgid = __float_as_uint(c.w);
            if (nb == B) {
              // full: release the nearer of the front entry and the new one
              // early (a later pair may still precede it: potential misorder)
              ++nmis;
              if (ct < bt[0]) {
                blend(ca, cgid);
                if (done) break;
                continue;
              }
              blend(ba[0], bg[0]);
              pop_front();
              if (done) break;
            }
            // sorted insert (ties keep arrival order)
#pragma unroll
            for (int i = 0; i < B; ++i) {
              const bool sw = ct < bt[i];
              const float t0 = bt[i], a0 = ba[i];
              const uint32_t g0 = bg[i];
              bt[i] = sw ? ct : t0;
              ba[i] = sw ? ca : a0;
              bg[i] = sw ? cgid : g0;
              ct = sw ? t0 : ct;
              ca = sw ? a0 : ca;
              cgid = sw ? g0 : cgid;
            }
            ++nb;
          }
        }
      }
    }
    __syncthreads();
  }
  // drain the buffer in order
  while (nb > 0 && !done) {
    blend(ba[0], bg[0]);
    pop_front();
  }

  if (in_image) {
    const size_t HW = (size_t)fc.W * fc.H;
    const size_t p = (size_t)py * fc.W + px;
    rgb[p] = Cr + T * fc.bg[0];
    rgb[HW + p] = Cg + T * fc.bg[1];
    rgb[2 * HW + p] = Cb + T * fc.bg[2];
    alpha[p] = 1.0f - T;
    final_T[p] = T;
    n_blended[p] = nblend;
  }
  // block-reduced counters
  unsigned long long e = neval, bl = nblend, mi = nmis;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    bl += __shfl_xor_sync(0xffffffffu, bl, o);
    mi += __shfl_xor_sync(0xffffffffu, mi, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicAdd(&stats[kStatEvaluations], e);
    if (bl) atomicAdd(&stats[kStatBlended], bl);
    if (mi) atomicAdd(&stats[kStatMisorders], mi);
  }
}

}  // namespace

aaag_status launch_render(aaag_workspace* ws, float* rgb, float* alpha, cudaStream_t st) {
  const int alt = ws->sorted_in_alt;
  render_kernel<kBuf><<<(unsigned)ws->n_tiles, kTilePixels, 0, st>>>(
      ws->ranges, ws->keys[alt], ws->vals[alt], ws->records, ws->fc, rgb, alpha, ws->final_T,
      ws->n_blended, ws->stats);
  return check_launch("render");
}

}  // namespace aaag
