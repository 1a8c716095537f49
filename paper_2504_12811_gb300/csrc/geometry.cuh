// Frustum tests in normalised Gaussian space (paper Sec. 3.4, Eq. 18).
//
// A screen-space plane pi_x = (1,0,0,-x) becomes, in the Gaussian's
// normalised space, pi' = T'^T pi_x = fx * t1 + (cx - x) * t3 (Eq. 4-5), with
// t_i the rows of T_view = V T.  Distance to the origin in that space is rho.
// The frustum of a screen rectangle is the intersection of four such
// half-spaces (optionally truncated by the view-space near plane z >= znear,
// the near-plane tile rule of Sec. 3.3).  rho^2 = |u|^2 is strictly convex, so
// its minimum over the frustum is 0 when the mean is inside, else it lies on a
// face, an edge or a vertex: the minimum-norm point of that feature's affine
// hull, provided the point lies in the frustum.  Faces and edges are the
// paper's candidates; near-plane vertices appear once the frustum is
// truncated.  Any feasible candidate is an upper bound of the minimum, so
// candidates are tried cheapest first and the test stops at the first one
// below the threshold.
#pragma once

#include "aaag_internal.cuh"

namespace aaag {

struct Plane {
  float3 n;   // unit normal in Gaussian space
  float h;    // signed distance of the Gaussian's mean (u = 0)
};

__device__ __forceinline__ Plane make_plane(float4 p, float sign) {
  const float3 n = sign * xyz(p);
  const float inv = rsqrtf(fmaxf(dot3(n, n), 1e-36f));
  Plane r;
  r.n = inv * n;
  r.h = sign * p.w * inv;
  return r;
}

// fx * t1 + cxm * t3 with cxm = cx - x0: the plane of screen column x0.
__device__ __forceinline__ float4 screen_plane(float4 ta, float4 t3, float f, float cm) {
  return make_float4(f * ta.x + cm * t3.x, f * ta.y + cm * t3.y, f * ta.z + cm * t3.z,
                     f * ta.w + cm * t3.w);
}

// Feasibility of a candidate with slack: accepting a point marginally outside
// the frustum only lowers the reported minimum, i.e. keeps more tiles.
__device__ __forceinline__ bool inside_plane(const Plane& p, float3 u) {
  return dot3(p.n, u) + p.h >= -1e-4f * (1.0f + fabsf(p.h));
}

// True when min over the frustum of rho^2 < tau.  Planes 0..3 bound
// x >= xlo, x <= xhi, y >= ylo, y <= yhi; plane 4 is z >= znear (NEAR only).
template <bool NEAR>
__device__ __forceinline__ bool frustum_hit(float4 t1, float4 t2, float4 t3, float fx, float fy,
                                            float cx, float cy, float znear, float xlo,
                                            float xhi, float ylo, float yhi, float tau) {
  constexpr int M = NEAR ? 5 : 4;
  Plane P[5];
  P[0] = make_plane(screen_plane(t1, t3, fx, cx - xlo), 1.0f);
  P[1] = make_plane(screen_plane(t1, t3, fx, cx - xhi), -1.0f);
  P[2] = make_plane(screen_plane(t2, t3, fy, cy - ylo), 1.0f);
  P[3] = make_plane(screen_plane(t2, t3, fy, cy - yhi), -1.0f);
  P[4] = make_plane(make_float4(t3.x, t3.y, t3.z, t3.w - znear), 1.0f);

  // mean inside the frustum: minimum 0
  bool all_in = true;
#pragma unroll
  for (int k = 0; k < M; ++k) all_in &= P[k].h >= 0.0f;
  if (all_in) return tau > 0.0f;

  // faces: projection of the origin onto each plane
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float v = P[j].h * P[j].h;
    if (v < tau) {
      const float3 u = (-P[j].h) * P[j].n;
      bool ok = true;
#pragma unroll
      for (int k = 0; k < M; ++k)
        if (k != j) ok &= inside_plane(P[k], u);
      if (ok) return true;
    }
  }

  // edges: intersection lines of adjacent planes
  constexpr int kEdges = NEAR ? 8 : 4;
  const int ea[8] = {0, 0, 1, 1, 0, 1, 2, 3};
  const int eb[8] = {2, 3, 2, 3, 4, 4, 4, 4};
#pragma unroll
  for (int e = 0; e < kEdges; ++e) {
    const Plane& A = P[ea[e]];
    const Plane& B = P[eb[e]];
    const float3 d = cross3(A.n, B.n);
    const float dd = dot3(d, d);
    if (dd > 1e-12f) {
      const float3 num = A.h * B.n - B.h * A.n;
      const float inv = 1.0f / dd;
      const float v = dot3(num, num) * inv;
      if (v < tau) {
        const float3 u = inv * cross3(d, num);
        bool ok = true;
#pragma unroll
        for (int k = 0; k < M; ++k)
          if (k != ea[e] && k != eb[e]) ok &= inside_plane(P[k], u);
        if (ok) return true;
      }
    }
  }

  if (NEAR) {
    // vertices: near plane with one x plane and one y plane
    const int va[4] = {0, 0, 1, 1};
    const int vb[4] = {2, 3, 2, 3};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const Plane& A = P[va[e]];
      const Plane& B = P[vb[e]];
      const Plane& C = P[4];
      const float3 bc = cross3(B.n, C.n), ca = cross3(C.n, A.n), ab = cross3(A.n, B.n);
      const float det = dot3(A.n, bc);
      if (fabsf(det) > 1e-6f) {
        const float3 u = (-1.0f / det) * (A.h * bc + B.h * ca + C.h * ab);
        if (dot3(u, u) < tau) {
          bool ok = true;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (k != va[e] && k != vb[e]) ok &= inside_plane(P[k], u);
          if (ok) return true;
        }
      }
    }
  }
  return false;
}

// Tile test for a Gaussian whose tau-ellipsoid lies entirely beyond the near
// plane (so in front of the camera).  A screen point (x, y) sees the
// Gaussian's maximum below tau exactly where
//     F(x, y) = |num(x, y)|^2 - tau |d(x, y)|^2 <= 0,
// with num = h1 n2 - h2 n1 and d = n1 x n2 the affine functions of the pixel
// planes of Eq. 4-5 (rho^2 = |num|^2 / |d|^2).  This region is the
// ellipsoid's silhouette, a convex ellipse, so min over the frustum of rho^2 <
// tau (Eq. 18) holds iff the tile rectangle meets it: iff the projected mean
// (rho = 0) lies in the tile or F <= 0 somewhere on one of the four edges.  F
// along an edge is a convex quadratic in the edge parameter, minimised at a
// clamped vertex.  Uniform work, no square roots; same decision as the
// frustum minimum up to rounding.
struct ConicTester {
  float3 Nx, Ny, Dx, Dy;   // d num/dx, d num/dy, d d/dx, d d/dy
  float4 t1, t2, t3;
  float fx, fy, cx, cy, tau, ax, ay, mx, my;

  __device__ __forceinline__ void init(float4 t1_, float4 t2_, float4 t3_, float fx_, float fy_, float cx_,
                                       float cy_, float tau_) {
    t1 = t1_;
    t2 = t2_;
    t3 = t3_;
    fx = fx_;
    fy = fy_;
    cx = cx_;
    cy = cy_;
    tau = tau_;
    // planes at x = 0, y = 0: U = fx t1 + cx t3, W = fy t2 + cy t3
    const float3 T3 = f3(t3.x, t3.y, t3.z);
    const float3 Uv = f3(fx * t1.x + cx * t3.x, fx * t1.y + cx * t3.y, fx * t1.z + cx * t3.z);
    const float Uw = fx * t1.w + cx * t3.w;
    const float3 Wv = f3(fy * t2.x + cy * t3.x, fy * t2.y + cy * t3.y, fy * t2.z + cy * t3.z);
    const float Ww = fy * t2.w + cy * t3.w;
    Nx = Ww * T3 - t3.w * Wv;
    Ny = t3.w * Uv - Uw * T3;
    Dx = cross3(Wv, T3);
    Dy = cross3(T3, Uv);
    ax = dot3(Nx, Nx) - tau * dot3(Dx, Dx);
    ay = dot3(Ny, Ny) - tau * dot3(Dy, Dy);
    mx = fx * t1.w / t3.w + cx;   // projected mean
    my = fy * t2.w / t3.w + cy;
  }

  // min over t in [0, len] of F(p + t e) = a t^2 + 2 b t + c <= 0, with
  // num(p) = n, d(p) = d: the minimum is at an end or at the clamped vertex
  __device__ __forceinline__ bool edge(float3 n, float3 d, float3 En, float3 Ed, float a, float len) const {
    const float b = dot3(n, En) - tau * dot3(d, Ed);
    const float c = dot3(n, n) - tau * dot3(d, d);
    float m = fminf(c, fmaf(fmaf(a, len, 2.0f * b), len, c));
    if (a > 0.0f) {
      const float t = fminf(fmaxf(-b / a, 0.0f), len);
      m = fminf(m, fmaf(fmaf(a, t, 2.0f * b), t, c));
    }
    return m <= 0.0f;
  }

  __device__ __forceinline__ bool hit(float x0, float y0, float x1, float y1) const {
    if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
    // num and d at the corner (x0, y0), from the planes of that corner
    const float3 T3 = f3(t3.x, t3.y, t3.z);
    const float cxm = cx - x0, cym = cy - y0;
    const float3 Uv = f3(fmaf(cxm, t3.x, fx * t1.x), fmaf(cxm, t3.y, fx * t1.y), fmaf(cxm, t3.z, fx * t1.z));
    const float Uw = fmaf(cxm, t3.w, fx * t1.w);
    const float3 Wv = f3(fmaf(cym, t3.x, fy * t2.x), fmaf(cym, t3.y, fy * t2.y), fmaf(cym, t3.z, fy * t2.z));
    const float Ww = fmaf(cym, t3.w, fy * t2.w);
    const float3 n00 = Uw * Wv - Ww * Uv;
    const float3 d00 = cross3(Uv, Wv);
    const float w = x1 - x0, h = y1 - y0;
    const float3 n10 = n00 + w * Nx, d10 = d00 + w * Dx;
    const float3 n01 = n00 + h * Ny, d01 = d00 + h * Dy;
    return edge(n00, d00, Ny, Dy, ay, h) || edge(n10, d10, Ny, Dy, ay, h) || edge(n00, d00, Nx, Dx, ax, w) ||
           edge(n01, d01, Nx, Dx, ax, w);
  }
};

// Cutoff used by the conservative geometric tests: tau slightly inflated so
// that float32 rounding never drops a tile or a Gaussian with alpha >= 1/255.
__device__ __forceinline__ float inflate_tau(float tau) { return tau * (1.0f + 1e-4f) + 1e-4f; }

// The aux word holds the inclusive pixel-centre ranges [x0, x1] x [y0, y1]
// (16 bits each) of a visible Gaussian; its tile rectangle is the tiles
// holding those pixels.
__device__ __forceinline__ void unpack_rect(uint4 a, int& tx0, int& ty0, int& tx1, int& ty1) {
  tx0 = (int)(a.x & 0xffffu) / kTile;
  ty0 = (int)(a.x >> 16) / kTile;
  tx1 = (int)(a.y & 0xffffu) / kTile;
  ty1 = (int)(a.y >> 16) / kTile;
}

}  // namespace aaag
