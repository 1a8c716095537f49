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

// Tile test for a Gaussian whose tau-ellipsoid reaches in front of z_near.
// A pixel receives such a Gaussian only where rho^2 <= tau and the depth t*
// of the maximum is not closer than the near plane (Sec. 3.3).  On the ray
// of screen point (x, y) the maximum is the foot u* = (d x num) / |d|^2 of
// the perpendicular from the mean (origin of normalised space), so
// t* = T3.u* + t3.w and, multiplying through by |d|^2 > 0,
//     F(x, y) = |num|^2 - tau |d|^2 <= 0   and
//     G(x, y) = (t3.w - z_near) |d|^2 + T3.(d x num) >= 0,
// both quadratic in (x, y).  A rectangle meets that set iff
//   (a) it holds one of two interior witnesses: the projected mean (rho = 0,
//       t* = t3.w) when t3.w >= z_near, or the screen point of smallest rho
//       on the curve t* = z_near.  The feet u* of all rays from the camera c
//       lie on the sphere with diameter [0, c], so that curve is the circle
//       where this sphere meets the plane z = z_near, and rho^2 = |u*|^2 has
//       a single local minimum on it.  A part of the set lying inside the
//       rectangle without touching its edges attains its smallest rho either
//       at the projected mean or at that circle point; or
//   (b) max(F, -G) <= 0 somewhere on one of its edges.  Along an edge both
//       are quadratics in the edge parameter, and the minimum of their
//       maximum lies at an end, at the vertex of F or of G, or where
//       F + G = 0.  Every candidate is a point of the edge, so evaluating a
//       spurious one (a vertex of a concave branch, a clamped root) never
//       accepts a tile wrongly; they are all evaluated without branches.
// Tighter than the frustum minimum truncated at z_near (Eq. 18), which also
// keeps tiles seeing only the cap of the ellipsoid in front of the plane,
// where every ray's maximum lies closer than z_near.  z_near is lowered by
// 1e-3 relative so that float32 rounding never drops a contributing tile.
struct NearTester {
  float3 Nx, Ny, Dx, Dy;   // d num/dx, d num/dy, d d/dx, d d/dy
  float4 t1, t2, t3;
  float fx, fy, cx, cy, tau, zr;
  float mx, my, wx, wy;    // witnesses; NaN when absent

  __device__ __forceinline__ void init(float4 t1_, float4 t2_, float4 t3_, float fx_, float fy_, float cx_,
                                       float cy_, float znear, float tau_) {
    t1 = t1_;
    t2 = t2_;
    t3 = t3_;
    fx = fx_;
    fy = fy_;
    cx = cx_;
    cy = cy_;
    tau = tau_;
    const float zn = znear * (1.0f - 1e-3f);
    const float3 T3 = f3(t3.x, t3.y, t3.z);
    const float3 Uv = f3(fx * t1.x + cx * t3.x, fx * t1.y + cx * t3.y, fx * t1.z + cx * t3.z);
    const float Uw = fx * t1.w + cx * t3.w;
    const float3 Wv = f3(fy * t2.x + cy * t3.x, fy * t2.y + cy * t3.y, fy * t2.z + cy * t3.z);
    const float Ww = fy * t2.w + cy * t3.w;
    Nx = Ww * T3 - t3.w * Wv;
    Ny = t3.w * Uv - Uw * T3;
    Dx = cross3(Wv, T3);
    Dy = cross3(T3, Uv);
    zr = t3.w - zn;
    const float nan = __int_as_float(0x7fffffff);
    // witness 1: the projected mean
    const bool mean_ok = t3.w >= zn;
    mx = mean_ok ? fx * t1.w / t3.w + cx : nan;
    my = mean_ok ? fy * t2.w / t3.w + cy : nan;
    // witness 2: camera c in normalised space (A c + m = 0, A with rows
    // t_i.xyz, m = view mean), then the circle point closest to the origin
    const float3 a1 = f3(t1.x, t1.y, t1.z), a2 = f3(t2.x, t2.y, t2.z);
    const float3 c23 = cross3(a2, T3), c31 = cross3(T3, a1), c12 = cross3(a1, a2);
    const float det = dot3(a1, c23);
    const float3 h = (-0.5f / det) * (t1.w * c23 + t2.w * c31 + t3.w * c12);   // c / 2
    const float iq = rsqrtf(dot3(T3, T3));
    const float3 k = iq * T3;
    const float hk = dot3(h, k);
    const float dist = hk - (zn - t3.w) * iq;   // sphere centre to the plane
    const float rc2 = dot3(h, h) - dist * dist;
    float3 hp = h - hk * k;                      // direction of the circle centre from the origin's foot
    float hpn = dot3(hp, hp);
    if (!(hpn > 1e-12f * dot3(h, h))) {
      // rho constant on the circle: any point of it will do
      hp = cross3(k, fabsf(k.x) < 0.9f ? f3(1.0f, 0.0f, 0.0f) : f3(0.0f, 1.0f, 0.0f));
      hpn = dot3(hp, hp);
    }
    const float3 w = (h - dist * k) - (sqrtf(fmaxf(rc2, 0.0f)) * rsqrtf(hpn)) * hp;
    const float wz = dot3(T3, w) + t3.w;
    const bool w_ok = rc2 >= 0.0f && dot3(w, w) <= tau && wz > 0.0f;
    wx = w_ok ? fx * (dot3(a1, w) + t1.w) / wz + cx : nan;
    wy = w_ok ? fy * (dot3(a2, w) + t2.w) / wz + cy : nan;
  }

  __device__ __forceinline__ float3 T3() const { return f3(t3.x, t3.y, t3.z); }
  __device__ __forceinline__ float F(float3 n, float3 d) const { return dot3(n, n) - tau * dot3(d, d); }
  __device__ __forceinline__ float G(float3 n, float3 d) const {
    return fmaf(zr, dot3(d, d), dot3(n, cross3(T3(), d)));
  }

  // Does max(F, -G) <= 0 hold at some point of the edge p + t e, t in
  // [0, len], with num(p) = n, d(p) = d, F(p) = fc, G(p) = gc, and
  // num' = En, d' = Ed along it?  F and G are a t^2 + 2 b t + c there, with
  // G's quadratic coefficient zr |Ed|^2 + T3.(Ed x En).
  __device__ __forceinline__ bool edge(float3 n, float3 d, float fc, float gc, float3 En, float3 Ed,
                                       float len) const {
    const float3 t3v = T3();
    const float ded = dot3(d, Ed);
    const float fa = F(En, Ed);
    const float ga = fmaf(zr, dot3(Ed, Ed), dot3(t3v, cross3(Ed, En)));
    const float fb = dot3(n, En) - tau * ded;
    const float gb = fmaf(zr, ded, 0.5f * (dot3(t3v, cross3(d, En)) + dot3(t3v, cross3(Ed, n))));
    const float a = fa + ga, b = fb + gb, c = fc + gc;
    const float q = -(b + copysignf(sqrtf(fmaxf(fmaf(b, b, -a * c), 0.0f)), b));
    const float cand[4] = {__fdividef(-fb, fa), __fdividef(-gb, ga), __fdividef(q, a), __fdividef(c, q)};
    bool hit = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float t = fminf(fmaxf(cand[j], 0.0f), len);
      const float Ft = fmaf(fmaf(fa, t, 2.0f * fb), t, fc);
      const float Gt = fmaf(fmaf(ga, t, 2.0f * gb), t, gc);
      hit |= (Ft <= 0.0f) & (Gt >= 0.0f);
    }
    return hit;
  }

  __device__ __forceinline__ bool hit(float x0, float y0, float x1, float y1) const {
    // NaN witnesses fail every comparison
    if ((mx >= x0) & (mx <= x1) & (my >= y0) & (my <= y1)) return true;
    if ((wx >= x0) & (wx <= x1) & (wy >= y0) & (wy <= y1)) return true;
    const float cxm = cx - x0, cym = cy - y0;
    const float3 Uv = f3(fmaf(cxm, t3.x, fx * t1.x), fmaf(cxm, t3.y, fx * t1.y), fmaf(cxm, t3.z, fx * t1.z));
    const float Uw = fmaf(cxm, t3.w, fx * t1.w);
    const float3 Wv = f3(fmaf(cym, t3.x, fy * t2.x), fmaf(cym, t3.y, fy * t2.y), fmaf(cym, t3.z, fy * t2.z));
    const float Ww = fmaf(cym, t3.w, fy * t2.w);
    const float w = x1 - x0, h = y1 - y0;
    // corner (x0, y0), then the top and left edges from it
    const float3 n00 = Uw * Wv - Ww * Uv, d00 = cross3(Uv, Wv);
    const float f00 = F(n00, d00), g00 = G(n00, d00);
    if ((f00 <= 0.0f) & (g00 >= 0.0f)) return true;
    if (edge(n00, d00, f00, g00, Nx, Dx, w) || edge(n00, d00, f00, g00, Ny, Dy, h)) return true;
    // corner (x1, y0) and the right edge
    const float3 n10 = n00 + w * Nx, d10 = d00 + w * Dx;
    const float f10 = F(n10, d10), g10 = G(n10, d10);
    if ((f10 <= 0.0f) & (g10 >= 0.0f)) return true;
    if (edge(n10, d10, f10, g10, Ny, Dy, h)) return true;
    // corner (x0, y1) and the bottom edge (its far end (x1, y1) is a candidate)
    const float3 n01 = n00 + h * Ny, d01 = d00 + h * Dy;
    const float f01 = F(n01, d01), g01 = G(n01, d01);
    if ((f01 <= 0.0f) & (g01 >= 0.0f)) return true;
    return edge(n01, d01, f01, g01, Nx, Dx, w);
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
