// K1: per-Gaussian preprocessing for one view (paper Sec. 3.2-3.4).
//
// One thread per Gaussian; reads the scene arrays once (colour coefficients
// only for Gaussians that survive), writes a 64-byte record and a 16-byte aux
// word per visible Gaussian.  Memory-bound by design: everything else is a few
// hundred FP32 operations per Gaussian.
#include <cmath>

#include <algorithm>

#include "aaag_internal.cuh"
#include "geometry.cuh"

namespace aaag {
namespace {

constexpr float kPi = 3.14159265358979f;

// Real SH (orthonormal, Condon-Shortley phase) expanded as polynomials in the
// unit direction (x, y, z).  Constants are the normalisations
// K_l^m * sqrt(2) (m != 0) of the associated-Legendre definition:
//   1/(2 sqrt(pi)); sqrt(3/(4 pi));
//   sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4;
//   sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4,
//   sqrt(105/pi)/4.
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

__device__ __forceinline__ void sh_basis(float x, float y, float z, int deg, float* Y) {
  Y[0] = kY00;
  if (deg < 1) return;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.0f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.0f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.0f * zz - xx - yy);
  Y[12] = kY3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[13] = -kY3c * x * (4.0f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.0f * yy);
}

// Screen interval of one axis from the view-space tangent planes (Sec. 3.3,
// Eq. 14-17).  Ai: row i of A = Rv R S' (view axis i of the Gaussian frame),
// A3: the z row; mi, mz: view-space mean.  Returns false when the interval is
// empty (the Gaussian lies behind the camera on this axis).  When the whole
// tau-ellipsoid lies in front of the camera plane (in_front), x/z is
// continuous over it and both tangent angles lie in (-pi/2, pi/2) around the
// mean's, so the rotation step of Eq. 16 only orders them: the bounds are the
// two slopes tan(theta) themselves, without the angles (the clamp of Eq. 17
// is left to the pixel ranges, which only widens the interval).
__device__ __forceinline__ bool axis_bounds(float3 Ai, float3 A3, float mi, float mz, float tau,
                                            float f, float c, float eps, bool in_front, float& p1, float& p2) {
  const float sii = tau * dot3(Ai, Ai) - mi * mi;
  const float si3 = tau * dot3(Ai, A3) - mi * mz;
  const float S33 = tau * dot3(A3, A3);
  const float s33 = S33 - mz * mz;
  // s13^2 - s11 s33 without the mu^4 cancellation:
  //   tau * (|Ai mz - A3 mi|^2 - tau |Ai x A3|^2)
  const float3 w = mz * Ai - mi * A3;
  const float3 cr = cross3(Ai, A3);
  const float D = tau * (dot3(w, w) - tau * dot3(cr, cr));
  const float lim = 0.5f * kPi - eps;
  float a1 = -lim, a2 = lim;
  const bool degenerate = !(D >= 0.0f) || fabsf(s33) <= 1e-5f * (S33 + mz * mz);
  if (!degenerate) {
    // roots of s33 tan^2 - 2 s13 tan + s11 = 0, numerically stable form
    const float sq = sqrtf(D);
    const float q = si3 + copysignf(sq, si3);
    if (q != 0.0f && in_front) {
      const float ta = q / s33, tb = sii / q;
      p1 = f * fminf(ta, tb) + c;
      p2 = f * fmaxf(ta, tb) + c;
      p1 -= 0.01f + 1e-5f * fabsf(p1);
      p2 += 0.01f + 1e-5f * fabsf(p2);
      return true;
    }
    if (q != 0.0f) {
      const float ra = atanf(q / s33);
      const float rb = atanf(sii / q);
      const float amu = atan2f(mi, mz);
      // representative of a root angle in (amu - pi, amu]
      auto lo = [&](float r) {
        const float dlt = amu - r;
        return amu - (dlt - kPi * floorf(dlt / kPi));
      };
      float b1 = lo(ra), b2 = lo(rb) + kPi;
      if (b2 - b1 >= kPi) {
        b1 = lo(rb);
        b2 = lo(ra) + kPi;
      }
      a1 = fmaxf(-lim, b1);
      a2 = fminf(lim, b2);
      if (a1 > a2) return false;
    }
  }
  p1 = f * tanf(a1) + c;
  p2 = f * tanf(a2) + c;
  // margin for float32 rounding of the angles
  p1 -= 0.01f + 1e-5f * fabsf(p1);
  p2 += 0.01f + 1e-5f * fabsf(p2);
  return true;
}

// Screen interval of one axis for a Gaussian whose tau-ellipsoid E reaches in
// front of z_near, intersected into [p1, p2].  Only E's part beyond the near
// plane is seen (Sec. 3.3), and the projection of that convex part is
// bounded, whereas the tangent-plane bounds above grow to the whole screen
// once E crosses the camera plane.  x/z over E and z >= z_near attains its
// extremes either on the rim (the disc of E in the plane z = z_near, centre
// s0 A3, s0 = (z_near - m_z)/|A3|^2, radius^2 tau - s0^2 |A3|^2) or at the
// contact point of a tangent plane x = s z (a root of
// (m_i - s m_z)^2 = tau |Ai - s A3|^2, Eq. 14 in tangent form) lying at
// z >= z_near; the interval spans all such candidates.  Roots are kept as
// fractions so that the contact depth is computed without the slope itself.
__device__ __forceinline__ void near_bounds(float3 Ai, float3 A3, float mi, float mz, float tau, float z_lo,
                                            float z_hi, float f, float c, float znear, float& p1, float& p2) {
  const float q = dot3(A3, A3), ai3 = dot3(Ai, A3), aii = dot3(Ai, Ai);
  const float s0 = (znear - mz) / q;
  const float r2 = fmaxf(fmaf(-s0 * s0, q, tau), 0.0f);
  const float perp2 = fmaxf(aii - ai3 * ai3 / q, 0.0f);
  const float xc = fmaf(s0, ai3, mi), ext = sqrtf(r2 * perp2);
  float lo = (xc - ext) / znear, hi = (xc + ext) / znear;
  const float3 w = mz * Ai - mi * A3;
  const float3 cr = cross3(Ai, A3);
  const float D = tau * (dot3(w, w) - tau * dot3(cr, cr));
  if (D >= 0.0f) {
    // a2 s^2 - 2 b s + a0 = 0 with a2 = m_z^2 - tau |A3|^2 = z_lo z_hi
    const float ei = sqrtf(tau * aii);
    const float a2 = z_lo * z_hi, a0 = (mi - ei) * (mi + ei);
    const float b = fmaf(mi, mz, -tau * ai3);
    const float qq = b + copysignf(sqrtf(D), b);
    const float num[2] = {qq, a0}, den[2] = {a2, qq};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      // tangent plane (den Ai - num A3).u + (den m_i - num m_z) = 0
      const float3 n = den[k] * Ai - num[k] * A3;
      const float h = den[k] * mi - num[k] * mz;
      const float nn = dot3(n, n);
      const float zc = mz - h * dot3(A3, n) / nn;
      if (nn > 0.0f && zc >= znear * (1.0f - 1e-3f)) {
        const float s = num[k] / den[k];
        lo = fminf(lo, s);
        hi = fmaxf(hi, s);
      }
    }
  }
  float q1 = f * lo + c, q2 = f * hi + c;
  q1 -= 0.01f + 1e-5f * fabsf(q1);
  q2 += 0.01f + 1e-5f * fabsf(q2);
  p1 = fmaxf(p1, q1);
  p2 = fminf(p2, q2);
}

// Pixels whose centre (i + 1/2) lies in the screen interval [p1, p2],
// clamped to the image: the only pixels of this axis that can see the
// Gaussian.  Returns false when there is none.
__device__ __forceinline__ bool pixel_range(float p1, float p2, int size, int& i0, int& i1) {
  const float lo = fmaxf(p1 - 0.5f, 0.0f);
  const float hi = fminf(p2 - 0.5f, (float)(size - 1));
  if (!(lo <= hi)) return false;   // also rejects NaN bounds
  i0 = (int)ceilf(lo);
  i1 = (int)floorf(hi);
  return i0 <= i1;
}

// Ablation without 3D evaluation (Sec. 5): the Gaussian is splatted in 2D.
// Its filtered view-space covariance A A^T (A = Rv R S') is projected with
// the Jacobian J of the perspective map at the mean (EWA), Sigma' = (J A)(J A)^T
// (2x2, no extra screen-space dilation), and the pixel (x, y) sees
// rho^2 = D^T Sigma'^-1 D, D = (x, y) - projected mean, at depth t* = z.
// With the rows (A1' | x_v), (A2' | y_v), (0 | z_v), the plane form of
// Eq. 4-5 used by every later stage gives exactly this: n1 = fx A1',
// h1 = z (m_x - x), n2 = fy A2', h2 = z (m_y - y), so d = n1 x n2 is constant,
// t* = G.d/|d|^2 = z and |num|^2/|d|^2 = |L^T D|^2 when A1' = |d| (l21, l22, 0)
// / (z fx), A2' = -|d| (l11, 0, 0) / (z fy), |d| = z^2 / (l11 l22), with
// L L^T = Sigma'^-1 (Cholesky).  Writes the rows and the pixel-centre ranges
// of the ellipse rho^2 <= tau; false when the splat is degenerate or off the
// image.
__device__ __forceinline__ bool ewa_record(float3 A1, float3 A2, float3 A3, float vx, float vy, float vz,
                                           float tau_c, const FrameConst& fc, float4& t1, float4& t2,
                                           float4& t3, int& ix0, int& ix1, int& iy0, int& iy1) {
  const float iz = 1.0f / vz;
  const float3 P1 = (fc.fx * iz) * (A1 - (vx * iz) * A3);
  const float3 P2 = (fc.fy * iz) * (A2 - (vy * iz) * A3);
  const float a = dot3(P1, P1), b = dot3(P1, P2), c = dot3(P2, P2);
  const float det = fmaf(a, c, -b * b);
  if (!(det > 0.0f) || !(c > 0.0f) || !isfinite(det)) return false;
  const float l11 = sqrtf(c / det), l21 = -b / sqrtf(c * det), l22 = rsqrtf(c);
  const float dn = vz * vz / (l11 * l22);
  const float s1 = dn / (vz * fc.fx), s2 = -dn / (vz * fc.fy);
  t1 = make_float4(s1 * l21, s1 * l22, 0.0f, vx);
  t2 = make_float4(s2 * l11, 0.0f, 0.0f, vy);
  t3 = make_float4(0.0f, 0.0f, 0.0f, vz);
  const float mx = fmaf(fc.fx, vx * iz, fc.cx), my = fmaf(fc.fy, vy * iz, fc.cy);
  const float hx = sqrtf(tau_c * a), hy = sqrtf(tau_c * c);
  const float ex = 0.01f + 1e-5f * fabsf(mx), ey = 0.01f + 1e-5f * fabsf(my);
  return pixel_range(mx - hx - ex, mx + hx + ex, fc.W, ix0, ix1) && pixel_range(my - hy - ey, my + hy + ey, fc.H, iy0, iy1);
}

// Activations, view-space mean and filtered variances of Gaussian i (the part
// every Gaussian needs before the early test).
struct Basic {
  float mx, my, mz;      // mean (world)
  float vx, vy, vz;      // mean (view)
  float s2x, s2y, s2z;   // variances s^2
  float hx, hy, hz;      // filtered variances s^2 + k / v'^2 (Eq. 6, 13)
  float opac;
};

__device__ __forceinline__ Basic basic_from(const float* m, const float* l, float logit, float vtrain,
                                            const FrameConst& fc) {
  Basic b;
  b.mx = m[0];
  b.my = m[1];
  b.mz = m[2];
  const float lx = l[0], ly = l[1], lz = l[2];
  // view-space mean
  b.vx = fc.Rv[0] * b.mx + fc.Rv[1] * b.my + fc.Rv[2] * b.mz + fc.tv[0];
  b.vy = fc.Rv[3] * b.mx + fc.Rv[4] * b.my + fc.Rv[5] * b.mz + fc.tv[1];
  b.vz = fc.Rv[6] * b.mx + fc.Rv[7] * b.my + fc.Rv[8] * b.mz + fc.tv[2];
  // activations (Sec. 3.1)
  const float sx = expf(lx), sy = expf(ly), sz = expf(lz);
  b.opac = 1.0f / (1.0f + expf(-logit));
  // adaptive filter (Eq. 6, 13)
  float kv = 0.0f;
  if (!(fc.flags & AAAG_FLAG_NO_FILTER)) {
    const float vhat = fc.fx / fmaxf(b.vz, fc.znear);
    const float veff = fminf(vtrain, vhat);
    kv = fc.k / (veff * veff);
  }
  b.s2x = sx * sx;
  b.s2y = sy * sy;
  b.s2z = sz * sz;
  b.hx = b.s2x + kv;
  b.hy = b.s2y + kv;
  b.hz = b.s2z + kv;
  return b;
}

__device__ __forceinline__ Basic load_basic(const SceneDev& s, const FrameConst& fc, int64_t i) {
  const float m[3] = {s.means[3 * i + 0], s.means[3 * i + 1], s.means[3 * i + 2]};
  const float l[3] = {s.log_scales[3 * i + 0], s.log_scales[3 * i + 1], s.log_scales[3 * i + 2]};
  return basic_from(m, l, s.opacity_logits[i], s.vhat_train[i], fc);
}

// The early test's inputs: only the largest filtered variance enters the
// test, so one exponential of the largest log-scale replaces three, and the
// activations use the fast intrinsics (relative errors of a few 1e-6, far
// inside the test's 0.1% radius margin; the opacity threshold is lowered by
// 1e-5 relative).  The full kernel recomputes everything exactly.
__device__ __forceinline__ Basic basic_early(const float* m, const float* l, float logit, float vtrain,
                                             const FrameConst& fc) {
  Basic b;
  b.mx = m[0];
  b.my = m[1];
  b.mz = m[2];
  b.vx = fc.Rv[0] * b.mx + fc.Rv[1] * b.my + fc.Rv[2] * b.mz + fc.tv[0];
  b.vy = fc.Rv[3] * b.mx + fc.Rv[4] * b.my + fc.Rv[5] * b.mz + fc.tv[1];
  b.vz = fc.Rv[6] * b.mx + fc.Rv[7] * b.my + fc.Rv[8] * b.mz + fc.tv[2];
  b.opac = __fdividef(1.0f, 1.0f + __expf(-logit));
  float kv = 0.0f;
  if (!(fc.flags & AAAG_FLAG_NO_FILTER)) {
    const float vhat = __fdividef(fc.fx, fmaxf(b.vz, fc.znear));
    const float veff = fminf(vtrain, vhat);
    kv = __fdividef(fc.k, veff * veff);
  }
  const float s2 = __expf(2.0f * fmaxf(l[0], fmaxf(l[1], l[2])));
  b.s2x = b.s2y = b.s2z = s2;
  b.hx = b.hy = b.hz = s2 + kv;
  return b;
}

// Conservative early test.  The tau-ellipsoid lies inside the sphere of
// radius sqrt(tau_max * max_i s_hat_i^2) around the mean, where tau_max =
// 2 ln(255 o) >= tau because the amplitude factor of Eq. 12 is at most 1.  A
// sphere wholly outside one side plane of the image frustum or in front of
// z_near holds no visible point.
// The same test with the fast logarithm and the lowered opacity threshold,
// for the inputs of basic_early (the vectorised path).  (Kept apart from the
// exact one: with a single function for both paths the vectorised loop
// compiled to code 15% slower at 16M Gaussians.)
__device__ __forceinline__ bool may_be_visible_fast(const Basic& b, const FrameConst& fc) {
  if (fc.flags & AAAG_FLAG_EVAL_2D) return b.vz >= fc.znear && b.opac > kAlphaMin * (1.0f - 1e-5f);
  const float tau_max = 2.0f * __logf(fmaxf(b.opac * 255.0f, 1.0f));
  const float rad = fmaf(sqrtf(inflate_tau(tau_max) * fmaxf(b.hx, fmaxf(b.hy, b.hz))), 1.001f, 1e-6f);
  bool near_view = b.vz + rad >= fc.znear && b.opac > kAlphaMin * (1.0f - 1e-5f);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    near_view &= fmaf(fc.side[j][0], b.vx, fmaf(fc.side[j][1], b.vy, fc.side[j][2] * b.vz)) >= -rad;
  return near_view;
}

__device__ __forceinline__ bool may_be_visible(const Basic& b, const FrameConst& fc) {
  // the EWA splat of the 2D-evaluation ablation is not bounded by the sphere
  if (fc.flags & AAAG_FLAG_EVAL_2D) return b.vz >= fc.znear && b.opac > kAlphaMin;
  const float tau_max = 2.0f * logf(fmaxf(b.opac * 255.0f, 1.0f));
  const float rad = fmaf(sqrtf(inflate_tau(tau_max) * fmaxf(b.hx, fmaxf(b.hy, b.hz))), 1.001f, 1e-6f);
  bool near_view = b.vz + rad >= fc.znear && b.opac > kAlphaMin;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    near_view &= fmaf(fc.side[j][0], b.vx, fmaf(fc.side[j][1], b.vy, fc.side[j][2] * b.vz)) >= -rad;
  return near_view;
}

// Full preprocessing of a Gaussian that passed the early test.  Writes its
// record, aux word and chunk count and returns true when it is visible;
// writes nothing otherwise.
__device__ __forceinline__ bool preprocess_one(const SceneDev& s, const FrameConst& fc, int64_t i,
                                               Record* __restrict__ rec, uint4* __restrict__ aux,
                                               uint32_t* __restrict__ chunks) {
  const Basic bb = load_basic(s, fc, i);
  const float mx = bb.mx, my = bb.my, mz = bb.mz, vx = bb.vx, vy = bb.vy, vz = bb.vz;
  const float s2x = bb.s2x, s2y = bb.s2y, s2z = bb.s2z, hx = bb.hx, hy = bb.hy, hz = bb.hz;
  const float opac = bb.opac;
  const float4 q4 = reinterpret_cast<const float4*>(s.quats)[i];
  float qn = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
  const float qi = qn > 0.0f ? rsqrtf(qn) : 0.0f;
  const float w = qn > 0.0f ? q4.x * qi : 1.0f;
  const float qx = q4.y * qi, qy = q4.z * qi, qz = q4.w * qi;
  float R[9];
  R[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
  R[1] = 2.0f * (qx * qy - w * qz);
  R[2] = 2.0f * (qx * qz + w * qy);
  R[3] = 2.0f * (qx * qy + w * qz);
  R[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
  R[5] = 2.0f * (qy * qz - w * qx);
  R[6] = 2.0f * (qx * qz - w * qy);
  R[7] = 2.0f * (qy * qz + w * qx);
  R[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
  bool visible = false;
  // d = unit vector camera -> mean; d' = R^T d
  const float dx0 = mx - fc.o[0], dy0 = my - fc.o[1], dz0 = mz - fc.o[2];
  const float dist = sqrtf(dx0 * dx0 + dy0 * dy0 + dz0 * dz0);
  const float idist = 1.0f / dist;
  const float ddx = dx0 * idist, ddy = dy0 * idist, ddz = dz0 * idist;
  const float p0 = R[0] * ddx + R[3] * ddy + R[6] * ddz;
  const float p1 = R[1] * ddx + R[4] * ddy + R[7] * ddz;
  const float p2 = R[2] * ddx + R[5] * ddy + R[8] * ddz;
  // Eq. 12 divided through by s_hat_1 s_hat_2 s_hat_3: a weighted mean of
  // r_j r_k with weights d'_i^2 / s_hat_i, r_j = s_j^2 / s_hat_j
  const float w0 = p0 * p0 / hx, w1 = p1 * p1 / hy, w2 = p2 * p2 / hz;
  const float r0 = s2x / hx, r1 = s2y / hy, r2 = s2z / hz;
  const float phi2 = (w0 * r1 * r2 + w1 * r0 * r2 + w2 * r0 * r1) / (w0 + w1 + w2);
  const float o_hat = opac * sqrtf(phi2);

  if (o_hat > kAlphaMin) {
    const float tau = 2.0f * logf(o_hat * 255.0f);
    const float spx = sqrtf(hx), spy = sqrtf(hy), spz = sqrtf(hz);
    // camera origin in normalised Gaussian space: S'^-1 R^T (o - mu)
    const float ux = -dist * p0 / spx, uy = -dist * p1 / spy, uz = -dist * p2 / spz;
    const bool inside = ux * ux + uy * uy + uz * uz < tau;
    // A = Rv R S': rows are the view axes expressed in the Gaussian frame
    float A[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float a0 = fc.Rv[3 * r + 0] * R[0] + fc.Rv[3 * r + 1] * R[3] + fc.Rv[3 * r + 2] * R[6];
      const float a1 = fc.Rv[3 * r + 0] * R[1] + fc.Rv[3 * r + 1] * R[4] + fc.Rv[3 * r + 2] * R[7];
      const float a2 = fc.Rv[3 * r + 0] * R[2] + fc.Rv[3 * r + 1] * R[5] + fc.Rv[3 * r + 2] * R[8];
      A[3 * r + 0] = a0 * spx;
      A[3 * r + 1] = a1 * spy;
      A[3 * r + 2] = a2 * spz;
    }
    const float3 A1 = f3(A[0], A[1], A[2]), A2 = f3(A[3], A[4], A[5]), A3 = f3(A[6], A[7], A[8]);
    const float tau_c = inflate_tau(tau);
    const float zext = sqrtf(tau_c * dot3(A3, A3));
    const float z_lo = vz - zext, z_hi = vz + zext;
    int ix0 = 1, ix1 = 0, iy0 = 1, iy1 = 0;   // pixel-centre ranges
    const bool eval2d = (fc.flags & AAAG_FLAG_EVAL_2D) != 0;
    bool ok = !inside && z_hi >= fc.znear;
    if (ok) {
      float px1, px2, py1, py2;
      const bool in_front = z_lo > 0.0f;
      ok = axis_bounds(A1, A3, vx, vz, tau_c, fc.fx, fc.cx, fc.eps, in_front, px1, px2) &&
           axis_bounds(A2, A3, vy, vz, tau_c, fc.fy, fc.cy, fc.eps, in_front, py1, py2);
      if (ok && z_lo < fc.znear && !eval2d) {
        near_bounds(A1, A3, vx, vz, tau_c, z_lo, z_hi, fc.fx, fc.cx, fc.znear, px1, px2);
        near_bounds(A2, A3, vy, vz, tau_c, z_lo, z_hi, fc.fy, fc.cy, fc.znear, py1, py2);
      }
      ok = ok && pixel_range(px1, px2, fc.W, ix0, ix1) && pixel_range(py1, py2, fc.H, iy0, iy1);
    }
    float4 t1 = make_float4(A[0], A[1], A[2], vx);
    float4 t2 = make_float4(A[3], A[4], A[5], vy);
    float4 t3 = make_float4(A[6], A[7], A[8], vz);
    if (eval2d) {
      // ablation without 3D evaluation: the record encodes the EWA splat
      ok = vz >= fc.znear && ewa_record(A1, A2, A3, vx, vy, vz, tau_c, fc, t1, t2, t3, ix0, ix1, iy0, iy1);
    } else if (ok) {
      // whole-image frustum cull (Sec. 3.4, last paragraph)
      const float W = (float)fc.W, H = (float)fc.H;
      ok = (z_lo < fc.znear)
               ? frustum_hit<true>(t1, t2, t3, fc.fx, fc.fy, fc.cx, fc.cy, fc.znear, 0.f, W, 0.f, H, tau_c)
               : frustum_hit<false>(t1, t2, t3, fc.fx, fc.fy, fc.cx, fc.cy, fc.znear, 0.f, W, 0.f, H, tau_c);
    }
    if (ok) {
      visible = true;
      // colour (view-dependent, real SH up to degree 3)
      const int K = (s.sh_degree + 1) * (s.sh_degree + 1);
      float Y[16];
      sh_basis(ddx, ddy, ddz, s.sh_degree, Y);
      float cr = 0.5f, cg = 0.5f, cb = 0.5f;
      const float* shp = s.sh + (size_t)i * K * 3;
      if (K == 16) {
        const float4* s4 = reinterpret_cast<const float4*>(shp);
        float c[48];
#pragma unroll
        for (int j = 0; j < 12; ++j) {
          const float4 v = s4[j];
          c[4 * j + 0] = v.x; c[4 * j + 1] = v.y; c[4 * j + 2] = v.z; c[4 * j + 3] = v.w;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          cr += Y[j] * c[3 * j + 0];
          cg += Y[j] * c[3 * j + 1];
          cb += Y[j] * c[3 * j + 2];
        }
      } else {
        for (int j = 0; j < K; ++j) {
          cr += Y[j] * shp[3 * j + 0];
          cg += Y[j] * shp[3 * j + 1];
          cb += Y[j] * shp[3 * j + 2];
        }
      }
      Record out;
      out.t1 = t1;
      out.t2 = t2;
      out.t3 = t3;
      out.rgba = make_float4(fmaxf(cr, 0.0f), fmaxf(cg, 0.0f), fmaxf(cb, 0.0f), o_hat);
      rec[i] = out;
      // Depth key: a lower bound of the depth t* of the maximum on every
      // contributing ray.  In normalised Gaussian space the maximum u* of a
      // ray from the camera c is the foot of the perpendicular from the
      // origin, so u*.(u* - c) = 0: u* lies on the sphere |u|^2 = u.c, and
      // contributing means |u*|^2 <= tau.  Hence u*.c_hat is in
      // [0, tau/|c|] and the part of u* orthogonal to c_hat has length
      // <= sqrt(tau); the view depth Z = A3.u + mu_z is then at least
      //   mu_z - sqrt(tau) |A3_perp| + min(0, A3.c_hat) tau / |c|,
      // with A3_perp the part of A3 orthogonal to c_hat.  This is never
      // below the front of the tau-ellipsoid (|A3_perp| <= |A3|) and is much
      // tighter for Gaussians seen head-on.  Quantised max(bound, znear),
      // rounded down.
      const float cn = sqrtf(ux * ux + uy * uy + uz * uz);
      const float3 ch = (1.0f / cn) * f3(ux, uy, uz);
      const float a3c = dot3(A3, ch);
      const float3 A3p = A3 - a3c * ch;
      float t_lo = vz - sqrtf(tau_c * dot3(A3p, A3p)) + fminf(a3c, 0.0f) * tau_c / cn;
      t_lo -= 1e-5f * fabsf(t_lo) + 1e-6f;
      // (sort, bounded-buffer and 2D-evaluation ablations: the depth of the mean)
      const float zk = (fc.flags & kMeanDepthKeyFlags) ? fmaxf(vz, fc.znear)
                                                                             : fmaxf(fmaxf(t_lo, z_lo), fc.znear);
      uint32_t dk = (__float_as_uint(zk) - fc.znear_bits) >> fc.depth_shift;
      const uint32_t dmax = (fc.depth_bits >= 32) ? 0xffffffffu : ((1u << fc.depth_bits) - 1u);
      dk = min(dk, dmax);
      // tau_rho, negated when the front of the ellipsoid reaches znear (the
      // tile test then truncates the frustum at the near plane)
      aux[i] = make_uint4((uint32_t)ix0 | ((uint32_t)iy0 << 16), (uint32_t)ix1 | ((uint32_t)iy1 << 16),
                          __float_as_uint(z_lo < fc.znear && !eval2d ? -tau : tau), dk);
      const uint32_t ntiles = (uint32_t)((ix1 / kTile) - (ix0 / kTile) + 1) *
                              (uint32_t)((iy1 / kTile) - (iy0 / kTile) + 1);
      chunks[i] = (ntiles + 31u) / 32u;
    }
  }
  return visible;
}

// Phase 1: the early test, four consecutive Gaussians per thread (their
// means, scales, opacities and training frequencies are loaded as float4
// vectors when the arrays are 16-byte aligned).  Every chunk count is zeroed
// (phase 2 writes those of visible Gaussians); survivors are appended to the
// candidate list (in a large scene only a few percent survive, scattered over
// the warps, so the full work runs in a second kernel on converged warps).
__global__ void __launch_bounds__(256)
preprocess_test_kernel(SceneDev s, const FrameConst* __restrict__ fcp, uint32_t* __restrict__ chunks,
                       uint32_t* __restrict__ cand, uint32_t* __restrict__ n_cand, int vec4) {
  pdl_begin();
  const FrameConst fc = *fcp;
  const int lane = threadIdx.x & 31;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  unsigned pass = 0u;   // bit j: Gaussian i0 + j survives
  if (vec4 && i0 + 3 < s.n) {
    const float4* m4 = reinterpret_cast<const float4*>(s.means + 3 * i0);
    const float4* l4 = reinterpret_cast<const float4*>(s.log_scales + 3 * i0);
    const float4 ma = m4[0], mb = m4[1], mc = m4[2], la = l4[0], lb = l4[1], lc = l4[2];
    const float4 op = *reinterpret_cast<const float4*>(s.opacity_logits + i0);
    const float4 vt = *reinterpret_cast<const float4*>(s.vhat_train + i0);
    const float mm[12] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w, mc.x, mc.y, mc.z, mc.w};
    const float ll[12] = {la.x, la.y, la.z, la.w, lb.x, lb.y, lb.z, lb.w, lc.x, lc.y, lc.z, lc.w};
    const float oo[4] = {op.x, op.y, op.z, op.w}, vv[4] = {vt.x, vt.y, vt.z, vt.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (may_be_visible_fast(basic_early(mm + 3 * j, ll + 3 * j, oo[j], vv[j], fc), fc)) pass |= 1u << j;
    *reinterpret_cast<uint4*>(chunks + i0) = make_uint4(0u, 0u, 0u, 0u);
  } else {
    for (int j = 0; j < 4; ++j) {
      const int64_t i = i0 + j;
      if (i < s.n) {
        if (may_be_visible(load_basic(s, fc, i), fc)) pass |= 1u << j;
        chunks[i] = 0u;
      }
    }
  }
  // append the survivors: scan of the per-thread counts over the block and
  // one atomic per block (one per warp serialised on the single counter:
  // 125k of them at 16M Gaussians)
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_base;
  const int warp = threadIdx.x >> 5;
  const uint32_t c = (uint32_t)__popc(pass);
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t sum = 0u;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const uint32_t t = s_warp[w];
      s_warp[w] = sum;
      sum += t;
    }
    s_base = sum ? atomicAdd(n_cand, sum) : 0u;
  }
  __syncthreads();
  uint32_t at = s_base + s_warp[warp] + incl - c;
  for (int j = 0; j < 4; ++j)
    if (pass >> j & 1u) cand[at++] = (uint32_t)(i0 + j);
}

// Phase 2: full preprocessing of the candidates (grid-stride over the count
// left in device memory by phase 1).  Two blocks per SM: with the registers
// of three (85 per thread) the kernel spilled and ran 9% slower at 16M
// Gaussians; four were slower still.
__global__ void __launch_bounds__(256, 2)
preprocess_kernel(SceneDev s, const FrameConst* __restrict__ fcp, const uint32_t* __restrict__ cand,
                  const uint32_t* __restrict__ n_cand, Record* __restrict__ rec, uint4* __restrict__ aux,
                  uint32_t* __restrict__ chunks, unsigned long long* __restrict__ stats) {
  pdl_begin();
  const FrameConst fc = *fcp;
  const uint32_t count = *n_cand;
  uint32_t nvis = 0;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j - threadIdx.x < count; j += gridDim.x * blockDim.x) {
    bool visible = false;
    if (j < count) {
      const int64_t g = cand[j];
      visible = preprocess_one(s, fc, g, rec, aux, chunks);   // count stays 0 when not
    }
    nvis += (uint32_t)__popc(__ballot_sync(0xffffffffu, visible));
  }
  if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(&stats[kStatVisible], (unsigned long long)nvis);
}

// Scenes of at least kPreFusedMin Gaussians: both phases in one kernel.
// Blocks take work items of kPreItem Gaussians (two runs of four consecutive
// ones per thread) from a counter and run the early test on them as phase 1
// does.  The survivors' indices go to a ring in shared memory, and whenever
// it holds a block's worth every thread runs the full preprocessing of one
// of them: the full work stays converged although only a few percent
// survive in a large scene, and the survivors' scene values, read by this
// block moments earlier, come back from cache instead of DRAM (phase 2 of
// the two-kernel form re-reads each from its own DRAM line).  Whatever the
// ring holds at the end is drained.  Two blocks per SM (the full work's
// registers).  Smaller scenes keep the two kernels: with few work items per
// block the fused form balances its load worse, and its test runs at two
// blocks per SM instead of four (1M Gaussians: 37 against 33 us, 2M: 50
// against 48; 4M: 79 against 84, 8M: 139 against 149, 16M: 243 against 262).
constexpr int kPreThreads = 256;
constexpr int kPreItem = 8 * kPreThreads;
constexpr uint32_t kPreRing = 4096;   // holds kPreThreads - 1 waiting plus one item's survivors
constexpr int64_t kPreFusedMin = 4 << 20;

__global__ void __launch_bounds__(kPreThreads, 2)
preprocess_fused_kernel(SceneDev s, const FrameConst* __restrict__ fcp, Record* __restrict__ rec,
                        uint4* __restrict__ aux, uint32_t* __restrict__ chunks, uint32_t* __restrict__ work,
                        unsigned long long* __restrict__ stats, int vec4) {
  pdl_begin();
  const FrameConst fc = *fcp;
  __shared__ uint32_t s_ring[kPreRing];
  __shared__ uint32_t s_warp[kPreThreads / 32];
  __shared__ uint32_t s_item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n_items = (s.n + kPreItem - 1) / kPreItem;
  uint32_t head = 0u, tail = 0u;   // ring positions, the same in every thread
  uint32_t nvis = 0u;
  bool more = true;                // work items left
  for (;;) {
    const uint32_t waiting = tail - head;
    if (waiting >= (uint32_t)kPreThreads || (!more && waiting > 0u)) {
      // full preprocessing of up to one survivor per thread
      const uint32_t cnt = min(waiting, (uint32_t)kPreThreads);
      bool visible = false;
      if (threadIdx.x < cnt)
        visible = preprocess_one(s, fc, s_ring[(head + threadIdx.x) & (kPreRing - 1u)], rec, aux, chunks);
      nvis += (uint32_t)__popc(__ballot_sync(0xffffffffu, visible));
      head += cnt;
      continue;
    }
    if (!more) break;
    __syncthreads();   // every thread has read the previous item number
    if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= n_items) {
      more = false;
      continue;
    }
    // the early test: Gaussians i0 + j and i0 + kPreItem / 2 + j, j < 4
    const int64_t i0 = item * kPreItem + (int64_t)threadIdx.x * 4;
    const int64_t i1 = i0 + kPreItem / 2;
    unsigned pass = 0u;   // bit j: Gaussian i0 + j survives; bit 4 + j: i1 + j
    if (vec4 && i1 + 3 < s.n) {
      const float4* m4 = reinterpret_cast<const float4*>(s.means + 3 * i0);
      const float4* l4 = reinterpret_cast<const float4*>(s.log_scales + 3 * i0);
      const float4* m5 = reinterpret_cast<const float4*>(s.means + 3 * i1);
      const float4* l5 = reinterpret_cast<const float4*>(s.log_scales + 3 * i1);
      const float4 ma = m4[0], mb = m4[1], mc = m4[2], la = l4[0], lb = l4[1], lc = l4[2];
      const float4 op = *reinterpret_cast<const float4*>(s.opacity_logits + i0);
      const float4 vt = *reinterpret_cast<const float4*>(s.vhat_train + i0);
      const float4 na = m5[0], nb = m5[1], nc = m5[2], ka = l5[0], kb = l5[1], kc = l5[2];
      const float4 oq = *reinterpret_cast<const float4*>(s.opacity_logits + i1);
      const float4 vu = *reinterpret_cast<const float4*>(s.vhat_train + i1);
      const float mm[24] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w, mc.x, mc.y, mc.z, mc.w,
                            na.x, na.y, na.z, na.w, nb.x, nb.y, nb.z, nb.w, nc.x, nc.y, nc.z, nc.w};
      const float ll[24] = {la.x, la.y, la.z, la.w, lb.x, lb.y, lb.z, lb.w, lc.x, lc.y, lc.z, lc.w,
                            ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w, kc.x, kc.y, kc.z, kc.w};
      const float oo[8] = {op.x, op.y, op.z, op.w, oq.x, oq.y, oq.z, oq.w};
      const float vv[8] = {vt.x, vt.y, vt.z, vt.w, vu.x, vu.y, vu.z, vu.w};
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (may_be_visible_fast(basic_early(mm + 3 * j, ll + 3 * j, oo[j], vv[j], fc), fc)) pass |= 1u << j;
      *reinterpret_cast<uint4*>(chunks + i0) = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(chunks + i1) = make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (int j = 0; j < 8; ++j) {
        const int64_t i = (j < 4 ? i0 : i1 - 4) + j;
        if (i < s.n) {
          if (may_be_visible(load_basic(s, fc, i), fc)) pass |= 1u << j;
          chunks[i] = 0u;
        }
      }
    }
    // append the survivors to the ring in index order (block-wide scan)
    const uint32_t c = (uint32_t)__popc(pass);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t before = 0u, total = 0u;
#pragma unroll
    for (int w = 0; w < kPreThreads / 32; ++w) {
      const uint32_t t = s_warp[w];
      before += w < warp ? t : 0u;
      total += t;
    }
    uint32_t at = tail + before + incl - c;
    for (int j = 0; j < 8; ++j)
      if (pass >> j & 1u) s_ring[(at++) & (kPreRing - 1u)] = (uint32_t)((j < 4 ? i0 : i1 - 4) + j);
    tail += total;
    __syncthreads();   // the ring entries are visible (and s_warp read by all)
  }
  if (lane == 0 && nvis) atomicAdd(&stats[kStatVisible], (unsigned long long)nvis);
}

}  // namespace

void configure_preprocess(LaunchConfig& c) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, preprocess_kernel, 256, 0);
  c.pre_per_sm = std::max(1, per_sm);
  per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, preprocess_fused_kernel, kPreThreads, 0);
  c.pre_fused_per_sm = std::max(1, per_sm);
}

aaag_status launch_preprocess(const SceneDev& s, aaag_workspace* ws, cudaStream_t st) {
  if (s.n == 0) return AAAG_OK;
  const LaunchConfig& lc = launch_config();
  const int64_t pre_blocks = (int64_t)lc.sms * lc.pre_per_sm;
  const int threads = 256;
  const int64_t blocks = (s.n + threads - 1) / threads;
  const int64_t tblocks = ((s.n + 3) / 4 + threads - 1) / threads;
  // the candidate count of the two kernels, or the work-item counter of the
  // fused one (zeroed with the frame's statistics)
  uint32_t* n_cand = reinterpret_cast<uint32_t*>(ws->stats + kStatCandidates);
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0u; };
  const int vec4 = a16(s.means) && a16(s.log_scales) && a16(s.opacity_logits) && a16(s.vhat_train) &&
                   a16(ws->counts);
  if (s.n >= kPreFusedMin) {
    const int64_t items = (s.n + kPreItem - 1) / kPreItem;
    const unsigned grid = (unsigned)std::min<int64_t>(items, (int64_t)lc.sms * lc.pre_fused_per_sm);
    launch_chained(preprocess_fused_kernel, grid, kPreThreads, 0, st, s, ws->fc_dev, ws->records, ws->aux,
                   ws->counts, n_cand, ws->stats, vec4);
    return check_launch("preprocess_fused");
  }
  launch_chained(preprocess_test_kernel, (unsigned)tblocks, threads, 0, st, s, ws->fc_dev, ws->counts, ws->candidates, n_cand,
                                                                vec4);
  aaag_status e = check_launch("preprocess_test");
  if (e != AAAG_OK) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(blocks, pre_blocks);
  launch_chained(preprocess_kernel, grid, threads, 0, st, s, ws->fc_dev, ws->candidates, n_cand, ws->records, ws->aux,
                                              ws->counts, ws->stats);
  return check_launch("preprocess");
}

}  // namespace aaag
