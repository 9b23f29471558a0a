// Exact meeting test of two triangles with float vertices (the distance of
// section 2.1 is 0 exactly when the closed triangles share a point).
//
// Orientation signs are exact: with float inputs, every term of the
// determinants expanded in the raw coordinates is a product of two or three
// floats; a product of two floats is exact in double (48 significant bits),
// and a third factor is taken exactly by a fused multiply-add (TwoProduct).
// The terms are summed exactly into a floating-point expansion (a sum of
// non-overlapping doubles, Knuth's TwoSum with zero elimination, after
// Shewchuk, "Adaptive precision floating-point arithmetic and fast robust
// geometric predicates", 1997), whose sign is that of its largest
// component.  No float input can underflow or overflow these products.
//
// The decision logic: two closed triangles meet iff an edge of one meets
// the other (in the non-coplanar case their common part is a segment of the
// planes' common line with its ends on edges; in the coplanar case the
// boundaries cross or one triangle holds the other's vertices).  An edge
// (segment) meets a triangle:
//   * never when both ends lie strictly on one side of its plane;
//   * when the ends lie strictly on opposite sides, iff the line through
//     them passes no edge of the triangle on the wrong side (the signs of
//     the three tetrahedra (a, b, t_j, t_j+1) are not mixed);
//   * when an end lies in the plane, iff the end lies in the triangle, or,
//     with both ends in the plane, iff an end lies in it or the segment
//     crosses one of its edges; decided in a coordinate plane onto which the
//     triangle projects with non-zero area (one-to-one on its plane);
//   * a triangle with collinear vertices is the union of its edges; two
//     segments meet iff they are coplanar and meet in all three coordinate
//     projections.
// Used only when the single-precision sign filter of the kernels is not
// certain, so it is out of line.
#pragma once
#include <cuda_runtime.h>

namespace pj {

// a + b = s + e exactly (s the rounded sum)
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bv = __dsub_rn(s, a);
  const double av = __dsub_rn(s, bv);
  e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// h (n components, increasing magnitude, non-overlapping) += b, in place;
// zero components are dropped.  Returns the new length (<= n + 1).
__device__ __forceinline__ int grow_expansion(double* h, int n, double b) {
  double q = b;
  int m = 0;
  for (int i = 0; i < n; ++i) {
    double s, e;
    two_sum(q, h[i], s, e);
    q = s;
    if (e != 0.0) h[m++] = e;
  }
  if (q != 0.0 || m == 0) h[m++] = q;
  return m;
}

// add the exact product a*b*c of three floats
__device__ __forceinline__ int add_prod3(double* h, int n, float a, float b, float c, bool neg) {
  const double ab = __dmul_rn((double)a, (double)b);   // exact: 48 bits
  const double p = __dmul_rn(ab, (double)c);
  const double e = __fma_rn(ab, (double)c, -p);         // ab c = p + e exactly
  n = grow_expansion(h, n, neg ? -e : e);
  return grow_expansion(h, n, neg ? -p : p);
}

__device__ __forceinline__ int exp_sign(const double* h, int n) {
  const double t = h[n - 1];
  return t > 0.0 ? 1 : (t < 0.0 ? -1 : 0);
}

// det [p; q; r] of three float points as the six signed triple products
__device__ __forceinline__ int add_det3(double* h, int n, float4 p, float4 q, float4 r, bool neg) {
  n = add_prod3(h, n, p.x, q.y, r.z, neg);
  n = add_prod3(h, n, p.x, q.z, r.y, !neg);
  n = add_prod3(h, n, p.y, q.x, r.z, !neg);
  n = add_prod3(h, n, p.y, q.z, r.x, neg);
  n = add_prod3(h, n, p.z, q.x, r.y, neg);
  n = add_prod3(h, n, p.z, q.y, r.x, !neg);
  return n;
}

// exact sign of (b - a) . ((c - a) x (d - a)); by multilinearity this is
// det(b,c,d) - det(a,c,d) - det(b,a,d) - det(b,c,a) in the raw coordinates
__device__ __forceinline__ int orient3_exact(float4 a, float4 b, float4 c, float4 d) {
  double h[48];
  int n = 0;
  n = add_det3(h, n, b, c, d, false);
  n = add_det3(h, n, a, c, d, true);
  n = add_det3(h, n, b, a, d, true);
  n = add_det3(h, n, b, c, a, true);
  return exp_sign(h, n);
}

// exact sign of (b - a) x (c - a) in the plane:
// bx cy - bx ay - ax cy - by cx + by ax + ay cx
__device__ __forceinline__ int orient2_exact(float2 a, float2 b, float2 c) {
  double h[8];
  int n = 0;
  n = grow_expansion(h, n, __dmul_rn((double)b.x, (double)c.y));
  n = grow_expansion(h, n, -__dmul_rn((double)b.x, (double)a.y));
  n = grow_expansion(h, n, -__dmul_rn((double)a.x, (double)c.y));
  n = grow_expansion(h, n, -__dmul_rn((double)b.y, (double)c.x));
  n = grow_expansion(h, n, __dmul_rn((double)b.y, (double)a.x));
  n = grow_expansion(h, n, __dmul_rn((double)a.y, (double)c.x));
  return exp_sign(h, n);
}

// drop coordinate k
__device__ __forceinline__ float2 proj2(float4 p, int k) {
  return k == 0 ? make_float2(p.y, p.z) : (k == 1 ? make_float2(p.x, p.z) : make_float2(p.x, p.y));
}

// x collinear with the 2-D segment [p, q]: inside its box?
__device__ __forceinline__ bool in_box2(float2 p, float2 q, float2 x) {
  return fminf(p.x, q.x) <= x.x && x.x <= fmaxf(p.x, q.x) && fminf(p.y, q.y) <= x.y && x.y <= fmaxf(p.y, q.y);
}

// closed 2-D segments [a, b] and [c, d] (possibly points) share a point
__device__ __forceinline__ bool segs_meet2(float2 a, float2 b, float2 c, float2 d) {
  const int s1 = orient2_exact(c, d, a), s2 = orient2_exact(c, d, b);
  const int s3 = orient2_exact(a, b, c), s4 = orient2_exact(a, b, d);
  if (s1 * s2 < 0 && s3 * s4 < 0) return true;
  return (s1 == 0 && in_box2(c, d, a)) || (s2 == 0 && in_box2(c, d, b)) || (s3 == 0 && in_box2(a, b, c)) ||
         (s4 == 0 && in_box2(a, b, d));
}

// closed 3-D segments share a point: coplanar, and meeting in every
// coordinate projection
__device__ __forceinline__ bool segs_meet3(float4 a, float4 b, float4 c, float4 d) {
  if (orient3_exact(a, b, c, d) != 0) return false;
  for (int k = 0; k < 3; ++k)
    if (!segs_meet2(proj2(a, k), proj2(b, k), proj2(c, k), proj2(d, k))) return false;
  return true;
}

// 2-D point in the closed triangle (t0, t1, t2) of orientation o != 0
__device__ __forceinline__ bool in_tri2(float2 p, float2 t0, float2 t1, float2 t2, int o) {
  return orient2_exact(t0, t1, p) * o >= 0 && orient2_exact(t1, t2, p) * o >= 0 &&
         orient2_exact(t2, t0, p) * o >= 0;
}

// closed segment [a, b] and closed triangle t share a point
__device__ __forceinline__ bool seg_meets_tri(float4 a, float4 b, const float4* t) {
  const int sa = orient3_exact(t[0], t[1], t[2], a), sb = orient3_exact(t[0], t[1], t[2], b);
  if (sa * sb > 0) return false;
  if (sa != 0 && sb != 0) {
    const int o1 = orient3_exact(a, b, t[0], t[1]), o2 = orient3_exact(a, b, t[1], t[2]),
              o3 = orient3_exact(a, b, t[2], t[0]);
    const bool pos = o1 > 0 || o2 > 0 || o3 > 0, neg = o1 < 0 || o2 < 0 || o3 < 0;
    return !(pos && neg);
  }
  int k = -1, o = 0;
  for (int kk = 0; kk < 3 && k < 0; ++kk) {
    o = orient2_exact(proj2(t[0], kk), proj2(t[1], kk), proj2(t[2], kk));
    if (o != 0) k = kk;
  }
  if (k < 0) return segs_meet3(a, b, t[0], t[1]) || segs_meet3(a, b, t[1], t[2]) || segs_meet3(a, b, t[2], t[0]);
  const float2 A = proj2(a, k), B = proj2(b, k);
  const float2 T0 = proj2(t[0], k), T1 = proj2(t[1], k), T2 = proj2(t[2], k);
  if (sa == 0 && sb == 0)
    return in_tri2(A, T0, T1, T2, o) || in_tri2(B, T0, T1, T2, o) || segs_meet2(A, B, T0, T1) ||
           segs_meet2(A, B, T1, T2) || segs_meet2(A, B, T2, T0);
  return in_tri2(sa == 0 ? A : B, T0, T1, T2, o);
}

// Do the closed triangles p, q (raw float vertices, .w ignored) meet?
static __device__ __noinline__ bool tri_meet_exact(const float4* p, const float4* q) {
  for (int side = 0; side < 2; ++side) {
    const float4* A = side ? q : p;
    const float4* B = side ? p : q;
    for (int i = 0; i < 3; ++i)
      if (seg_meets_tri(A[i], A[(i + 1) % 3], B)) return true;
  }
  return false;
}

}  // namespace pj
