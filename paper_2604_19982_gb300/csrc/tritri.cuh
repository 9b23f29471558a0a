// Triangle-triangle minimum distance on the GPU (section 2.2: the Moller
// decomposition into 6 vertex-to-triangle and 9 edge-to-edge distances, plus
// an edge-crosses-triangle test for the meeting case the 15 distances miss).
//
// Formulation (branch-light, one thread per facet pair):
//  * Each facet is pre-processed once into a record: vertices v_i, edges
//    e_i = v_{i+1} - v_i, |e_i|^2 and its inverse, unit normal n, in-plane
//    inward edge normals m_i = n x e_i, its Hausdorff bounds hd / ph, and
//    hoff (0, or +inf for a zero-area facet, which has no interior case).
//  * vertex-to-triangle: only the case where the vertex projects inside the
//    other triangle (all m_j . (p - q_j) >= 0) contributes, as the plane
//    distance n . (p - q_0); when the projection falls outside, the nearest
//    point is on an edge and that distance is one of the edge-edge cases.
//  * edge-to-edge: closest parameters of the two segments by one unclamped
//    solve, then t re-optimised for s and s re-optimised for the clamped t
//    (any s, t in [0, 1] is a true point pair, so the value never
//    underestimates); the distance is taken from the difference vector
//    r + s d1 - t d2 itself.
//  * meeting: when both triangles straddle each other's planes, each edge is
//    tested against the other triangle with the heights h and the in-plane
//    dots g already formed above: the crossing point of edge (a, b) is inside
//    iff every (h_b g_aj - h_a g_bj) sign(h_b - h_a) >= 0.  With error
//    margins (single precision) the test yields `possible` (cannot be
//    excluded) and `certain` (holds for the exact input).
//
// The register-side record (P) stores n and m negated so that every dot
// product reads the same difference vectors D_ij = p_i - q_j.
#pragma once
#include <math.h>

#include "common.cuh"

namespace pj {

template <class T>
struct Rec {
  T v[3][3];
  T e[3][3];
  T ee[3];
  T iee[3];
  T n[3];
  T m[3][3];
  T hd, ph, hoff;
};

// ---------------------------------------------------------------- scalar ops
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float sat_(float x) { return __saturatef(x); }
__device__ __forceinline__ double sat_(double x) { return fmin(fmax(x, 0.0), 1.0); }
// x / y for the segment parameter: any value is acceptable (it is clamped
// and re-optimised), so the single-precision path uses the fast reciprocal.
__device__ __forceinline__ float pdiv_(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double pdiv_(double x, double y) { return x / y; }
__device__ __forceinline__ float inf_(float) { return __int_as_float(0x7f800000); }
__device__ __forceinline__ double inf_(double) { return __longlong_as_double(0x7ff0000000000000LL); }
__device__ __forceinline__ float sqrt_test(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double sqrt_test(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double sqrt_rn(double x) { return __dsqrt_rn(x); }
__device__ __forceinline__ float add_ru(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ double add_ru(double a, double b) { return __dadd_ru(a, b); }
__device__ __forceinline__ float sub_rd(float a, float b) { return __fsub_rd(a, b); }
__device__ __forceinline__ double sub_rd(double a, double b) { return __dsub_rd(a, b); }

template <class T>
__device__ __forceinline__ T dot3(const T* a, const T* b) {
  return fma_(a[2], b[2], fma_(a[1], b[1], a[0] * b[0]));
}

// ---------------------------------------------------------------- records
// Build a record from three (already translated) vertices.  `neg` flips n
// and m for the register side.  sin_min (optional) receives the facet's
// conditioning |e0 x e1| / (|e0| |e1|).
template <class T>
__device__ __forceinline__ void make_rec(Rec<T>& R, const T a[3], const T b[3], const T c[3], T hd, T ph,
                                         bool neg) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R.v[0][k] = a[k];
    R.v[1][k] = b[k];
    R.v[2][k] = c[k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 3; ++k) R.e[i][k] = R.v[(i + 1) % 3][k] - R.v[i][k];
    R.ee[i] = dot3(R.e[i], R.e[i]);
    R.iee[i] = R.ee[i] > T(0) ? T(1) / R.ee[i] : T(0);
  }
  T cx = R.e[0][1] * R.e[1][2] - R.e[0][2] * R.e[1][1];
  T cy = R.e[0][2] * R.e[1][0] - R.e[0][0] * R.e[1][2];
  T cz = R.e[0][0] * R.e[1][1] - R.e[0][1] * R.e[1][0];
  T c2 = cx * cx + cy * cy + cz * cz;
  T sgn = neg ? T(-1) : T(1);
  if (c2 > T(0)) {
    T inv = sgn / sqrt_rn(c2);
    R.n[0] = cx * inv;
    R.n[1] = cy * inv;
    R.n[2] = cz * inv;
    R.hoff = T(0);
  } else {
    R.n[0] = R.n[1] = R.n[2] = T(0);
    R.hoff = inf_(T(0));
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    // m_i = n x e_i (n already carries the sign)
    R.m[i][0] = R.n[1] * R.e[i][2] - R.n[2] * R.e[i][1];
    R.m[i][1] = R.n[2] * R.e[i][0] - R.n[0] * R.e[i][2];
    R.m[i][2] = R.n[0] * R.e[i][1] - R.n[1] * R.e[i][0];
  }
  R.hd = hd;
  R.ph = ph;
}

// |e0 x e1| / (|e0| |e1|) of a facet (its sine; small for slivers)
template <class T>
__device__ __forceinline__ T facet_sin(const T a[3], const T b[3], const T c[3]) {
  T e0[3], e1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e0[k] = b[k] - a[k];
    e1[k] = c[k] - b[k];
  }
  T cx = e0[1] * e1[2] - e0[2] * e1[1], cy = e0[2] * e1[0] - e0[0] * e1[2], cz = e0[0] * e1[1] - e0[1] * e1[0];
  T den = sqrt_rn(dot3(e0, e0) * dot3(e1, e1));
  return den > T(0) ? sqrt_rn(cx * cx + cy * cy + cz * cz) / den : T(0);
}

// Shared-memory image of a record: 40 values, vector-loadable.
template <class T>
struct RecSmem {
  T x[40];
};

template <class T>
__device__ __forceinline__ void store_rec(RecSmem<T>& S, const Rec<T>& R) {
  T* x = S.x;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      x[4 * i + k] = R.v[i][k];
      x[12 + 4 * i + k] = R.e[i][k];
      x[28 + 4 * i + k] = R.m[i][k];
    }
  x[3] = R.hd;
  x[7] = R.ph;
  x[11] = R.hoff;
  x[15] = R.ee[0];
  x[19] = R.ee[1];
  x[23] = R.ee[2];
  x[24] = R.n[0];
  x[25] = R.n[1];
  x[26] = R.n[2];
  x[27] = R.iee[0];
  x[31] = R.iee[1];
  x[35] = R.iee[2];
  x[39] = T(0);
}

template <class T>
__device__ __forceinline__ void load_rec(Rec<T>& R, const RecSmem<T>& S);

template <>
__device__ __forceinline__ void load_rec<float>(Rec<float>& R, const RecSmem<float>& S) {
  const float4* q = reinterpret_cast<const float4*>(S.x);
  float4 a[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) a[k] = q[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R.v[i][0] = a[i].x; R.v[i][1] = a[i].y; R.v[i][2] = a[i].z;
    R.e[i][0] = a[3 + i].x; R.e[i][1] = a[3 + i].y; R.e[i][2] = a[3 + i].z; R.ee[i] = a[3 + i].w;
    R.m[i][0] = a[7 + i].x; R.m[i][1] = a[7 + i].y; R.m[i][2] = a[7 + i].z;
  }
  R.hd = a[0].w; R.ph = a[1].w; R.hoff = a[2].w;
  R.n[0] = a[6].x; R.n[1] = a[6].y; R.n[2] = a[6].z;
  R.iee[0] = a[6].w; R.iee[1] = a[7].w; R.iee[2] = a[8].w;
}

template <>
__device__ __forceinline__ void load_rec<double>(Rec<double>& R, const RecSmem<double>& S) {
  const double2* q = reinterpret_cast<const double2*>(S.x);
  double x[40];
#pragma unroll
  for (int k = 0; k < 20; ++k) {
    double2 t = q[k];
    x[2 * k] = t.x;
    x[2 * k + 1] = t.y;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      R.v[i][k] = x[4 * i + k];
      R.e[i][k] = x[12 + 4 * i + k];
      R.m[i][k] = x[28 + 4 * i + k];
    }
  R.hd = x[3]; R.ph = x[7]; R.hoff = x[11];
  R.ee[0] = x[15]; R.ee[1] = x[19]; R.ee[2] = x[23];
  R.n[0] = x[24]; R.n[1] = x[25]; R.n[2] = x[26];
  R.iee[0] = x[27]; R.iee[1] = x[31]; R.iee[2] = x[35];
}

// ---------------------------------------------------------------- the test
// Squared minimum over the 15 candidate distances of P (register record,
// negated n / m) and Q.  `maybe` is set when both triangles straddle the
// other's plane (within eh), the precondition of a crossing.
template <class T>
__device__ __forceinline__ T tri_d2(const Rec<T>& P, const Rec<T>& Q, T eh, bool& maybe) {
  T D[3][3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) D[i][j][k] = P.v[i][k] - Q.v[j][k];

  const T INF = inf_(T(0));
  T d2 = INF;
  T hP[3], hQ[3];
  // vertices of P against Q's interior
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    hP[i] = fma_(Q.n[2], D[i][0][2], fma_(Q.n[1], D[i][0][1], fma_(Q.n[0], D[i][0][0], Q.hoff)));
    T g0 = dot3(Q.m[0], D[i][0]);
    T g1 = dot3(Q.m[1], D[i][1]);
    T g2 = dot3(Q.m[2], D[i][2]);
    T gmin = min(g0, min(g1, g2));
    T c = gmin >= T(0) ? hP[i] * hP[i] : INF;
    d2 = min(d2, c);
  }
  // vertices of Q against P's interior (P.n, P.m are negated)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    hQ[j] = fma_(P.n[2], D[0][j][2], fma_(P.n[1], D[0][j][1], fma_(P.n[0], D[0][j][0], P.hoff)));
    T g0 = dot3(P.m[0], D[0][j]);
    T g1 = dot3(P.m[1], D[1][j]);
    T g2 = dot3(P.m[2], D[2][j]);
    T gmin = min(g0, min(g1, g2));
    T c = gmin >= T(0) ? hQ[j] * hQ[j] : INF;
    d2 = min(d2, c);
  }
  // edge i of P against edge j of Q
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T* r = D[i][j];
      const T* d1 = P.e[i];
      const T* dq = Q.e[j];
      T b = dot3(d1, dq);
      T c = dot3(d1, r);
      T f = dot3(dq, r);
      T den = fma_(P.ee[i], Q.ee[j], -b * b);
      T num = fma_(b, f, -c * Q.ee[j]);
      T s = sat_(pdiv_(num, den));
      T t = sat_(fma_(b, s, f) * Q.iee[j]);
      s = sat_(fma_(b, t, -c) * P.iee[i]);
      T wx = fma_(-t, dq[0], fma_(s, d1[0], r[0]));
      T wy = fma_(-t, dq[1], fma_(s, d1[1], r[1]));
      T wz = fma_(-t, dq[2], fma_(s, d1[2], r[2]));
      d2 = min(d2, fma_(wz, wz, fma_(wy, wy, wx * wx)));
    }
  T pmin = min(hP[0], min(hP[1], hP[2])), pmax = max(hP[0], max(hP[1], hP[2]));
  T qmin = min(hQ[0], min(hQ[1], hQ[2])), qmax = max(hQ[0], max(hQ[1], hQ[2]));
  maybe = (pmin <= eh) && (pmax >= -eh) && (qmin <= eh) && (qmax >= -eh);
  return d2;
}

// Edge (a, b) with heights ha, hb over the other triangle's plane and the
// in-plane dots ga[j], gb[j]: can it cross / does it certainly cross?
template <class T>
__device__ __forceinline__ void edge_cross(T ha, T hb, const T ga[3], const T gb[3], T eh, T ew, bool& possible,
                                           bool& certain) {
  bool same_pos = ha > eh && hb > eh;
  bool same_neg = ha < -eh && hb < -eh;
  if (same_pos || same_neg) return;
  bool opposite = (ha > eh && hb < -eh) || (ha < -eh && hb > eh);
  T dh = hb - ha;
  bool sgn_known = dh > T(2) * eh || dh < -T(2) * eh;
  T sg = dh > T(0) ? T(1) : T(-1);
  bool all_nonneg = true, all_pos = true;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    T w = (hb * ga[j] - ha * gb[j]) * sg;
    all_nonneg = all_nonneg && (w >= -ew);
    all_pos = all_pos && (w > ew);
  }
  // with zero margins (double precision) "certain" reduces to the exact-
  // arithmetic crossing test evaluated as computed
  if (!sgn_known || all_nonneg) possible = true;
  if (opposite && sgn_known && all_pos) certain = true;
}

// The crossing test of all six edges (only run when `maybe`).  Recomputes
// the heights and in-plane dots to keep the common path's registers low.
template <class T>
__device__ void tri_cross(const Rec<T>& P, const Rec<T>& Q, T eh, T ew, bool& possible, bool& certain) {
  T D[3][3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) D[i][j][k] = P.v[i][k] - Q.v[j][k];
  T hP[3], hQ[3], gP[3][3], gQ[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    hP[i] = fma_(Q.n[2], D[i][0][2], fma_(Q.n[1], D[i][0][1], fma_(Q.n[0], D[i][0][0], Q.hoff)));
#pragma unroll
    for (int j = 0; j < 3; ++j) gP[i][j] = dot3(Q.m[j], D[i][j]);      // m_Qj . (p_i - q_j)
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    hQ[j] = fma_(P.n[2], D[0][j][2], fma_(P.n[1], D[0][j][1], fma_(P.n[0], D[0][j][0], P.hoff)));
#pragma unroll
    for (int i = 0; i < 3; ++i) gQ[j][i] = dot3(P.m[i], D[i][j]);      // m_Pi . (q_j - p_i)
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int k = (i + 1) % 3;
    edge_cross(hP[i], hP[k], gP[i], gP[k], eh, ew, possible, certain);
    edge_cross(hQ[i], hQ[k], gQ[i], gQ[k], eh, ew, possible, certain);
  }
}

// Forward error margins of the single-precision test for coordinates
// bounded by rho (pair-local, per axis), maximal edge length L and minimal
// facet sine smin (see the error analysis in the design notes):
//   heights   |h~ - h| <= 128 u rho / smin
//   crossing  |w~ - w| <= 2048 u rho^2 L / smin
//   distance  |d~ - d| <= 256 u rho / smin + 8 sqrt(u) L
struct Margins {
  float eps, eh, ew;
};

__host__ __device__ __forceinline__ Margins fp32_margins(float rho, float L, float smin) {
  const float u = 5.9604644775390625e-08f;          // 2^-24
  const float su = 2.44140625e-04f;                 // sqrt(2^-24) = 2^-12
  float s = smin > 1e-6f ? smin : 1e-6f;
  Margins m;
  m.eh = 128.0f * u * rho / s;
  m.ew = 2048.0f * u * rho * rho * L / s;
  m.eps = 256.0f * u * rho / s + 8.0f * su * L;
  return m;
}

}  // namespace pj
