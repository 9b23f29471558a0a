// Triangle-triangle minimum distance on the GPU (section 2.2: the Moller
// decomposition into 6 vertex-to-triangle and 9 edge-to-edge distances, plus
// an edge-crosses-triangle test for the meeting case the 15 distances miss).
//
// Formulation (branch-light, one thread per facet pair):
//  * Each facet is pre-processed once into a record: vertices v_i, edges
//    e_i = v_{i+1} - v_i, |e_i|^2 and its inverse, unit normal n, in-plane
//    inward edge normals m_i = n x e_i, its Hausdorff bounds hd / ph, and
//    hoff (0, or NaN for a zero-area facet, which has no interior case).
//  * vertex-to-triangle: only the case where the vertex projects inside the
//    other triangle (all m_j . (p - q_j) >= 0) contributes, as the plane
//    distance n . (p - q_0); when the projection falls outside, the nearest
//    point is on an edge and that distance is one of the edge-edge cases.
//  * edge-to-edge: closest parameters of the two segments by one unclamped
//    solve, then t re-optimised for s and s re-optimised for the clamped t
//    (any s, t in [0, 1] is a true point pair, so the value never
//    underestimates); the distance is taken from the difference vector
//    r + s d1 - t d2 itself.
//  * meeting: only when both triangles straddle each other's planes (within
//    the height error margin) can they meet; that case gets the exact
//    decision from the float vertices (cross_decide: single-precision signs
//    wherever an error bound makes them certain, else exact expansion
//    arithmetic, exact.cuh), in both precisions of the path.  A facet with
//    zero computed area has a NaN plane offset: it has no interior case, and
//    its straddle test always passes, so it always gets the exact test.
//
// The register-side record (P) stores n and m negated so that every dot
// product reads the same difference vectors D_ij = p_i - q_j.
#pragma once
#include <math.h>

#include "common.cuh"
#include "exact.cuh"

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
  T sc[3], sr;   // a ball holding the facet: centroid, radius rounded well up
};

// Facet balls apart by more than `bound` (see the float overload below).
__device__ __forceinline__ bool balls_apart(const double pc[3], double pr, const double qc[3], double qr,
                                            double bound) {
  const double dx = pc[0] - qc[0], dy = pc[1] - qc[1], dz = pc[2] - qc[2];
  const double dist2 = fma(dz, dz, fma(dy, dy, dx * dx));
  const double lim = bound + pr + qr;
  return lim >= 0.0 && dist2 * (1.0 - 1e-12) > lim * lim * (1.0 + 1e-12);
}

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
__device__ __forceinline__ float nan_(float) { return __int_as_float(0x7fffffff); }
__device__ __forceinline__ double nan_(double) { return __longlong_as_double(0x7fffffffffffffffLL); }
// the smallest positive value: the distance of facets that do not meet
// where the candidates round to 0 (0 is kept for facets that meet)
__device__ __forceinline__ float tiny_(float) { return __int_as_float(1); }
__device__ __forceinline__ double tiny_(double) { return __longlong_as_double(1LL); }
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
__device__ __forceinline__ float sub_ru(float a, float b) { return __fsub_ru(a, b); }
__device__ __forceinline__ double sub_ru(double a, double b) { return __dsub_ru(a, b); }
__device__ __forceinline__ float add_rd(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ double add_rd(double a, double b) { return __dadd_rd(a, b); }
__device__ __forceinline__ float sqrt_ru(float x) { return __fsqrt_ru(x); }
__device__ __forceinline__ double sqrt_ru(double x) { return __dsqrt_ru(x); }

template <class T>
__device__ __forceinline__ T dot3(const T* a, const T* b) {
  return fma_(a[2], b[2], fma_(a[1], b[1], a[0] * b[0]));
}

// ---------------------------------------------------------------- records
// A ball holding the facet (a, b, c): the centroid and the largest vertex
// distance, rounded well up (relative 1e-5 plus 1e-6 of the largest
// coordinate), so that it holds the exact facet despite the rounding of the
// translation and of the centroid.
template <class T>
__device__ __forceinline__ void facet_ball(const T a[3], const T b[3], const T c[3], T sc[3], T& sr) {
  T rmax = T(0), amax = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) sc[k] = (a[k] + b[k] + c[k]) * (T(1) / T(3));
  const T* v[3] = {a, b, c};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T q2 = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T dv = v[i][k] - sc[k];
      q2 = fma_(dv, dv, q2);
      amax = max(amax, abs(v[i][k]));
    }
    rmax = max(rmax, q2);
  }
  sr = sqrt(rmax) * T(1.00001) + amax * T(1e-6) + T(1e-30);
}

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
    R.hoff = nan_(T(0));
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
  facet_ball(a, b, c, R.sc, R.sr);
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
  T x[44];
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
  x[40] = R.sc[0];
  x[41] = R.sc[1];
  x[42] = R.sc[2];
  x[43] = R.sr;
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
  double x[44];
#pragma unroll
  for (int k = 0; k < 22; ++k) {
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
  R.sc[0] = x[40]; R.sc[1] = x[41]; R.sc[2] = x[42]; R.sr = x[43];
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
  // (NaN heights of a zero-area facet fail every comparison: maybe)
  maybe = !((pmin > eh) || (pmax < -eh) || (qmin > eh) || (qmax < -eh));
  return d2;
}

// Are the boxes of the two facets strictly apart on some axis?  Then they
// cannot meet.  Rounding of the pair-local translation is monotone, so a
// strict separation of the computed coordinates implies one of the exact.
template <class R>
__device__ __forceinline__ bool boxes_apart(const R& P, const R& Q) {
  bool apart = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    auto pmin = min(P.v[0][k], min(P.v[1][k], P.v[2][k])), pmax = max(P.v[0][k], max(P.v[1][k], P.v[2][k]));
    auto qmin = min(Q.v[0][k], min(Q.v[1][k], Q.v[2][k])), qmax = max(Q.v[0][k], max(Q.v[1][k], Q.v[2][k]));
    apart = apart || (pmax < qmin) || (qmax < pmin);
  }
  return apart;
}

// ---------------------------------------------------------------- FP32 form
// The single-precision kernels evaluate the same 15 candidates without the
// 27 vertex differences: every plane, inside and edge product against a
// vertex x of the other facet is taken as (a . x) - k with the constant k
// of the record, so that only the three differences an edge pair's closest
// points need are formed, when they are needed.  Record constants:
//   c = n . v0 - hoff,   mc_i = m_i . v_i,   ev_i = e_i . v_i.
// Both sides use the same orientation (n, m_i = n x e_i, not negated).  The
// rounding of (a . x) - k is a few u rho (rho: coordinate bound of the pair
// frame), far inside the margins eh / eps of fp32_margins.
struct RecL {
  float v[3][3];
  float e[3][3];
  float ee[3], iee[3];
  float n[3];
  float m[3][3];
  float c, mc[3], ev[3];
  float hd, ph;
  float sc[3], sr;   // a ball holding the facet: centroid, radius rounded well up
};

// Lower bound of the distance of two facets from their balls, as a test on
// squares: true when |c_P - c_Q| - r_P - r_Q > bound for the exact values
// (relative slack covers the rounding of the centre distance).
__device__ __forceinline__ bool balls_apart(const float pc[3], float pr, const float qc[3], float qr, float bound) {
  const float dx = pc[0] - qc[0], dy = pc[1] - qc[1], dz = pc[2] - qc[2];
  const float dist2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const float lim = bound + pr + qr;
  return lim >= 0.f && dist2 * 0.99996f > lim * lim * 1.00002f;
}

__device__ __forceinline__ void make_rec(RecL& R, const float a[3], const float b[3], const float c[3], float hd,
                                         float ph, bool) {
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
    R.iee[i] = R.ee[i] > 0.f ? 1.f / R.ee[i] : 0.f;
  }
  float cx = R.e[0][1] * R.e[1][2] - R.e[0][2] * R.e[1][1];
  float cy = R.e[0][2] * R.e[1][0] - R.e[0][0] * R.e[1][2];
  float cz = R.e[0][0] * R.e[1][1] - R.e[0][1] * R.e[1][0];
  float c2 = cx * cx + cy * cy + cz * cz;
  float hoff;
  if (c2 > 0.f) {
    float inv = 1.f / sqrt_rn(c2);
    R.n[0] = cx * inv;
    R.n[1] = cy * inv;
    R.n[2] = cz * inv;
    hoff = 0.f;
  } else {
    R.n[0] = R.n[1] = R.n[2] = 0.f;
    hoff = nan_(0.f);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R.m[i][0] = R.n[1] * R.e[i][2] - R.n[2] * R.e[i][1];
    R.m[i][1] = R.n[2] * R.e[i][0] - R.n[0] * R.e[i][2];
    R.m[i][2] = R.n[0] * R.e[i][1] - R.n[1] * R.e[i][0];
    R.mc[i] = dot3(R.m[i], R.v[i]);
    R.ev[i] = dot3(R.e[i], R.v[i]);
  }
  R.c = dot3(R.n, R.v[0]) - hoff;
  R.hd = hd;
  R.ph = ph;
  facet_ball(a, b, c, R.sc, R.sr);
}

// Shared-memory image of a RecL: 48 floats, 12 float4 loads.
struct RecSmemL {
  float x[52];
};

__device__ __forceinline__ void store_rec(RecSmemL& S, const RecL& R) {
  float4* q = reinterpret_cast<float4*>(S.x);
  q[0] = make_float4(R.v[0][0], R.v[0][1], R.v[0][2], R.hd);
  q[1] = make_float4(R.v[1][0], R.v[1][1], R.v[1][2], R.ph);
  q[2] = make_float4(R.v[2][0], R.v[2][1], R.v[2][2], R.c);
  q[3] = make_float4(R.e[0][0], R.e[0][1], R.e[0][2], R.ee[0]);
  q[4] = make_float4(R.e[1][0], R.e[1][1], R.e[1][2], R.ee[1]);
  q[5] = make_float4(R.e[2][0], R.e[2][1], R.e[2][2], R.ee[2]);
  q[6] = make_float4(R.n[0], R.n[1], R.n[2], R.iee[0]);
  q[7] = make_float4(R.m[0][0], R.m[0][1], R.m[0][2], R.iee[1]);
  q[8] = make_float4(R.m[1][0], R.m[1][1], R.m[1][2], R.iee[2]);
  q[9] = make_float4(R.m[2][0], R.m[2][1], R.m[2][2], R.mc[0]);
  q[10] = make_float4(R.ev[0], R.ev[1], R.ev[2], R.mc[1]);
  q[11] = make_float4(R.sc[0], R.sc[1], R.sc[2], R.sr);   // the ball: one aligned load
  q[12] = make_float4(R.mc[2], R.hd, R.ph, 0.f);          // hd, ph again beside it for the ball test
}

__device__ __forceinline__ void load_rec(RecL& R, const RecSmemL& S) {
  const float4* q = reinterpret_cast<const float4*>(S.x);
  float4 a[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) a[k] = q[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R.v[i][0] = a[i].x; R.v[i][1] = a[i].y; R.v[i][2] = a[i].z;
    R.e[i][0] = a[3 + i].x; R.e[i][1] = a[3 + i].y; R.e[i][2] = a[3 + i].z; R.ee[i] = a[3 + i].w;
    R.m[i][0] = a[7 + i].x; R.m[i][1] = a[7 + i].y; R.m[i][2] = a[7 + i].z;
  }
  R.hd = a[0].w; R.ph = a[1].w; R.c = a[2].w;
  R.n[0] = a[6].x; R.n[1] = a[6].y; R.n[2] = a[6].z;
  R.iee[0] = a[6].w; R.iee[1] = a[7].w; R.iee[2] = a[8].w;
  R.mc[0] = a[9].w; R.mc[1] = a[10].w; R.mc[2] = a[12].x;
  R.ev[0] = a[10].x; R.ev[1] = a[10].y; R.ev[2] = a[10].z;
  R.sc[0] = a[11].x; R.sc[1] = a[11].y; R.sc[2] = a[11].z; R.sr = a[11].w;
}

// (a . x) - k as one FMA chain
__device__ __forceinline__ float affine3(const float a[3], const float x[3], float k) {
  return fmaf(a[2], x[2], fmaf(a[1], x[1], fmaf(a[0], x[0], -k)));
}

// Squared minimum over the 15 candidate distances of P and Q (as tri_d2),
// with `maybe` set when both facets straddle the other's plane within eh.
__device__ __forceinline__ float tri_d2(const RecL& P, const RecL& Q, float eh, bool& maybe) {
  const float INF = inf_(0.f);
  float d2 = INF;
  float hP[3], hQ[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {   // vertices of P against Q's interior
    hP[i] = affine3(Q.n, P.v[i], Q.c);
    const float g = min(affine3(Q.m[0], P.v[i], Q.mc[0]),
                        min(affine3(Q.m[1], P.v[i], Q.mc[1]), affine3(Q.m[2], P.v[i], Q.mc[2])));
    d2 = min(d2, g >= 0.f ? hP[i] * hP[i] : INF);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {   // vertices of Q against P's interior
    hQ[j] = affine3(P.n, Q.v[j], P.c);
    const float g = min(affine3(P.m[0], Q.v[j], P.mc[0]),
                        min(affine3(P.m[1], Q.v[j], P.mc[1]), affine3(P.m[2], Q.v[j], P.mc[2])));
    d2 = min(d2, g >= 0.f ? hQ[j] * hQ[j] : INF);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)     // edge i of P against edge j of Q
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float* d1 = P.e[i];
      const float* dq = Q.e[j];
      const float b = dot3(d1, dq);
      const float c = -affine3(d1, Q.v[j], P.ev[i]);   // d1 . (p_i - q_j)
      const float f = affine3(dq, P.v[i], Q.ev[j]);    // dq . (p_i - q_j)
      const float den = fmaf(P.ee[i], Q.ee[j], -b * b);
      const float num = fmaf(b, f, -c * Q.ee[j]);
      float s = __saturatef(__fdividef(num, den));
      const float t = __saturatef(fmaf(b, s, f) * Q.iee[j]);
      s = __saturatef(fmaf(b, t, -c) * P.iee[i]);
      const float wx = fmaf(s, d1[0], P.v[i][0]) - fmaf(t, dq[0], Q.v[j][0]);
      const float wy = fmaf(s, d1[1], P.v[i][1]) - fmaf(t, dq[1], Q.v[j][1]);
      const float wz = fmaf(s, d1[2], P.v[i][2]) - fmaf(t, dq[2], Q.v[j][2]);
      d2 = min(d2, fmaf(wz, wz, fmaf(wy, wy, wx * wx)));
    }
  const float pmin = min(hP[0], min(hP[1], hP[2])), pmax = max(hP[0], max(hP[1], hP[2]));
  const float qmin = min(hQ[0], min(hQ[1], hQ[2])), qmax = max(hQ[0], max(hQ[1], hQ[2]));
  maybe = !((pmin > eh) || (pmax < -eh) || (qmin > eh) || (qmax < -eh));
  return d2;
}

// Coarse-LoD culling of a facet pair from its balls: true when the pair can
// lower neither the running lower bound lbm (its terms are d - ph - ph) nor
// the running upper bound ubu (d + hd + hd), i.e. when the balls are apart
// by more than both lbm + ph + ph and ubu - hd - hd (the test of
// balls_apart for both bounds, sharing the centre distance: both hold iff
// the smaller limit is >= 0 and the squared distance beats the larger one).
__device__ __forceinline__ bool coarse_cull(const float pc[3], float pr, float pph, float phd, const float qc[3],
                                            float qr, float qph, float qhd, float lbm, float ubu) {
  const float dx = pc[0] - qc[0], dy = pc[1] - qc[1], dz = pc[2] - qc[2];
  const float dist2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const float rr = pr + qr;
  const float l1 = __fadd_ru(lbm, __fadd_ru(pph, qph)) + rr;
  const float l2 = __fsub_ru(ubu, __fadd_rd(phd, qhd)) + rr;
  const float lo = fminf(l1, l2), hi = fmaxf(l1, l2);
  return lo >= 0.f && dist2 * 0.99996f > hi * hi * 1.00002f;
}
__device__ __forceinline__ bool coarse_cull(const double*, double, double, double, const double*, double, double,
                                            double, double, double) {
  return false;   // double precision: coarse steps do not cull
}

// Ball, hd and ph of a shared-memory record (read before the record itself).
__device__ __forceinline__ void rec_ball(const RecSmemL& S, float c[3], float& r, float& hd, float& ph) {
  const float4 b = reinterpret_cast<const float4*>(S.x)[11];
  const float2 h = *reinterpret_cast<const float2*>(S.x + 49);   // hd, ph
  c[0] = b.x;
  c[1] = b.y;
  c[2] = b.z;
  r = b.w;
  hd = h.x;
  ph = h.y;
}
__device__ __forceinline__ void rec_ball(const RecSmem<double>& S, double c[3], double& r, double& hd, double& ph) {
  c[0] = S.x[40];
  c[1] = S.x[41];
  c[2] = S.x[42];
  r = S.x[43];
  hd = S.x[3];
  ph = S.x[7];
}

// Record types per precision: FP32 kernels use the form above, FP64 the
// difference form (which reproduces the oracle's arithmetic).
template <class T>
struct RecOf {
  using R = Rec<T>;
  using S = RecSmem<T>;
};
template <>
struct RecOf<float> {
  using R = RecL;
  using S = RecSmemL;
};

// Sign of the orientation determinant of (a, b, c, d) from single-precision
// differences of the raw float coordinates, or 0 when the sign is not
// certain.  Each difference carries a relative rounding error of at most
// u = 2^-24, and the evaluation of the 3x3 determinant adds a few u of the
// permanent Pm (the same sum with absolute values), so the computed value is
// within 12 u Pm of the exact one; a value beyond 2^-19 Pm (32 u Pm) has the
// exact sign.  A semi-static filter in the manner of adaptive-precision
// geometric predicates; uncertain signs go to exact arithmetic.
__device__ __forceinline__ int orient_sign32(const float4& a, const float4& b, const float4& c, const float4& d) {
  const float x0 = b.x - a.x, x1 = b.y - a.y, x2 = b.z - a.z;
  const float y0 = c.x - a.x, y1 = c.y - a.y, y2 = c.z - a.z;
  const float z0 = d.x - a.x, z1 = d.y - a.y, z2 = d.z - a.z;
  const float c0 = y1 * z2 - y2 * z1, c1 = y2 * z0 - y0 * z2, c2 = y0 * z1 - y1 * z0;
  const float det = x0 * c0 + x1 * c1 + x2 * c2;
  const float p0 = fabsf(y1 * z2) + fabsf(y2 * z1), p1 = fabsf(y2 * z0) + fabsf(y0 * z2),
              p2 = fabsf(y0 * z1) + fabsf(y1 * z0);
  const float perm = fabsf(x0) * p0 + fabsf(x1) * p1 + fabsf(x2) * p2;
  const float bound = perm * 1.9073486e-06f;   // 2^-19
  // outside [1e-20, 1e30] (tiny facets whose products may be subnormal,
  // overflow, NaN) the sign is left to double precision
  if (!(perm > 1e-20f && perm < 1e30f)) return 0;
  return det > bound ? 1 : (det < -bound ? -1 : 0);
}

// The same sign from double-precision differences of the float coordinates
// (exact for coordinates within 2^29 of each other, else rounded once),
// trusted beyond 16 u_64 Pm: the first-order error of the rounded
// differences, products and sums stays below 8 u_64 Pm.  0 when not
// certain (also outside [1e-200, 1e200]).
__device__ __forceinline__ int orient_sign64(const float4& a, const float4& b, const float4& c, const float4& d) {
  const double x0 = (double)b.x - a.x, x1 = (double)b.y - a.y, x2 = (double)b.z - a.z;
  const double y0 = (double)c.x - a.x, y1 = (double)c.y - a.y, y2 = (double)c.z - a.z;
  const double z0 = (double)d.x - a.x, z1 = (double)d.y - a.y, z2 = (double)d.z - a.z;
  const double c0 = y1 * z2 - y2 * z1, c1 = y2 * z0 - y0 * z2, c2 = y0 * z1 - y1 * z0;
  const double det = x0 * c0 + x1 * c1 + x2 * c2;
  const double p0 = fabs(y1 * z2) + fabs(y2 * z1), p1 = fabs(y2 * z0) + fabs(y0 * z2),
               p2 = fabs(y0 * z1) + fabs(y1 * z0);
  const double perm = fabs(x0) * p0 + fabs(x1) * p1 + fabs(x2) * p2;
  if (!(perm > 1e-200 && perm < 1e200)) return 0;
  const double bound = perm * 1.7763568394002505e-15;   // 2^-49 = 16 u_64
  return det > bound ? 1 : (det < -bound ? -1 : 0);
}

// The meeting decision from filtered signs (SIGN: orient_sign32 or
// orient_sign64): 1 when an edge
// of one facet certainly crosses the other strictly inside, 0 when every
// edge certainly misses (both ends strictly on one side of the plane, or
// the line passing an edge strictly on the wrong side), -1 when some sign
// is not certain (tri_meet_exact then decides; touching, coplanar and
// degenerate configurations always land there, since the filter never
// certifies a zero sign).
template <int (*SIGN)(const float4&, const float4&, const float4&, const float4&)>
__device__ __forceinline__ int cross_filter(const float4* fp, const float4* fq) {
  bool unsure = false;
  for (int side = 0; side < 2; ++side) {
    const float4* A = side ? fq : fp;
    const float4* B = side ? fp : fq;
    int h[3];
    for (int i = 0; i < 3; ++i) h[i] = SIGN(B[0], B[1], B[2], A[i]);
    for (int i = 0; i < 3; ++i) {
      const int k = (i + 1) % 3;
      if (h[i] == 0 || h[k] == 0) {
        unsure = true;   // the edge may or may not cross B's plane
        continue;
      }
      if (h[i] == h[k]) continue;   // both ends on one side
      const int o1 = SIGN(A[i], A[k], B[0], B[1]);
      const int o2 = SIGN(A[i], A[k], B[1], B[2]);
      const int o3 = SIGN(A[i], A[k], B[2], B[0]);
      if (o1 == 0 || o2 == 0 || o3 == 0) {
        unsure = true;
        continue;
      }
      if (o1 == o2 && o2 == o3) return 1;
    }
  }
  return unsure ? -1 : 0;
}

// The meeting decision where filtered signs make it certain: single
// precision, then double precision; -1 when neither is certain (touching,
// coplanar and degenerate configurations, or signs within rounding).
__device__ __forceinline__ int cross_filtered(const float4* fp, const float4* fq) {
  const int f = cross_filter<orient_sign32>(fp, fq);
  return f >= 0 ? f : cross_filter<orient_sign64>(fp, fq);
}

// Do the closed facets (raw float vertices) meet?  Exact: filtered signs
// where they are certain, else exact expansion arithmetic.  The refinement
// kernels use cross_filtered alone and queue the uncertain pairs for a
// separate kernel, so that the expansion arithmetic (and its local memory)
// stays out of their code.
static __device__ __forceinline__ bool cross_decide(const float4* fp, const float4* fq) {
  const int f = cross_filtered(fp, fq);
  return f >= 0 ? f == 1 : tri_meet_exact(fp, fq);
}

// Forward error margins of the single-precision test for coordinates
// bounded by rho (pair-local, per axis), maximal edge length L and minimal
// facet sine smin:
//   heights   |h~ - h| <= 128 u rho / smin   (straddle pre-filter)
//   distance  |d~ - d| <= 256 u rho / smin + 8 sqrt(u) L
// (u = 2^-24; the sqrt(u) L term covers nearly parallel edges, where the
// segment parameter is ill-conditioned but any clamped value is a true
// point pair).
struct Margins {
  float eps, eh, ew;
};

// Below a sine of 1e-6 (slivers) no margin is claimed: eh = eps = +inf, so
// every straddle test passes (the exact meeting test decides) and the unit
// decides nothing in single precision (its pairs go to double precision).
__host__ __device__ __forceinline__ Margins fp32_margins(float rho, float L, float smin) {
  const float u = 5.9604644775390625e-08f;          // 2^-24
  const float su = 2.44140625e-04f;                 // sqrt(2^-24) = 2^-12
  Margins m;
  m.ew = 0.0f;
  if (!(smin >= 1e-6f)) {
    m.eh = m.eps = INFINITY;
    return m;
  }
  m.eh = 128.0f * u * rho / smin;
  m.eps = 256.0f * u * rho / smin + 8.0f * su * L;
  return m;
}

// The double-precision kernels take their distances as exact (eps = 0) but
// need the straddle margin of their heights for the meeting test: the same
// derivation with u = 2^-53 (the single-precision margin times 2^-29).
__host__ __device__ __forceinline__ float fp64_height_margin(const Margins& m32) {
  return m32.eh * 1.862645149230957e-09f;   // 2^-29 (inf stays inf)
}

}  // namespace pj
