// Two triangle tests per lane and instruction: the single-precision test of
// tritri.cuh (the RecL form) evaluated for one r facet against two s facets
// at once with the packed FP32x2 instructions of sm_100-class GPUs
// (fma / mul / add / sub .rn.f32x2).  Each packed instruction does the work
// of two scalar ones in one issue slot, which the refinement loop -- bound
// by instruction issue, not by the FMA pipes -- turns into throughput.
// Saturation, min / max and the reciprocal have no packed form and stay
// scalar on the two halves.  Every half computes what the scalar RecL test
// computes, in the same order and rounding, except the denominator of the
// first segment parameter (one rounding more): that parameter is clamped and
// re-optimised, and any clamped value gives a true point pair, so the
// candidate distances keep the error bound of the scalar test.
#pragma once
#include "tritri.cuh"

namespace pj {

typedef unsigned long long f2;   // two floats: low half = first s facet

__device__ __forceinline__ f2 pk2(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2 dup2(float x) { return pk2(x, x); }
__device__ __forceinline__ float lo2(f2 x) { return __uint_as_float((unsigned)x); }
__device__ __forceinline__ float hi2(f2 x) { return __uint_as_float((unsigned)(x >> 32)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sat2(f2 x) { return pk2(__saturatef(lo2(x)), __saturatef(hi2(x))); }
__device__ __forceinline__ f2 min2(f2 a, f2 b) { return pk2(fminf(lo2(a), lo2(b)), fminf(hi2(a), hi2(b))); }

// (a . x) - k with k given negated (nk = -k), as in affine3
__device__ __forceinline__ f2 affine3x2(const f2 a[3], const f2 x[3], f2 nk) {
  return fma2(a[2], x[2], fma2(a[1], x[1], fma2(a[0], x[0], nk)));
}
__device__ __forceinline__ f2 dot3x2(const f2 a[3], const f2 b[3]) {
  return fma2(a[2], b[2], fma2(a[1], b[1], mul2(a[0], b[0])));
}

// A RecL with every field as a pair; the constants are kept negated.
struct RecL2 {
  f2 v[3][3];
  f2 e[3][3];
  f2 ee[3], iee[3];
  f2 n[3];
  f2 m[3][3];
  f2 nc, nmc[3], nev[3];
};

// the register side: one facet duplicated into both halves
__device__ __forceinline__ void dup_rec(RecL2& D, const RecL& R) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      D.v[i][k] = dup2(R.v[i][k]);
      D.e[i][k] = dup2(R.e[i][k]);
      D.m[i][k] = dup2(R.m[i][k]);
    }
    D.ee[i] = dup2(R.ee[i]);
    D.iee[i] = dup2(R.iee[i]);
    D.n[i] = dup2(R.n[i]);
    D.nmc[i] = dup2(-R.mc[i]);
    D.nev[i] = dup2(-R.ev[i]);
  }
  D.nc = dup2(-R.c);
}

// Shared-memory image of two s facets: field f of facet h (0 / 1) at float
// 2 f + h, 49 fields, padded to 102 floats so that the 16 records of a block
// start on different banks.
constexpr int REC2_FLOATS = 102;
struct RecSmem2 {
  float x[REC2_FLOATS];
};
// field numbers
enum : int {
  F_V = 0,      // v[i][k] at F_V + 3 i + k
  F_E = 9,      // e[i][k]
  F_M = 18,     // m[i][k]
  F_N = 27,     // n[k]
  F_EE = 30,    // ee[i]
  F_IEE = 33,   // iee[i]
  F_NMC = 36,   // -mc[i]
  F_NEV = 39,   // -ev[i]
  F_NC = 42,
  F_HD = 43,
  F_PH = 44,
  F_SC = 45,    // ball centre [k]
  F_SR = 48     // ball radius
};

__device__ __forceinline__ void store_half(RecSmem2& S, int h, const RecL& R) {
  float* x = S.x + h;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      x[2 * (F_V + 3 * i + k)] = R.v[i][k];
      x[2 * (F_E + 3 * i + k)] = R.e[i][k];
      x[2 * (F_M + 3 * i + k)] = R.m[i][k];
    }
    x[2 * (F_N + i)] = R.n[i];
    x[2 * (F_EE + i)] = R.ee[i];
    x[2 * (F_IEE + i)] = R.iee[i];
    x[2 * (F_NMC + i)] = -R.mc[i];
    x[2 * (F_NEV + i)] = -R.ev[i];
  }
  x[2 * F_NC] = -R.c;
  x[2 * F_HD] = R.hd;
  x[2 * F_PH] = R.ph;
#pragma unroll
  for (int k = 0; k < 3; ++k) x[2 * (F_SC + k)] = R.sc[k];
  x[2 * F_SR] = R.sr;
}

__device__ __forceinline__ f2 ld2(const RecSmem2& S, int f) {
  return *reinterpret_cast<const f2*>(S.x + 2 * f);
}

__device__ __forceinline__ void load_pair(RecL2& Q, const RecSmem2& S) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Q.v[i][k] = ld2(S, F_V + 3 * i + k);
      Q.e[i][k] = ld2(S, F_E + 3 * i + k);
      Q.m[i][k] = ld2(S, F_M + 3 * i + k);
    }
    Q.n[i] = ld2(S, F_N + i);
    Q.ee[i] = ld2(S, F_EE + i);
    Q.iee[i] = ld2(S, F_IEE + i);
    Q.nmc[i] = ld2(S, F_NMC + i);
    Q.nev[i] = ld2(S, F_NEV + i);
  }
  Q.nc = ld2(S, F_NC);
}

// The RecL test of P (duplicated) against the two facets of Q: squared
// minimum per half, and per half whether both facets straddle the other's
// plane within eh.
__device__ __forceinline__ f2 tri_d2x2(const RecL2& P, const RecL2& Q, float eh, bool& maybe0, bool& maybe1) {
  const float INF = inf_(0.f);
  f2 d2 = dup2(INF);
  f2 hP[3], hQ[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {   // vertices of P against Q's interior
    hP[i] = affine3x2(Q.n, P.v[i], Q.nc);
    const f2 g0 = affine3x2(Q.m[0], P.v[i], Q.nmc[0]);
    const f2 g1 = affine3x2(Q.m[1], P.v[i], Q.nmc[1]);
    const f2 g2 = affine3x2(Q.m[2], P.v[i], Q.nmc[2]);
    const f2 h2 = mul2(hP[i], hP[i]);
    const float ga = fminf(lo2(g0), fminf(lo2(g1), lo2(g2))), gb = fminf(hi2(g0), fminf(hi2(g1), hi2(g2)));
    d2 = min2(d2, pk2(ga >= 0.f ? lo2(h2) : INF, gb >= 0.f ? hi2(h2) : INF));
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {   // vertices of Q against P's interior
    hQ[j] = affine3x2(P.n, Q.v[j], P.nc);
    const f2 g0 = affine3x2(P.m[0], Q.v[j], P.nmc[0]);
    const f2 g1 = affine3x2(P.m[1], Q.v[j], P.nmc[1]);
    const f2 g2 = affine3x2(P.m[2], Q.v[j], P.nmc[2]);
    const f2 h2 = mul2(hQ[j], hQ[j]);
    const float ga = fminf(lo2(g0), fminf(lo2(g1), lo2(g2))), gb = fminf(hi2(g0), fminf(hi2(g1), hi2(g2)));
    d2 = min2(d2, pk2(ga >= 0.f ? lo2(h2) : INF, gb >= 0.f ? hi2(h2) : INF));
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)     // edge i of P against edge j of Q
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const f2* d1 = P.e[i];
      const f2* dq = Q.e[j];
      const f2 b = dot3x2(d1, dq);
      const f2 cn = affine3x2(d1, Q.v[j], P.nev[i]);   // -c = d1 . q_j - d1 . p_i
      const f2 f = affine3x2(dq, P.v[i], Q.nev[j]);    // dq . (p_i - q_j)
      const f2 den = sub2(mul2(P.ee[i], Q.ee[j]), mul2(b, b));
      const f2 num = fma2(b, f, mul2(cn, Q.ee[j]));    // b f - c ee_q
      const f2 s0 = sat2(mul2(num, pk2(__fdividef(1.f, lo2(den)), __fdividef(1.f, hi2(den)))));
      const f2 t = sat2(mul2(fma2(b, s0, f), Q.iee[j]));
      const f2 s = sat2(mul2(fma2(b, t, cn), P.iee[i]));   // (b t - c) / ee_p
      const f2 wx = sub2(fma2(s, d1[0], P.v[i][0]), fma2(t, dq[0], Q.v[j][0]));
      const f2 wy = sub2(fma2(s, d1[1], P.v[i][1]), fma2(t, dq[1], Q.v[j][1]));
      const f2 wz = sub2(fma2(s, d1[2], P.v[i][2]), fma2(t, dq[2], Q.v[j][2]));
      d2 = min2(d2, fma2(wz, wz, fma2(wy, wy, mul2(wx, wx))));
    }
  {
    const float p0 = fminf(lo2(hP[0]), fminf(lo2(hP[1]), lo2(hP[2])));
    const float p1 = fmaxf(lo2(hP[0]), fmaxf(lo2(hP[1]), lo2(hP[2])));
    const float q0 = fminf(lo2(hQ[0]), fminf(lo2(hQ[1]), lo2(hQ[2])));
    const float q1 = fmaxf(lo2(hQ[0]), fmaxf(lo2(hQ[1]), lo2(hQ[2])));
    maybe0 = !((p0 > eh) || (p1 < -eh) || (q0 > eh) || (q1 < -eh));   // NaN (zero area): maybe
  }
  {
    const float p0 = fminf(hi2(hP[0]), fminf(hi2(hP[1]), hi2(hP[2])));
    const float p1 = fmaxf(hi2(hP[0]), fmaxf(hi2(hP[1]), hi2(hP[2])));
    const float q0 = fminf(hi2(hQ[0]), fminf(hi2(hQ[1]), hi2(hQ[2])));
    const float q1 = fmaxf(hi2(hQ[0]), fmaxf(hi2(hQ[1]), hi2(hQ[2])));
    maybe1 = !((p0 > eh) || (p1 < -eh) || (q0 > eh) || (q1 < -eh));
  }
  return d2;
}

// Are the boxes of P and of facet h of the pair strictly apart on an axis?
__device__ __forceinline__ bool boxes_apart_half(const RecL2& P, const RecSmem2& S, int h) {
  bool apart = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a = S.x[2 * (F_V + k) + h], b = S.x[2 * (F_V + 3 + k) + h], c = S.x[2 * (F_V + 6 + k) + h];
    const float qmin = fminf(a, fminf(b, c)), qmax = fmaxf(a, fmaxf(b, c));
    const float pmin = fminf(lo2(P.v[0][k]), fminf(lo2(P.v[1][k]), lo2(P.v[2][k])));
    const float pmax = fmaxf(lo2(P.v[0][k]), fmaxf(lo2(P.v[1][k]), lo2(P.v[2][k])));
    apart = apart || (pmax < qmin) || (qmax < pmin);
  }
  return apart;
}

}  // namespace pj
