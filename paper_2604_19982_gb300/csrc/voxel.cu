// Voxels of a loaded set (section 2.1, "Object Voxelization", "Consistent
// Voxelization across LoDs", "Object and Voxel Centers") and voxel-pair
// filtering of object pairs (section 3.2: Algorithm 1 bounds every voxel
// pair, Algorithm 2 keeps those whose lower bound does not exceed the object
// pair's upper bound, by count / scan / compact).
//
// Voxelization runs once per object at load (one CTA per object):
//   * k = round(2 % of the original facets), at least 1 and at most the
//     coarsest LoD's facets; none without coarsest facets;
//   * the initial centres are the coarsest vertex array's entries at the
//     evenly spaced positions floor((2j + 1) V / 2k);
//   * two k-means updates over the coarsest facets' centroids;
//   * every facet of every LoD is labelled with its nearest final centre,
//     which keeps the partition consistent across LoDs;
//   * boxes and anchors come from the original LoD's facets.
// All of it is double precision and every expression is rounded in a fixed
// order (__dadd_rn / __dmul_rn / __ddiv_rn: no contraction into FMA), so the
// labels, centres, boxes and anchors are the same doubles as a plain
// evaluation of the same formulas on the CPU.
//
// Voxel-pair filtering (one CTA per object pair, grid-stride):
//   k_vp_bound   Algorithm 1: lb = MINDIST of the voxel boxes, ub = distance
//                of the voxel anchors (in double, or in single precision
//                rounded outward); their minima are the object pair's
//                [lb, ub]; with tau >= 0 the pair is a result (ub <= tau),
//                pruned (lb > tau) or undecided;
//   k_vp_count   Algorithm 2 step 1: surviving voxel pairs per undecided pair;
//   scan_i64     step 2: their offsets;
//   k_vp_compact step 3: the survivors (i, j) in row-major order.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pj {

namespace {

constexpr int VOX_T = 256;          // threads of every voxel kernel
constexpr int VOX_WARPS = VOX_T / 32;

__device__ __forceinline__ double dsq3(double x, double y, double z) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

// centroid ((v0 + v1) + v2) / 3 of facet f
__device__ __forceinline__ void centroid(const float4* fac, int64_t f, double& x, double& y, double& z) {
  const float4 a = fac[3 * f], b = fac[3 * f + 1], c = fac[3 * f + 2];
  x = __ddiv_rn(__dadd_rn(__dadd_rn((double)a.x, (double)b.x), (double)c.x), 3.0);
  y = __ddiv_rn(__dadd_rn(__dadd_rn((double)a.y, (double)b.y), (double)c.y), 3.0);
  z = __ddiv_rn(__dadd_rn(__dadd_rn((double)a.z, (double)b.z), (double)c.z), 3.0);
}

// index of the centre (cs: [3k] in shared memory) nearest to (x, y, z); the
// lowest index among equal distances
__device__ __forceinline__ int nearest(const double* cs, int k, double x, double y, double z) {
  double best = 0.0;
  int bj = 0;
  for (int j = 0; j < k; ++j) {
    const double d = dsq3(__dsub_rn(x, cs[3 * j]), __dsub_rn(y, cs[3 * j + 1]), __dsub_rn(z, cs[3 * j + 2]));
    if (j == 0 || d < best) {
      best = d;
      bj = j;
    }
  }
  return bj;
}

// Float order as signed integers (negative floats reversed) for shared
// atomicMin / atomicMax; -0.0 sorts just below +0.0.
__device__ __forceinline__ int ford(float x) {
  const int i = __float_as_int(x);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float fdec(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// k-means of each object's coarsest facets: centres out [3 V_total]; lab
// (the coarsest LoD's label array) holds the assignments of the last update
// and is overwritten by k_vox_label afterwards.
__global__ void __launch_bounds__(VOX_T) k_vox_kmeans(int n, const float4* fac, const int64_t* foff,
                                                      const float* verts, const int64_t* voff,
                                                      const int64_t* vox_off, int updates, int32_t* lab,
                                                      double* centre_out) {
  extern __shared__ double cs[];   // [3k]
  for (int o = blockIdx.x; o < n; o += gridDim.x) {
    const int64_t f0 = foff[o];
    const int F = (int)(foff[o + 1] - f0);
    const int64_t c0 = vox_off[o];
    const int k = (int)(vox_off[o + 1] - c0);
    const int64_t v0 = voff[o];
    const int64_t V = voff[o + 1] - v0;
    if (k == 0 || V <= 0) continue;   // the same for every thread of the block
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      const int64_t idx = ((2 * (int64_t)j + 1) * V) / (2 * (int64_t)k);   // < V
      const float* p = verts + 3 * (v0 + idx);
      cs[3 * j] = (double)p[0];
      cs[3 * j + 1] = (double)p[1];
      cs[3 * j + 2] = (double)p[2];
    }
    __syncthreads();
    for (int u = 0; u < updates; ++u) {
      for (int f = threadIdx.x; f < F; f += blockDim.x) {
        double x, y, z;
        centroid(fac, f0 + f, x, y, z);
        lab[f0 + f] = nearest(cs, k, x, y, z);
      }
      __syncthreads();
      // each centre becomes the running sum of its members in facet order
      // divided by their count (a centre without members stays)
      for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        int cnt = 0;
        for (int f = 0; f < F; ++f) {
          if (lab[f0 + f] != j) continue;
          double x, y, z;
          centroid(fac, f0 + f, x, y, z);
          if (cnt == 0) {
            sx = x;
            sy = y;
            sz = z;
          } else {
            sx = __dadd_rn(sx, x);
            sy = __dadd_rn(sy, y);
            sz = __dadd_rn(sz, z);
          }
          ++cnt;
        }
        if (cnt > 0) {
          cs[3 * j] = __ddiv_rn(sx, (double)cnt);
          cs[3 * j + 1] = __ddiv_rn(sy, (double)cnt);
          cs[3 * j + 2] = __ddiv_rn(sz, (double)cnt);
        }
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < 3 * k; j += blockDim.x) centre_out[3 * c0 + j] = cs[j];
    __syncthreads();
  }
}

// every facet of one LoD labelled with its object's nearest final centre
// (-1 for objects without voxels)
__global__ void __launch_bounds__(VOX_T) k_vox_label(int n, const float4* fac, const int64_t* foff,
                                                     const int64_t* vox_off, const double* centre, int32_t* lab) {
  extern __shared__ double cs[];   // [3k]
  for (int o = blockIdx.x; o < n; o += gridDim.x) {
    const int64_t f0 = foff[o];
    const int F = (int)(foff[o + 1] - f0);
    const int64_t c0 = vox_off[o];
    const int k = (int)(vox_off[o + 1] - c0);
    if (k == 0) {
      for (int f = threadIdx.x; f < F; f += blockDim.x) lab[f0 + f] = -1;
      continue;
    }
    for (int j = threadIdx.x; j < 3 * k; j += blockDim.x) cs[j] = centre[3 * c0 + j];
    __syncthreads();
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
      double x, y, z;
      centroid(fac, f0 + f, x, y, z);
      lab[f0 + f] = nearest(cs, k, x, y, z);
    }
    __syncthreads();
  }
}

// Boxes of each voxel's original facets, and its anchor: the corner closest
// to the box centre, the first in (facet, corner) order among equals.
// box out [6 V_total] (lo.xyz, hi.xyz; +inf / -inf for a voxel without
// original facets), anchor out [3 V_total] (NaN for such a voxel).
__global__ void __launch_bounds__(VOX_T) k_vox_box(int n, const float4* fac, const int64_t* foff,
                                                   const int64_t* vox_off, const int32_t* lab, float* box,
                                                   float* anchor, int* err) {
  extern __shared__ unsigned long long sb[];   // bd [k] | lo [3k] | hi [3k] | bi [k]
  for (int o = blockIdx.x; o < n; o += gridDim.x) {
    const int64_t f0 = foff[o];
    const int F = (int)(foff[o + 1] - f0);
    const int64_t c0 = vox_off[o];
    const int k = (int)(vox_off[o + 1] - c0);
    if (k == 0) continue;
    unsigned long long* bd = sb;
    int* lo = reinterpret_cast<int*>(sb + k);
    int* hi = lo + 3 * k;
    int* bi = hi + 3 * k;
    const int inf_lo = ford(__int_as_float(0x7f800000));    // +inf
    const int inf_hi = ford(__int_as_float((int)0xff800000));   // -inf
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      bd[j] = ~0ull;
      bi[j] = INT_MAX;
      for (int a = 0; a < 3; ++a) {
        lo[3 * j + a] = inf_lo;
        hi[3 * j + a] = inf_hi;
      }
    }
    __syncthreads();
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
      const int j = lab[f0 + f];
      if (j < 0 || j >= k) {
        set_err(err, ERR_BOUNDS);
        continue;
      }
      for (int c = 0; c < 3; ++c) {
        const float4 v = fac[3 * (f0 + f) + c];
        atomicMin(&lo[3 * j], ford(v.x));
        atomicMin(&lo[3 * j + 1], ford(v.y));
        atomicMin(&lo[3 * j + 2], ford(v.z));
        atomicMax(&hi[3 * j], ford(v.x));
        atomicMax(&hi[3 * j + 1], ford(v.y));
        atomicMax(&hi[3 * j + 2], ford(v.z));
      }
    }
    __syncthreads();
    // two passes: the least squared distance to the box centre, then the
    // first corner that reaches it
    for (int pass = 0; pass < 2; ++pass) {
      for (int f = threadIdx.x; f < F; f += blockDim.x) {
        const int j = lab[f0 + f];
        if (j < 0 || j >= k) continue;
        const double cx = __dmul_rn(0.5, __dadd_rn((double)fdec(lo[3 * j]), (double)fdec(hi[3 * j])));
        const double cy = __dmul_rn(0.5, __dadd_rn((double)fdec(lo[3 * j + 1]), (double)fdec(hi[3 * j + 1])));
        const double cz = __dmul_rn(0.5, __dadd_rn((double)fdec(lo[3 * j + 2]), (double)fdec(hi[3 * j + 2])));
        for (int c = 0; c < 3; ++c) {
          const float4 v = fac[3 * (f0 + f) + c];
          const double d = dsq3(__dsub_rn((double)v.x, cx), __dsub_rn((double)v.y, cy), __dsub_rn((double)v.z, cz));
          const unsigned long long b = d2bits(d);
          if (pass == 0)
            atomicMin(&bd[j], b);
          else if (b == bd[j])
            atomicMin(&bi[j], 3 * f + c);
        }
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      float* bx = box + 6 * (c0 + j);
      for (int a = 0; a < 3; ++a) {
        bx[a] = fdec(lo[3 * j + a]);
        bx[3 + a] = fdec(hi[3 * j + a]);
      }
      float* an = anchor + 3 * (c0 + j);
      if (bi[j] != INT_MAX) {
        const float4 v = fac[3 * (f0 + bi[j] / 3) + bi[j] % 3];
        an[0] = v.x;
        an[1] = v.y;
        an[2] = v.z;
      } else {
        an[0] = an[1] = an[2] = __int_as_float(0x7fc00000);
      }
    }
    __syncthreads();
  }
}

}  // namespace

namespace {

// box (lo.xyz, hi.xyz) of a voxel is empty when lo.x > hi.x (+inf / -inf)
__device__ __forceinline__ bool box_empty(const float* b) { return !(b[0] <= b[3]); }

// block-wide minimum of v (every thread gets it); red: [VOX_WARPS] shared
__device__ __forceinline__ double block_min(double v, double* red) {
  v = warp_min(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = red[0];
  for (int i = 1; i < VOX_WARPS; ++i) m = fmin(m, red[i]);
  return m;
}

__device__ __forceinline__ long long block_sum(long long v, long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  long long s = 0;
  for (int i = 0; i < VOX_WARPS; ++i) s += red[i];
  return s;
}

struct VoxView {
  const int64_t* off;   // [n+1]
  const float* box;     // [6 V]
  const float* anc;     // [3 V]
  int n;
};

// One voxel pair's bounds: lb = MINDIST of boxes a, b (lo.xyz, hi.xyz), ub =
// distance of anchors ua, ub_.  F64: double precision rounded to nearest in
// a fixed order.  Otherwise single precision with outward rounding: every
// step of lb rounds down and every step of ub rounds up (|x - y| bounded
// by the larger magnitude of its two directed differences), so lb never
// exceeds the exact MINDIST and ub is never below the exact distance.
template <bool F64>
struct VpPrec {
  using T = double;
};
template <>
struct VpPrec<false> {
  using T = float;
};

__device__ __forceinline__ void vp_bounds(const float* a, const float* b, const float* ua, const float* ub_, double& lb,
                                          double& ub) {
  double g[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const double d1 = __dsub_rn((double)b[e], (double)a[3 + e]);
    const double d2 = __dsub_rn((double)a[e], (double)b[3 + e]);
    g[e] = fmax(0.0, fmax(d1, d2));
  }
  lb = __dsqrt_rn(dsq3(g[0], g[1], g[2]));
  ub = __dsqrt_rn(dsq3(__dsub_rn((double)ua[0], (double)ub_[0]), __dsub_rn((double)ua[1], (double)ub_[1]),
                       __dsub_rn((double)ua[2], (double)ub_[2])));
}

__device__ __forceinline__ void vp_bounds(const float* a, const float* b, const float* ua, const float* ub_, float& lb,
                                          float& ub) {
  float g[3], h[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    g[e] = fmaxf(0.f, fmaxf(__fsub_rd(b[e], a[3 + e]), __fsub_rd(a[e], b[3 + e])));
    h[e] = fmaxf(fabsf(__fsub_ru(ua[e], ub_[e])), fabsf(__fsub_rd(ua[e], ub_[e])));
  }
  lb = __fsqrt_rd(__fadd_rd(__fadd_rd(__fmul_rd(g[0], g[0]), __fmul_rd(g[1], g[1])), __fmul_rd(g[2], g[2])));
  ub = __fsqrt_ru(__fadd_ru(__fadd_ru(__fmul_ru(h[0], h[0]), __fmul_ru(h[1], h[1])), __fmul_ru(h[2], h[2])));
}

// The double of a float x >= 0 (or +inf), exactly, by integer operations
// (exponent rebiased from 127 to 1023, significand shifted up by 29 bits),
// so that the single-precision path issues no double-precision operation
// per voxel pair; subnormal x take the conversion instruction.
__device__ __forceinline__ double widen(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = u >> 23;
  const unsigned long long f = (unsigned long long)(u & 0x7fffffu) << 29;
  if (u == 0) return 0.0;
  if (e == 0) return (double)x;
  if (e == 0xffu) return __longlong_as_double((long long)(0x7ff0000000000000ull | f));
  return __longlong_as_double((long long)(((unsigned long long)(e + 896u) << 52) | f));
}
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }

// Algorithm 1: one CTA per object pair, its n_r x n_s voxel pairs flattened
// over the threads (row-major t = i n_s + j); vp_off [n+1] holds each
// pair's first slot.  Pairs whose ids lie outside the sets are skipped
// (ERR_BOUNDS), slots at or past cap are not written (ERR_CAPACITY).
template <bool F64>
__global__ void __launch_bounds__(VOX_T) k_vp_bound(int64_t n, const int32_t* pr, const int32_t* ps, VoxView R,
                                                    VoxView S, const int64_t* vp_off, int64_t cap, double tau,
                                                    double* vp_lb, double* vp_ub, double* op_lb, double* op_ub,
                                                    uint8_t* status, int* err) {
  __shared__ double red[VOX_WARPS];
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    const int r = pr[p], s = ps[p];
    if (r < 0 || r >= R.n || s < 0 || s >= S.n) {
      if (threadIdx.x == 0) {
        set_err(err, ERR_BOUNDS);
        op_lb[p] = op_ub[p] = __longlong_as_double(0x7ff0000000000000LL);
        status[p] = 2;
      }
      continue;
    }
    const int64_t i0 = R.off[r], j0 = S.off[s];
    const int64_t nr = R.off[r + 1] - i0, ns = S.off[s + 1] - j0;
    const int64_t m = nr * ns;
    const int64_t base = vp_off[p];
    const bool room = base + m <= cap;
    if (!room && threadIdx.x == 0) set_err(err, ERR_CAPACITY);
    using V = typename VpPrec<F64>::T;
    const V inf = (V)INFINITY;
    V tl = inf, tu = inf;
    if (m > 0) {
      // 32-bit row / column of t, advanced without a division per step
      // (m <= PJ_VOXEL_MAX^2 < 2^31)
      const int nsi = (int)ns, mi = (int)m, step = (int)blockDim.x;
      const int q = step / nsi, rr = step - q * nsi;
      int t = (int)threadIdx.x, i = t / nsi, j = t - i * nsi;
      for (; t < mi; t += step) {
        const float* a = R.box + 6 * (i0 + i);
        const float* b = S.box + 6 * (j0 + j);
        V lb = inf, ub = inf;   // a voxel without facets bounds nothing
        if (!box_empty(a) && !box_empty(b)) vp_bounds(a, b, R.anc + 3 * (i0 + i), S.anc + 3 * (j0 + j), lb, ub);
        if (room) {
          vp_lb[base + t] = widen(lb);
          vp_ub[base + t] = widen(ub);
        }
        tl = vmin(tl, lb);
        tu = vmin(tu, ub);
        i += q;
        j += rr;
        if (j >= nsi) {
          j -= nsi;
          ++i;
        }
      }
    }
    const double olb = block_min(widen(tl), red);
    const double oub = block_min(widen(tu), red);
    if (threadIdx.x == 0) {
      op_lb[p] = olb;
      op_ub[p] = oub;
      uint8_t stt = 0;
      if (tau >= 0.0) stt = oub <= tau ? 1 : (olb > tau ? 2 : 0);
      status[p] = stt;
    }
  }
}

// Algorithm 2, step 1: per undecided pair, its voxel pairs with lb <= the
// pair's ub (0 for decided pairs and pairs without room)
__global__ void __launch_bounds__(VOX_T) k_vp_count(int64_t n, const int64_t* vp_off, int64_t cap,
                                                    const double* vp_lb, const double* op_ub, const uint8_t* status,
                                                    int64_t* cnt) {
  __shared__ long long red[VOX_WARPS];
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    const int64_t base = vp_off[p], m = vp_off[p + 1] - base;
    long long c = 0;
    if (status[p] == 0 && base + m <= cap) {
      const double u = op_ub[p];
      for (int64_t t = threadIdx.x; t < m; t += blockDim.x) c += vp_lb[base + t] <= u;
    }
    c = block_sum(c, red);
    if (threadIdx.x == 0) cnt[p] = c;
  }
}

// Algorithm 2, step 3: the surviving voxel pairs (i, j) of each undecided
// pair at kept_off[p], in row-major order (a stable block-wide compaction)
__global__ void __launch_bounds__(VOX_T) k_vp_compact(int64_t n, const int32_t* ps, VoxView S,
                                                      const int64_t* vp_off, int64_t cap,
                                                      const double* vp_lb, const double* op_ub,
                                                      const uint8_t* status, const int64_t* kept_off,
                                                      int32_t* kept) {
  __shared__ int wsum[VOX_WARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    const int64_t base = vp_off[p], m = vp_off[p + 1] - base;
    if (status[p] != 0 || base + m > cap) continue;   // the same for the whole block
    const int s = ps[p];
    const int64_t ns = S.off[s + 1] - S.off[s];
    const double u = op_ub[p];
    int64_t out = kept_off[p];
    for (int64_t t0 = 0; t0 < m; t0 += blockDim.x) {
      const int64_t t = t0 + threadIdx.x;
      const bool keep = t < m && vp_lb[base + t] <= u;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) wsum[w] = __popc(bal);
      __syncthreads();
      int before = 0, total = 0;
      for (int i = 0; i < VOX_WARPS; ++i) {
        before += i < w ? wsum[i] : 0;
        total += wsum[i];
      }
      if (keep) {
        const int64_t q = out + before + __popc(bal & ((1u << lane) - 1u));
        const int i = (int)t / (int)ns;
        kept[2 * q] = i;
        kept[2 * q + 1] = (int)t - i * (int)ns;
      }
      out += total;
      __syncthreads();
    }
  }
}

// voxel pairs per object pair (n_r n_s; 0 for ids out of range)
__global__ void k_vp_sizes(int64_t n, const int32_t* pr, const int32_t* ps, VoxView R, VoxView S, int64_t* sz) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int r = pr[p], s = ps[p];
  if (r < 0 || r >= R.n || s < 0 || s >= S.n) {
    sz[p] = 0;
    return;
  }
  sz[p] = (R.off[r + 1] - R.off[r]) * (S.off[s + 1] - S.off[s]);
}

}  // namespace

namespace {

constexpr int VOX_UPDATES = 2;   // centroid updates of the k-means (section 2.1)

template <class K>
void smem_attr(K kern, size_t bytes) {
  if (bytes > 48 * 1024) PJ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

VoxView view(const pj_set* s) { return VoxView{s->vox_off, s->vox_box, s->vox_anchor, s->n}; }

}  // namespace

void free_voxels(pj_set* s) {
  cudaFree(s->vox_off);
  cudaFree(s->vox_centre);
  cudaFree(s->vox_box);
  cudaFree(s->vox_anchor);
  for (int l = 0; l < PJ_MAX_LODS; ++l) {
    cudaFree(s->vox_label[l]);
    s->vox_label[l] = nullptr;
  }
  s->vox_off = nullptr;
  s->vox_centre = nullptr;
  s->vox_box = s->vox_anchor = nullptr;
  s->vox_off_h.clear();
  s->V = 0;
  s->voxels = false;
}

void voxelize_set(pj_ctx* ctx, pj_set* s, const float* verts0, const int64_t* voff0, cudaStream_t st) {
  const int n = s->n, L = s->L;
  const LodData& c = s->lod[0];
  const LodData& o = s->lod[L - 1];
  s->vox_off_h.assign((size_t)n + 1, 0);
  int64_t kmax = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t fc = c.foff_h[i + 1] - c.foff_h[i];
    const int64_t fo = o.foff_h[i + 1] - o.foff_h[i];
    // round(F / 50) with halves up, at least 1, at most the coarsest facets
    const int64_t k = fc <= 0 ? 0 : std::max<int64_t>(1, std::min<int64_t>((fo + 25) / 50, fc));
    if (k > PJ_VOXEL_MAX) throw ApiError{PJ_EINVAL, "an object needs more voxels than PJ_VOXEL_MAX"};
    kmax = std::max(kmax, k);
    s->vox_off_h[i + 1] = s->vox_off_h[i] + k;
  }
  s->V = s->vox_off_h[n];
  s->vox_kmax = (int)kmax;
  auto alloc = [&](void** p, size_t bytes) {
    note_alloc();
    PJ_CK(cudaMallocAsync(p, std::max<size_t>(bytes, 16), st));
  };
  alloc((void**)&s->vox_off, ((size_t)n + 1) * 8);
  PJ_CK(cudaMemcpyAsync(s->vox_off, s->vox_off_h.data(), ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, st));
  alloc((void**)&s->vox_centre, (size_t)s->V * 3 * 8);
  alloc((void**)&s->vox_box, (size_t)s->V * 6 * 4);
  alloc((void**)&s->vox_anchor, (size_t)s->V * 3 * 4);
  for (int l = 0; l < L; ++l) alloc((void**)&s->vox_label[l], (size_t)s->lod[l].F * 4);
  if (s->V > 0) PJ_CK(cudaMemsetAsync(s->vox_centre, 0, (size_t)s->V * 3 * 8, st));
  s->voxels = true;
  if (n == 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>(n, (int64_t)ctx->sm_count * 8);
  const size_t sm_c = std::max<size_t>(8, (size_t)kmax * 3 * 8);
  const size_t sm_b = std::max<size_t>(8, (size_t)kmax * (8 + 24 + 4));
  smem_attr(k_vox_kmeans, sm_c);
  smem_attr(k_vox_label, sm_c);
  smem_attr(k_vox_box, sm_b);
  if (s->V > 0) {
    k_vox_kmeans<<<grid, VOX_T, sm_c, st>>>(n, c.fac, c.foff, verts0, voff0, s->vox_off, VOX_UPDATES,
                                            s->vox_label[0], s->vox_centre);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
  for (int l = 0; l < L; ++l) {
    k_vox_label<<<grid, VOX_T, sm_c, st>>>(n, s->lod[l].fac, s->lod[l].foff, s->vox_off, s->vox_centre,
                                           s->vox_label[l]);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
  if (s->V > 0) {
    k_vox_box<<<grid, VOX_T, sm_b, st>>>(n, o.fac, o.foff, s->vox_off, s->vox_label[L - 1], s->vox_box,
                                         s->vox_anchor, ctx->d_err);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
}

void voxel_filter(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps, int64_t n,
                  double tau, bool fp64, double* op_lb, double* op_ub, uint8_t* status, int64_t* vp_off, double* vp_lb,
                  double* vp_ub, int64_t vp_cap, int64_t* kept_off, int32_t* kept, int64_t* n_kept,
                  cudaStream_t st) {
  struct Temps {
    std::vector<void*> v;
    cudaStream_t st;
    ~Temps() {
      for (void* p : v) cudaFreeAsync(p, st);
    }
  } temps{{}, st};
  cudaEvent_t ev[6] = {};
  struct Events {
    cudaEvent_t* e;
    ~Events() {
      for (int i = 0; i < 6; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } evs{ev};
  for (int i = 0; i < 6; ++i) PJ_CK(cudaEventCreate(&ev[i]));
  int64_t* sz = nullptr;
  int64_t* cnt = nullptr;
  note_alloc();
  PJ_CK(cudaMallocAsync((void**)&sz, (size_t)std::max<int64_t>(n, 1) * 8, st));
  temps.v.push_back(sz);
  note_alloc();
  PJ_CK(cudaMallocAsync((void**)&cnt, (size_t)std::max<int64_t>(n, 1) * 8, st));
  temps.v.push_back(cnt);
  PJ_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  const VoxView vr = view(R), vs = view(S);
  const unsigned g1 = (unsigned)std::max<int64_t>(1, (n + VOX_T - 1) / VOX_T);
  const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)ctx->sm_count * 8));
  PJ_CK(cudaEventRecord(ev[0], st));
  if (n > 0) {
    k_vp_sizes<<<g1, VOX_T, 0, st>>>(n, pr, ps, vr, vs, sz);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
  scan_i64(ctx, sz, vp_off, n, st);
  PJ_CK(cudaEventRecord(ev[1], st));
  if (n > 0) {
    auto kern = fp64 ? k_vp_bound<true> : k_vp_bound<false>;
    kern<<<gp, VOX_T, 0, st>>>(n, pr, ps, vr, vs, vp_off, vp_cap, tau, vp_lb, vp_ub, op_lb, op_ub, status,
                               ctx->d_err);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
  PJ_CK(cudaEventRecord(ev[2], st));
  if (n > 0) {
    k_vp_count<<<gp, VOX_T, 0, st>>>(n, vp_off, vp_cap, vp_lb, op_ub, status, cnt);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
  PJ_CK(cudaEventRecord(ev[3], st));
  scan_i64(ctx, cnt, kept_off, n, st);
  PJ_CK(cudaEventRecord(ev[4], st));
  if (n > 0) {
    k_vp_compact<<<gp, VOX_T, 0, st>>>(n, ps, vs, vp_off, vp_cap, vp_lb, op_ub, status, kept_off, kept);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
  PJ_CK(cudaEventRecord(ev[5], st));
  int64_t tot[2] = {0, 0};
  int herr = 0;
  PJ_CK(cudaMemcpyAsync(&tot[0], vp_off + n, 8, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaMemcpyAsync(&tot[1], kept_off + n, 8, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  if (herr & ERR_BOUNDS) throw ApiError{PJ_EBOUNDS, "an object id of a pair lies outside its set"};
  if ((herr & ERR_CAPACITY) || tot[0] > vp_cap)
    throw ApiError{PJ_EINVAL, "vp_cap is below the voxel pairs of the object pairs (" + std::to_string(tot[0]) + ")"};
  *n_kept = tot[1];
  float ms[5];
  for (int i = 0; i < 5; ++i) PJ_CK(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
  char buf[512];
  snprintf(buf, sizeof buf,
           "{\"prec\": \"%s\", \"op_pairs\": %lld, \"voxel_pairs\": %lld, \"kept\": %lld, \"ms_sizes\": %.6f, \"ms_bound\": %.6f, "
           "\"ms_count\": %.6f, \"ms_scan\": %.6f, \"ms_compact\": %.6f}",
           fp64 ? "f64" : "f32", (long long)n, (long long)tot[0], (long long)tot[1], ms[0], ms[1], ms[2], ms[3],
           ms[4]);
  ctx->stats = buf;
}

}  // namespace pj
