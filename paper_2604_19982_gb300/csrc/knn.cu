// k-NN join on the GPU (section 3.1 "MBB-based Object Filtering" for k-NN
// and section 3.4, Algorithm 6).
//
// Candidates: theta_r = the k-th smallest anchor distance from r to S (an
// upper bound of the k-th smallest d(r, s), since anchors lie on the
// surfaces); every s with box MINDIST(r, s) <= theta_r is a candidate.  A
// warp per r finds theta_r by searching grid shells around r's anchor (each
// s is counted in the cell that holds its anchor), then the candidates are
// gathered with a per-r radius, grouped by r and sorted by s.
//
// Refinement: LoD by LoD, the undecided candidates are refined with units
// pruned against theta_r; one CTA per r then applies Algorithm 6 in the
// corrected reading (n precedes m iff (ub_n, id_n) < (lb_m, id_m); m is
// REMOVED when at least kLeft undecided candidates precede it, CONFIRMED
// when fewer than kLeft others might precede it; decisions of one round use
// the statuses at its start) and lowers theta_r to the k-th smallest upper
// bound of the non-removed candidates (the shrinking bound).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pj {

struct KGrid {
  float g0[3];
  float inv_h;
  float h;
  int dim[3];
  int64_t ncell;
};

__device__ __forceinline__ int kcell1(float x, float g0, float inv_h, int dim) {
  float f = floorf((x - g0) * inv_h);
  return f < 0.f ? 0 : (f >= (float)dim ? dim - 1 : (int)f);
}
__device__ __forceinline__ int64_t kcell_id(const KGrid& G, int x, int y, int z) {
  return ((int64_t)z * G.dim[1] + y) * G.dim[0] + x;
}

__global__ void k_kgrid_count(int nS, const float* mbb, KGrid G, int64_t* cnt) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nS) return;
  const float* b = mbb + 6LL * s;
  int c0[3], c1[3];
  for (int k = 0; k < 3; ++k) {
    c0[k] = kcell1(b[k], G.g0[k], G.inv_h, G.dim[k]);
    c1[k] = kcell1(b[3 + k], G.g0[k], G.inv_h, G.dim[k]);
  }
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) atomicAdd((unsigned long long*)&cnt[kcell_id(G, x, y, z)], 1ULL);
}

__global__ void k_kgrid_fill(int nS, const float* mbb, KGrid G, const int64_t* off, int64_t* cursor, int32_t* ids) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nS) return;
  const float* b = mbb + 6LL * s;
  int c0[3], c1[3];
  for (int k = 0; k < 3; ++k) {
    c0[k] = kcell1(b[k], G.g0[k], G.inv_h, G.dim[k]);
    c1[k] = kcell1(b[3 + k], G.g0[k], G.inv_h, G.dim[k]);
  }
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        int64_t c = kcell_id(G, x, y, z);
        unsigned long long pos = atomicAdd((unsigned long long*)&cursor[c], 1ULL);
        ids[off[c] + (int64_t)pos] = s;
      }
}

constexpr int KMAX = 32;   // largest k of the GPU k-NN join

// theta_r: warp per r; shells of cells of growing Chebyshev radius around
// r's anchor cell; each s is taken from the cell holding its anchor.  The
// search stops once k anchors are known and the k-th distance is at most the
// distance from r's anchor to the outside of the searched cube.
__global__ void k_theta(int nR, const float* ancR, const float* ancS, KGrid G, const int64_t* off, const int32_t* ids,
                        int k, double* theta) {
  __shared__ double topd[8][KMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + warp;
  if (r >= nR) return;
  const float ax = ancR[3LL * r], ay = ancR[3LL * r + 1], az = ancR[3LL * r + 2];
  const int cx = kcell1(ax, G.g0[0], G.inv_h, G.dim[0]);
  const int cy = kcell1(ay, G.g0[1], G.inv_h, G.dim[1]);
  const int cz = kcell1(az, G.g0[2], G.inv_h, G.dim[2]);
  double* top = topd[warp];
  if (lane < k) top[lane] = INFINITY;
  __syncwarp();
  int have = 0;
  const int maxs = max(G.dim[0], max(G.dim[1], G.dim[2]));
  for (int sh = 0; sh <= maxs; ++sh) {
    for (int z = cz - sh; z <= cz + sh; ++z) {
      if (z < 0 || z >= G.dim[2]) continue;
      for (int y = cy - sh; y <= cy + sh; ++y) {
        if (y < 0 || y >= G.dim[1]) continue;
        // the shell's cells of this row: all of it on the two faces, else
        // its two ends
        const bool face = abs(z - cz) == sh || abs(y - cy) == sh;
        const int xstep = face || sh == 0 ? 1 : 2 * sh;
        for (int x = cx - sh; x <= cx + sh; x += xstep) {
          if (x < 0 || x >= G.dim[0]) continue;
          const int64_t c = kcell_id(G, x, y, z);
          for (int64_t q0 = off[c]; q0 < off[c + 1]; q0 += 32) {
            const int64_t q = q0 + lane;
            double dd = INFINITY;
            if (q < off[c + 1]) {
              const int s = ids[q];
              const float* as = ancS + 3LL * s;
              if (kcell1(as[0], G.g0[0], G.inv_h, G.dim[0]) == x && kcell1(as[1], G.g0[1], G.inv_h, G.dim[1]) == y &&
                  kcell1(as[2], G.g0[2], G.inv_h, G.dim[2]) == z) {
                double gx = (double)as[0] - ax, gy = (double)as[1] - ay, gz = (double)as[2] - az;
                dd = __dsqrt_ru(__dadd_ru(__dadd_ru(__dmul_ru(gx, gx), __dmul_ru(gy, gy)), __dmul_ru(gz, gz)));
              }
            }
            have += __popc(__ballot_sync(0xffffffffu, dd < INFINITY));
            // only the lanes that beat the current k-th enter the list
            unsigned m = __ballot_sync(0xffffffffu, dd < top[k - 1]);
            while (m) {
              const int l = __ffs(m) - 1;
              m &= m - 1u;
              const double v = __shfl_sync(0xffffffffu, dd, l);
              if (lane == 0 && v < top[k - 1]) {
                int pos = k - 1;
                while (pos > 0 && top[pos - 1] > v) {
                  top[pos] = top[pos - 1];
                  --pos;
                }
                top[pos] = v;
              }
              __syncwarp();
            }
            __syncwarp();
          }
        }
      }
    }
    __syncwarp();
    const double kth = top[k - 1];
    // every anchor outside the searched cube is farther than sh * h
    if (have >= k && kth <= (double)sh * (double)G.h) break;
  }
  if (lane == 0) theta[r] = top[k - 1];
}

// box MINDIST^2 (exact differences, sum rounded down) <= lim2
__device__ __forceinline__ bool kbox_within(const float* a, const float* b, double lim2) {
  double s2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double g = 0.0;
    if ((double)b[k] > (double)a[3 + k]) g = (double)b[k] - (double)a[3 + k];
    else if ((double)a[k] > (double)b[3 + k]) g = (double)a[k] - (double)b[3 + k];
    s2 = __dadd_rd(s2, __dmul_rd(g, g));
  }
  return s2 <= lim2;
}

// Candidates of r: s with MINDIST(r, s) <= theta_r; r's box grown by
// theta_r probes the grid; (r, s) is taken in the cell of the low corner of
// the overlap of the grown box and s's box.
template <bool EMIT>
__global__ void k_kprobe(int nR, const float* mbbR, const float* mbbS, const double* theta, KGrid G,
                         const int64_t* off, const int32_t* ids, int64_t* rcount, const int64_t* roff, int32_t* out_r,
                         int32_t* out_s) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nR) return;
  const float* a = mbbR + 6LL * w;
  const double th = theta[w];
  const float fth = __double2float_ru(th);
  const double lim = th * (1.0 + 1e-9), lim2 = lim * lim;
  float lo[3], hi[3];
  int c0[3], c1[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = __fsub_rd(a[k], fth);
    hi[k] = __fadd_ru(a[3 + k], fth);
    c0[k] = kcell1(lo[k], G.g0[k], G.inv_h, G.dim[k]);
    c1[k] = kcell1(hi[k], G.g0[k], G.inv_h, G.dim[k]);
  }
  int64_t found = 0;
  const int64_t base = EMIT ? roff[w] : 0;
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        const int64_t c = kcell_id(G, x, y, z);
        const int64_t b0 = off[c], b1 = off[c + 1];
        for (int64_t q0 = b0; q0 < b1; q0 += 32) {
          const int64_t q = q0 + lane;
          bool keep = false;
          int s = -1;
          if (q < b1) {
            s = ids[q];
            const float* b = mbbS + 6LL * s;
            int rx = kcell1(fmaxf(lo[0], b[0]), G.g0[0], G.inv_h, G.dim[0]);
            int ry = kcell1(fmaxf(lo[1], b[1]), G.g0[1], G.inv_h, G.dim[1]);
            int rz = kcell1(fmaxf(lo[2], b[2]), G.g0[2], G.inv_h, G.dim[2]);
            keep = rx == x && ry == y && rz == z && kbox_within(a, b, lim2);
          }
          unsigned m = __ballot_sync(0xffffffffu, keep);
          if (EMIT && keep) {
            int64_t pos = base + found + __popc(m & ((1u << lane) - 1u));
            out_r[pos] = w;
            out_s[pos] = s;
          }
          found += __popc(m);
        }
      }
  if (!EMIT && lane == 0) rcount[w] = found;
}

__global__ void k_seg_sort(int nR, const int64_t* roff, int32_t* s);   // filter.cu

static KGrid make_kgrid(const pj_set* R, const pj_set* S) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double ext = 0;
  for (const pj_set* X : {R, S})
    for (int o = 0; o < X->n; ++o) {
      const float* b = &X->mbb_h[6 * o];
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], b[k]);
        hi[k] = std::max(hi[k], b[3 + k]);
        if (X == S) ext += (double)b[3 + k] - b[k];
      }
    }
  ext /= std::max(1, 3 * S->n);
  for (int k = 0; k < 3; ++k) {
    lo[k] -= 1.f;
    hi[k] += 1.f;
  }
  double vol = 1.0;
  for (int k = 0; k < 3; ++k) vol *= std::max(1e-6, (double)hi[k] - lo[k]);
  // cells a quarter of the width that would hold two objects on average
  // (clustered sets are far denser than that average), never below the
  // mean box size
  double h = std::max(ext, 0.25 * std::cbrt(vol * 2.0 / std::max(1, S->n)));
  KGrid G;
  for (;;) {
    int64_t tot = 1;
    for (int k = 0; k < 3; ++k) {
      G.dim[k] = (int)std::max<double>(1.0, std::ceil(((double)hi[k] - lo[k]) / h));
      tot *= G.dim[k];
    }
    if (tot <= (1LL << 22)) {
      G.ncell = tot;
      break;
    }
    h *= 1.25;
  }
  for (int k = 0; k < 3; ++k) G.g0[k] = lo[k];
  G.h = (float)h;
  G.inv_h = (float)(1.0 / h);
  return G;
}

FilterOut filter_knn(pj_ctx* ctx, const pj_set* R, const pj_set* S, int k, cudaStream_t st) {
  FilterOut out;
  if (R->n == 0 || S->n == 0) return out;
  KGrid G = make_kgrid(R, S);
  ctx->sgrid.valid = false;   // the grid slots are reused here
  auto cnt = (int64_t*)ws_get(ctx, WS_GRID, (G.ncell + 1) * 8, st);
  auto off = (int64_t*)ws_get(ctx, WS_MISC, (G.ncell + 1) * 8, st);
  PJ_CK(cudaMemsetAsync(cnt, 0, (G.ncell + 1) * 8, st));
  int th = 256;
  k_kgrid_count<<<(S->n + th - 1) / th, th, 0, st>>>(S->n, S->mbb, G, cnt);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, cnt, off, G.ncell, st);
  int64_t nids = 0;
  for (int o = 0; o < S->n; ++o) {
    const float* b = &S->mbb_h[6 * o];
    int64_t c = 1;
    for (int q = 0; q < 3; ++q) {
      double a0 = std::floor(((double)b[q] - G.g0[q]) * G.inv_h), a1 = std::floor(((double)b[3 + q] - G.g0[q]) * G.inv_h);
      c *= (int64_t)std::min<double>(G.dim[q], std::max(1.0, a1 - a0 + 3.0));
    }
    nids += c;
  }
  auto ids = (int32_t*)ws_get(ctx, WS_GRIDIDS, std::max<int64_t>(1, nids) * 4, st);
  PJ_CK(cudaMemsetAsync(cnt, 0, (G.ncell + 1) * 8, st));
  k_kgrid_fill<<<(S->n + th - 1) / th, th, 0, st>>>(S->n, S->mbb, G, off, cnt, ids);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  auto theta = (double*)ws_get(ctx, WS_KNN, (size_t)R->n * 8, st);
  const int kk = std::min(k, S->n);
  unsigned g8 = (unsigned)((R->n + 7) / 8);
  k_theta<<<g8, 256, 0, st>>>(R->n, R->anchor, S->anchor, G, off, ids, kk, theta);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  auto rcount = (int64_t*)ws_get(ctx, WS_RCOUNT, ((int64_t)R->n + 1) * 8, st);
  auto roff = (int64_t*)ws_get(ctx, WS_ROFF, ((int64_t)R->n + 1) * 8, st);
  unsigned g = (unsigned)(((int64_t)R->n * 32 + th - 1) / th);
  k_kprobe<false><<<g, th, 0, st>>>(R->n, R->mbb, S->mbb, theta, G, off, ids, rcount, nullptr, nullptr, nullptr);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, rcount, roff, R->n, st);
  int64_t total = 0;
  PJ_CK(cudaMemcpyAsync(&total, roff + R->n, 8, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  out.n_pairs = total;
  if (total == 0) return out;
  auto pr = (int32_t*)ws_get(ctx, WS_PR, total * 4, st);
  auto ps = (int32_t*)ws_get(ctx, WS_PS, total * 4, st);
  k_kprobe<true><<<g, th, 0, st>>>(R->n, R->mbb, S->mbb, theta, G, off, ids, nullptr, roff, pr, ps);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  k_seg_sort<<<R->n, 256, 0, st>>>(R->n, roff, ps);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  return out;
}

// ------------------------------------------------------------------ prune

// Pruning thresholds sit strictly above theta_r: a unit skipped against one
// holds no facet pair at distance <= theta_r, and a pair whose lower bound
// is clamped to one is certainly beyond the k-th neighbour.
__device__ __forceinline__ float thr_above(double t) {
  return nextafterf(__double2float_ru(t), INFINITY);
}

__global__ void k_theta_to_pairs(int64_t n, const int32_t* pr, const double* theta, float* thr) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) thr[p] = thr_above(theta[pr[p]]);
}

template <bool F64>
__device__ __forceinline__ double kload(const void* a, int64_t p) {
  if (F64) return bits2d(((const unsigned long long*)a)[p]);
  return (double)bits2f(((const unsigned*)a)[p]);
}

constexpr int KPRUNE_SMEM = 2048;   // candidates of one r kept in shared memory

struct PruneArgs {
  const int64_t* roff;
  const int32_t* ps;
  uint8_t* status;
  uint8_t* stnew;
  uint8_t* lod0;
  const void* lbw;
  const void* ubw;
  const void* midw;
  float* thr;
  double* theta;
  double* dlo;
  double* dhi;
  double* d;
  uint8_t* exact;
  unsigned long long* cnt;
  int nR;
  int k;
  int fresh_st;    // status whose pairs were refined now (with lod0 <= step); -1: none
  int step;
  int clamp;       // the refinement pruned units against thr
  int full;        // the refinement ran at full resolution
};

// Algorithm 6 (corrected) for one r per CTA, then the shrinking bound.  The
// candidates in state UNDECIDED or WAVE compete; the ones refined at this
// step take their fresh lb / ub words, the others keep their bracket.  A
// first-wave candidate left undecided returns to UNDECIDED with lod0 =
// step + 1, so the second wave of the same step does not refine it again.
template <bool F64>
__global__ void __launch_bounds__(256) k_knn_prune(PruneArgs A) {
  __shared__ double s_lb[KPRUNE_SMEM], s_ub[KPRUNE_SMEM];
  __shared__ int s_id[KPRUNE_SMEM];
  __shared__ uint8_t s_st[KPRUNE_SMEM];
  __shared__ int s_conf;
  const int r = blockIdx.x;
  if (r >= A.nR) return;
  const int64_t a = A.roff[r], C = A.roff[r + 1] - a;
  if (C == 0) return;
  if (threadIdx.x == 0) s_conf = 0;
  __syncthreads();
  const bool in_smem = C <= KPRUNE_SMEM;
  auto fresh_at = [&](int64_t p, uint8_t stt) { return (int)stt == A.fresh_st && (int)A.lod0[p] <= A.step; };
  for (int64_t i = threadIdx.x; i < C; i += blockDim.x) {
    const int64_t p = a + i;
    const uint8_t stt = A.status[p];
    double l, u;
    if (fresh_at(p, stt)) {
      l = kload<F64>(A.lbw, p);
      if (A.clamp) l = fmin(l, (double)A.thr[p]);   // pruned units lie above thr
      u = kload<F64>(A.ubw, p);
      A.dlo[p] = l;
      A.dhi[p] = u;
    } else {
      l = A.dlo[p];
      u = A.dhi[p];
    }
    if (stt == CONFIRMED) atomicAdd(&s_conf, 1);
    if (in_smem) {
      s_lb[i] = l;
      s_ub[i] = u;
      s_id[i] = A.ps[p];
      s_st[i] = stt;
    }
  }
  __syncthreads();
  const int k_left = A.k - s_conf;
  auto LB = [&](int64_t i) { return in_smem ? s_lb[i] : A.dlo[a + i]; };
  auto UB = [&](int64_t i) { return in_smem ? s_ub[i] : A.dhi[a + i]; };
  auto ID = [&](int64_t i) { return in_smem ? s_id[i] : A.ps[a + i]; };
  auto ST = [&](int64_t i) { return in_smem ? s_st[i] : A.status[a + i]; };
  auto live = [](uint8_t x) { return x == UNDECIDED || x == WAVE; };
  // (xv, xi) < (yv, yi) lexicographically
  auto before = [](double xv, int xi, double yv, int yi) { return xv < yv || (xv == yv && xi < yi); };
  // decisions against the statuses at the start of the round
  for (int64_t m = threadIdx.x; m < C; m += blockDim.x) {
    uint8_t ns = ST(m);
    if (live(ns)) {
      if (k_left <= 0) {
        ns = REMOVED;
      } else {
        const double lm = LB(m), um = UB(m);
        const int im = ID(m);
        int64_t prec = 0, maybe = 0;
        for (int64_t j = 0; j < C; ++j) {
          if (j == m || !live(ST(j))) continue;
          const double lj = LB(j), uj = UB(j);
          const int ij = ID(j);
          if (before(uj, ij, lm, im)) ++prec;     // j certainly before m
          if (!before(um, im, lj, ij)) ++maybe;   // j possibly before m
        }
        if (prec >= k_left) ns = REMOVED;
        else if (maybe < k_left) ns = CONFIRMED;
      }
    }
    A.stnew[a + m] = ns;
  }
  __syncthreads();
  for (int64_t m = threadIdx.x; m < C; m += blockDim.x) {
    const int64_t p = a + m;
    const uint8_t old = ST(m), ns = A.stnew[p];
    const bool fr = fresh_at(p, old);
    if (ns == WAVE) {   // first wave, still undecided
      A.status[p] = UNDECIDED;
      A.lod0[p] = (uint8_t)min(A.step + 1, STEP_ALL);
      continue;
    }
    if (ns == old) continue;
    A.status[p] = ns;
    if (ns == CONFIRMED) {
      atomicAdd(&A.cnt[2], 1ULL);
      if (A.full && fr) {
        A.exact[p] = F64 ? 1 : 2;
        A.d[p] = F64 ? UB(m) : kload<F64>(A.midw, p);
      } else {
        A.exact[p] = 0;
        A.d[p] = 0.5 * (LB(m) + UB(m));
      }
    } else if (ns == REMOVED) {
      atomicAdd(&A.cnt[3], 1ULL);
    }
  }
  __syncthreads();
  // shrinking bound: k-th smallest upper bound of the candidates not removed
  if (threadIdx.x == 0) {
    double top[KMAX];
    int nt = 0;
    const int kk = min(A.k, KMAX);
    for (int64_t i = 0; i < C; ++i) {
      if (A.status[a + i] == REMOVED) continue;
      const double u = A.dhi[a + i];
      if (nt < kk || u < top[nt - 1]) {
        int pos = nt < kk ? nt++ : kk - 1;
        while (pos > 0 && top[pos - 1] > u) {
          top[pos] = top[pos - 1];
          --pos;
        }
        top[pos] = u;
      }
    }
    double t = nt >= kk ? top[kk - 1] : INFINITY;
    t = fmin(t, A.theta[r]);
    A.theta[r] = t;
    const float th = thr_above(t);
    for (int64_t i = 0; i < C; ++i) A.thr[a + i] = th;
  }
}

// First wave of a step: per r (one warp), the k_left undecided candidates
// with the smallest key become WAVE; the key is the proposal's predicted
// distance when one is given (step 0), else the midpoint of the current
// bracket.  Ties go to the smaller s id.
__global__ void k_knn_wave(int nR, const int64_t* roff, const int32_t* ps, uint8_t* status, const uint8_t* lod0,
                           int step, const float* pred, const double* dlo, const double* dhi, int k) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nR) return;
  const int64_t a = roff[r], C = roff[r + 1] - a;
  int conf = 0;
  for (int64_t i = lane; i < C; i += 32) conf += status[a + i] == CONFIRMED;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) conf += __shfl_xor_sync(0xffffffffu, conf, o);
  const int k_left = k - conf;
  for (int t = 0; t < k_left; ++t) {
    double bk = INFINITY;
    int bid = INT_MAX;
    int64_t bi = -1;
    for (int64_t i = lane; i < C; i += 32) {
      const int64_t p = a + i;
      if (status[p] != UNDECIDED || (int)lod0[p] > step) continue;
      const double key = pred ? (double)pred[p] : 0.5 * (dlo[p] + dhi[p]);
      const int id = ps[p];
      if (key < bk || (key == bk && id < bid)) {
        bk = key;
        bid = id;
        bi = p;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oid = __shfl_xor_sync(0xffffffffu, bid, o);
      const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
      if (ok < bk || (ok == bk && oid < bid)) {
        bk = ok;
        bid = oid;
        bi = oi;
      }
    }
    if (bi < 0) break;
    if (lane == 0) status[bi] = WAVE;
    __syncwarp();
  }
}

static void knn_prune_launch(pj_ctx* ctx, int nR, int k, bool full, bool fp64, int fresh_st, int step, bool clamp,
                             cudaStream_t st) {
  PruneArgs A;
  A.roff = (const int64_t*)ctx->ws[WS_ROFF].p;
  A.ps = (const int32_t*)ctx->ws[WS_PS].p;
  A.status = (uint8_t*)ctx->ws[WS_STATUS].p;
  A.stnew = (uint8_t*)ctx->ws[WS_KNN2].p;
  A.lod0 = (uint8_t*)ctx->ws[WS_LOD0].p;
  A.lbw = ctx->ws[WS_LB].p;
  A.ubw = ctx->ws[WS_UB].p;
  A.midw = ctx->ws[WS_MID].p;
  A.thr = (float*)ctx->ws[WS_THR].p;
  A.theta = (double*)ctx->ws[WS_KNN].p;
  A.dlo = (double*)ctx->ws[WS_DLO].p;
  A.dhi = (double*)ctx->ws[WS_DHI].p;
  A.d = (double*)ctx->ws[WS_D].p;
  A.exact = (uint8_t*)ctx->ws[WS_EXACT].p;
  A.cnt = ctx->d_counters;
  A.nR = nR;
  A.k = k;
  A.fresh_st = fresh_st;
  A.step = step;
  A.clamp = clamp ? 1 : 0;
  A.full = full ? 1 : 0;
  if (fp64) k_knn_prune<true><<<nR, 256, 0, st>>>(A);
  else k_knn_prune<false><<<nR, 256, 0, st>>>(A);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

static void knn_wave(pj_ctx* ctx, int nR, int k, int step, const float* pred, cudaStream_t st) {
  const int wpb = 8;
  k_knn_wave<<<(nR + wpb - 1) / wpb, wpb * 32, 0, st>>>(
      nR, (const int64_t*)ctx->ws[WS_ROFF].p, (const int32_t*)ctx->ws[WS_PS].p, (uint8_t*)ctx->ws[WS_STATUS].p,
      (const uint8_t*)ctx->ws[WS_LOD0].p, step, pred, (const double*)ctx->ws[WS_DLO].p,
      (const double*)ctx->ws[WS_DHI].p, k);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// ------------------------------------------------------------------ driver

static pj_status join_knn_once(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                               cudaStream_t st, std::string& stats) {
  Timer tall;
  const unsigned long long launches0 = ctx->launches;
  const int k = q->k;
  if (k > KMAX) throw ApiError{PJ_EINVAL, "k above 32 is not supported by the GPU k-NN join"};
  const bool fp64 = q->prec == PJ_PREC_FP64;
  const bool cull = (q->flags & PJ_TILE_PRUNE) != 0;
  const bool use_mlp = (q->flags & PJ_USE_MLP) != 0;
  if (use_mlp && !ctx->mlp_ready) throw ApiError{PJ_EINVAL, "PJ_USE_MLP needs trained or loaded proposal weights"};
  PJ_CK(cudaMemsetAsync(ctx->d_counters, 0, 15 * sizeof(unsigned long long), st));
  PJ_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  Timer tf;
  FilterOut fo = filter_knn(ctx, R, S, k, st);
  const int64_t n = fo.n_pairs;
  setup_pairs(ctx, R, S, n, 0.0, false, st);
  const float* pred = nullptr;
  if (n > 0) {
    int th = 256;
    k_theta_to_pairs<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, (const int32_t*)ctx->ws[WS_PR].p,
                                                                   (const double*)ctx->ws[WS_KNN].p,
                                                                   (float*)ctx->ws[WS_THR].p);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    // the box / anchor bracket is the first round of Algorithm 6
    ws_get(ctx, WS_KNN2, (size_t)n, st);
    knn_prune_launch(ctx, R->n, k, false, false, -1, 0, false, st);
    if (use_mlp) pred = propose(ctx, R, S, n, st);
  }
  const double ms_filter = tf.ms();
  const int Lmax = std::max(R->L, S->L);
  ctx->ev_used = 0;
  StepLog log;
  // one refinement pass over the pairs in state `want` and its pruning round
  auto pass = [&](StepSpec sp, int fresh_st) {
    init_bounds(ctx, n, sp, st);
    UnitCount uc = build_tiles(ctx, R, S, n, sp, st);
    log.add(ctx, uc, run_refine(ctx, R, S, uc, sp, st), sp, st);
    knn_prune_launch(ctx, R->n, k, sp.full, sp.fp64, fresh_st, sp.step, sp.cull, st);
  };
  for (int step = 0; step < Lmax && n > 0; ++step) {
    if (q->timeout_s > 0 && tall.ms() > q->timeout_s * 1000.0) return PJ_ETIMEOUT;
    StepSpec sp;
    sp.rerun_ok = true;
    sp.lodR = std::max(0, step - (Lmax - R->L));
    sp.lodS = std::max(0, step - (Lmax - S->L));
    sp.full = step == Lmax - 1;
    sp.fp64 = fp64;
    sp.cull = cull;
    sp.step = step;
    // first wave: the k most promising candidates of every r tighten theta_r
    // before the others are refined against it
    knn_wave(ctx, R->n, k, step, step == 0 ? pred : nullptr, st);
    sp.want = WAVE;
    pass(sp, WAVE);
    sp.want = UNDECIDED;
    pass(sp, UNDECIDED);
  }
  if (!fp64 && n > 0) {
    // candidates whose single-precision brackets still tie: FP64 at full
    // resolution, units pruned against the strict threshold, then the last
    // pruning round resolves everything
    StepSpec sp;
    sp.rerun_ok = true;
    sp.lodR = R->L - 1;
    sp.lodS = S->L - 1;
    sp.full = true;
    sp.fp64 = true;
    sp.cull = cull;
    sp.want = UNDECIDED;
    sp.step = STEP_ALL;
    pass(sp, UNDECIDED);
  }
  if ((q->flags & PJ_EXACT_DIST) && n > 0) {
    mark_exact(ctx, n, st);
    StepSpec sp;
    sp.rerun_ok = true;
    sp.lodR = R->L - 1;
    sp.lodS = S->L - 1;
    sp.full = true;
    sp.fp64 = true;
    sp.cull = cull;   // result pairs lie within theta_r < thr
    sp.want = MAKE_EXACT;
    sp.step = STEP_ALL;
    init_bounds(ctx, n, sp, st);
    UnitCount uc = build_tiles(ctx, R, S, n, sp, st);
    log.add(ctx, uc, run_refine(ctx, R, S, uc, sp, st), sp, st);
    decide_within(ctx, n, 0.0, sp, st);
  }
  {
    // a step whose units overflowed the buffer voids the join (rerun)
    int e0 = 0;
    PJ_CK(cudaMemcpyAsync(&e0, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PJ_CK(cudaStreamSynchronize(st));
    check_units(ctx, e0);
  }
  Timer tg;
  int64_t m = gather_results(ctx, n, out, st);
  if (q->flags & PJ_EXACT_DIST) {
    // order each r's neighbours by (d, s)
    std::vector<int64_t> idx(m);
    for (int64_t i = 0; i < m; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
      if (out->r[x] != out->r[y]) return out->r[x] < out->r[y];
      if (out->d[x] != out->d[y]) return out->d[x] < out->d[y];
      return out->s[x] < out->s[y];
    });
    pj_result tmp;
    memset(&tmp, 0, sizeof tmp);
    alloc_result(&tmp, m);
    for (int64_t i = 0; i < m; ++i) {
      tmp.r[i] = out->r[idx[i]];
      tmp.s[i] = out->s[idx[i]];
      tmp.d_lo[i] = out->d_lo[idx[i]];
      tmp.d_hi[i] = out->d_hi[idx[i]];
      tmp.d[i] = out->d[idx[i]];
      tmp.exact[i] = out->exact[idx[i]];
    }
    free(out->priv);
    *out = tmp;
  }
  int herr = 0;
  PJ_CK(cudaMemcpy(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  unsigned long long cnt[8];
  PJ_CK(cudaMemcpy(cnt, ctx->d_counters, sizeof cnt, cudaMemcpyDeviceToHost));
  double rms32 = 0, rms64 = 0;
  int64_t units = 0;
  const std::string steps = log.json(ctx, &rms32, &rms64, &units);
  char buf[1500];
  snprintf(buf, sizeof buf,
           "{\"pred\":\"knn\",\"k\":%d,\"prec\":\"%s\",\"mlp\":%d,\"candidates\":%lld,\"results\":%lld,\"tests_fp32\":%llu,"
           "\"tests_fp64\":%llu,\"tests_culled\":%llu,\"tests_needed\":%llu,\"confirmed\":%llu,\"removed\":%llu,"
           "\"tiles\":%lld,\"ms_filter\":%.3f,"
           "\"ms_gather\":%.3f,\"ms_total\":%.3f,\"refine_ms_fp32\":%.4f,\"refine_ms_fp64\":%.4f,"
           "\"launches\":%llu,\"steps\":",
           k, fp64 ? "fp64" : "fp32", use_mlp ? 1 : 0, (long long)n, (long long)m, cnt[0], cnt[1], cnt[5], cnt[6], cnt[2], cnt[3],
           (long long)units,
           ms_filter, tg.ms(), tall.ms(), rms32, rms64, ctx->launches - launches0);
  stats = std::string(buf) + steps + "}";
  JoinSummary& js = ctx->last_sum;
  js.candidates = n;
  js.results = m;
  js.units = units;
  js.tests32 = cnt[0];
  js.tests64 = cnt[1];
  js.confirmed = cnt[2];
  js.removed = cnt[3];
  js.ms_filter = ms_filter;
  js.ms_total = tall.ms();
  js.refine_ms32 = rms32;
  js.refine_ms64 = rms64;
  js.launches = ctx->launches - launches0;
  if (herr & ERR_MBAR_TIMEOUT) return PJ_ETIMEOUT;
  if (herr & ERR_CAPACITY) throw ApiError{PJ_ENOMEM, "refinement units above the unit buffer"};
  if (herr & ERR_NONFINITE) return PJ_ENONFINITE;   // data of a LoD built on demand
  return PJ_OK;
}

// A k-NN join; reruns (at most three times) when a step's refinement units
// did not fit the unit buffer, which is then grown to the count needed.
pj_status join_knn(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                   cudaStream_t st, std::string& stats) {
  for (int attempt = 0;; ++attempt) {
    try {
      return join_knn_once(ctx, R, S, q, out, st, stats);
    } catch (const UnitsOverflow& e) {
      if (attempt >= 3) throw ApiError{PJ_ENOMEM, "refinement units above the unit buffer after resizing"};
      grow_units(ctx, e.units, st);
    }
  }
}

}  // namespace pj
