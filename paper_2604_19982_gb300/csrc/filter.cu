// MBB candidate filter on the GPU (section 3.1, "MBB-based Object
// Filtering"; the paper walks an R-tree on the CPU).  A uniform grid is
// built over the S boxes grown by tau; every r probes the cells its box
// overlaps, each (r, s) is reported once from the cell holding the low
// corner of the overlap of the two boxes, and kept when the box MINDIST is
// at most tau (a lower bound of d, so no result is lost).  Output: pairs
// grouped by r, each group sorted by s.
#include <algorithm>
#include <cstring>
#include <cmath>

#include "internal.h"
#include "common.cuh"

namespace pj {

struct Grid {
  float g0[3];
  float inv_h;
  int dim[3];
  int64_t ncell;
};

__device__ __forceinline__ int cell1(float x, float g0, float inv_h, int dim) {
  float f = floorf((x - g0) * inv_h);
  int c = f < 0.f ? 0 : (f >= (float)dim ? dim - 1 : (int)f);
  return c;
}

__device__ __forceinline__ int64_t cell_id(const Grid& G, int cx, int cy, int cz) {
  return ((int64_t)cz * G.dim[1] + cy) * G.dim[0] + cx;
}

__global__ void k_grid_count(int nS, const float* mbbS, float tau, Grid G, int64_t* cnt) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nS) return;
  const float* b = mbbS + 6LL * s;
  int c0[3], c1[3];
  for (int k = 0; k < 3; ++k) {
    c0[k] = cell1(b[k] - tau, G.g0[k], G.inv_h, G.dim[k]);
    c1[k] = cell1(b[3 + k] + tau, G.g0[k], G.inv_h, G.dim[k]);
  }
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) atomicAdd((unsigned long long*)&cnt[cell_id(G, x, y, z)], 1ULL);
}

__global__ void k_grid_fill(int nS, const float* mbbS, float tau, Grid G, const int64_t* off, int64_t* cursor,
                            int32_t* ids) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nS) return;
  const float* b = mbbS + 6LL * s;
  int c0[3], c1[3];
  for (int k = 0; k < 3; ++k) {
    c0[k] = cell1(b[k] - tau, G.g0[k], G.inv_h, G.dim[k]);
    c1[k] = cell1(b[3 + k] + tau, G.g0[k], G.inv_h, G.dim[k]);
  }
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        int64_t c = cell_id(G, x, y, z);
        unsigned long long pos = atomicAdd((unsigned long long*)&cursor[c], 1ULL);
        ids[off[c] + (int64_t)pos] = s;
      }
}

// box MINDIST^2 (exact differences in double, sum rounded down) <= lim2
__device__ __forceinline__ bool box_within(const float* a, const float* b, double lim2) {
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

constexpr int PROBE_SLOT = 64;   // candidates of one r kept by the counting probe

// One warp per r: lanes stride over the candidates of each probed cell.
// The counting pass (EMIT = false) also keeps the first PROBE_SLOT
// candidates of each r in slot[r][.] (when slot is set) and raises
// *overflow when an r has more.
template <bool EMIT>
__global__ void k_probe(int nR, const float* mbbR, const float* mbbS, float tau, double lim2, Grid G,
                        const int64_t* off, const int32_t* ids, int64_t* rcount, const int64_t* roff,
                        int32_t* out_r, int32_t* out_s, int32_t* slot = nullptr, int* overflow = nullptr) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= nR) return;
  const float* a = mbbR + 6LL * w;
  int c0[3], c1[3];
  for (int k = 0; k < 3; ++k) {
    c0[k] = cell1(a[k], G.g0[k], G.inv_h, G.dim[k]);
    c1[k] = cell1(a[3 + k], G.g0[k], G.inv_h, G.dim[k]);
  }
  int64_t found = 0;
  int64_t base = EMIT ? roff[w] : 0;
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        int64_t c = cell_id(G, x, y, z);
        int64_t b0 = off[c], b1 = off[c + 1];
        for (int64_t q0 = b0; q0 < b1; q0 += 32) {
          int64_t q = q0 + lane;
          bool keep = false;
          int s = -1;
          if (q < b1) {
            s = ids[q];
            const float* b = mbbS + 6LL * s;
            // report from the cell of the low corner of the overlap of
            // r's box and s's box grown by tau
            int rx = cell1(fmaxf(a[0], b[0] - tau), G.g0[0], G.inv_h, G.dim[0]);
            int ry = cell1(fmaxf(a[1], b[1] - tau), G.g0[1], G.inv_h, G.dim[1]);
            int rz = cell1(fmaxf(a[2], b[2] - tau), G.g0[2], G.inv_h, G.dim[2]);
            keep = (rx == x && ry == y && rz == z) && box_within(a, b, lim2);
          }
          unsigned m = __ballot_sync(0xffffffffu, keep);
          if (EMIT && keep) {
            int64_t pos = base + found + __popc(m & ((1u << lane) - 1u));
            out_r[pos] = w;
            out_s[pos] = s;
          }
          if (!EMIT && slot && keep) {
            const int64_t pos = found + __popc(m & ((1u << lane) - 1u));
            if (pos < PROBE_SLOT) slot[(int64_t)w * PROBE_SLOT + pos] = s;
          }
          found += __popc(m);
        }
      }
  if (!EMIT && lane == 0) {
    rcount[w] = found;
    if (slot && found > PROBE_SLOT) *overflow = 1;
  }
}

// Candidate lists of at most PROBE_SLOT entries per r, from the counting
// probe's slots: one warp per r ranks its s ids (each appears once; ties would
// go by position) and writes them in ascending order at roff[r] -- the output of the emitting probe followed by
// the per-r sort, without probing the grid a second time.
// With cap >= 0 (a speculative capacity), an r whose list would end past
// cap writes nothing and sets bit 1 of *over (the join then runs again with
// the capacity the count asks for).
__global__ void k_slot_emit(int nR, const int32_t* slot, const int64_t* roff, int32_t* out_r, int32_t* out_s,
                            int64_t cap, int* over) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nR) return;   // warp-uniform
  const int64_t base = roff[w];
  const int n = (int)(roff[w + 1] - base);
  if (n == 0) return;
  if (cap >= 0 && roff[w + 1] > cap) {
    if (lane == 0) atomicOr(over, 2);
    return;
  }
  const int32_t* sl = slot + (int64_t)w * PROBE_SLOT;
  const int32_t v0 = lane < n ? sl[lane] : 0x7fffffff;
  const int32_t v1 = lane + 32 < n ? sl[lane + 32] : 0x7fffffff;
  int r0 = 0, r1 = 0;
  for (int j = 0; j < n; ++j) {
    const int32_t u = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
    r0 += u < v0 || (u == v0 && j < lane);   // ties by position: ranks stay distinct
    r1 += u < v1 || (u == v1 && j < lane + 32);
  }
  if (lane < n) {
    out_r[base + r0] = w;
    out_s[base + r0] = v0;
  }
  if (lane + 32 < n) {
    out_r[base + r1] = w;
    out_s[base + r1] = v1;
  }
}

// Sort each r's candidate list by s (one CTA per r; bitonic in shared
// memory up to 4096, odd-even transposition in global memory above).
__global__ void k_seg_sort(int nR, const int64_t* roff, int32_t* s) {
  __shared__ int32_t buf[4096];
  const int r = blockIdx.x;
  if (r >= nR) return;
  const int64_t a = roff[r], n = roff[r + 1] - a;
  if (n <= 1) return;
  int32_t* v = s + a;
  if (n <= 4096) {
    int P = 32;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) buf[i] = i < n ? v[i] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          int l = i ^ j;
          if (l > i) {
            bool up = (i & k) == 0;
            int32_t x = buf[i], y = buf[l];
            if ((x > y) == up) {
              buf[i] = y;
              buf[l] = x;
            }
          }
        }
        __syncthreads();
      }
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = buf[i];
  } else {
    for (int64_t round = 0; round < n; ++round) {
      for (int64_t i = 2 * threadIdx.x + (round & 1); i + 1 < n; i += 2 * blockDim.x) {
        int32_t x = v[i], y = v[i + 1];
        if (x > y) {
          v[i] = y;
          v[i + 1] = x;
        }
      }
      __syncthreads();
    }
  }
}

// With R == nullptr the grid spans S's boxes alone (for a streamed R, whose
// chunks then share one grid): an R box outside it probes the clamped edge
// cells, which hold every S box (grown by tau) that can reach it.
static Grid make_grid(const pj_set* R, const pj_set* S, double tau) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double extS = 0, extR = 0;
  auto acc = [&](const pj_set* X, double& ext) {
    for (int o = 0; o < X->n; ++o) {
      const float* b = &X->mbb_h[6 * o];
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], b[k]);
        hi[k] = std::max(hi[k], b[3 + k]);
        ext += (double)b[3 + k] - b[k];
      }
    }
    ext /= std::max(1, 3 * X->n);
  };
  if (R) acc(R, extR);
  acc(S, extS);
  for (int k = 0; k < 3; ++k) {
    lo[k] -= (float)tau + 1.f;
    hi[k] += (float)tau + 1.f;
  }
  // cells at least one S box (+tau) and one R box wide, and about four
  // cells per S object (sparser grids only add empty cells to clear and scan)
  double vol = 1.0;
  for (int k = 0; k < 3; ++k) vol *= std::max(1e-3, (double)hi[k] - lo[k]);
  double h = std::max({extS + 2 * tau, extR, std::cbrt(vol / (4.0 * std::max(1, S->n))), 1e-3});
  Grid G;
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
  G.inv_h = (float)(1.0 / h);
  return G;
}

// Grid parameters and the bound on grid entries depend only on the two
// sets and tau: kept per (R, S, tau) for repeated joins (sets are
// immutable once loaded; streamed chunk views have uid 0 and are not kept).
static bool grid_cached(pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau, Grid* G, int64_t* nids) {
  if (!R->uid || !S->uid) return false;
  for (auto& e : ctx->grid_cache)
    if (e.rid == R->uid && e.sid == S->uid && e.tau == tau) {
      memcpy(G, e.grid, sizeof(Grid));
      *nids = e.nids;
      return true;
    }
  return false;
}

static void grid_keep(pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau, const Grid& G, int64_t nids) {
  if (!R->uid || !S->uid) return;
  static_assert(sizeof(Grid) <= sizeof(GridCacheEntry::grid), "grid cache entry");
  if (ctx->grid_cache.size() >= 8) ctx->grid_cache.erase(ctx->grid_cache.begin());
  GridCacheEntry e;
  e.rid = R->uid;
  e.sid = S->uid;
  e.tau = tau;
  memcpy(e.grid, &G, sizeof(Grid));
  e.nids = nids;
  ctx->grid_cache.push_back(e);
}

FilterOut filter_within(pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau, cudaStream_t st) {
  FilterOut out;
  if (R->n == 0 || S->n == 0) return out;
  Grid G;
  int64_t nids = 0;
  float ftau = (float)tau;
  if ((double)ftau < tau) ftau = nextafterf(ftau, INFINITY);
  double lim = tau * (1.0 + 1e-9);
  double lim2 = lim * lim;
  int th = 256;
  // a streamed R's chunks (views with uid 0) share one grid over S, kept
  // in the workspace while no other grid replaces it
  const bool s_only = R->uid == 0 && S->uid != 0;
  const bool kept = s_only && ctx->sgrid.valid && ctx->sgrid.sid == S->uid && ctx->sgrid.tau == tau;
  int64_t* off;
  int32_t* ids;
  if (kept) {
    memcpy(&G, ctx->sgrid.grid, sizeof(Grid));
    off = (int64_t*)ctx->ws[WS_MISC].p;
    ids = (int32_t*)ctx->ws[WS_GRIDIDS].p;
  } else {
    ctx->sgrid.valid = false;
    const bool cached = !s_only && grid_cached(ctx, R, S, tau, &G, &nids);
    if (!cached) G = make_grid(s_only ? nullptr : R, S, tau);
    auto cnt = (int64_t*)ws_get(ctx, WS_GRID, (G.ncell + 1) * 8, st);
    off = (int64_t*)ws_get(ctx, WS_MISC, (G.ncell + 1) * 8, st);
    PJ_CK(cudaMemsetAsync(cnt, 0, (G.ncell + 1) * 8, st));
    k_grid_count<<<(S->n + th - 1) / th, th, 0, st>>>(S->n, S->mbb, ftau, G, cnt);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    scan_i64(ctx, cnt, off, G.ncell, st);
    // grid entries bounded on the host (one extra cell per axis absorbs
    // host/device rounding of the cell index), so no synchronization here
    if (!cached) {
      for (int o = 0; o < S->n; ++o) {
        const float* b = &S->mbb_h[6 * o];
        int64_t c = 1;
        for (int k = 0; k < 3; ++k) {
          double a0 = std::floor(((double)b[k] - tau - G.g0[k]) * G.inv_h);
          double a1 = std::floor(((double)b[3 + k] + tau - G.g0[k]) * G.inv_h);
          int64_t w = (int64_t)std::min<double>(G.dim[k], std::max(1.0, a1 - a0 + 3.0));
          c *= w;
        }
        nids += c;
      }
      if (!s_only) grid_keep(ctx, R, S, tau, G, nids);
    }
    ids = (int32_t*)ws_get(ctx, WS_GRIDIDS, std::max<int64_t>(1, nids) * 4, st);
    PJ_CK(cudaMemsetAsync(cnt, 0, (G.ncell + 1) * 8, st));
    k_grid_fill<<<(S->n + th - 1) / th, th, 0, st>>>(S->n, S->mbb, ftau, G, off, cnt, ids);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    if (s_only) {
      ctx->sgrid.valid = true;
      ctx->sgrid.sid = S->uid;
      ctx->sgrid.tau = tau;
      static_assert(sizeof(Grid) <= sizeof(ctx->sgrid.grid), "kept grid");
      memcpy(ctx->sgrid.grid, &G, sizeof(Grid));
    }
  }
  auto rcount = (int64_t*)ws_get(ctx, WS_RCOUNT, ((int64_t)R->n + 1) * 8, st);
  auto roff = (int64_t*)ws_get(ctx, WS_ROFF, ((int64_t)R->n + 1) * 8, st);
  int64_t warps_threads = (int64_t)R->n * 32;
  unsigned g = (unsigned)((warps_threads + th - 1) / th);
  // the counting probe also keeps up to PROBE_SLOT candidates per r; if no
  // r has more, they are ranked into place instead of probing again
  auto slot = (int32_t*)ws_get(ctx, WS_FSLOT, (int64_t)R->n * PROBE_SLOT * 4, st);
  int* overflow = (int*)(ctx->d_counters + 12);
  PJ_CK(cudaMemsetAsync(overflow, 0, sizeof(int), st));
  k_probe<false><<<g, th, 0, st>>>(R->n, R->mbb, S->mbb, ftau, lim2, G, off, ids, rcount, nullptr, nullptr,
                                   nullptr, slot, overflow);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, rcount, roff, R->n, st, (int64_t*)ws_get(ctx, WS_FSCAN, (scan_tmp_words(R->n) + 8) * 8, st));
  int64_t total = 0;
  int over = 0;
  PJ_CK(cudaMemcpyAsync(&total, roff + R->n, 8, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaMemcpyAsync(&over, overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  out.n_pairs = total;
  if (total == 0) return out;
  // capacity of the pair arrays: the next power of two (a fixed-capacity
  // join pads to it without reallocating the filter's output)
  int64_t cap = 256;
  while (cap < total) cap <<= 1;
  auto pr = (int32_t*)ws_get(ctx, WS_PR, cap * 4, st);
  auto ps = (int32_t*)ws_get(ctx, WS_PS, cap * 4, st);
  if (!over) {
    k_slot_emit<<<g, th, 0, st>>>(R->n, slot, roff, pr, ps, -1, nullptr);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    return out;
  }
  k_probe<true><<<g, th, 0, st>>>(R->n, R->mbb, S->mbb, ftau, lim2, G, off, ids, nullptr, roff, pr, ps);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  k_seg_sort<<<R->n, 256, 0, st>>>(R->n, roff, ps);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  return out;
}

// Whether the grid over S alone is kept for this (R, S, tau): a streamed
// chunk's filter then needs no host work before its launches.
bool filter_grid_kept(const pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau) {
  return R->uid == 0 && S->uid != 0 && ctx->sgrid.valid && ctx->sgrid.sid == S->uid && ctx->sgrid.tau == tau;
}

// The filter with the kept grid and a capacity fixed in advance (no host
// synchronization): count probe keeping up to PROBE_SLOT candidates per r,
// scan (the count lands in WS_ROFF[R->n]), ranked emit into pair arrays of
// `cap` entries.  *over (a device word the caller clears) gets bit 0 when
// some r has more than PROBE_SLOT candidates and bit 1 when the pairs
// exceed cap; either voids the join, which then runs the synchronous filter.
void filter_within_enqueue(pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau, int64_t cap, int* over,
                           cudaStream_t st) {
  Grid G;
  memcpy(&G, ctx->sgrid.grid, sizeof(Grid));
  const int64_t* off = (const int64_t*)ctx->ws[WS_MISC].p;
  const int32_t* ids = (const int32_t*)ctx->ws[WS_GRIDIDS].p;
  float ftau = (float)tau;
  if ((double)ftau < tau) ftau = nextafterf(ftau, INFINITY);
  const double lim = tau * (1.0 + 1e-9);
  const int th = 256;
  auto rcount = (int64_t*)ws_get(ctx, WS_RCOUNT, ((int64_t)R->n + 1) * 8, st);
  auto roff = (int64_t*)ws_get(ctx, WS_ROFF, ((int64_t)R->n + 1) * 8, st);
  auto slot = (int32_t*)ws_get(ctx, WS_FSLOT, (int64_t)R->n * PROBE_SLOT * 4, st);
  auto pr = (int32_t*)ws_get(ctx, WS_PR, cap * 4, st);
  auto ps = (int32_t*)ws_get(ctx, WS_PS, cap * 4, st);
  const unsigned g = (unsigned)(((int64_t)R->n * 32 + th - 1) / th);
  k_probe<false><<<g, th, 0, st>>>(R->n, R->mbb, S->mbb, ftau, lim * lim, G, off, ids, rcount, nullptr, nullptr,
                                   nullptr, slot, over);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, rcount, roff, R->n, st, (int64_t*)ws_get(ctx, WS_FSCAN, (scan_tmp_words(R->n) + 8) * 8, st));
  k_slot_emit<<<g, th, 0, st>>>(R->n, slot, roff, pr, ps, cap, over);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

}  // namespace pj
