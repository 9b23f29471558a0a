// Facet-level refinement (section 3.3, Algorithm 4 and Eq. 1 / Eq. 2),
// re-designed for sm_103a:
//  * unit = one 32-facet block of r x one 32-facet block of s of one
//    candidate pair at one LoD (replaces the paper's thread block per voxel
//    pair); units are built on the device (k_items / k_emit_units) and
//    consumed by a persistent kernel, one launch per LoD step;
//  * every warp works alone through a pipeline of its own: units are claimed
//    ahead (the first two by warp index, dealt across the SMs), a unit's tile
//    is fetched by a bulk copy, and its pair origin / threshold, r block and
//    s block are staged by TMA (cp.async.bulk, mbarrier completion, bounded
//    waits) into the warp's other buffer while the current unit computes;
//    the s facets are expanded once into shared-memory records, each lane
//    holds one r facet in registers and tests it against the broadcast s
//    records;
//  * facet balls skip facet pairs that cannot improve the lane's bounds;
//    at full resolution k_unit_masks first records which s facets a unit
//    needs at all and drops the units that need none;
//  * per-lane running minima, a warp minimum and one atomicMin per unit and
//    pair on the order-preserving bits (replaces the block-wide Hillis-Steele
//    scan and shared-memory aggregation of section 2.2);
//  * facet pairs whose planes straddle each other get the meeting test after
//    the loop (warp list, overflow to a global queue and k_cross_fix):
//    single-precision signs where an error bound makes them certain, double
//    precision otherwise;
//  * optional pruning (PJ_TILE_PRUNE): block pairs whose box distance minus
//    the Hausdorff terms exceeds the pair's threshold are never built.
#include <algorithm>
#include <stdexcept>

#include <type_traits>

#include "internal.h"
#include "tritri.cuh"
#include "tritri2.cuh"

namespace pj {

// ------------------------------------------------------------------ setup

__global__ void k_setup_pairs(int64_t n, const int32_t* pr, const int32_t* ps, const float* mbbR,
                              const float* mbbS, const float* ancR, const float* ancS, double tau, int within,
                              float4* origin, float* thr, double* box_lb, double* anc_ub, uint8_t* status,
                              uint8_t* lod0, uint8_t* exact, double* dlo, double* dhi, double* d,
                              const int64_t* n_live) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (n_live && p >= *n_live) {   // padding of a fixed-capacity (graph) join
    status[p] = REMOVED;
    lod0[p] = 0;
    return;
  }
  const int r = pr[p], s = ps[p];
  const float* a = mbbR + 6LL * r;
  const float* b = mbbS + 6LL * s;
  // pair-local frame: centre of the smaller box
  float da = (a[3] - a[0]) + (a[4] - a[1]) + (a[5] - a[2]);
  float db = (b[3] - b[0]) + (b[4] - b[1]) + (b[5] - b[2]);
  const float* c = da <= db ? a : b;
  origin[p] = make_float4(0.5f * (c[0] + c[3]), 0.5f * (c[1] + c[4]), 0.5f * (c[2] + c[5]), 0.f);
  // box MINDIST, rounded down (differences of floats are exact in double)
  double s2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double g = 0.0;
    if ((double)b[k] > (double)a[3 + k]) g = (double)b[k] - (double)a[3 + k];
    else if ((double)a[k] > (double)b[3 + k]) g = (double)a[k] - (double)b[3 + k];
    s2 = __dadd_rd(s2, __dmul_rd(g, g));
  }
  double lo = __dsqrt_rd(s2);
  // anchor distance, rounded up
  double u2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double g = (double)ancR[3LL * r + k] - (double)ancS[3LL * s + k];
    u2 = __dadd_ru(u2, __dmul_ru(g, g));
  }
  double hi = __dsqrt_ru(u2);
  box_lb[p] = lo;
  anc_ub[p] = hi;
  thr[p] = __double2float_ru(tau);
  lod0[p] = 0;
  exact[p] = 0;
  dlo[p] = lo;
  dhi[p] = hi;
  d[p] = hi;
  status[p] = (within && hi <= tau) ? CONFIRMED : UNDECIDED;
}

void setup_pairs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, double tau, bool within,
                 cudaStream_t st, const int64_t* n_live) {
  if (n == 0) return;
  auto pr = (int32_t*)ws_get(ctx, WS_PR, n * 4, st);
  auto ps = (int32_t*)ws_get(ctx, WS_PS, n * 4, st);
  auto origin = (float4*)ws_get(ctx, WS_ORIGIN, n * 16, st);
  auto thr = (float*)ws_get(ctx, WS_THR, ((n + 3) & ~int64_t(3)) * 4, st);   // 16-byte groups (k_refine)
  auto box_lb = (double*)ws_get(ctx, WS_BOXLB, n * 8, st);
  auto anc_ub = (double*)ws_get(ctx, WS_ANCUB, n * 8, st);
  auto status = (uint8_t*)ws_get(ctx, WS_STATUS, n, st);
  auto lod0 = (uint8_t*)ws_get(ctx, WS_LOD0, n, st);
  auto exact = (uint8_t*)ws_get(ctx, WS_EXACT, n, st);
  auto dlo = (double*)ws_get(ctx, WS_DLO, n * 8, st);
  auto dhi = (double*)ws_get(ctx, WS_DHI, n * 8, st);
  auto d = (double*)ws_get(ctx, WS_D, n * 8, st);
  int th = 256;
  k_setup_pairs<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, pr, ps, R->mbb, S->mbb, R->anchor, S->anchor,
                                                              tau, within ? 1 : 0, origin, thr, box_lb, anc_ub,
                                                              status, lod0, exact, dlo, dhi, d, n_live);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// ------------------------------------------------------------------ units
// A refinement unit is one 32-facet block of r x one 32-facet block of s of
// one candidate pair at one LoD.  A work item of the builder is one (pair,
// r block, 256-facet s chunk): the r block's box is tested against the s
// chunk's box, then against each of the chunk's (up to 8) s blocks; a box
// pair whose distance minus the Hausdorff terms exceeds the pair's
// threshold is skipped (PJ_TILE_PRUNE; without it every block pair is a
// unit).  The live units of a warp are appended with one atomic add.

struct BoxView {
  const float4* chunk;   // [3C] chunk boxes
  const int64_t* coff;   // [n+1]
  const float4* blk;     // [3B] block boxes
  const int64_t* boff;   // [n+1]
  const int64_t* foff;   // [n+1]
};

// lower bound of the distance of two boxes (rounded down)
__device__ __forceinline__ float box_gap_rd(float4 alo, float4 ahi, float4 blo, float4 bhi) {
  float gx = fmaxf(0.f, fmaxf(__fsub_rd(blo.x, ahi.x), __fsub_rd(alo.x, bhi.x)));
  float gy = fmaxf(0.f, fmaxf(__fsub_rd(blo.y, ahi.y), __fsub_rd(alo.y, bhi.y)));
  float gz = fmaxf(0.f, fmaxf(__fsub_rd(blo.z, ahi.z), __fsub_rd(alo.z, bhi.z)));
  float s = __fadd_rd(__fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy)), __fmul_rd(gz, gz));
  return __fsqrt_rd(s);
}

__device__ __forceinline__ float absmax_rel(float4 lo, float4 hi, float4 o) {
  float m = fmaxf(fmaxf(fabsf(lo.x - o.x), fabsf(hi.x - o.x)), fmaxf(fabsf(lo.y - o.y), fabsf(hi.y - o.y)));
  return fmaxf(m, fmaxf(fabsf(lo.z - o.z), fabsf(hi.z - o.z)));
}

// Margins of a box pair (chunks or blocks) in the pair-local frame.
__device__ __forceinline__ Margins box_margins(const float4* cr, const float4* cs, float4 o) {
  float rho = fmaxf(absmax_rel(cr[0], cr[1], o), absmax_rel(cs[0], cs[1], o));
  rho = rho * 1.0001f + 1e-30f;
  float L = fmaxf(cr[2].x, cs[2].x);
  float smin = fminf(cr[2].y, cs[2].y);
  return fp32_margins(rho, L, smin);
}

// Can a facet pair of these two boxes reach the threshold?  Every facet pair
// has true distance >= the box gap; the single-precision lower bound loses
// at most 2 eps; Eq. 2 subtracts at most the max ph of each side.
__device__ __forceinline__ bool box_pair_live(const float4* cr, const float4* cs, float thr, float eps) {
  float g = box_gap_rd(cr[0], cr[1], cs[0], cs[1]);
  float lb = __fsub_rd(__fsub_rd(__fsub_rd(g, cr[1].w), cs[1].w), 2.f * eps);
  return !(lb > thr);
}

__device__ __forceinline__ int64_t find_pair(const int64_t* off, int64_t n, int64_t w) {
  // largest p with off[p] <= w
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Work items of every selected pair: r blocks x s chunks.  Also clears the
// unit counter that k_emit_units appends to.
__global__ void k_items(int64_t n, const int32_t* pr, const int32_t* ps, const uint8_t* status,
                        const uint8_t* lod0, uint8_t want, int step, const int64_t* boffR, const int64_t* coffS,
                        int64_t* cnt, int64_t* ucount) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p == 0) *ucount = 0;
  if (p >= n) return;
  const bool sel = status[p] == want && lod0[p] <= step;
  cnt[p] = sel ? (boffR[pr[p] + 1] - boffR[pr[p]]) * (coffS[ps[p] + 1] - coffS[ps[p]]) : 0;
}

// EMIT = false: only count the live units into *ucount; EMIT = true: also
// write them (at most cap; more sets ERR_CAPACITY and drops the excess).
// Work items w < off1[n] (read on the device), walked in warp-uniform
// strides so the warp-wide append is safe.
template <bool EMIT>
__global__ void __launch_bounds__(256) k_emit_units(int64_t n, const int32_t* pr, const int32_t* ps,
                                                    const int64_t* off1, BoxView R, BoxView S,
                                                    const float4* origin, const float* thr, int cull, int fp64,
                                                    Tile* tiles, int64_t cap, int64_t* ucount, int* err) {
  constexpr int SB = CHUNK / BLK;
  const int64_t W = off1[n];
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); w0 < W; w0 += stride) {
    const int64_t w = w0 + lane;
    unsigned mask = 0;
    float eps[SB], eh[SB];
    int sl[SB];
    int32_t pair = 0, fr = 0, fs0 = 0;
    int rl = 0;
#pragma unroll
    for (int j = 0; j < SB; ++j) {
      eps[j] = eh[j] = 0.f;
      sl[j] = 0;
    }
    if (w < W) {
      const int64_t p = find_pair(off1, n, w);
      const int r = pr[p], s = ps[p];
      const int64_t loc = w - off1[p];
      const int64_t nsc = S.coff[s + 1] - S.coff[s];
      const int64_t rb = R.boff[r] + loc / nsc;
      const int64_t sc = S.coff[s] + loc % nsc;
      const int64_t sb0 = S.boff[s] + (sc - S.coff[s]) * SB;
      const int nsb = (int)min((int64_t)SB, S.boff[s + 1] - sb0);
      const float4 o = origin[p];
      const float t = thr[p];
      const float4* ba = R.blk + 3 * rb;
      const int64_t fr64 = R.foff[r] + (rb - R.boff[r]) * BLK;
      const int64_t fs64 = S.foff[s] + (sb0 - S.boff[s]) * BLK;
      pair = (int32_t)p;
      fr = (int32_t)fr64;
      fs0 = (int32_t)fs64;
      rl = (int)min((int64_t)BLK, R.foff[r + 1] - fr64);
      const int64_t send = S.foff[s + 1];
      bool live = true;
      if (cull) {
        const float4* cb = S.chunk + 3 * sc;
        live = box_pair_live(ba, cb, t, fp64 ? 0.f : box_margins(ba, cb, o).eps);
      }
      if (live) {
#pragma unroll
        for (int j = 0; j < SB; ++j) {
          if (j < nsb) {
            const float4* bb = S.blk + 3 * (sb0 + j);
            Margins m = box_margins(ba, bb, o);
            if (fp64) m.eps = m.eh = 0.f;
            if (!cull || box_pair_live(ba, bb, t, m.eps)) {
              mask |= 1u << j;
              eps[j] = m.eps;
              eh[j] = m.eh;
              sl[j] = (int)min((int64_t)BLK, send - (fs64 + (int64_t)j * BLK));
            }
          }
        }
      }
    }
    const int c = __popc(mask);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total)
      base = atomicAdd(reinterpret_cast<unsigned long long*>(ucount), (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (EMIT && mask) {
      int64_t pos = (int64_t)base + incl - c;
      if (pos + c > cap) {
        set_err(err, ERR_CAPACITY);
      } else {
#pragma unroll
        for (int j = 0; j < SB; ++j) {
          if (mask & (1u << j)) {
            Tile tl;
            tl.pair = pair;
            tl.rb = fr;
            tl.sb = fs0 + j * BLK;
            tl.rl = (uint16_t)rl;
            tl.sl = (uint16_t)sl[j];
            tl.eps = eps[j];
            tl.eh = eh[j];
            tl.ew = 0.f;
            tl.pad = 0;
            tiles[pos++] = tl;
          }
        }
      }
    }
  }
}

static BoxView box_view(const LodData& L) { return BoxView{L.chunk, L.coff, L.blk, L.boff, L.foff}; }

// Shared by the workspace path and the explicit-buffer path.
constexpr size_t UNIT_BUDGET_BYTES = size_t(512) << 20;

static UnitCount build_units(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                             const int32_t* pr, const int32_t* ps, const uint8_t* status, const uint8_t* lod0,
                             const float4* origin, const float* thr, int64_t* cnt1, int64_t* off1, int64_t* ucount,
                             Tile** tiles_io, int64_t tiles_cap, bool grow, int64_t* scan_tmp, int* err,
                             cudaStream_t st) {
  const LodData& LR = R->lod[sp.lodR];
  const LodData& LS = S->lod[sp.lodS];
  BoxView vr = box_view(LR), vs = box_view(LS);
  int th = 256;
  k_items<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, pr, ps, status, lod0, sp.want, sp.step, LR.boff, LS.coff,
                                                        cnt1, ucount);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, cnt1, off1, n, st, scan_tmp);   // off1[n] = work items
  const int64_t bR = (LR.maxF + BLK - 1) / BLK, bS = (LS.maxF + BLK - 1) / BLK;
  const int64_t cS = std::max<int64_t>(1, (LS.maxF + CHUNK - 1) / CHUNK);
  const int64_t items_max = n * bR * cS;
  const unsigned g =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((items_max + th - 1) / th, (int64_t)ctx->sm_count * 16));
  const int64_t worst = n * bR * bS;
  UnitCount uc{-1, ucount};
  int64_t cap = tiles_cap;
  if (worst <= tiles_cap || (grow && (size_t)worst * sizeof(Tile) <= UNIT_BUDGET_BYTES)) {
    if (worst > tiles_cap) {
      *tiles_io = (Tile*)ws_get(ctx, WS_TILES, worst * sizeof(Tile), st);
      cap = worst;
    }
  } else {
    // the worst case does not fit: count first, then size the buffer
    k_emit_units<false><<<g, th, 0, st>>>(n, pr, ps, off1, vr, vs, origin, thr, sp.cull, sp.fp64, nullptr, 0,
                                          ucount, err);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    int64_t total = 0;
    PJ_CK(cudaMemcpyAsync(&total, ucount, 8, cudaMemcpyDeviceToHost, st));
    PJ_CK(cudaStreamSynchronize(st));
    uc.count = total;
    if (total == 0) return uc;
    if (total > tiles_cap) {
      if (!grow) throw ApiError{PJ_EINVAL, "refinement units above the scratch capacity"};
      *tiles_io = (Tile*)ws_get(ctx, WS_TILES, total * sizeof(Tile), st);
      cap = total;
    }
    PJ_CK(cudaMemsetAsync(ucount, 0, 8, st));
  }
  k_emit_units<true><<<g, th, 0, st>>>(n, pr, ps, off1, vr, vs, origin, thr, sp.cull, sp.fp64, *tiles_io, cap,
                                       ucount, err);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  return uc;
}

UnitCount build_tiles(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                      cudaStream_t st) {
  if (n == 0) return UnitCount{0, nullptr};
  auto pr = (int32_t*)ws_get(ctx, WS_PR, n * 4, st);
  auto ps = (int32_t*)ws_get(ctx, WS_PS, n * 4, st);
  auto status = (uint8_t*)ws_get(ctx, WS_STATUS, n, st);
  auto lod0 = (uint8_t*)ws_get(ctx, WS_LOD0, n, st);
  auto origin = (float4*)ws_get(ctx, WS_ORIGIN, n * 16, st);
  auto thr = (float*)ws_get(ctx, WS_THR, ((n + 3) & ~int64_t(3)) * 4, st);   // 16-byte groups (k_refine)
  auto cnt1 = (int64_t*)ws_get(ctx, WS_TCOUNT, (n + 1) * 8, st);
  auto off1 = (int64_t*)ws_get(ctx, WS_SCAN, (n + 1) * 8, st);
  auto ucount = (int64_t*)ws_get(ctx, WS_MISC4, 64, st);
  auto tmp = (int64_t*)ws_get(ctx, WS_MISC5, (scan_tmp_words(n) + 8) * 8, st);
  Tile* tiles = (Tile*)ctx->ws[WS_TILES].p;
  const int64_t cap = (int64_t)(ctx->ws[WS_TILES].cap / sizeof(Tile));
  return build_units(ctx, R, S, n, sp, pr, ps, status, lod0, origin, thr, cnt1, off1, ucount, &tiles, cap, true,
                     tmp, ctx->d_err, st);
}

__global__ void k_init_bounds(int64_t n, const uint8_t* status, const uint8_t* lod0, uint8_t want, int step,
                              int fp64, void* lb, void* ub, void* mid, uint8_t* flag) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (!(status[p] == want && lod0[p] <= step)) return;
  if (flag) flag[p] = 0;
  if (fp64) {
    const unsigned long long inf = 0x7ff0000000000000ULL;
    ((unsigned long long*)lb)[p] = inf;
    ((unsigned long long*)ub)[p] = inf;
    ((unsigned long long*)mid)[p] = inf;
  } else {
    const unsigned inf = 0x7f800000u;
    ((unsigned*)lb)[p] = inf;
    ((unsigned*)ub)[p] = inf;
    ((unsigned*)mid)[p] = inf;
  }
}

void init_bounds(pj_ctx* ctx, int64_t n, const StepSpec& sp, cudaStream_t st) {
  if (n == 0) return;
  auto status = (uint8_t*)ws_get(ctx, WS_STATUS, n, st);
  auto lod0 = (uint8_t*)ws_get(ctx, WS_LOD0, n, st);
  auto lb = ws_get(ctx, WS_LB, n * 8, st);
  auto ub = ws_get(ctx, WS_UB, n * 8, st);
  auto mid = ws_get(ctx, WS_MID, n * 8, st);
  auto flag = (uint8_t*)ws_get(ctx, WS_FLAG, n, st);
  int th = 256;
  k_init_bounds<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, status, lod0, sp.want, sp.step, sp.fp64, lb,
                                                               ub, mid, flag);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// ------------------------------------------------------------------ refine

struct RefineArgs {
  const Tile* tiles;
  int64_t n_tiles;
  const int64_t* n_tiles_dev;   // if set, the unit count lives here
  int* counter;
  const float4* facR;
  const float4* facS;
  const float4* origin;
  const float* thr;
  void* lb;
  void* ub;
  void* mid;
  unsigned long long* ntests;
  unsigned long long* nculled;   // facet pairs skipped by the ball test (may be null)
  unsigned long long* nneeded;   // executed tests whose lane's own ball test asked for them (may be null)
  int* err;
  int4* queue;       // straddling facet pairs: (pair, r facet, s facet, eps bits)
  unsigned* qcount;
  unsigned qcap;
  uint8_t* flag;     // per pair: a unit proved ub <= threshold (early exit)
  int early;         // skip the units of flagged pairs
  int exact_cross;   // decide every straddling pair's meeting test (bounds entry points)
  const double* ub_prev;   // per pair: a valid upper bound of d known before this step (may be null)
  int cull;                // units were pruned against thr (values above thr are not needed)
  int split_k;             // tail units are handed out as split_k sub-units (1: no splitting)
  int64_t split_tail;      // how many of the last units are split
  int masked;              // full resolution: Tile::pad holds the unit's s-facet mask (k_unit_masks)
};

// Tail splitting.  Units are taken from one counter over a virtual index
// space: the first NT - T indices are whole units, the rest are the
// split_k parts of the last T units (part q covers s facets
// [q 32/K, (q+1) 32/K) of its unit, and the matching bits of its s-facet
// mask), so that the last units of a launch are short and the warps finish
// together.  Parts past a ragged unit's s facets are empty (sl = 0).
struct UnitSpace {
  int64_t NT, T, NV;
  int K;
};
__host__ __device__ __forceinline__ UnitSpace unit_space(int64_t NT, int K, int64_t tail) {
  UnitSpace u;
  u.NT = NT;
  u.K = K > 1 ? K : 1;
  u.T = u.K > 1 ? (NT < tail ? NT : tail) : 0;
  u.NV = NT + u.T * (u.K - 1);
  return u;
}
// the unit array entry of virtual index v, and which part of it (-1: whole)
__device__ __forceinline__ int64_t unit_index(const UnitSpace& u, int64_t v, int& part) {
  const int64_t head = u.NT - u.T;
  if (v < head) {
    part = -1;
    return v;
  }
  part = (int)((v - head) % u.K);
  return head + (v - head) / u.K;
}
__device__ __forceinline__ Tile unit_part(Tile t, const UnitSpace& u, int part) {
  if (part < 0) return t;
  const int w = BLK / u.K, s0 = part * w;
  t.sb += s0;
  t.sl = (uint16_t)max(0, min(w, (int)t.sl - s0));
  t.pad = (int32_t)(((uint32_t)t.pad >> s0) & (w >= 32 ? 0xffffffffu : ((1u << w) - 1u)));   // s-facet mask
  return t;
}
__device__ __forceinline__ Tile unit_at(const Tile* tiles, const UnitSpace& u, int64_t v) {
  int part;
  const int64_t i = unit_index(u, v, part);
  return unit_part(tiles[i], u, part);
}

template <class T>
__device__ __forceinline__ void translate(const float4& A, const float4& o, T out[3]) {
  out[0] = T(A.x) - T(o.x);
  out[1] = T(A.y) - T(o.y);
  out[2] = T(A.z) - T(o.z);
}

constexpr uint32_t MBAR_POLL_LIMIT = 1u << 20;
constexpr int REFINE_WARPS = REFINE_THREADS / 32;
// k_refine's warps per CTA: 12 in single precision (166 registers), 8 in
// double precision (its records need up to 255 registers)
template <class T>
constexpr int kref_warps() {
  return sizeof(T) == 4 ? REFINE_WARPS : 8;
}

constexpr int WARP_LIST = 128;   // straddling facet pairs kept per warp and unit

// k_refine's per-warp shared memory: two stages (header: the unit's tile,
// its pair's origin and threshold; the unit's r facets; its s facets), the s-facet
// records, the straddling-pair list, and the slot the next unit's tile is
// fetched into.
struct StageHdr {
  Tile tile;
  float4 origin;
  float thr4[4];   // thr[pair & ~3 ..]: the pair's threshold at [pair & 3]
};
constexpr size_t STAGE_BYTES = sizeof(StageHdr) + 2 * BLK * 48;
static_assert(sizeof(StageHdr) == 64 && STAGE_BYTES % 16 == 0, "stage layout");
template <class T>
constexpr size_t warp_smem_bytes() {
  return 2 * STAGE_BYTES + (size_t)BLK * sizeof(typename RecOf<T>::S) + (size_t)WARP_LIST * 8 + sizeof(Tile);
}
template <class T>
constexpr size_t refine_smem_bytes() {
  return kref_warps<T>() * warp_smem_bytes<T>();
}

template <class T>
struct ListOut {
  T lbm, ubu, ubc, d2m;
  bool anyposs;
};

// Contributions of the straddling facet pairs a warp listed during one
// unit: lane k takes entries k, k+32, ...; the meeting test is decided in
// double precision (cross_decide: single-precision filtered signs, else
// cross_exact64).  Out of line so that its double-precision
// registers do not weigh on the unit's inner loop; called only when the
// warp's list is non-empty.
template <class T, bool FULL>
__device__ __noinline__ ListOut<T> process_list(const uint2* list, unsigned nl, int lane, const float4* fr0,
                                                const float4* raw, float4 o4) {
  const T INF = inf_(T(0));
  ListOut<T> out{INF, INF, INF, INF, false};
  for (unsigned k = lane; k < nl; k += 32) {
    const uint2 e = list[k];
    const int li = e.x & 255, lj = e.x >> 8;
    const float4* fr = fr0 + 3 * li;
    const bool cert = cross_decide(fr, raw + 3 * lj, o4);
    const T phs = add_ru(T(fr[1].w), T(raw[3 * lj + 1].w)), hds = add_ru(T(fr[0].w), T(raw[3 * lj].w));
    if (cert) {
      out.lbm = min(out.lbm, -phs);
      out.ubc = min(out.ubc, hds);
      if (FULL) out.anyposs = true;
    } else {
      const T d2e = T(__uint_as_float(e.y));
      if (FULL) {
        out.d2m = min(out.d2m, d2e);
      } else {
        T d = sqrt_test(d2e);
        out.lbm = min(out.lbm, sub_rd(d, phs));
        out.ubu = min(out.ubu, add_ru(d, hds));
      }
    }
  }
  return out;
}

// Full-resolution steps: which s facets of a unit some r facet may still
// need.  A facet pair whose balls are farther apart than the pair's bound
// (its upper bound from the previous step and, when units were pruned, its
// threshold: the same bound k_refine starts from) cannot lower the
// distance, so it is skipped.  One warp per unit: lane i holds the ball of r
// facet i and of s facet i; the union of the lanes' needs goes into
// Tile::pad and the bound into Tile::ew (rounded up to float).  With `out`,
// units that need nothing are dropped and the rest
// compacted into `out` (count at *n_out); without it, the masks are written
// in place.  The skipped facet pairs are added to *nculled (if set).  Light
// on registers, so it runs at full occupancy and hides the loads that the
// refinement kernel would otherwise wait on per unit.
struct MaskArgs {
  Tile* tiles;
  int64_t n_tiles;
  const int64_t* n_tiles_dev;
  const float4* facR;
  const float4* facS;
  const float4* origin;
  const float* thr;
  const double* ub_prev;
  int cull;
  Tile* out;
  int64_t* n_out;
  unsigned long long* nculled;
};

template <class T>
__global__ void __launch_bounds__(256) k_unit_masks(MaskArgs m) {
  using T4 = typename std::conditional<sizeof(T) == 4, float4, double4>::type;
  __shared__ T4 sball[8][32];   // per warp: the s facets' balls (centre, radius)
  const int lane = threadIdx.x & 31;
  T4* sb = sball[threadIdx.x >> 5];
  const unsigned FULLM = 0xffffffffu;
  const int64_t NT = m.n_tiles_dev ? *m.n_tiles_dev : m.n_tiles;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long culled = 0;
  Tile keep;            // lane k: the k-th kept unit not yet written
  int nkeep = 0;
  auto flush = [&]() {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(m.n_out), (unsigned long long)nkeep);
    base = __shfl_sync(FULLM, base, 0);
    if (lane < nkeep) m.out[base + lane] = keep;
    nkeep = 0;
  };
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < NT; u += nw) {
    const Tile t = m.tiles[u];
    const float4 o4 = m.origin[t.pair];
    const bool ract = lane < t.rl, sact = lane < t.sl;
    T rc[3], rr, sc[3], sr;
    {
      const float4* f = m.facR + 3LL * (t.rb + (ract ? lane : 0));
      T va[3], vb[3], vc[3];
      translate(f[0], o4, va);
      translate(f[1], o4, vb);
      translate(f[2], o4, vc);
      facet_ball(va, vb, vc, rc, rr);
    }
    {
      const float4* f = m.facS + 3LL * (t.sb + (sact ? lane : 0));
      T va[3], vb[3], vc[3];
      translate(f[0], o4, va);
      translate(f[1], o4, vb);
      translate(f[2], o4, vc);
      facet_ball(va, vb, vc, sc, sr);
    }
    T bound = inf_(T(0));
    if (m.ub_prev) bound = sizeof(T) == 4 ? T(__double2float_ru(m.ub_prev[t.pair])) : T(m.ub_prev[t.pair]);
    if (m.cull) bound = min(bound, T(m.thr[t.pair]));
    uint32_t mine = 0;
    T4 mb;
    mb.x = sc[0];
    mb.y = sc[1];
    mb.z = sc[2];
    mb.w = sr;
    sb[lane] = mb;
    __syncwarp();
    for (int j = 0; j < t.sl; ++j) {
      const T4 q = sb[j];   // broadcast read
      const T qc[3] = {q.x, q.y, q.z};
      if (ract && !balls_apart(rc, rr, qc, q.w, bound)) mine |= 1u << j;
    }
    __syncwarp();   // the balls are read before the next unit writes them
    const uint32_t need = __reduce_or_sync(FULLM, mine);
    const uint32_t all = t.sl >= 32 ? 0xffffffffu : ((1u << t.sl) - 1u);
    if (ract) culled += (unsigned long long)__popc(all & ~need);
    // the unit's starting bound for k_refine, rounded up to float
    const float bf = sizeof(T) == 4 ? float(bound) : __double2float_ru(double(bound));
    if (!m.out) {
      if (lane == 0) {
        m.tiles[u].pad = (int32_t)need;
        m.tiles[u].ew = bf;
      }
    } else if (need) {
      if (lane == nkeep) {
        keep = t;
        keep.pad = (int32_t)need;
        keep.ew = bf;
      }
      if (++nkeep == 32) flush();
    }
  }
  if (nkeep) flush();
  culled = warp_sum_u64(culled);
  if (lane == 0 && culled && m.nculled) atomicAdd(m.nculled, culled);
}

// Minimum over the warp: floats through __reduce_min_sync on an
// order-preserving map of their bits (one instruction instead of a shuffle
// tree), doubles by shuffles.
__device__ __forceinline__ float warp_min_fast(float v) {
  unsigned u = __float_as_uint(v);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  u = __reduce_min_sync(0xffffffffu, u);
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ double warp_min_fast(double v) { return warp_min(v); }

// Persistent, warp-granular refinement.  Every warp takes units (its first
// two by its index, then from a global counter) and runs a three-deep
// pipeline of its own: a unit is claimed two iterations before it is
// computed, its tile is fetched by a bulk copy one iteration before, and
// then its pair origin and threshold, r facets and s facets are staged by
// TMA into the warp's second buffer while the current unit computes; so the
// compute of a unit waits on no global load.  The s facets are expanded into
// records in the warp's shared-memory slice, one r facet per lane is kept in
// registers.  No barrier couples the warps of a CTA.
template <class T, bool FULL>
__global__ void __launch_bounds__(kref_warps<T>() * 32, 1) k_refine(RefineArgs a) {
  constexpr int WARPS = kref_warps<T>();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[WARPS][3];
  __shared__ unsigned list_n[WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wbase = smem + warp * warp_smem_bytes<T>();
  using RecT = typename RecOf<T>::R;
  using RecS = typename RecOf<T>::S;
  RecS* rec = reinterpret_cast<RecS*>(wbase + 2 * STAGE_BYTES);
  uint2* list = reinterpret_cast<uint2*>(wbase + 2 * STAGE_BYTES + BLK * sizeof(RecS));
  Tile* tslot = reinterpret_cast<Tile*>(wbase + 2 * STAGE_BYTES + BLK * sizeof(RecS) + WARP_LIST * 8);
  uint64_t* bar = bars[warp];   // [0], [1]: stages; [2]: the tile slot
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    fence_mbar_init();
    list_n[warp] = 0;
  }
  __syncwarp();
  const T INF = inf_(T(0));
  const unsigned FULLM = 0xffffffffu;
  const UnitSpace us = unit_space(a.n_tiles_dev ? *a.n_tiles_dev : a.n_tiles, a.split_k, a.split_tail);
  uint32_t ph0 = 0, ph1 = 0, ph2 = 0;
  unsigned ntest = 0, nskip = 0, nneed = 0;   // per lane (a lane sees far fewer than 2^32)
  bool failed = false;
  unsigned pend = 0;   // lane 0: barriers with copies in flight (bit k: stage k, bit 2: tile slot)

  // lane 0: stage unit t into buffer k (header by a store, the rest by TMA)
  auto stage = [&](int k, const Tile& t) {
    unsigned char* sb = wbase + k * STAGE_BYTES;
    StageHdr* h = reinterpret_cast<StageHdr*>(sb);
    h->tile = t;
    if (t.sl == 0) {   // an empty part: nothing to copy
      mbar_arrive_expect_tx(&bar[k], 0);
      return;
    }
    pend |= 1u << k;
    fence_proxy_async();
    const uint32_t rb = (uint32_t)t.rl * 48u, sbytes = (uint32_t)t.sl * 48u;
    mbar_arrive_expect_tx(&bar[k], 32u + rb + sbytes);
    tma_load_1d(&h->origin, a.origin + t.pair, 16u, &bar[k]);
    tma_load_1d(h->thr4, a.thr + (t.pair & ~3), 16u, &bar[k]);
    tma_load_1d(sb + sizeof(StageHdr), a.facR + 3LL * t.rb, rb, &bar[k]);
    tma_load_1d(sb + sizeof(StageHdr) + BLK * 48, a.facS + 3LL * t.sb, sbytes, &bar[k]);
  };
  // lane 0: fetch the tile of virtual unit v into the slot
  auto fetch = [&](int v) {
    int part;
    const int64_t i = unit_index(us, v, part);
    pend |= 4u;
    fence_proxy_async();
    mbar_arrive_expect_tx(&bar[2], (uint32_t)sizeof(Tile));
    tma_load_1d(tslot, a.tiles + i, (uint32_t)sizeof(Tile), &bar[2]);
  };

  // the first two units of every warp are assigned statically (warp w: w
  // and w + NW, with w counted CTA-minor so that consecutive units land on
  // different SMs), later ones come from the counter, offset by 2 NW; so a
  // launch with few units spreads them over the SMs
  const int NV = (int)us.NV;
  const int NW = (int)gridDim.x * WARPS, gw = warp * (int)gridDim.x + (int)blockIdx.x;
  int cur = gw, vnext = 0, vclaim = 0;   // virtual unit indices; vnext, vclaim: lane 0 only
  if (lane == 0) {
    if (cur < NV) stage(0, unit_at(a.tiles, us, cur));
    vnext = gw + NW;
    if (vnext < NV) fetch(vnext);
    vclaim = 2 * NW + atomicAdd(a.counter, 1);
  }
  cur = __shfl_sync(FULLM, cur, 0);
  int b = 0;
  while (cur < NV) {
    // lane 0: the next unit into the other stage, the tile after it into the
    // slot, and one more claim
    int nxt = 0;
    if (lane == 0) {
      nxt = vnext;
      if (vnext < NV) {
        if (mbar_wait_bounded(&bar[2], ph2, MBAR_POLL_LIMIT)) {
          ph2 ^= 1u;
          pend &= ~4u;
          int part;
          unit_index(us, vnext, part);
          stage(b ^ 1, unit_part(*tslot, us, part));
          vnext = vclaim;
          if (vnext < NV) fetch(vnext);
          vclaim = 2 * NW + atomicAdd(a.counter, 1);
        } else {
          failed = true;
          nxt = NV;
        }
      }
    }
    nxt = __shfl_sync(FULLM, nxt, 0);
    // this unit's stage
    const bool ok = mbar_wait_bounded(b ? &bar[1] : &bar[0], b ? ph1 : ph0, MBAR_POLL_LIMIT);
    if (__any_sync(FULLM, !ok) || __any_sync(FULLM, failed)) {
      failed = true;
      break;
    }
    if (b) ph1 ^= 1u;
    else ph0 ^= 1u;
    pend &= ~(1u << b);
    const unsigned char* sbuf = wbase + b * STAGE_BYTES;
    const StageHdr* hdr = reinterpret_cast<const StageHdr*>(sbuf);
    const Tile tl = hdr->tile;
    const int rl = tl.rl, sl = tl.sl;
    const bool act = lane < rl;
    // the decided flag (written by other warps) and the threshold, loaded
    // now and used after the records are built
    const uint8_t decided = (a.early && sl) ? __ldcg(a.flag + tl.pair) : (uint8_t)0;
    if (sl == 0 || (FULL && a.masked && tl.pad == 0)) {   // an empty part or mask
      __syncwarp();
      cur = nxt;
      b ^= 1;
      continue;
    }
    const float4 o4 = hdr->origin;
    const float4* rfac = reinterpret_cast<const float4*>(sbuf + sizeof(StageHdr));
    const float4* raw = reinterpret_cast<const float4*>(sbuf + sizeof(StageHdr) + BLK * 48);
    RecT P;
    {
      const float4* f = rfac + 3 * (act ? lane : 0);
      float4 A = f[0], B = f[1], C = f[2];
      T va[3], vb[3], vc[3];
      translate(A, o4, va);
      translate(B, o4, vb);
      translate(C, o4, vc);
      make_rec(P, va, vb, vc, T(A.w), T(B.w), true);
    }
    if (lane < sl) {
      float4 A = raw[3 * lane], B = raw[3 * lane + 1], C = raw[3 * lane + 2];
      T va[3], vb[3], vc[3];
      translate(A, o4, va);
      translate(B, o4, vb);
      translate(C, o4, vc);
      RecT Q;
      make_rec(Q, va, vb, vc, T(A.w), T(B.w), false);
      store_rec(rec[lane], Q);
    }
    __syncwarp();
    if (decided) {   // the pair is already decided
      __syncwarp();
      cur = nxt;
      b ^= 1;
      continue;
    }

    T lbm = INF, ubu = INF, d2m = INF;
    bool anyposs = false;
    const T eh = T(tl.eh);
    // facet pairs whose balls are farther apart than what the lane can
    // still improve are skipped (when the whole warp agrees): always in
    // single precision, in double precision when units were pruned.  At
    // full resolution only the s facets of the unit's mask are visited
    // (k_unit_masks), and the bound starts at the mask pass's bound.
    const bool balls = sizeof(T) == 4 || a.cull;
    T dcur = INF;
    uint32_t cand = sl >= 32 ? 0xffffffffu : ((1u << sl) - 1u);
    if (FULL && balls && a.masked) {
      cand &= (uint32_t)tl.pad;
      dcur = T(tl.ew);
    }
    while (cand) {
      const int j = __ffs(cand) - 1;
      cand &= cand - 1u;
      if (balls) {
        // the ball (and hd / ph) first; the record only when needed
        T qc[3], qr, qhd, qph;
        rec_ball(rec[j], qc, qr, qhd, qph);
        bool need = act;
        if (need) {
          if (FULL) need = !balls_apart(P.sc, P.sr, qc, qr, dcur);
          else need = !coarse_cull(P.sc, P.sr, P.ph, P.hd, qc, qr, qph, qhd, lbm, ubu);
        }
        if (!__any_sync(FULLM, need)) {
          nskip += act;
          continue;
        }
        nneed += need;
      } else {
        nneed += act;
      }
      if (!act) continue;
      RecT Q;
      load_rec(Q, rec[j]);
      ++ntest;
      bool maybe;
      T d2 = tri_d2(P, Q, eh, maybe);
      if (maybe && boxes_apart(P, Q)) maybe = false;   // straddling planes, but apart
      if (!maybe) {
        if (FULL) {
          if (d2 < d2m) {
            d2m = d2;
            if (balls) dcur = min(dcur, sqrt_ru(d2m));
          }
        } else {
          T d = sqrt_test(d2);
          lbm = min(lbm, sub_rd(d, add_ru(P.ph, Q.ph)));
          ubu = min(ubu, add_ru(d, add_ru(P.hd, Q.hd)));
        }
      } else if (!FULL && sizeof(T) == 4 && !a.exact_cross) {
        // coarse LoD: a crossing is taken as possible (lower term -ph-ph,
        // upper term d+hd+hd); both stay valid and are only ~d looser
        T d = sqrt_test(d2);
        lbm = min(lbm, -add_ru(P.ph, Q.ph));
        ubu = min(ubu, add_ru(d, add_ru(P.hd, Q.hd)));
      } else {
        // rare at full resolution: both triangles straddle each other's
        // planes; decided after the loop (warp list), or by k_cross_fix
        // when the list is full
        unsigned li = atomicAdd(&list_n[warp], 1u);
        if (li < WARP_LIST) {
          list[li] = make_uint2((unsigned)(lane | (j << 8)), __float_as_uint((float)d2));
        } else {
          unsigned qk = atomicAdd(a.qcount, 1u);
          if (qk < a.qcap) {
            a.queue[qk] = make_int4(tl.pair, tl.rb + lane, tl.sb + j, __float_as_int(tl.eps));
          } else if (FULL) {
            anyposs = true;   // a crossing is possible: lower bound 0 stays valid
            d2m = min(d2m, d2);
          } else {
            T d = sqrt_test(d2);
            lbm = min(lbm, -add_ru(P.ph, Q.ph));
            ubu = min(ubu, add_ru(d, add_ru(P.hd, Q.hd)));
          }
        }
      }
    }
    // the warp's straddling pairs: meeting test in double precision
    __syncwarp();
    const unsigned nl = min(list_n[warp], (unsigned)WARP_LIST);
    T ubc = INF;
    if (nl) {
      ListOut<T> lo = process_list<T, FULL>(list, nl, lane, rfac, raw, o4);
      lbm = min(lbm, lo.lbm);
      ubu = min(ubu, lo.ubu);
      ubc = lo.ubc;
      d2m = min(d2m, lo.d2m);
      anyposs = anyposs || lo.anyposs;
    }
    __syncwarp();
    if (lane == 0) list_n[warp] = 0;
    T lbv, ubv, midv = INF;
    if (FULL) {
      T d = d2m < INF ? sqrt_rn(d2m) : INF;
      midv = ubc < INF ? T(0) : d;
      lbv = anyposs ? T(0) : d;
      ubv = d;
    } else {
      lbv = lbm;
      ubv = ubu;
    }
    lbv = warp_min_fast(lbv);
    ubv = warp_min_fast(ubv);
    ubc = warp_min_fast(ubc);
    if (FULL) midv = warp_min_fast(midv);
    if (lane == 0) {
      const T eps = T(tl.eps);
      T lb = lbv < INF ? sub_rd(lbv, eps) : INF;
      lb = max(lb, T(0));
      T ub = ubv < INF ? add_ru(ubv, eps) : INF;
      ub = min(ub, ubc);
      using Bt = Bits<T>;
      if (lb < INF) atomicMin(&((typename Bt::U*)a.lb)[tl.pair], Bt::enc(lb));
      if (ub < INF) atomicMin(&((typename Bt::U*)a.ub)[tl.pair], Bt::enc(ub));
      if (FULL && midv < INF) atomicMin(&((typename Bt::U*)a.mid)[tl.pair], Bt::enc(midv));
      if (a.early && ub <= hdr->thr4[tl.pair & 3]) a.flag[tl.pair] = 1;
    }
    __syncwarp();   // records of this unit are read; the next unit overwrites them
    cur = nxt;
    b ^= 1;
  }
  if (failed && lane == 0) {
    set_err(a.err, ERR_MBAR_TIMEOUT);
    // let the copies in flight land (bounded) before the warp leaves
    if (pend & 1u) mbar_wait_bounded(&bar[0], ph0, MBAR_POLL_LIMIT);
    if (pend & 2u) mbar_wait_bounded(&bar[1], ph1, MBAR_POLL_LIMIT);
    if (pend & 4u) mbar_wait_bounded(&bar[2], ph2, MBAR_POLL_LIMIT);
  }
  const unsigned long long nt = warp_sum_u64(ntest), ns = warp_sum_u64(nskip), nn = warp_sum_u64(nneed);
  if (lane == 0 && nt) atomicAdd(a.ntests, nt);
  if (lane == 0 && ns && a.nculled) atomicAdd(a.nculled, ns);
  if (lane == 0 && nn && a.nneeded) atomicAdd(a.nneeded, nn);
}

// Bounds contribution of the queued straddling facet pairs: the 15-candidate
// distance as in k_refine, the meeting test in double precision (exact
// translation of the float vertices), then the same atomicMin updates.
// ---------------------------------------------------------------- packed FP32
// k_refine2: the single-precision refinement with two s facets per lane and
// loop iteration (tritri2.cuh).  The s block is expanded into 16 paired
// records; an odd last facet is paired with a copy of itself and the copy's
// half is masked.  Unit scheduling, staging, the straddle list and the
// reductions are those of k_refine.
constexpr size_t warp_smem_bytes2() {
  return (size_t)2 * BLK * 48 + (size_t)(BLK / 2) * sizeof(RecSmem2) + (size_t)WARP_LIST * 8;
}
constexpr size_t refine_smem_bytes2() { return REFINE_WARPS * warp_smem_bytes2(); }

template <bool FULL>
__global__ void __launch_bounds__(REFINE_THREADS, 1) k_refine2(RefineArgs a) {
  using T = float;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[REFINE_WARPS][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wbase = smem + warp * warp_smem_bytes2();
  float4* raw0 = reinterpret_cast<float4*>(wbase);
  float4* raw1 = raw0 + 3 * BLK;
  RecSmem2* rec = reinterpret_cast<RecSmem2*>(wbase + 2 * BLK * 48);
  uint2* list = reinterpret_cast<uint2*>(wbase + 2 * BLK * 48 + (BLK / 2) * sizeof(RecSmem2));
  __shared__ unsigned list_n[REFINE_WARPS];
  uint64_t* bar0 = &bars[warp][0];
  uint64_t* bar1 = &bars[warp][1];
  if (lane == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    fence_mbar_init();
    list_n[warp] = 0;
  }
  __syncwarp();
  const T INF = inf_(T(0));
  const unsigned FULLM = 0xffffffffu;
  const UnitSpace us = unit_space(a.n_tiles_dev ? *a.n_tiles_dev : a.n_tiles, a.split_k, a.split_tail);
  uint32_t ph0 = 0, ph1 = 0;
  int b = 0;
  unsigned long long ntest = 0, nskip = 0;

  int64_t cur = 0;
  if (lane == 0) {
    cur = atomicAdd(a.counter, 1);
    if (cur < us.NV) {
      const Tile t0 = unit_at(a.tiles, us, cur);
      mbar_arrive_expect_tx(bar0, (uint32_t)t0.sl * 48u);
      if (t0.sl) tma_load_1d(raw0, a.facS + 3LL * t0.sb, (uint32_t)t0.sl * 48u, bar0);
    }
  }
  cur = __shfl_sync(FULLM, cur, 0);
  while (cur < us.NV) {
    int64_t nxt = 0;
    if (lane == 0) {
      nxt = atomicAdd(a.counter, 1);
      if (nxt < us.NV) {
        const Tile tn = unit_at(a.tiles, us, nxt);
        fence_proxy_async();
        uint64_t* bn = b ? bar0 : bar1;
        mbar_arrive_expect_tx(bn, (uint32_t)tn.sl * 48u);
        if (tn.sl) tma_load_1d(b ? raw0 : raw1, a.facS + 3LL * tn.sb, (uint32_t)tn.sl * 48u, bn);
      }
    }
    nxt = __shfl_sync(FULLM, nxt, 0);
    const Tile tl = unit_at(a.tiles, us, cur);
    const int rl = tl.rl, sl = tl.sl;
    const float4 o4 = a.origin[tl.pair];
    const bool act = lane < rl;
    RecL2 P;
    T Pph, Phd;
    float Psc[3], Psr;
    {
      const float4* f = a.facR + 3LL * (tl.rb + (act ? lane : 0));
      float4 A = f[0], B = f[1], C = f[2];
      T va[3], vb[3], vc[3];
      translate(A, o4, va);
      translate(B, o4, vb);
      translate(C, o4, vc);
      RecL R;
      make_rec(R, va, vb, vc, T(A.w), T(B.w), true);
      dup_rec(P, R);
      Pph = R.ph;
      Phd = R.hd;
      Psc[0] = R.sc[0];
      Psc[1] = R.sc[1];
      Psc[2] = R.sc[2];
      Psr = R.sr;
    }
    const bool ok = mbar_wait_bounded(b ? bar1 : bar0, b ? ph1 : ph0, MBAR_POLL_LIMIT);
    if (__any_sync(FULLM, !ok)) {
      if (lane == 0) {
        set_err(a.err, ERR_MBAR_TIMEOUT);
        if (nxt < us.NV) mbar_wait_bounded(b ? bar0 : bar1, b ? ph0 : ph1, MBAR_POLL_LIMIT);
      }
      break;
    }
    if (b) ph1 ^= 1u;
    else ph0 ^= 1u;
    const float4* raw = b ? raw1 : raw0;
    if (sl == 0 || (FULL && a.masked && tl.pad == 0) || (a.early && __ldcg(a.flag + tl.pair))) {
      __syncwarp();
      cur = nxt;
      b ^= 1;
      continue;
    }
    const int sl2 = (sl + 1) & ~1;   // facets in paired records (odd: last one twice)
    if (lane < sl2) {
      const int fi = min(lane, sl - 1);
      float4 A = raw[3 * fi], B = raw[3 * fi + 1], C = raw[3 * fi + 2];
      T va[3], vb[3], vc[3];
      translate(A, o4, va);
      translate(B, o4, vb);
      translate(C, o4, vc);
      RecL Q;
      make_rec(Q, va, vb, vc, T(A.w), T(B.w), false);
      store_half(rec[lane >> 1], lane & 1, Q);
    }
    __syncwarp();

    T lbm = INF, ubu = INF, d2m = INF;
    bool anyposs = false;
    const T eh = T(tl.eh);
    // facet pairs whose balls are farther apart than what the lane can
    // still improve are skipped (a record pair when the whole warp agrees)
    float dcur = FULL && a.ub_prev ? __double2float_ru(a.ub_prev[tl.pair]) : INF;
    if (FULL && a.cull) dcur = fminf(dcur, a.thr[tl.pair]);
    {
      for (int jp = 0; jp < (sl2 >> 1); ++jp) {
        if (FULL && a.masked && !((((uint32_t)tl.pad) >> (2 * jp)) & 3u)) continue;   // counted by k_unit_masks
        bool need = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!act || 2 * jp + h >= sl) continue;
          const RecSmem2& S2 = rec[jp];
          const float qc[3] = {S2.x[2 * F_SC + h], S2.x[2 * (F_SC + 1) + h], S2.x[2 * (F_SC + 2) + h]};
          const float qr = S2.x[2 * F_SR + h];
          bool nh;
          if (FULL) {
            nh = !balls_apart(Psc, Psr, qc, qr, dcur);
          } else {
            const float qph = S2.x[2 * F_PH + h], qhd = S2.x[2 * F_HD + h];
            nh = !(balls_apart(Psc, Psr, qc, qr, __fadd_ru(lbm, __fadd_ru(Pph, qph))) &&
                   balls_apart(Psc, Psr, qc, qr, __fsub_ru(ubu, __fadd_rd(Phd, qhd))));
          }
          need = need || nh;
        }
        if (!__any_sync(FULLM, need)) {
          if (act) nskip += min(2, sl - 2 * jp);
          continue;
        }
        if (!act) continue;
        RecL2 Q;
        load_pair(Q, rec[jp]);
        bool m0, m1;
        const f2 d2p = tri_d2x2(P, Q, eh, m0, m1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * jp + h;
          if (j >= sl) continue;
          ++ntest;
          const T d2 = h ? hi2(d2p) : lo2(d2p);
          bool maybe = h ? m1 : m0;
          if (maybe && boxes_apart_half(P, rec[jp], h)) maybe = false;
          const T qph = rec[jp].x[2 * F_PH + h], qhd = rec[jp].x[2 * F_HD + h];
          if (!maybe) {
            if (FULL) {
              if (d2 < d2m) {
                d2m = d2;
                dcur = fminf(dcur, __fsqrt_ru(d2m));
              }
            } else {
              T d = sqrt_test(d2);
              lbm = min(lbm, sub_rd(d, add_ru(Pph, qph)));
              ubu = min(ubu, add_ru(d, add_ru(Phd, qhd)));
            }
          } else if (!FULL && !a.exact_cross) {
            T d = sqrt_test(d2);
            lbm = min(lbm, -add_ru(Pph, qph));
            ubu = min(ubu, add_ru(d, add_ru(Phd, qhd)));
          } else {
            unsigned li = atomicAdd(&list_n[warp], 1u);
            if (li < WARP_LIST) {
              list[li] = make_uint2((unsigned)(lane | (j << 8)), __float_as_uint((float)d2));
            } else {
              unsigned qk = atomicAdd(a.qcount, 1u);
              if (qk < a.qcap) {
                a.queue[qk] = make_int4(tl.pair, tl.rb + lane, tl.sb + j, __float_as_int(tl.eps));
              } else if (FULL) {
                anyposs = true;
                d2m = min(d2m, d2);
              } else {
                T d = sqrt_test(d2);
                lbm = min(lbm, -add_ru(Pph, qph));
                ubu = min(ubu, add_ru(d, add_ru(Phd, qhd)));
              }
            }
          }
        }
      }
    }
    __syncwarp();
    const unsigned nl = min(list_n[warp], (unsigned)WARP_LIST);
    T ubc = INF;
    if (nl) {
      ListOut<T> lo = process_list<T, FULL>(list, nl, lane, a.facR + 3LL * tl.rb, raw, o4);
      lbm = min(lbm, lo.lbm);
      ubu = min(ubu, lo.ubu);
      ubc = lo.ubc;
      d2m = min(d2m, lo.d2m);
      anyposs = anyposs || lo.anyposs;
    }
    __syncwarp();
    if (lane == 0) list_n[warp] = 0;
    T lbv, ubv, midv = INF;
    if (FULL) {
      T d = d2m < INF ? sqrt_rn(d2m) : INF;
      midv = ubc < INF ? T(0) : d;
      lbv = anyposs ? T(0) : d;
      ubv = d;
    } else {
      lbv = lbm;
      ubv = ubu;
    }
    lbv = warp_min(lbv);
    ubv = warp_min(ubv);
    ubc = warp_min(ubc);
    if (FULL) midv = warp_min(midv);
    if (lane == 0) {
      const T eps = T(tl.eps);
      T lb = lbv < INF ? sub_rd(lbv, eps) : INF;
      lb = max(lb, T(0));
      T ub = ubv < INF ? add_ru(ubv, eps) : INF;
      ub = min(ub, ubc);
      using Bt = Bits<T>;
      if (lb < INF) atomicMin(&((typename Bt::U*)a.lb)[tl.pair], Bt::enc(lb));
      if (ub < INF) atomicMin(&((typename Bt::U*)a.ub)[tl.pair], Bt::enc(ub));
      if (FULL && midv < INF) atomicMin(&((typename Bt::U*)a.mid)[tl.pair], Bt::enc(midv));
      if (a.early && ub <= a.thr[tl.pair]) a.flag[tl.pair] = 1;
    }
    __syncwarp();
    cur = nxt;
    b ^= 1;
  }
  ntest = warp_sum_u64(ntest);
  if (lane == 0 && ntest) atomicAdd(a.ntests, ntest);
  nskip = warp_sum_u64(nskip);
  if (lane == 0 && nskip && a.nculled) atomicAdd(a.nculled, nskip);
}

template <class T, bool FULL>
__global__ void __launch_bounds__(256) k_cross_fix(RefineArgs a) {
  const unsigned n = min(*a.qcount, a.qcap);
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int4 e = a.queue[k];
    const int pair = e.x;
    const float eps = __int_as_float(e.w);
    const float4 o4 = a.origin[pair];
    const float4* fr = a.facR + 3LL * e.y;
    const float4* fs = a.facS + 3LL * e.z;
    float4 r0 = fr[0], r1 = fr[1], r2 = fr[2], s0 = fs[0], s1 = fs[1], s2 = fs[2];
    T va[3], vb[3], vc[3], wa[3], wb[3], wc[3];
    translate(r0, o4, va);
    translate(r1, o4, vb);
    translate(r2, o4, vc);
    translate(s0, o4, wa);
    translate(s1, o4, wb);
    translate(s2, o4, wc);
    typename RecOf<T>::R P, Q;
    make_rec(P, va, vb, vc, T(r0.w), T(r1.w), true);
    make_rec(Q, wa, wb, wc, T(s0.w), T(s1.w), false);
    bool maybe;
    T d2 = tri_d2(P, Q, T(0), maybe);
    float4 rr[3] = {r0, r1, r2}, ss[3] = {s0, s1, s2};
    const bool cert = cross_decide(rr, ss, o4);
    const T phs = add_ru(P.ph, Q.ph), hds = add_ru(P.hd, Q.hd);
    T lb, ub, mid;
    if (cert) {
      lb = -phs;
      ub = hds;
      mid = T(0);
    } else {
      T d = FULL ? sqrt_rn(d2) : sqrt_test(d2);
      lb = sub_rd(sub_rd(d, phs), T(eps));
      ub = add_ru(add_ru(d, hds), T(eps));
      mid = d;
    }
    lb = max(lb, T(0));
    using B = Bits<T>;
    atomicMin(&((typename B::U*)a.lb)[pair], B::enc(lb));
    atomicMin(&((typename B::U*)a.ub)[pair], B::enc(ub));
    if (FULL) atomicMin(&((typename B::U*)a.mid)[pair], B::enc(mid));
  }
}

// The last refine_tail units per resident warp are split refine_split ways.
static void set_split(const pj_ctx* ctx, RefineArgs& args, int64_t resident_warps) {
  args.split_k = ctx->refine_split;
  args.split_tail = ctx->refine_split > 1 ? (int64_t)ctx->refine_tail * resident_warps : 0;
}

template <class T, bool FULL>
static void launch_refine(pj_ctx* ctx, RefineArgs& args, int64_t n_tiles, cudaStream_t st) {
  auto kern = k_refine<T, FULL>;
  const size_t smem = refine_smem_bytes<T>();
  PJ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the stages of a 12-warp CTA need most of the shared memory
  PJ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int occ = 0;
  constexpr int threads = kref_warps<T>() * 32;
  PJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
  if (occ < 1) occ = 1;
  if (ctx->ctas_per_sm > 0) occ = std::min(occ, ctx->ctas_per_sm);
  int64_t grid = (int64_t)occ * ctx->sm_count;
  set_split(ctx, args, grid * kref_warps<T>());
  // few units: one CTA per unit up to the resident limit, so that they
  // spread over the SMs (units are dealt CTA-minor)
  if (n_tiles >= 0) grid = std::min<int64_t>(unit_space(n_tiles, args.split_k, args.split_tail).NV, grid);
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, threads, smem, st>>>(args);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  if (args.qcap > 0) {
    k_cross_fix<T, FULL><<<ctx->sm_count * 4, 256, 0, st>>>(args);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
}

template <bool FULL>
static void launch_refine2(pj_ctx* ctx, RefineArgs& args, int64_t n_tiles, cudaStream_t st) {
  auto kern = k_refine2<FULL>;
  const size_t smem = refine_smem_bytes2();
  PJ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  PJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, REFINE_THREADS, smem));
  if (occ < 1) occ = 1;
  if (ctx->ctas_per_sm > 0) occ = std::min(occ, ctx->ctas_per_sm);
  int64_t grid = (int64_t)occ * ctx->sm_count;
  set_split(ctx, args, grid * REFINE_WARPS);
  if (n_tiles >= 0) grid = std::min<int64_t>(unit_space(n_tiles, args.split_k, args.split_tail).NV, grid);
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, REFINE_THREADS, smem, st>>>(args);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  if (args.qcap > 0) {
    k_cross_fix<float, FULL><<<ctx->sm_count * 4, 256, 0, st>>>(args);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
}

// FP64 steps use k_refine<double>; FP32 steps the scalar kernel (variant 1,
// default) or the packed one (variant 2), chosen per context or autotuned.
static void dispatch_refine(pj_ctx* ctx, RefineArgs& a, int64_t n_tiles, const StepSpec& sp, cudaStream_t st) {
  if (sp.fp64) {
    if (sp.full) launch_refine<double, true>(ctx, a, n_tiles, st);
    else launch_refine<double, false>(ctx, a, n_tiles, st);
  } else if (ctx->refine_variant == 1) {
    if (sp.full) launch_refine<float, true>(ctx, a, n_tiles, st);
    else launch_refine<float, false>(ctx, a, n_tiles, st);
  } else {
    if (sp.full) launch_refine2<true>(ctx, a, n_tiles, st);
    else launch_refine2<false>(ctx, a, n_tiles, st);
  }
}

static void launch_masks(pj_ctx* ctx, const MaskArgs& m, int64_t n_tiles, bool fp64, cudaStream_t st) {
  int64_t grid = (int64_t)ctx->sm_count * 8;
  if (n_tiles >= 0) grid = std::max<int64_t>(1, std::min<int64_t>(grid, (n_tiles + 7) / 8));
  if (fp64) k_unit_masks<double><<<(unsigned)grid, 256, 0, st>>>(m);
  else k_unit_masks<float><<<(unsigned)grid, 256, 0, st>>>(m);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

float refine_ms(pj_ctx* ctx, int ev) {
  if (ev < 0) return 0.f;
  float ms = 0.f;
  PJ_CK(cudaEventElapsedTime(&ms, ctx->ev[ev], ctx->ev[ev + 1]));
  return ms;
}

int run_refine(pj_ctx* ctx, const pj_set* R, const pj_set* S, UnitCount units, const StepSpec& sp,
               cudaStream_t st) {
  const int64_t n_tiles = units.count;
  if (n_tiles == 0) return -1;
  int ev = -1;
  // no timing events inside a captured graph (a replay is timed as a whole)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  PJ_CK(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusNone && ctx->ev_used + 2 <= 60 && ctx->ev[ctx->ev_used]) {
    ev = ctx->ev_used;
    ctx->ev_used += 2;
  }
  RefineArgs a;
  a.tiles = (const Tile*)ctx->ws[WS_TILES].p;
  a.n_tiles = n_tiles;
  a.n_tiles_dev = n_tiles < 0 ? units.dev : nullptr;
  a.counter = (int*)(ctx->d_counters + 15);
  PJ_CK(cudaMemsetAsync(a.counter, 0, sizeof(int), st));
  a.facR = R->lod[sp.lodR].fac;
  a.facS = S->lod[sp.lodS].fac;
  a.origin = (const float4*)ctx->ws[WS_ORIGIN].p;
  a.thr = (const float*)ctx->ws[WS_THR].p;
  a.ub_prev = (const double*)ctx->ws[WS_DHI].p;
  a.lb = ctx->ws[WS_LB].p;
  a.ub = ctx->ws[WS_UB].p;
  a.mid = ctx->ws[WS_MID].p;
  a.ntests = ctx->d_counters + (sp.fp64 ? 1 : 0);
  a.nculled = ctx->d_counters + 5;
  a.nneeded = ctx->d_counters + 6;
  a.err = ctx->d_err;
  a.qcap = CROSS_QUEUE_CAP;
  a.queue = (int4*)ws_get(ctx, WS_MISC2, (size_t)a.qcap * sizeof(int4), st);
  a.qcount = (unsigned*)(ctx->d_counters + 14);
  PJ_CK(cudaMemsetAsync(a.qcount, 0, sizeof(unsigned), st));
  a.flag = (uint8_t*)ctx->ws[WS_FLAG].p;
  a.early = sp.early ? 1 : 0;
  a.exact_cross = sp.exact_cross ? 1 : 0;
  a.cull = sp.cull ? 1 : 0;
  a.masked = 0;
  if (ev >= 0) PJ_CK(cudaEventRecord(ctx->ev[ev], st));
  int64_t n_run = n_tiles;
  if (sp.full && (!sp.fp64 || sp.cull)) {
    // full resolution with facet balls: per-unit s masks first, the units
    // that need nothing dropped (timed with the refinement)
    Tile* out = (Tile*)ws_get(ctx, WS_TILES2, std::max<size_t>(ctx->ws[WS_TILES].cap, sizeof(Tile)), st);
    int64_t* n_out = (int64_t*)(ctx->d_counters + 13);
    PJ_CK(cudaMemsetAsync(n_out, 0, sizeof(int64_t), st));
    MaskArgs m{(Tile*)ctx->ws[WS_TILES].p, a.n_tiles, a.n_tiles_dev, a.facR, a.facS, a.origin, a.thr, a.ub_prev,
               a.cull, out, n_out, a.nculled};
    launch_masks(ctx, m, n_tiles, sp.fp64, st);
    a.tiles = out;
    a.n_tiles = -1;
    a.n_tiles_dev = n_out;
    a.masked = 1;
    n_run = -1;
  }
  dispatch_refine(ctx, a, n_run, sp, st);
  if (ev >= 0) PJ_CK(cudaEventRecord(ctx->ev[ev + 1], st));
  return ev;
}

// ------------------------------------------------------------------ explicit buffers

void setup_pairs_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const PairBufs& b,
                      cudaStream_t st) {
  if (n == 0) return;
  int th = 256;
  k_setup_pairs<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, b.pr, b.ps, R->mbb, S->mbb, R->anchor, S->anchor,
                                                              0.0, 0, b.origin, b.thr, b.box_lb, b.anc_ub, b.status,
                                                              b.lod0, b.exact, b.dlo, b.dhi, b.d, nullptr);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

UnitCount build_tiles_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                           const PairBufs& b, int64_t tiles_cap, cudaStream_t st) {
  if (n == 0) return UnitCount{0, nullptr};
  Tile* tiles = b.tiles;
  return build_units(ctx, R, S, n, sp, b.pr, b.ps, b.status, b.lod0, b.origin, b.thr, b.tcount, b.toff, b.ucount,
                     &tiles, tiles_cap, false, b.scan_tmp, b.err, st);
}

void init_bounds_bufs(pj_ctx* ctx, int64_t n, const StepSpec& sp, const PairBufs& b, cudaStream_t st) {
  if (n == 0) return;
  int th = 256;
  k_init_bounds<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, b.status, b.lod0, sp.want, sp.step, sp.fp64, b.lb,
                                                               b.ub, b.mid, b.flag);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

void run_refine_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, UnitCount units, const StepSpec& sp,
                     const PairBufs& b, int* err, cudaStream_t st) {
  const int64_t n_tiles = units.count;
  if (n_tiles == 0) return;
  RefineArgs a;
  a.tiles = b.tiles;
  a.n_tiles = n_tiles;
  a.n_tiles_dev = n_tiles < 0 ? units.dev : nullptr;
  a.counter = (int*)(b.counters + 1);
  PJ_CK(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st));
  a.facR = R->lod[sp.lodR].fac;
  a.facS = S->lod[sp.lodS].fac;
  a.origin = b.origin;
  a.thr = b.thr;
  a.ub_prev = b.dhi;
  a.lb = b.lb;
  a.ub = b.ub;
  a.mid = b.mid;
  a.ntests = b.counters;
  a.nculled = nullptr;
  a.nneeded = nullptr;
  a.err = err;
  a.queue = b.queue;
  a.qcap = b.qcap;
  a.qcount = (unsigned*)(b.counters + 2);
  PJ_CK(cudaMemsetAsync(a.qcount, 0, sizeof(unsigned), st));
  a.flag = b.flag;
  a.early = 0;
  a.exact_cross = sp.exact_cross ? 1 : 0;
  a.cull = sp.cull ? 1 : 0;
  a.masked = 0;
  if (sp.full && (!sp.fp64 || sp.cull)) {
    // per-unit s masks in place (no buffer to compact into)
    MaskArgs m{b.tiles, a.n_tiles, a.n_tiles_dev, a.facR, a.facS, a.origin, a.thr, a.ub_prev, a.cull, nullptr,
               nullptr, nullptr};
    launch_masks(ctx, m, n_tiles, sp.fp64, st);
    a.masked = 1;
  }
  dispatch_refine(ctx, a, n_tiles, sp, st);
}

// ------------------------------------------------------------------ batch

template <class T>
__global__ void k_tri_dist(const float* P, const float* Q, int64_t n, double* out, double* err) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float* a = P + 9 * p;
  const float* b = Q + 9 * p;
  // local frame: centre of P's box
  float o[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float lo = fminf(a[k], fminf(a[3 + k], a[6 + k])), hi = fmaxf(a[k], fmaxf(a[3 + k], a[6 + k]));
    o[k] = 0.5f * (lo + hi);
  }
  T pv[3][3], qv[3][3];
  float rho = 0.f, L = 0.f;
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      pv[v][k] = T(a[3 * v + k]) - T(o[k]);
      qv[v][k] = T(b[3 * v + k]) - T(o[k]);
      rho = fmaxf(rho, fmaxf(fabsf(a[3 * v + k] - o[k]), fabsf(b[3 * v + k] - o[k])));
    }
  typename RecOf<T>::R RP, RQ;
  make_rec(RP, pv[0], pv[1], pv[2], T(0), T(0), true);
  make_rec(RQ, qv[0], qv[1], qv[2], T(0), T(0), false);
#pragma unroll
  for (int i = 0; i < 3; ++i) L = fmaxf(L, fmaxf(sqrtf(float(RP.ee[i])), sqrtf(float(RQ.ee[i]))));
  float smin = fminf(float(facet_sin(pv[0], pv[1], pv[2])), float(facet_sin(qv[0], qv[1], qv[2])));
  Margins m = fp32_margins(rho * 1.0001f + 1e-30f, L, smin);
  T eh = sizeof(T) == 8 ? T(0) : T(m.eh), ew = sizeof(T) == 8 ? T(0) : T(m.ew);
  bool maybe;
  T d2 = tri_d2(RP, RQ, eh, maybe);
  float4 fp[3] = {make_float4(a[0], a[1], a[2], 0.f), make_float4(a[3], a[4], a[5], 0.f),
                  make_float4(a[6], a[7], a[8], 0.f)};
  float4 fq[3] = {make_float4(b[0], b[1], b[2], 0.f), make_float4(b[3], b[4], b[5], 0.f),
                  make_float4(b[6], b[7], b[8], 0.f)};
  const bool cert = maybe && cross_decide(fp, fq, make_float4(o[0], o[1], o[2], 0.f));
  (void)ew;
  T d = sqrt_rn(d2);
  out[p] = cert ? 0.0 : double(d);
  if (err) err[p] = (cert || sizeof(T) == 8) ? 0.0 : (double)m.eps;
}

void tri_dist_batch(pj_ctx* ctx, const float* P, const float* Q, int64_t n, bool fp64, double* out, double* err,
                    cudaStream_t st) {
  (void)ctx;
  if (n == 0) return;
  int th = 128;
  unsigned g = (unsigned)((n + th - 1) / th);
  if (fp64) k_tri_dist<double><<<g, th, 0, st>>>(P, Q, n, out, err);
  else k_tri_dist<float><<<g, th, 0, st>>>(P, Q, n, out, err);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

}  // namespace pj
