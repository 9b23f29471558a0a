// Facet-level refinement (section 3.3, Algorithm 4 and Eq. 1 / Eq. 2),
// re-designed for sm_103a:
//  * unit = one 32-facet block of r x one 32-facet block of s of one
//    candidate pair at one LoD (replaces the paper's thread block per voxel
//    pair); units are built on the device (k_emit_units, a warp per pair) and
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

#include "refine_kern.cuh"

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
// one candidate pair at one LoD.  The builder takes one warp per selected
// pair and walks the box hierarchy: the lanes test the pair's (256-facet r
// chunk, 256-facet s chunk) box pairs, and for each live chunk pair the
// warp tests its (up to 8 x 8) block pairs; a box pair whose distance minus
// the Hausdorff terms exceeds the pair's threshold is skipped
// (PJ_TILE_PRUNE; without it every block pair is a unit).  A block box lies
// inside its chunk's box and the chunk's Hausdorff and shape terms bound the
// block's, so the chunk test only ever skips block pairs the block test
// would skip: the units are exactly the live block pairs.  The live units of
// 32 block-pair tests are appended with one atomic add.

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


// EMIT = false: only count the live units into *ucount (zeroed by the
// caller); EMIT = true: also write them (at most cap; more sets
// ERR_CAPACITY and drops the excess).  The pair loop, the chunk loop and
// the block loop are warp-uniform, so the ballots are over full warps.
template <bool EMIT>
__global__ void __launch_bounds__(256, 4) k_emit_units(int64_t n, const int32_t* pr, const int32_t* ps,
                                                    const uint8_t* status, const uint8_t* lod0, uint8_t want,
                                                    int step, BoxView R, BoxView S, const float4* origin,
                                                    const float* thr, int cull, int fp64, Tile* tiles, int64_t cap,
                                                    int64_t* ucount, int* err) {
  constexpr int SB = CHUNK / BLK;   // blocks per chunk
  constexpr unsigned FULLW = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += nw) {
    // the selection and the ids are loaded together (the ids do not wait
    // for the selection), then the per-object offsets in one more round
    const uint8_t stv = status[p], l0v = lod0[p];
    const int r = pr[p], s = ps[p];
    if (!(stv == want && l0v <= step)) continue;
    const float4 o = origin[p];
    const float t = thr[p];
    // facet, block and chunk indices are below 2^31 (a LoD holds fewer facets)
    const int rc0 = (int)R.coff[r], nrc = (int)R.coff[r + 1] - rc0;
    const int sc0 = (int)S.coff[s], nsc = (int)S.coff[s + 1] - sc0;
    const int rb0 = (int)R.boff[r], nrbo = (int)R.boff[r + 1] - rb0;
    const int sbase = (int)S.boff[s], nsbo = (int)S.boff[s + 1] - sbase;
    const int64_t items = (int64_t)nrc * nsc;   // chunk pairs
    for (int64_t i0 = 0; i0 < items; i0 += 32) {
      const int64_t i = i0 + lane;
      int rc = 0, sc = 0;   // chunk indices within the objects
      bool live = false;
      if (i < items) {
        rc = (int)(i / nsc);
        sc = (int)(i - (int64_t)rc * nsc);
        live = true;
        if (cull) {
          const float4* ca = R.chunk + 3 * (int64_t)(rc0 + rc);
          const float4* cb = S.chunk + 3 * (int64_t)(sc0 + sc);
          live = box_pair_live(ca, cb, t, fp64 ? 0.f : box_margins(ca, cb, o).eps);
        }
      }
      unsigned lm = __ballot_sync(FULLW, live);
      while (lm) {
        const int src = __ffs(lm) - 1;
        lm &= lm - 1;
        const int crc = __shfl_sync(FULLW, rc, src), csc = __shfl_sync(FULLW, sc, src);
        const int nrb = min(SB, nrbo - crc * SB), nsb = min(SB, nsbo - csc * SB);
        const int nbp = nrb * nsb;   // <= 64 block pairs
        for (int j0 = 0; j0 < nbp; j0 += 32) {
          const int j = j0 + lane;
          bool ul = false;
          float eps = 0.f, eh = 0.f;
          int jr = 0, js = 0;
          if (j < nbp) {
            jr = crc * SB + j / nsb;   // block indices within the objects
            js = csc * SB + j % nsb;
            const float4* ba = R.blk + 3 * (int64_t)(rb0 + jr);
            const float4* bb = S.blk + 3 * (int64_t)(sbase + js);
            Margins m = box_margins(ba, bb, o);
            if (fp64) {   // exact distances, but the straddle margin of the heights
              m.eh = fp64_height_margin(m);
              m.eps = 0.f;
            }
            ul = !cull || box_pair_live(ba, bb, t, m.eps);
            eps = m.eps;
            eh = m.eh;
          }
          const unsigned um = __ballot_sync(FULLW, ul);
          if (um == 0u) continue;
          unsigned long long base = 0;
          if (lane == 0)
            base = atomicAdd(reinterpret_cast<unsigned long long*>(ucount), (unsigned long long)__popc(um));
          base = __shfl_sync(FULLW, base, 0);
          if (EMIT && ul) {
            const int64_t pos = (int64_t)base + __popc(um & below);
            if (pos < cap) {
              const int fr0 = (int)R.foff[r], fs0 = (int)S.foff[s];
              const int fr = fr0 + jr * BLK, fs = fs0 + js * BLK;
              Tile tl;
              tl.pair = (int32_t)p;
              tl.rb = fr;
              tl.sb = fs;
              tl.rl = (uint16_t)min(BLK, (int)R.foff[r + 1] - fr);
              tl.sl = (uint16_t)min(BLK, (int)S.foff[s + 1] - fs);
              tl.eps = eps;
              tl.eh = eh;
              tl.ew = 0.f;
              tl.pad = 0;
              tiles[pos] = tl;
            } else {
              set_err(err, ERR_CAPACITY);
            }
          }
        }
      }
    }
  }
}

static BoxView box_view(const LodData& L) { return BoxView{L.chunk, L.coff, L.blk, L.boff, L.foff}; }


static UnitCount build_units(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                             const int32_t* pr, const int32_t* ps, const uint8_t* status, const uint8_t* lod0,
                             const float4* origin, const float* thr, int64_t* ucount, Tile** tiles_io,
                             int64_t tiles_cap, bool grow, int* err, cudaStream_t st) {
  const LodData& LR = R->lod[sp.lodR];
  const LodData& LS = S->lod[sp.lodS];
  BoxView vr = box_view(LR), vs = box_view(LS);
  const int th = 256;
  // a LoD built on demand: lay out the objects this step needs first (the
  // FP64 re-decide refines pairs that the full-resolution step before it
  // refined, so their objects are laid out already)
  if (sp.want != REDECIDE) ensure_lod(ctx, R, sp.lodR, n, pr, status, lod0, sp.want, sp.step, st);
  PJ_CK(cudaMemsetAsync(ucount, 0, 8, st));
  // one warp per pair; one wave of 4 blocks of 8 warps per SM (the
  // kernel's register bound) walks the pairs
  const unsigned g = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n + th / 32 - 1) / (th / 32), (int64_t)ctx->sm_count * 4));
  const int64_t bR = (LR.maxF + BLK - 1) / BLK, bS = (LS.maxF + BLK - 1) / BLK;
  const int64_t worst = n * bR * bS;
  UnitCount uc{-1, ucount};
  int64_t cap = tiles_cap;
  if (worst <= tiles_cap || (grow && (size_t)worst * sizeof(Tile) <= ctx->unit_budget)) {
    if (worst > tiles_cap) {
      *tiles_io = (Tile*)ws_get(ctx, WS_TILES, worst * sizeof(Tile), st);
      cap = worst;
    }
  } else if (grow && sp.rerun_ok && ctx->trial_unit_cap == 0) {
    // the worst case does not fit: emit into the buffer as it is (at least
    // the budget); an overflow is flagged, the join records the count it
    // needed, grows the buffer and runs again (so after the first joins of
    // a workload no step pays for a counting pass and a synchronization)
    const int64_t floor_units = (int64_t)(ctx->unit_budget / sizeof(Tile));
    if (tiles_cap < floor_units) {
      *tiles_io = (Tile*)ws_get(ctx, WS_TILES, floor_units * sizeof(Tile), st);
      cap = floor_units;
    }
  } else {
    // the worst case does not fit: count first, then size the buffer
    k_emit_units<false><<<g, th, 0, st>>>(n, pr, ps, status, lod0, sp.want, sp.step, vr, vs, origin, thr, sp.cull,
                                          sp.fp64, nullptr, 0, ucount, err);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    int64_t total = 0;
    PJ_CK(cudaMemcpyAsync(&total, ucount, 8, cudaMemcpyDeviceToHost, st));
    PJ_CK(cudaStreamSynchronize(st));
    uc.count = total;
    if (total == 0) return uc;
    if (ctx->trial_unit_cap > 0 && total > ctx->trial_unit_cap) throw TrialTooLarge{total};
    if (total > tiles_cap) {
      if (!grow) throw ApiError{PJ_EINVAL, "refinement units above the scratch capacity"};
      *tiles_io = (Tile*)ws_get(ctx, WS_TILES, total * sizeof(Tile), st);
      cap = total;
    }
    PJ_CK(cudaMemsetAsync(ucount, 0, 8, st));
  }
  k_emit_units<true><<<g, th, 0, st>>>(n, pr, ps, status, lod0, sp.want, sp.step, vr, vs, origin, thr, sp.cull,
                                       sp.fp64, *tiles_io, cap, ucount, err);
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
  auto ucount = (int64_t*)ws_get(ctx, WS_MISC4, 64, st);
  Tile* tiles = (Tile*)ctx->ws[WS_TILES].p;
  const int64_t cap = (int64_t)(ctx->ws[WS_TILES].cap / sizeof(Tile));
  return build_units(ctx, R, S, n, sp, pr, ps, status, lod0, origin, thr, ucount, &tiles, cap, true, ctx->d_err,
                     st);
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
  int64_t tiles_cap;               // units the tile array holds
  unsigned long long* units_max;   // largest device unit count seen (may be null)
};

template <class T>
__global__ void __launch_bounds__(256) k_unit_masks(MaskArgs m) {
  using T4 = typename std::conditional<sizeof(T) == 4, float4, double4>::type;
  __shared__ T4 sball[8][32];   // per warp: the s facets' balls (centre, radius)
  const int lane = threadIdx.x & 31;
  T4* sb = sball[threadIdx.x >> 5];
  const unsigned FULLM = 0xffffffffu;
  const int64_t NT = launch_units(m.n_tiles_dev, m.n_tiles, m.tiles_cap, m.units_max);
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


// FP64 steps use k_refine<double>; FP32 steps the scalar kernel (variant 1,
// default) or the packed one (variant 2), chosen per context or autotuned.
static void dispatch_refine(pj_ctx* ctx, RefineArgs& a, int64_t n_tiles, const StepSpec& sp, cudaStream_t st) {
  if (sp.fp64) launch_refine_f64(ctx, a, n_tiles, sp.full, st);
  else launch_refine_f32(ctx, a, n_tiles, sp.full, ctx->refine_variant, st);
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
  a.tiles_cap = (int64_t)(ctx->ws[WS_TILES].cap / sizeof(Tile));
  a.units_max = ctx->d_counters + CNT_UNITS_MAX;
  if (ev >= 0) PJ_CK(cudaEventRecord(ctx->ev[ev], st));
  int64_t n_run = n_tiles;
  if (sp.full && (!sp.fp64 || sp.cull)) {
    // full resolution with facet balls: per-unit s masks first, the units
    // that need nothing dropped (timed with the refinement)
    Tile* out = (Tile*)ws_get(ctx, WS_TILES2, std::max<size_t>(ctx->ws[WS_TILES].cap, sizeof(Tile)), st);
    int64_t* n_out = (int64_t*)(ctx->d_counters + 13);
    PJ_CK(cudaMemsetAsync(n_out, 0, sizeof(int64_t), st));
    MaskArgs m{(Tile*)ctx->ws[WS_TILES].p, a.n_tiles, a.n_tiles_dev, a.facR, a.facS, a.origin, a.thr, a.ub_prev,
               a.cull, out, n_out, a.nculled, a.tiles_cap, a.units_max};
    launch_masks(ctx, m, n_tiles, sp.fp64, st);
    a.tiles = out;
    a.n_tiles = -1;
    a.n_tiles_dev = n_out;
    a.masked = 1;
    a.tiles_cap = (int64_t)(ctx->ws[WS_TILES2].cap / sizeof(Tile));
    n_run = -1;
  }
  dispatch_refine(ctx, a, n_run, sp, st);
  if (ev >= 0) PJ_CK(cudaEventRecord(ctx->ev[ev + 1], st));
  return ev;
}

// After a join's final synchronization: was a unit buffer too small?  Then
// the join's results are void; UnitsOverflow asks for a rerun with the
// buffer grown to the largest count a step needed.
void check_units(pj_ctx* ctx, int herr) {
  if (!(herr & ERR_CAPACITY)) return;
  unsigned long long need = 0;
  PJ_CK(cudaMemcpy(&need, ctx->d_counters + CNT_UNITS_MAX, sizeof need, cudaMemcpyDeviceToHost));
  const int64_t have = (int64_t)(ctx->ws[WS_TILES].cap / sizeof(Tile));
  if ((int64_t)need <= have) throw ApiError{PJ_ENOMEM, "refinement units above the unit buffer"};
  throw UnitsOverflow{(int64_t)need};
}

void grow_units(pj_ctx* ctx, int64_t units, cudaStream_t st) {
  const int64_t want = units + units / 4 + 1024;
  PJ_CK(cudaStreamSynchronize(st));
  ws_get(ctx, WS_TILES, (size_t)want * sizeof(Tile), st);
  ws_get(ctx, WS_TILES2, (size_t)want * sizeof(Tile), st);
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
  return build_units(ctx, R, S, n, sp, b.pr, b.ps, b.status, b.lod0, b.origin, b.thr, b.ucount, &tiles, tiles_cap,
                     false, b.err, st);
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
  a.tiles_cap = b.tiles_cap;
  a.units_max = nullptr;
  if (sp.full && (!sp.fp64 || sp.cull)) {
    // per-unit s masks in place (no buffer to compact into)
    MaskArgs m{b.tiles, a.n_tiles, a.n_tiles_dev, a.facR, a.facS, a.origin, a.thr, a.ub_prev, a.cull, nullptr,
               nullptr, nullptr, b.tiles_cap, nullptr};
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
  const T eh = sizeof(T) == 8 ? T(fp64_height_margin(m)) : T(m.eh);
  bool maybe;
  T d2 = tri_d2(RP, RQ, eh, maybe);
  float4 fp[3] = {make_float4(a[0], a[1], a[2], 0.f), make_float4(a[3], a[4], a[5], 0.f),
                  make_float4(a[6], a[7], a[8], 0.f)};
  float4 fq[3] = {make_float4(b[0], b[1], b[2], 0.f), make_float4(b[3], b[4], b[5], 0.f),
                  make_float4(b[6], b[7], b[8], 0.f)};
  const bool cert = maybe && !boxes_apart(RP, RQ) && cross_decide(fp, fq);
  T d = d2 > T(0) ? sqrt_rn(d2) : tiny_(T(0));
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
