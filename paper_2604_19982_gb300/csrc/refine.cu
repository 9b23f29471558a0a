// Facet-level refinement (section 3.3, Algorithm 4 and Eq. 1 / Eq. 2),
// re-designed for sm_103a:
//  * work unit = tile: one 256-facet chunk of r x one 256-facet chunk of s of
//    one candidate pair at one LoD (replaces the paper's block per voxel
//    pair); tiles are built on the device and consumed by a persistent
//    kernel through an atomic counter (one launch per LoD step);
//  * the s chunk is staged into shared memory with a TMA bulk copy
//    (cp.async.bulk, mbarrier completion, bounded wait), then expanded once
//    into per-facet records; r facets live in registers (one per thread,
//    several s stripes when the r chunk is short), s records are read by
//    warp-wide broadcast;
//  * per-thread running minima, warp-shuffle + one shared word per warp,
//    then one atomicMin per tile and pair on the order-preserving bits
//    (replaces the block-wide Hillis-Steele scan of section 2.2);
//  * optional pruning (PJ_TILE_PRUNE): chunk pairs and 32-facet blocks whose
//    box distance minus the Hausdorff terms exceeds the pair's threshold are
//    skipped; they cannot change the decision (see build_tiles).
#include <algorithm>
#include <stdexcept>

#include "internal.h"
#include "tritri.cuh"

namespace pj {

// ------------------------------------------------------------------ setup

__global__ void k_setup_pairs(int64_t n, const int32_t* pr, const int32_t* ps, const float* mbbR,
                              const float* mbbS, const float* ancR, const float* ancS, double tau, int within,
                              float4* origin, float* thr, double* box_lb, double* anc_ub, uint8_t* status,
                              uint8_t* lod0, uint8_t* exact, double* dlo, double* dhi, double* d) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
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
                 cudaStream_t st) {
  if (n == 0) return;
  auto pr = (int32_t*)ws_get(ctx, WS_PR, n * 4, st);
  auto ps = (int32_t*)ws_get(ctx, WS_PS, n * 4, st);
  auto origin = (float4*)ws_get(ctx, WS_ORIGIN, n * 16, st);
  auto thr = (float*)ws_get(ctx, WS_THR, n * 4, st);
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
                                                              status, lod0, exact, dlo, dhi, d);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// ------------------------------------------------------------------ tiles

struct ChunkView {
  const float4* chunk;   // [3C]
  const int64_t* coff;   // [n+1]
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

// Margins of a chunk pair in the pair-local frame.
__device__ __forceinline__ Margins chunk_margins(const float4* cr, const float4* cs, float4 o) {
  float rho = fmaxf(absmax_rel(cr[0], cr[1], o), absmax_rel(cs[0], cs[1], o));
  rho = rho * 1.0001f + 1e-30f;
  float L = fmaxf(cr[2].x, cs[2].x);
  float smin = fminf(cr[2].y, cs[2].y);
  return fp32_margins(rho, L, smin);
}

// Can a facet pair of these two chunks reach the threshold?  Every facet
// pair has true distance >= box gap; the single-precision lower bound adds
// at most 2 eps of error; Eq. 2 subtracts at most max ph of each side.
__device__ __forceinline__ bool chunk_pair_live(const float4* cr, const float4* cs, float thr, float eps) {
  float g = box_gap_rd(cr[0], cr[1], cs[0], cs[1]);
  float lb = __fsub_rd(__fsub_rd(__fsub_rd(g, cr[1].w), cs[1].w), 2.f * eps);
  return !(lb > thr);
}

__global__ void k_count_tiles(int64_t n, const int32_t* pr, const int32_t* ps, const uint8_t* status,
                              const uint8_t* lod0, uint8_t want, int step, ChunkView R, ChunkView S,
                              const float4* origin, const float* thr, int cull, int fp64, int64_t* count) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t c = 0;
  if (status[p] == want && lod0[p] <= step) {
    const int r = pr[p], s = ps[p];
    int64_t r0 = R.coff[r], r1 = R.coff[r + 1], s0 = S.coff[s], s1 = S.coff[s + 1];
    if (!cull) {
      c = (r1 - r0) * (s1 - s0);
    } else {
      const float4 o = origin[p];
      const float t = thr[p];
      for (int64_t a = r0; a < r1; ++a)
        for (int64_t b = s0; b < s1; ++b) {
          const float4* ca = R.chunk + 3 * a;
          const float4* cb = S.chunk + 3 * b;
          float eps = fp64 ? 0.f : chunk_margins(ca, cb, o).eps;
          c += chunk_pair_live(ca, cb, t, eps);
        }
    }
  }
  count[p] = c;
}

__global__ void k_emit_tiles(int64_t n, const int32_t* pr, const int32_t* ps, const uint8_t* status,
                             const uint8_t* lod0, uint8_t want, int step, ChunkView R, ChunkView S,
                             const float4* origin, const float* thr, int cull, int fp64, const int64_t* off,
                             Tile* tiles) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (!(status[p] == want && lod0[p] <= step)) return;
  const int r = pr[p], s = ps[p];
  const int64_t r0 = R.coff[r], r1 = R.coff[r + 1], s0 = S.coff[s], s1 = S.coff[s + 1];
  const int64_t fr0 = R.foff[r], fr1 = R.foff[r + 1], fs0 = S.foff[s], fs1 = S.foff[s + 1];
  const float4 o = origin[p];
  const float t = thr[p];
  int64_t w = off[p];
  for (int64_t a = r0; a < r1; ++a)
    for (int64_t b = s0; b < s1; ++b) {
      const float4* ca = R.chunk + 3 * a;
      const float4* cb = S.chunk + 3 * b;
      Margins m = chunk_margins(ca, cb, o);
      if (fp64) m.eps = m.eh = m.ew = 0.f;
      if (cull && !chunk_pair_live(ca, cb, t, m.eps)) continue;
      Tile tl;
      int64_t rb = fr0 + (a - r0) * CHUNK, sb = fs0 + (b - s0) * CHUNK;
      tl.pair = (int32_t)p;
      tl.rb = (int32_t)rb;
      tl.sb = (int32_t)sb;
      tl.rl = (uint16_t)(fr1 - rb < CHUNK ? fr1 - rb : CHUNK);
      tl.sl = (uint16_t)(fs1 - sb < CHUNK ? fs1 - sb : CHUNK);
      tl.eps = m.eps;
      tl.eh = m.eh;
      tl.ew = m.ew;
      tl.pad = 0;
      tiles[w++] = tl;
    }
}

int64_t build_tiles(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                    cudaStream_t st) {
  if (n == 0) return 0;
  auto pr = (int32_t*)ws_get(ctx, WS_PR, n * 4, st);
  auto ps = (int32_t*)ws_get(ctx, WS_PS, n * 4, st);
  auto status = (uint8_t*)ws_get(ctx, WS_STATUS, n, st);
  auto lod0 = (uint8_t*)ws_get(ctx, WS_LOD0, n, st);
  auto origin = (float4*)ws_get(ctx, WS_ORIGIN, n * 16, st);
  auto thr = (float*)ws_get(ctx, WS_THR, n * 4, st);
  auto cnt = (int64_t*)ws_get(ctx, WS_TCOUNT, (n + 1) * 8, st);
  auto off = (int64_t*)ws_get(ctx, WS_SCAN, (n + 1) * 8, st);
  const LodData& LR = R->lod[sp.lodR];
  const LodData& LS = S->lod[sp.lodS];
  ChunkView cr{LR.chunk, LR.coff, LR.foff}, cs{LS.chunk, LS.coff, LS.foff};
  int th = 128;
  unsigned g = (unsigned)((n + th - 1) / th);
  k_count_tiles<<<g, th, 0, st>>>(n, pr, ps, status, lod0, sp.want, sp.step, cr, cs, origin, thr, sp.cull,
                                   sp.fp64, cnt);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, cnt, off, n, st);
  int64_t total = 0;
  PJ_CK(cudaMemcpyAsync(&total, off + n, 8, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  if (total == 0) return 0;
  auto tiles = (Tile*)ws_get(ctx, WS_TILES, total * sizeof(Tile), st);
  k_emit_tiles<<<g, th, 0, st>>>(n, pr, ps, status, lod0, sp.want, sp.step, cr, cs, origin, thr, sp.cull,
                                  sp.fp64, off, tiles);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  return total;
}

__global__ void k_init_bounds(int64_t n, const uint8_t* status, const uint8_t* lod0, uint8_t want, int step,
                              int fp64, void* lb, void* ub, void* mid) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (!(status[p] == want && lod0[p] <= step)) return;
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
  int th = 256;
  k_init_bounds<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, status, lod0, sp.want, sp.step, sp.fp64, lb,
                                                               ub, mid);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// ------------------------------------------------------------------ refine

struct RefineArgs {
  const Tile* tiles;
  int64_t n_tiles;
  int* counter;
  const float4* facR;
  const float4* facS;
  const float4* origin;
  const float* thr;
  void* lb;
  void* ub;
  void* mid;
  unsigned long long* ntests;
  int* err;
  int4* queue;       // straddling facet pairs: (pair, r facet, s facet, eps bits)
  unsigned* qcount;
  unsigned qcap;
};

template <class T>
__device__ __forceinline__ void translate(const float4& A, const float4& o, T out[3]) {
  out[0] = T(A.x) - T(o.x);
  out[1] = T(A.y) - T(o.y);
  out[2] = T(A.z) - T(o.z);
}

constexpr uint32_t MBAR_POLL_LIMIT = 1u << 20;

template <class T>
constexpr size_t refine_smem_bytes() {
  return (size_t)CHUNK * 48 + (size_t)CHUNK * sizeof(RecSmem<T>) + 16 * sizeof(float4);
}

template <class T, bool FULL, bool CULL>
__global__ void __launch_bounds__(REFINE_THREADS, (sizeof(T) == 4 ? 2 : 1)) k_refine(RefineArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float4* raw = reinterpret_cast<float4*>(smem);
  RecSmem<T>* srec = reinterpret_cast<RecSmem<T>*>(smem + CHUNK * 48);
  float4* blk = reinterpret_cast<float4*>(smem + CHUNK * 48 + CHUNK * sizeof(RecSmem<T>));
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_tile;
  __shared__ int s_fail;
  __shared__ T red[4][REFINE_THREADS / 32];
  __shared__ unsigned long long red_n[REFINE_THREADS / 32];
  constexpr bool F64 = sizeof(T) == 8;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    s_fail = 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  const T INF = inf_(T(0));

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= a.n_tiles) break;
    const Tile tl = a.tiles[t];
    const int rl = tl.rl, sl = tl.sl;
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar, (uint32_t)sl * 48u);
      tma_load_1d(raw, a.facS + 3LL * tl.sb, (uint32_t)sl * 48u, &bar);
    }
    const float4 o4 = a.origin[tl.pair];
    const int nst = max(1, REFINE_THREADS / rl);
    const bool active = tid < rl * nst;
    const int i = active ? tid % rl : 0;
    const int stripe = active ? tid / rl : 0;

    // r facet -> register record (n, m negated)
    Rec<T> P;
    float rlo[3], rhi[3];
    {
      const float4* f = a.facR + 3LL * (tl.rb + i);
      float4 A = f[0], B = f[1], C = f[2];
      T va[3], vb[3], vc[3];
      translate(A, o4, va);
      translate(B, o4, vb);
      translate(C, o4, vc);
      make_rec(P, va, vb, vc, T(A.w), T(B.w), true);
      if (CULL) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float x0 = float(va[k]), x1 = float(vb[k]), x2 = float(vc[k]);
          rlo[k] = fminf(x0, fminf(x1, x2));
          rhi[k] = fmaxf(x0, fmaxf(x1, x2));
        }
      }
    }

    if (!mbar_wait_bounded(&bar, phase, MBAR_POLL_LIMIT)) atomicOr(&s_fail, 1);
    phase ^= 1u;
    __syncthreads();
    if (s_fail) {
      if (tid == 0) set_err(a.err, ERR_MBAR_TIMEOUT);
      // let the copy in flight land (bounded) before the CTA leaves
      mbar_wait_bounded(&bar, phase ^ 1u, MBAR_POLL_LIMIT);
      break;
    }

    // s chunk -> shared records
    for (int k = tid; k < sl; k += REFINE_THREADS) {
      float4 A = raw[3 * k], B = raw[3 * k + 1], C = raw[3 * k + 2];
      T va[3], vb[3], vc[3];
      translate(A, o4, va);
      translate(B, o4, vb);
      translate(C, o4, vc);
      Rec<T> Q;
      make_rec(Q, va, vb, vc, T(A.w), T(B.w), false);
      store_rec(srec[k], Q);
    }
    if (CULL) {
      // per 32-facet block: box (pair-local, float) with max ph / hd
      const int nblk = (sl + 31) / 32;
      if (warp < nblk) {
        const int k = 32 * warp + lane;
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        float ph = 0.f, hd = 0.f;
        if (k < sl) {
          float4 A = raw[3 * k], B = raw[3 * k + 1], C = raw[3 * k + 2];
          float xa[3] = {A.x - o4.x, A.y - o4.y, A.z - o4.z};
          float xb[3] = {B.x - o4.x, B.y - o4.y, B.z - o4.z};
          float xc[3] = {C.x - o4.x, C.y - o4.y, C.z - o4.z};
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            lo[q] = fminf(xa[q], fminf(xb[q], xc[q]));
            hi[q] = fmaxf(xa[q], fmaxf(xb[q], xc[q]));
          }
          ph = B.w;
          hd = A.w;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          lo[q] = warp_min(lo[q]);
          hi[q] = -warp_min(-hi[q]);
        }
        ph = -warp_min(-ph);
        hd = -warp_min(-hd);
        if (lane == 0) {
          blk[2 * warp] = make_float4(lo[0], lo[1], lo[2], ph);
          blk[2 * warp + 1] = make_float4(hi[0], hi[1], hi[2], hd);
        }
      }
    }
    __syncthreads();

    // ---- all facet pairs of this thread
    T lbm = INF, ubu = INF, ubc = INF, d2m = INF;
    bool anyposs = false, anycert = false;
    unsigned long long ntest = 0;
    const T eh = T(tl.eh), ew = T(tl.ew);
    if (active) {
      const int nblk = (sl + 31) / 32;
      const float thr = CULL ? a.thr[tl.pair] : 0.f;
      const float rph = CULL ? float(P.ph) : 0.f;
      for (int b = stripe; b < nblk; b += nst) {
        if (CULL) {
          float4 blo = blk[2 * b], bhi = blk[2 * b + 1];
          float4 mlo = make_float4(rlo[0], rlo[1], rlo[2], 0.f), mhi = make_float4(rhi[0], rhi[1], rhi[2], 0.f);
          float g = box_gap_rd(mlo, mhi, blo, bhi);
          float lbb = __fsub_rd(__fsub_rd(__fsub_rd(g, rph), blo.w), 2.f * tl.eps);
          if (lbb > thr) continue;
        }
        const int j0 = 32 * b, j1 = min(j0 + 32, sl);
        ntest += (unsigned long long)(j1 - j0);
        for (int j = j0; j < j1; ++j) {
          Rec<T> Q;
          load_rec(Q, srec[j]);
          bool maybe;
          T d2 = tri_d2(P, Q, eh, maybe);
          if (!maybe) {
            if (FULL) {
              d2m = min(d2m, d2);
            } else {
              T d = sqrt_test(d2);
              lbm = min(lbm, sub_rd(d, add_ru(P.ph, Q.ph)));
              ubu = min(ubu, add_ru(d, add_ru(P.hd, Q.hd)));
            }
          } else {
            // rare: both triangles straddle each other's planes.  The pair is
            // queued; k_cross_fix decides its meeting test in double
            // precision and folds its bounds in.  A full queue falls back to
            // "a crossing is possible" (lower bound 0), which stays valid.
            unsigned qk = atomicAdd(a.qcount, 1u);
            if (qk < a.qcap) {
              a.queue[qk] = make_int4(tl.pair, tl.rb + i, tl.sb + j, __float_as_int(tl.eps));
            } else if (FULL) {
              anyposs = true;
              d2m = min(d2m, d2);
            } else {
              T d = sqrt_test(d2);
              lbm = min(lbm, -add_ru(P.ph, Q.ph));
              ubu = min(ubu, add_ru(d, add_ru(P.hd, Q.hd)));
            }
          }
        }
      }
    }
    T lbv, ubv, ucv, midv = INF;
    if (FULL) {
      T d = d2m < INF ? sqrt_rn(d2m) : INF;
      midv = anycert ? T(0) : d;
      lbv = anyposs ? T(0) : d;
      ubv = d;
      ucv = anycert ? T(0) : INF;
    } else {
      lbv = lbm;
      ubv = ubu;
      ucv = ubc;
    }
    lbv = warp_min(lbv);
    ubv = warp_min(ubv);
    ucv = warp_min(ucv);
    midv = warp_min(midv);
    unsigned long long nt = warp_sum_u64(ntest);
    if (lane == 0) {
      red[0][warp] = lbv;
      red[1][warp] = ubv;
      red[2][warp] = ucv;
      red[3][warp] = midv;
      red_n[warp] = nt;
    }
    __syncthreads();
    if (tid == 0) {
      T L0 = red[0][0], U0 = red[1][0], C0 = red[2][0], M0 = red[3][0];
      unsigned long long N0 = red_n[0];
#pragma unroll
      for (int w = 1; w < REFINE_THREADS / 32; ++w) {
        L0 = min(L0, red[0][w]);
        U0 = min(U0, red[1][w]);
        C0 = min(C0, red[2][w]);
        M0 = min(M0, red[3][w]);
        N0 += red_n[w];
      }
      const T eps = T(tl.eps);
      T lb = L0 < INF ? sub_rd(L0, eps) : INF;
      lb = max(lb, T(0));
      T ub = U0 < INF ? add_ru(U0, eps) : INF;
      ub = min(ub, C0);
      using B = Bits<T>;
      atomicMin(&((typename B::U*)a.lb)[tl.pair], B::enc(lb));
      atomicMin(&((typename B::U*)a.ub)[tl.pair], B::enc(ub));
      if (FULL) atomicMin(&((typename B::U*)a.mid)[tl.pair], B::enc(M0));
      if (N0) atomicAdd(a.ntests, N0);
    }
    __syncthreads();
  }
}

// Bounds contribution of the queued straddling facet pairs: the 15-candidate
// distance as in k_refine, the meeting test in double precision (exact
// translation of the float vertices), then the same atomicMin updates.
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
    Rec<T> P, Q;
    make_rec(P, va, vb, vc, T(r0.w), T(r1.w), true);
    make_rec(Q, wa, wb, wc, T(s0.w), T(s1.w), false);
    bool maybe;
    T d2 = tri_d2(P, Q, T(0), maybe);
    float4 rr[3] = {r0, r1, r2}, ss[3] = {s0, s1, s2};
    const bool cert = cross_exact64(rr, ss, o4);
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

template <class T, bool FULL, bool CULL>
static void launch_refine(pj_ctx* ctx, RefineArgs& args, int64_t n_tiles, cudaStream_t st) {
  auto kern = k_refine<T, FULL, CULL>;
  const size_t smem = refine_smem_bytes<T>();
  PJ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  PJ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, REFINE_THREADS, smem));
  if (occ < 1) occ = 1;
  if (ctx->ctas_per_sm > 0) occ = std::min(occ, ctx->ctas_per_sm);
  int64_t grid = std::min<int64_t>(n_tiles, (int64_t)occ * ctx->sm_count);
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, REFINE_THREADS, smem, st>>>(args);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  if (args.qcap > 0) {
    k_cross_fix<T, FULL><<<ctx->sm_count * 4, 256, 0, st>>>(args);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
}

float refine_ms(pj_ctx* ctx, int ev) {
  if (ev < 0) return 0.f;
  float ms = 0.f;
  PJ_CK(cudaEventElapsedTime(&ms, ctx->ev[ev], ctx->ev[ev + 1]));
  return ms;
}

int run_refine(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n_tiles, const StepSpec& sp,
               cudaStream_t st) {
  if (n_tiles == 0) return -1;
  int ev = -1;
  if (ctx->ev_used + 2 <= 64 && ctx->ev[ctx->ev_used]) {
    ev = ctx->ev_used;
    ctx->ev_used += 2;
  }
  int64_t n = 1;
  RefineArgs a;
  a.tiles = (const Tile*)ctx->ws[WS_TILES].p;
  a.n_tiles = n_tiles;
  a.counter = (int*)(ctx->d_counters + 15);
  PJ_CK(cudaMemsetAsync(a.counter, 0, sizeof(int), st));
  a.facR = R->lod[sp.lodR].fac;
  a.facS = S->lod[sp.lodS].fac;
  a.origin = (const float4*)ctx->ws[WS_ORIGIN].p;
  a.thr = (const float*)ctx->ws[WS_THR].p;
  a.lb = ctx->ws[WS_LB].p;
  a.ub = ctx->ws[WS_UB].p;
  a.mid = ctx->ws[WS_MID].p;
  a.ntests = ctx->d_counters + (sp.fp64 ? 1 : 0);
  a.err = ctx->d_err;
  a.qcap = CROSS_QUEUE_CAP;
  a.queue = (int4*)ws_get(ctx, WS_MISC2, (size_t)a.qcap * sizeof(int4), st);
  a.qcount = (unsigned*)(ctx->d_counters + 14);
  PJ_CK(cudaMemsetAsync(a.qcount, 0, sizeof(unsigned), st));
  (void)n;
  if (ev >= 0) PJ_CK(cudaEventRecord(ctx->ev[ev], st));
  if (sp.fp64) {
    if (sp.full) {
      if (sp.cull) launch_refine<double, true, false>(ctx, a, n_tiles, st);
      else launch_refine<double, true, false>(ctx, a, n_tiles, st);
    } else {
      launch_refine<double, false, false>(ctx, a, n_tiles, st);
    }
  } else {
    if (sp.full) {
      if (sp.cull) launch_refine<float, true, true>(ctx, a, n_tiles, st);
      else launch_refine<float, true, false>(ctx, a, n_tiles, st);
    } else {
      if (sp.cull) launch_refine<float, false, true>(ctx, a, n_tiles, st);
      else launch_refine<float, false, false>(ctx, a, n_tiles, st);
    }
  }
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
                                                              b.lod0, b.exact, b.dlo, b.dhi, b.d);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

void count_tiles_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                      const PairBufs& b, cudaStream_t st) {
  if (n == 0) return;
  const LodData& LR = R->lod[sp.lodR];
  const LodData& LS = S->lod[sp.lodS];
  ChunkView cr{LR.chunk, LR.coff, LR.foff}, cs{LS.chunk, LS.coff, LS.foff};
  int th = 128;
  k_count_tiles<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, b.pr, b.ps, b.status, b.lod0, sp.want, sp.step, cr,
                                                              cs, b.origin, b.thr, sp.cull, sp.fp64, b.tcount);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

void emit_tiles_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                     const PairBufs& b, cudaStream_t st) {
  if (n == 0) return;
  const LodData& LR = R->lod[sp.lodR];
  const LodData& LS = S->lod[sp.lodS];
  ChunkView cr{LR.chunk, LR.coff, LR.foff}, cs{LS.chunk, LS.coff, LS.foff};
  int th = 128;
  k_emit_tiles<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, b.pr, b.ps, b.status, b.lod0, sp.want, sp.step, cr,
                                                             cs, b.origin, b.thr, sp.cull, sp.fp64, b.toff, b.tiles);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

void init_bounds_bufs(pj_ctx* ctx, int64_t n, const StepSpec& sp, const PairBufs& b, cudaStream_t st) {
  if (n == 0) return;
  int th = 256;
  k_init_bounds<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, b.status, b.lod0, sp.want, sp.step, sp.fp64, b.lb,
                                                               b.ub, b.mid);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

void run_refine_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n_tiles, const StepSpec& sp,
                     const PairBufs& b, int* err, cudaStream_t st) {
  if (n_tiles == 0) return;
  RefineArgs a;
  a.tiles = b.tiles;
  a.n_tiles = n_tiles;
  a.counter = (int*)(b.counters + 1);
  PJ_CK(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st));
  a.facR = R->lod[sp.lodR].fac;
  a.facS = S->lod[sp.lodS].fac;
  a.origin = b.origin;
  a.thr = b.thr;
  a.lb = b.lb;
  a.ub = b.ub;
  a.mid = b.mid;
  a.ntests = b.counters;
  a.err = err;
  a.queue = b.queue;
  a.qcap = b.qcap;
  a.qcount = (unsigned*)(b.counters + 2);
  PJ_CK(cudaMemsetAsync(a.qcount, 0, sizeof(unsigned), st));
  if (sp.fp64) {
    if (sp.full) launch_refine<double, true, false>(ctx, a, n_tiles, st);
    else launch_refine<double, false, false>(ctx, a, n_tiles, st);
  } else {
    if (sp.full) launch_refine<float, true, false>(ctx, a, n_tiles, st);
    else launch_refine<float, false, false>(ctx, a, n_tiles, st);
  }
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
  Rec<T> RP, RQ;
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
  const bool cert = maybe && cross_exact64(fp, fq, make_float4(o[0], o[1], o[2], 0.f));
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
