// The persistent refinement kernels (k_refine, k_refine2, k_cross_fix) and
// their launchers, shared by the translation units that instantiate them:
// refine_f32.cu (single precision) and refine_f64.cu (double precision), so
// that the two compile in parallel.  refine.cu builds the units and calls
// launch_refine_f32 / launch_refine_f64.
#pragma once
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "tritri.cuh"
#include "tritri2.cuh"

namespace pj {

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
  int64_t tiles_cap;       // units the tile array holds (a device count above it was truncated)
  unsigned long long* units_max;   // largest device unit count seen (may be null)
};

// The unit count of a launch: the host's, or the device's clamped to the
// tile array (a builder that overflowed flags the join, which reruns).
__device__ __forceinline__ int64_t launch_units(const int64_t* dev, int64_t host, int64_t cap,
                                                unsigned long long* units_max) {
  if (!dev) return host;
  const int64_t n = *dev;
  if (units_max && blockIdx.x == 0 && threadIdx.x == 0) atomicMax(units_max, (unsigned long long)n);
  return n < cap ? n : cap;
}

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
#ifdef PJ_REFINE_WARPS_F32
  return sizeof(T) == 4 ? PJ_REFINE_WARPS_F32 : 8;
#else
  return sizeof(T) == 4 ? REFINE_WARPS : 8;
#endif
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

// Where a listed pair goes when filtered signs cannot decide its meeting
// test: the global queue of k_cross_fix, which decides it exactly.
struct QueueRef {
  int4* queue;
  unsigned* qcount;
  unsigned qcap;
  int pair, rb, sb;
  float eps;
};

// Contributions of the straddling facet pairs a warp listed during one
// unit: lane k takes entries k, k+32, ...; the meeting test from filtered
// signs (cross_filtered: single, then double precision), and the rare pair
// neither makes certain goes to k_cross_fix's queue (exact arithmetic,
// where it adds its own contribution; a full queue keeps a meeting
// possible).  The list holds the single-precision squared distance; in
// double precision it is recomputed from the facets (the same records, so
// the same value as in the unit's loop).  Out of line so that its
// registers do not weigh on the unit's inner loop; called only when the
// warp's list is non-empty.
template <class T, bool FULL>
__device__ __noinline__ ListOut<T> process_list(const uint2* list, unsigned nl, int lane, const float4* fr0,
                                                const float4* raw, float4 o4, QueueRef q) {
  const T INF = inf_(T(0));
  ListOut<T> out{INF, INF, INF, INF, false};
  for (unsigned k = lane; k < nl; k += 32) {
    const uint2 e = list[k];
    const int li = e.x & 255, lj = e.x >> 8;
    const float4* fr = fr0 + 3 * li;
    const float4* fs = raw + 3 * lj;
    const int f = cross_filtered(fr, fs);
    if (f < 0) {
      const unsigned qk = atomicAdd(q.qcount, 1u);
      if (qk < q.qcap) {
        q.queue[qk] = make_int4(q.pair, q.rb + li, q.sb + lj, __float_as_int(q.eps));
        continue;
      }
    }
    const T phs = add_ru(T(fr[1].w), T(fs[1].w)), hds = add_ru(T(fr[0].w), T(fs[0].w));
    if (f == 1) {
      out.lbm = min(out.lbm, -phs);
      out.ubc = min(out.ubc, hds);
      if (FULL) out.anyposs = true;
      continue;
    }
    T d2e = T(__uint_as_float(e.y));
    if (sizeof(T) == 8) {
      T va[3], vb[3], vc[3], wa[3], wb[3], wc[3];
      translate(fr[0], o4, va);
      translate(fr[1], o4, vb);
      translate(fr[2], o4, vc);
      translate(fs[0], o4, wa);
      translate(fs[1], o4, wb);
      translate(fs[2], o4, wc);
      typename RecOf<T>::R P, Q;
      make_rec(P, va, vb, vc, T(fr[0].w), T(fr[1].w), true);
      make_rec(Q, wa, wb, wc, T(fs[0].w), T(fs[1].w), false);
      bool mb;
      d2e = tri_d2(P, Q, T(0), mb);
    }
    if (f < 0) {   // undecided and the queue is full: a meeting stays possible
      if (FULL) {
        out.anyposs = true;
        out.d2m = min(out.d2m, d2e);
      } else {
        out.lbm = min(out.lbm, -phs);
        out.ubu = min(out.ubu, add_ru(sqrt_test(d2e), hds));
      }
    } else if (FULL) {
      out.d2m = min(out.d2m, d2e);
    } else {
      T d = sqrt_test(d2e);
      out.lbm = min(out.lbm, sub_rd(d, phs));
      out.ubu = min(out.ubu, add_ru(d, hds));
    }
  }
  return out;
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
  const UnitSpace us =
      unit_space(launch_units(a.n_tiles_dev, a.n_tiles, a.tiles_cap, a.units_max), a.split_k, a.split_tail);
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
      ListOut<T> lo = process_list<T, FULL>(
          list, nl, lane, rfac, raw, o4, QueueRef{a.queue, a.qcount, a.qcap, tl.pair, tl.rb, tl.sb, tl.eps});
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
      // 0 only from a meeting test; candidates that round to 0 give the
      // smallest positive value
      T d = d2m < INF ? (d2m > T(0) ? sqrt_rn(d2m) : tiny_(T(0))) : INF;
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
  const UnitSpace us =
      unit_space(launch_units(a.n_tiles_dev, a.n_tiles, a.tiles_cap, a.units_max), a.split_k, a.split_tail);
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
      ListOut<T> lo = process_list<T, FULL>(list, nl, lane, a.facR + 3LL * tl.rb, raw, o4,
                                            QueueRef{a.queue, a.qcount, a.qcap, tl.pair, tl.rb, tl.sb, tl.eps});
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
      // 0 only from a meeting test; candidates that round to 0 give the
      // smallest positive value
      T d = d2m < INF ? (d2m > T(0) ? sqrt_rn(d2m) : tiny_(T(0))) : INF;
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
    typename RecOf<T>::R P, Q;
    make_rec(P, va, vb, vc, T(r0.w), T(r1.w), true);
    make_rec(Q, wa, wb, wc, T(s0.w), T(s1.w), false);
    bool maybe;
    T d2 = tri_d2(P, Q, T(0), maybe);
    float4 rr[3] = {r0, r1, r2}, ss[3] = {s0, s1, s2};
    const bool cert = cross_decide(rr, ss);
    const T phs = add_ru(P.ph, Q.ph), hds = add_ru(P.hd, Q.hd);
    T lb, ub, mid;
    if (cert) {
      lb = -phs;
      ub = hds;
      mid = T(0);
    } else {
      T d = FULL ? (d2 > T(0) ? sqrt_rn(d2) : tiny_(T(0))) : sqrt_test(d2);
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


// Launch the refinement of one LoD step over the built units (and the
// fix-up of the queued straddling pairs): single precision (variant 1
// scalar, 2 packed) or double precision.
void launch_refine_f32(pj_ctx* ctx, RefineArgs& a, int64_t n_tiles, bool full, int variant, cudaStream_t st);
void launch_refine_f64(pj_ctx* ctx, RefineArgs& a, int64_t n_tiles, bool full, cudaStream_t st);

}  // namespace pj
