// Autotuning of the join (PJ_AUTOTUNE): per workload key -- predicate,
// precision, flags, tau or k, and the shapes of R and S (objects, LoDs,
// largest facet count per LoD) -- the first join runs candidate
// configurations, keeps the fastest, and later joins with the same key use
// it.  Three dimensions:
//   * tests per lane: the single-precision refinement variant, one triangle
//     test per lane and instruction (scalar) or two (packed FP32x2), unless
//     the context fixed it with the "refine_variant" option;
//   * the LoD schedule of within-tau / intersection joins: every pair starts
//     at step 0, 1, ... or at full resolution (a fixed schedule: the
//     proposal network is not run), or, with PJ_USE_MLP, at its learned
//     per-pair start;
//   * the unit tile: 32 r facets x 32, 16 or 8 s facets (every unit of a
//     launch handed out as 1, 2 or 4 parts; small launches fill more warps
//     with shorter parts), unless the context fixed "refine_split".
// The first two are searched jointly, then the tile with the best of them
// (coordinate search); every candidate is timed twice, the faster run
// counts.  Configurations only change how the work is
// scheduled, never a result.  Choices persist across contexts in the
// "autotune_cache" file of pj_create, one "key choice" line each.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pj {

pj_status join_within(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                      cudaStream_t st, std::string& stats);
pj_status join_knn(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                   cudaStream_t st, std::string& stats);

namespace {

struct Choice {
  int variant;   // 1 scalar, 2 packed
  int start;     // -1: the query's own schedule; >= 0: every pair starts at that step
  int split;     // 0: the context's tail splitting; 1, 2, 4: every unit in that many parts
  int encode() const { return split * 4096 + variant * 64 + (start + 1); }
  static Choice decode(int c) { return Choice{(c % 4096) / 64, c % 64 - 1, c / 4096}; }
  int tile_s() const { return split > 0 ? BLK / split : BLK; }
};

std::string key_of(const pj_set* R, const pj_set* S, const pj_query* q) {
  std::ostringstream k;
  k.precision(17);
  k << "p" << (int)q->pred << ".x" << (int)q->prec << ".f" << (q->flags & ~(uint32_t)PJ_AUTOTUNE);
  if (q->pred == PJ_KNN) k << ".k" << q->k;
  else k << ".t" << q->tau;
  for (const pj_set* X : {R, S}) {
    k << ".n" << X->n << ".L" << X->L;
    for (int l = 0; l < X->L; ++l) k << "." << X->lod[l].maxF;
  }
  return k.str();
}

bool lookup(pj_ctx* ctx, const std::string& key, Choice* c) {
  for (auto& e : ctx->tuned)
    if (e.first == key) {
      *c = Choice::decode(e.second);
      return true;
    }
  if (!ctx->autotune_cache.empty()) {
    std::ifstream f(ctx->autotune_cache);
    std::string k;
    int v;
    while (f >> k >> v)
      if (k == key) {
        ctx->tuned.emplace_back(k, v);
        *c = Choice::decode(v);
        return true;
      }
  }
  return false;
}

void store(pj_ctx* ctx, const std::string& key, const Choice& c) {
  ctx->tuned.emplace_back(key, c.encode());
  if (!ctx->autotune_cache.empty()) {
    std::ofstream f(ctx->autotune_cache, std::ios::app);
    if (f) f << key << " " << c.encode() << "\n";
  }
}

// A trial that needs more refinement units in one step than this is far
// slower than the alternatives (e.g. starting blobs against long tubes at
// full resolution): it is abandoned at the unit count, before any refinement.
constexpr int64_t TRIAL_UNIT_CAP = int64_t(1) << 26;
// refine_tail value whose tail holds every unit of a launch (units per
// resident warp; launches of more units than this are not split whole)
constexpr int ALL_UNITS_TAIL = 1 << 16;

pj_status run_with(pj_ctx* ctx, const Choice& c, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                   cudaStream_t st, std::string& stats, int64_t unit_cap = 0) {
  const int v0 = ctx->refine_variant, s0 = ctx->sched_start, k0 = ctx->refine_split, t0 = ctx->refine_tail;
  auto restore = [&]() {
    ctx->refine_variant = v0;
    ctx->sched_start = s0;
    ctx->refine_split = k0;
    ctx->refine_tail = t0;
    ctx->trial_unit_cap = 0;
  };
  ctx->refine_variant = c.variant;
  ctx->sched_start = c.start;
  if (c.split > 0) {
    // every unit of a launch split (the tail covers all of them)
    ctx->refine_split = c.split;
    ctx->refine_tail = ALL_UNITS_TAIL;
  }
  ctx->trial_unit_cap = unit_cap;
  pj_status rc;
  try {
    rc = q->pred == PJ_KNN ? join_knn(ctx, R, S, q, out, st, stats) : join_within(ctx, R, S, q, out, st, stats);
  } catch (...) {
    restore();
    throw;
  }
  restore();
  return rc;
}

std::string with_tuning(const std::string& stats, const std::string& extra) {
  if (stats.size() < 2 || stats.back() != '}') return stats;
  return stats.substr(0, stats.size() - 1) + ",\"autotune\":" + extra + "}";
}

}  // namespace

// Whether the stored choice for this workload fixes the LoD schedule (every
// pair from one step, no learned start); false when nothing is stored yet.
bool tuned_schedule_fixed(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q) {
  Choice c{0, -1, 0};
  return lookup(ctx, key_of(R, S, q), &c) && c.start >= 0;
}

// Set the choice stored in `from` for this workload on `to` (it stays
// set); false when nothing is stored yet.
bool tuned_apply(pj_ctx* from, pj_ctx* to, const pj_set* R, const pj_set* S, const pj_query* q) {
  Choice c{0, -1, 0};
  if (!lookup(from, key_of(R, S, q), &c)) return false;
  to->refine_variant = c.variant;
  to->sched_start = c.start;
  if (c.split > 0) {
    to->refine_split = c.split;
    to->refine_tail = ALL_UNITS_TAIL;
  }
  return true;
}

// A join of a resident R (or one streamed chunk) with PJ_AUTOTUNE.
pj_status join_autotuned(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                         cudaStream_t st, std::string& stats) {
  const std::string key = key_of(R, S, q);
  Choice best{ctx->refine_variant, -1, 0};
  char buf[192];
  if (lookup(ctx, key, &best)) {
    pj_status rc = run_with(ctx, best, R, S, q, out, st, stats);
    snprintf(buf, sizeof buf, "{\"cached\":1,\"variant\":%d,\"start\":%d,\"tile_s\":%d}", best.variant, best.start,
             best.tile_s());
    stats = with_tuning(stats, buf);
    ctx->last_tune = buf;
    return rc;
  }
  std::vector<Choice> cand;
  const int Lmax = std::max(R->L, S->L);
  // FP64 joins have one refinement kernel; a variant fixed at context
  // creation is kept, only the schedule is tuned
  const std::vector<int> variants = (q->prec == PJ_PREC_FP64 || ctx->variant_fixed)
                                        ? std::vector<int>{ctx->refine_variant}
                                        : std::vector<int>{2, 1};
  for (int v : variants) {
    if (q->pred == PJ_KNN) {
      cand.push_back(Choice{v, -1, 0});
    } else {
      for (int s = 0; s < Lmax; ++s) cand.push_back(Choice{v, s, 0});
      if (q->flags & PJ_USE_MLP) cand.push_back(Choice{v, -1, 0});
    }
  }
  std::string tried = "[";
  double best_ms = 1e300;
  pj_result keep;
  memset(&keep, 0, sizeof keep);
  std::string keep_stats;
  JoinSummary keep_sum;
  {
    // one untimed run first: workspace growth would bias the first candidate
    pj_result warm;
    memset(&warm, 0, sizeof warm);
    std::string st_w;
    pj_status rc = run_with(ctx, cand[0], R, S, q, &warm, st, st_w);
    free(warm.priv);
    if (rc != PJ_OK) return rc;
  }
  int n_tried = 0;
  // one timed trial; false on an error status (returned through rc)
  auto trial = [&](const Choice& c, pj_status& rc) -> bool {
    pj_result res;
    memset(&res, 0, sizeof res);
    std::string st_i;
    Timer t;
    const char* sep = n_tried++ ? "," : "";
    try {
      // the first candidate (the warmed one) always completes
      rc = run_with(ctx, c, R, S, q, &res, st, st_i, n_tried > 1 ? TRIAL_UNIT_CAP : 0);
    } catch (const TrialTooLarge& e) {
      PJ_CK(cudaStreamSynchronize(st));
      snprintf(buf, sizeof buf, "%s{\"variant\":%d,\"start\":%d,\"tile_s\":%d,\"skipped_units\":%lld}", sep,
               c.variant, c.start, c.tile_s(), (long long)e.units);
      tried += buf;
      rc = PJ_OK;
      return true;
    }
    double ms = t.ms();
    if (rc != PJ_OK) {
      free(res.priv);
      return false;
    }
    {
      // a second timed run: the faster of the two (one run alone is at the
      // mercy of a late first-use cost)
      pj_result again;
      memset(&again, 0, sizeof again);
      std::string st_a;
      Timer t2;
      rc = run_with(ctx, c, R, S, q, &again, st, st_a);
      ms = std::min(ms, t2.ms());
      free(again.priv);
      if (rc != PJ_OK) {
        free(res.priv);
        return false;
      }
    }
    snprintf(buf, sizeof buf, "%s{\"variant\":%d,\"start\":%d,\"tile_s\":%d,\"ms\":%.3f}", sep, c.variant,
             c.start, c.tile_s(), ms);
    tried += buf;
    if (keep.priv && res.n != keep.n) {
      free(res.priv);
      throw ApiError{PJ_ECUDA, "autotuning: configurations disagree on the number of results"};
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
      free(keep.priv);
      keep = res;
      keep_stats = st_i;
      keep_sum = ctx->last_sum;
    } else {
      free(res.priv);
    }
    return true;
  };
  try {
    pj_status rc = PJ_OK;
    // tests per lane x schedule, with the context's tile
    for (const Choice& c : cand)
      if (!trial(c, rc)) {
        free(keep.priv);
        return rc;
      }
    // then the tile, with the best of those
    if (!ctx->split_fixed) {
      for (int k : {2, 4}) {
        Choice c = best;
        c.split = k;
        if (!trial(c, rc)) {
          free(keep.priv);
          return rc;
        }
      }
      // the whole-unit tile (32 s facets) wins ties: it is the default
      if (best.split == 0) best.split = 1;
    }
  } catch (...) {
    free(keep.priv);
    throw;
  }
  tried += "]";
  store(ctx, key, best);
  *out = keep;
  ctx->last_sum = keep_sum;
  snprintf(buf, sizeof buf, "{\"cached\":0,\"variant\":%d,\"start\":%d,\"tile_s\":%d,\"tried\":", best.variant,
           best.start, best.tile_s());
  ctx->last_tune = std::string(buf) + tried + "}";
  stats = with_tuning(keep_stats, std::string(buf) + tried + "}");
  return PJ_OK;
}

}  // namespace pj
