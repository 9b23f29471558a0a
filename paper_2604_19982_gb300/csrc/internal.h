// Host-side internals of the join library: context, device-resident sets,
// growable device buffers and the launchers each translation unit exports.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <chrono>
#include <string>
#include <vector>

#include "../../include/pj.h"

namespace pj {

// Pair status codes (per candidate object pair).
// MAKE_EXACT (4): a result pair queued for its FP64 distance; WAVE (5): a
// k-NN candidate in the current step's first wave.
enum : uint8_t { UNDECIDED = 0, CONFIRMED = 1, REMOVED = 2, REDECIDE = 3, MAKE_EXACT = 4, WAVE = 5 };
// lod0 gate value that admits every pair (passes after the LoD loop).
constexpr int STEP_ALL = 255;

struct CudaError {
  cudaError_t e;
  const char* what;
};

#define PJ_COUNT_LAUNCH count_launch(ctx)

#define PJ_CK(call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) throw ::pj::CudaError{e_, #call};          \
  } while (0)

struct ApiError {
  pj_status st;
  std::string msg;
};

// Thrown when an autotuning trial exceeds its unit budget (the tuner
// skips that configuration).
struct TrialTooLarge {
  int64_t units;
};

// Thrown at the end of a join whose unit buffer was too small for some
// step (its results are discarded): the buffer is grown to `units` and the
// join runs again.
struct UnitsOverflow {
  int64_t units;
};

// device counter slot of the largest unit count a join's steps asked for
constexpr int CNT_UNITS_MAX = 11;

// Grow-only device buffer (stream-ordered allocation on the context stream).
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// One LoD of a device-resident set.
struct LodData {
  int64_t F = 0;                  // facets of all objects
  float4* fac = nullptr;          // [3F]: (v0, hd), (v1, ph), (v2, 0)
  int64_t* foff = nullptr;        // device [n+1] facet offsets
  std::vector<int64_t> foff_h;    // host copy
  int64_t C = 0;                  // chunks of <= CHUNK facets
  float4* chunk = nullptr;        // [3C]: (lo, max hd), (hi, max ph), (max edge, min sine, 0, 0)
  int64_t* coff = nullptr;        // device [n+1] chunk offsets
  std::vector<int64_t> coff_h;
  int64_t B = 0;                  // blocks of <= BLK facets (same layout as chunks)
  float4* blk = nullptr;          // [3B]
  int64_t* boff = nullptr;        // device [n+1] block offsets
  std::vector<int64_t> boff_h;
  int64_t maxF = 0;               // largest facet count of one object
};

// Host-side grid parameters of the within filter for one (R, S, tau).
struct GridCacheEntry {
  uint64_t rid = 0, sid = 0;
  double tau = 0;
  unsigned char grid[64];
  int64_t nids = 0;
};

// The host-side record of a join's refinement steps (see StepLog).
struct StepLogData {
  int n = 0;
  int ev[16];
  int64_t units[16];
  bool f64[16];
  bool full[16];
  bool masked[16];   // full-resolution step whose units went through k_unit_masks
};

// Raw device arrays of one LoD as given by the caller (faces: shared
// template of nfs rows when nfs > 0, else per-object rows).
struct RawLod {
  const float* verts;
  const int64_t* voff;
  const int32_t* faces;
  int nfs;
  const float* hd;
  const float* ph;
};

// Totals of the last join (also in its JSON stats).
struct JoinSummary {
  int64_t candidates = 0, results = 0, units = 0;
  unsigned long long tests32 = 0, tests64 = 0, confirmed = 0, removed = 0;
  double ms_filter = 0, ms_total = 0, refine_ms32 = 0, refine_ms64 = 0;
  unsigned long long launches = 0;
  int graph = 0;   // within joins: 1 captured, 2 replayed from a graph
  double ms_seq = 0;   // within joins: the post-filter sequence from issue to completion (host clock)
  double graph_ms = 0;  // within joins: device time of a replayed graph (events around its launch)
  int spec = 0;         // within joins: the filter ran inside the speculative sequence
};

}  // namespace pj

struct pj_set {
  pj_ctx* ctx = nullptr;
  int device = 0;                 // CUDA device of the storage
  int n = 0;
  int L = 0;
  pj::LodData lod[PJ_MAX_LODS];
  float* mbb = nullptr;           // device [n][6] original-surface boxes
  float* anchor = nullptr;        // device [n][3]
  std::vector<float> mbb_h;       // host copy
  uint64_t uid = 0;               // unique per loaded set (0: a temporary view)
  // streamed chunk views: the LoDs from lazy_from on (the finer ones,
  // most of the facets) are laid out only for the objects whose pairs
  // reach them.  Per lazy LoD l: lazy_state[(l - lazy_from) * n + o] is 0
  // (not built) or 1 (built); lazy_list / lazy_count hold the objects a
  // step adds.
  int lazy_from = PJ_MAX_LODS;
  pj::RawLod lazy_raw[PJ_MAX_LODS] = {};
  unsigned* lazy_state = nullptr;
  int32_t* lazy_list = nullptr;
  unsigned* lazy_count = nullptr;
  // voxels (section 2.1), built at load when the context voxelizes:
  // vox_off [n+1] (host copy vox_off_h), centres [V][3] double, boxes
  // [V][6] (lo.xyz, hi.xyz of the voxel's original facets), anchors [V][3],
  // and per LoD the object-local voxel of every facet (-1: none)
  bool voxels = false;
  int64_t V = 0;
  int vox_kmax = 0;
  int64_t* vox_off = nullptr;
  std::vector<int64_t> vox_off_h;
  double* vox_centre = nullptr;
  float* vox_box = nullptr;
  float* vox_anchor = nullptr;
  int32_t* vox_label[PJ_MAX_LODS] = {};
  // streamed R: the chunks are loaded inside pj_join
  bool streamed = false;
  int64_t n_total = 0;
  int n_chunks = 0;
  pj_fill_fn fill = nullptr;
  void* user = nullptr;
};

namespace pj {
class PackPool;   // host threads that pack streamed chunks (stream.cu)
void destroy_pack_pool(pj::PackPool* p);
}  // namespace pj

struct pj_ctx {
  int device = 0;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  cudaStream_t stream = nullptr;   // default work stream
  cudaStream_t copy_stream = nullptr;
  cudaStream_t build_stream = nullptr;   // set building of streamed chunks
  cudaStream_t join_stream = nullptr;    // streamed chunk joins: the device's greatest priority, so
                                         // their small launches go ahead of the next chunk's build
  // the within filter's grid over S alone, kept in its workspace slots
  // across the chunks of a streamed R (valid until another grid is built)
  struct {
    bool valid = false;
    uint64_t sid = 0;
    double tau = 0;
    unsigned char grid[64];
  } sgrid;
  int* d_err = nullptr;            // device error word
  unsigned long long* d_counters = nullptr;  // [16] device counters
  std::string last_error;
  std::string stats;
  pj::JoinSummary last_sum;
  std::vector<pj::GridCacheEntry> grid_cache;
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    int64_t cap = 0;
    unsigned long long kernels = 0;   // library kernels in the graph
    pj::StepLogData log;
  };
  std::vector<GraphEntry> graphs;   // captured joins (PJ_USE_GRAPH), oldest first
  int ctas_per_sm = 0;             // 0 = from occupancy
  int refine_variant = 1;          // FP32 refinement: 1 scalar, 2 packed (two s facets per lane)
  bool variant_fixed = false;      // refine_variant was given at creation: autotuning keeps it
  bool zero_copy = false;          // pj_load_set reads pinned host arrays in place (no staging copy)
  int refine_split = 1;            // the last units of a refinement launch are split this many ways
  int refine_tail = 2;             // ... that many units per resident warp
  bool split_fixed = false;        // refine_split / refine_tail given at creation: autotuning keeps them
  int sched_start = -1;            // within joins: every pair starts at this LoD step (-1: query's own)
  int64_t trial_unit_cap = 0;      // > 0 while autotuning: a step needing more units abandons the trial
  size_t unit_budget = size_t(512) << 20;   // unit buffer sized for the worst case up to this many bytes
  std::string autotune_cache;
  // per-query workspace
  pj::DevBuf ws[56];
  // learned proposal (bf16 MLP), float master weights on the device
  float* mlp_w = nullptr;          // packed: W1 64x16, b1 64, W2 64x64, b2 64, W3 64, b3 1
  bool mlp_ready = false;
  // autotuned launch choices (per workload key)
  std::vector<std::pair<std::string, int>> tuned;
  // instrumentation: kernel launches issued by the library, and CUDA events
  // bracketing the refinement launches of the current join
  unsigned long long launches = 0;
  cudaEvent_t ev[64] = {};
  int ev_used = 0;
  long long* d_snap = nullptr;     // [64][4] per-step counter snapshots
  // pinned staging of result copies (grow-only)
  void* h_stage = nullptr;
  size_t h_stage_cap = 0;
  std::string last_tune;            // the autotuner's choice for the last join (JSON), if it ran
  // candidate capacity of the last join per (R objects, R LoDs, S, tau), for
  // the speculative graph mode of streamed chunks
  struct SpecCap {
    int64_t nR;
    int LR;
    uint64_t sid;
    double tau;
    int64_t cap;
  };
  std::vector<SpecCap> spec_caps;
  unsigned long long spec_misses = 0;   // speculative joins that ran again unspeculated
  pj::PackPool* pack_pool = nullptr;   // created by the first streamed join, kept until pj_destroy
  // a second join context (own workspace, counters, stage, graphs and join
  // stream; the proposal weights borrowed) that takes every other chunk of a
  // streamed within join, so that two chunks' joins overlap on the device
  pj_ctx* twin = nullptr;
  bool borrowed_mlp = false;         // mlp_w belongs to another context
  bool chunk_overlap = true;         // option "chunk_overlap": streamed within joins use the twin
  bool host_read = true;             // option "host_read": middle-LoD pinned chunk arrays read in place
  bool voxelize = false;             // option "voxels": pj_load_set voxelizes every object it loads
  void* stream_pinned[2] = {};      // pinned staging slots of streamed chunks
  size_t stream_pinned_cap[2] = {};
  void* stream_box_pinned[2] = {};  // pinned copies of a chunk's object boxes and error word
  size_t stream_box_cap[2] = {};
};

namespace pj {

// Packed MLP weight layout (floats).
// capacity of the queue of straddling facet pairs per refine launch
constexpr unsigned CROSS_QUEUE_CAP = 1u << 22;

constexpr int MLP_IN = 16, MLP_H = 64;
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H,
              MLP_B2 = MLP_W2 + MLP_H * MLP_H, MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_H,
              MLP_NW = MLP_B3 + 1;

// workspace slots
enum Slot {
  WS_PR, WS_PS, WS_ORIGIN, WS_THR, WS_BOXLB, WS_ANCUB, WS_STATUS, WS_LOD0, WS_LB, WS_UB, WS_MID,
  WS_DLO, WS_DHI, WS_D, WS_EXACT, WS_TCOUNT, WS_TILES, WS_SCAN, WS_GRID, WS_GRIDIDS, WS_RCOUNT,
  WS_ROFF, WS_TMP, WS_RES, WS_KNN, WS_FEAT, WS_PRED, WS_MISC, WS_MISC2, WS_MISC3, WS_MISC4, WS_MISC5,
  WS_FLAG, WS_KNN2, WS_KNN3, WS_KNN4, WS_KNN5, WS_MLP, WS_MLP2, WS_MLP3, WS_STREAM, WS_STREAM2, WS_STREAM3, WS_STREAM4, WS_STREAM5,
  WS_STREAM6, WS_STREAM7, WS_STREAM8, WS_TILES2, WS_FSLOT, WS_FSCAN,
  WS_COUNT
};

static_assert(WS_COUNT <= 56, "workspace slots");
void* ws_get(pj_ctx* ctx, int slot, size_t bytes, cudaStream_t st);

// ---- set layout (api.cu)
void free_set_storage(pj_set* s);

// ---- voxels (voxel.cu)
// Voxels of every object of a set being loaded: verts0 / voff0 are the
// device copies of its coarsest LoD's vertex array and offsets (the initial
// k-means centres are taken from them), the facet arrays must be built.
void voxelize_set(pj_ctx* ctx, pj_set* s, const float* verts0, const int64_t* voff0, cudaStream_t st);
void free_voxels(pj_set* s);
// Algorithms 1 and 2 over object pairs pr / ps (device); every output a
// caller device buffer (see pj_voxel_filter); synchronizes st at the end.
void voxel_filter(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps, int64_t n,
                  double tau, bool fp64, double* op_lb, double* op_ub, uint8_t* status, int64_t* vp_off, double* vp_lb,
                  double* vp_ub, int64_t vp_cap, int64_t* kept_off, int32_t* kept, int64_t* n_kept,
                  cudaStream_t st);

// ---- scan (join.cu): exclusive prefix sum of n int64 values into out[0..n],
// out[n] = total.  tmp is workspace.
// With tmp == nullptr the temporaries are allocated stream-ordered; otherwise
// tmp must hold scan_tmp_words(n) words and nothing is allocated.
void scan_i64(pj_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, int64_t* tmp = nullptr);
int64_t scan_tmp_words(int64_t n);

// ---- filter (filter.cu)
struct FilterOut {
  int64_t n_pairs = 0;
};
// Candidate pairs (r, s) with box MINDIST <= tau, grouped by r and sorted by
// s; results land in WS_PR / WS_PS.
FilterOut filter_within(pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau, cudaStream_t st);
// The within filter's grid over S alone is kept for (R, S, tau) (a streamed
// chunk R against a resident S after the first chunk).
bool filter_grid_kept(const pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau);
// With the kept grid: the filter's launches with a capacity fixed in
// advance and no host synchronization (count in WS_ROFF[R->n]; *over bit 0:
// an r with too many candidates for the ranked emit, bit 1: more than cap
// pairs; either voids the pairs).
void filter_within_enqueue(pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau, int64_t cap, int* over,
                           cudaStream_t st);
// k-NN candidates: per r all s with MINDIST <= theta_r (theta_r = k-th
// smallest anchor distance); roff (WS_ROFF, n_R+1) is the CSR of the result.
FilterOut filter_knn(pj_ctx* ctx, const pj_set* R, const pj_set* S, int k, cudaStream_t st);

// ---- refine (refine.cu)
struct Tile {
  int32_t pair, rb, sb;
  uint16_t rl, sl;
  float eps, eh, ew;
  int32_t pad;
};
static_assert(sizeof(Tile) == 32, "tile is two int4");

struct StepSpec {
  int lodR, lodS;
  bool early = false;  // units of a pair already proven ub <= threshold are skipped
  bool exact_cross = false;  // coarse single-precision steps also decide crossings exactly
  bool full;        // both at the original surfaces (hd = ph = 0)
  bool fp64;
  bool cull;        // skip chunk pairs / blocks that cannot reach the threshold
  uint8_t want;     // status of the pairs to refine (UNDECIDED or REDECIDE)
  int step;         // LoD step index (pairs with lod0 > step wait)
  // the caller checks the unit count after its final synchronization and
  // reruns on an overflow (check_units): the builder may then emit into the
  // buffer as it is instead of counting first
  bool rerun_ok = false;
};

// Count + emit refinement units for the pairs in state `want`.  count >= 0:
// the host knows the number; count < 0: it stays on the device at *dev
// (the unit buffer was sized for the worst case), nothing was synchronized.
struct UnitCount {
  int64_t count;
  const int64_t* dev;
};
UnitCount build_tiles(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n_pairs, const StepSpec& sp,
                      cudaStream_t st);
// Reset the per-pair lb / ub words of the pairs being refined.
void init_bounds(pj_ctx* ctx, int64_t n_pairs, const StepSpec& sp, cudaStream_t st);
// Run the persistent refinement kernel over the built tiles.  Returns the
// index of the CUDA event pair (ctx->ev) bracketing the launch on `st`, or -1.
int run_refine(pj_ctx* ctx, const pj_set* R, const pj_set* S, UnitCount units, const StepSpec& sp,
               cudaStream_t st);
// After a join's final synchronization (herr: its error word): throws
// UnitsOverflow when a step's units did not fit the unit buffer.
void check_units(pj_ctx* ctx, int herr);
// Grow the unit buffers to hold `units` (and a margin) before a rerun.
void grow_units(pj_ctx* ctx, int64_t units, cudaStream_t st);
// Elapsed milliseconds of an event pair returned by run_refine (0 if -1).
float refine_ms(pj_ctx* ctx, int ev);
// Per-step record of a join: units, tests and refinement time of every
// refinement launch, read back once after the join's final synchronization.
struct StepLog : StepLogData {
  static constexpr int MAX = 16;
  // Record one refinement step (after run_refine on `st`).
  void add(pj_ctx* ctx, const UnitCount& uc, int event, const StepSpec& sp, cudaStream_t st);
  // JSON array of the steps; also sums refinement ms per precision and units.
  // host_snap: the step snapshots already copied to the host (else read
  // from the device here)
  std::string json(pj_ctx* ctx, double* ms32, double* ms64, int64_t* units_total,
                   const long long* host_snap = nullptr) const;
};
// Pair-setup: origin (pair-local frame), box MINDIST, anchor distance.
// n_live (device, may be null): pairs at or past *n_live are padding of a
// fixed-capacity join and are marked REMOVED.
void setup_pairs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n_pairs, double tau, bool within,
                 cudaStream_t st, const int64_t* n_live = nullptr);

// ---- explicit-buffer launchers (refine.cu / join.cu), used by entry points
// that bring their own scratch instead of the context workspace
struct PairBufs {
  const int32_t* pr;
  const int32_t* ps;
  float4* origin;
  float* thr;
  double* box_lb;
  double* anc_ub;
  uint8_t* status;
  uint8_t* lod0;
  uint8_t* exact;
  double* dlo;
  double* dhi;
  double* d;
  void* lb;
  void* ub;
  void* mid;
  int64_t* ucount;   // [1] unit counter of the builder
  int* err;          // device error word
  Tile* tiles;
  unsigned long long* counters;  // [3]: tests, tile counter, straddle-queue count
  int4* queue;                   // straddling facet pairs (see k_cross_fix)
  unsigned qcap;
  uint8_t* flag;                 // [n] pair proven (early exit), may be null
  int64_t tiles_cap;             // units the tile array holds
};
void setup_pairs_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const PairBufs& b,
                      cudaStream_t st);
UnitCount build_tiles_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const StepSpec& sp,
                           const PairBufs& b, int64_t tiles_cap, cudaStream_t st);
void init_bounds_bufs(pj_ctx* ctx, int64_t n, const StepSpec& sp, const PairBufs& b, cudaStream_t st);
void run_refine_bufs(pj_ctx* ctx, const pj_set* R, const pj_set* S, UnitCount units, const StepSpec& sp,
                     const PairBufs& b, int* err, cudaStream_t st);
// single-block exclusive scan, n <= 4096, no allocation
void scan_small_i64(pj_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);

// ---- results (join.cu)
void alloc_result(pj_result* res, int64_t n);
int64_t gather_results(pj_ctx* ctx, int64_t n, pj_result* res, cudaStream_t st);
// gather_results in two halves: the device part (compaction and the copy of
// capacity n into pinned staging, no synchronization) and, after the
// stream is synchronized, the host part.
void gather_device(pj_ctx* ctx, int64_t n, cudaStream_t st);
// Destroy the captured join graphs of a context.
void graphs_clear(pj_ctx* ctx);
int64_t gather_host(pj_ctx* ctx, int64_t n, pj_result* res);
void mark_exact(pj_ctx* ctx, int64_t n, cudaStream_t st);

// ---- decide (join.cu)
void decide_within(pj_ctx* ctx, int64_t n_pairs, double tau, const StepSpec& sp, cudaStream_t st);

// ---- set building (api.cu)
// Facet records, chunk and block boxes of LoDs [0, lod_end) (default: all)
// and the object boxes, into the set's allocated buffers (foff / coff / boff
// already on the device); kernel errors go to ctx->d_err.
void build_set_kernels(pj_ctx* ctx, pj_set* s, const RawLod* raw, cudaStream_t st, int* err = nullptr,
                       int lod_end = -1);
// The per-chunk maxima of hd and ph of LoD l (the .w words of its chunk
// boxes) from the raw arrays alone, for a LoD whose records are built on
// demand (the learned start LoD reads them for every pair).
void chunk_hd_ph(pj_ctx* ctx, pj_set* s, int l, const RawLod& raw, cudaStream_t st);
// A set whose LoDs from s->lazy_from on are built on demand: the records
// and boxes of the R objects of the pairs a step selects (status `want`,
// lod0 <= step) that are not built yet; no-op for other sets and LoDs.
void ensure_lod(pj_ctx* ctx, const pj_set* R, int lod, int64_t n_pairs, const int32_t* pr, const uint8_t* status,
                const uint8_t* lod0, uint8_t want, int step, cudaStream_t st);

// ---- triangle distance batch (refine.cu)
void tri_dist_batch(pj_ctx* ctx, const float* P, const float* Q, int64_t n, bool fp64, double* out,
                    double* err, cudaStream_t st);

// ---- kNN (knn.cu)

// ---- MLP (mlp.cu)
void mlp_forward(pj_ctx* ctx, const float* feats, int64_t n, float* out, cudaStream_t st);
// Predicted log1p(d) of the candidate pairs in WS_PR / WS_PS (into WS_PRED).
// n_live: the live pair count of a fixed-capacity (graph) join, rows at or
// beyond it are padding (nullptr: all n rows are pairs)
const float* propose(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, cudaStream_t st,
                     const int64_t* n_live = nullptr);
// lod0 of the undecided pairs from the predictions (within-tau start LoD).
void start_lod(pj_ctx* ctx, const pj_set* R, const pj_set* S, int64_t n, const float* pred, double tau,
               cudaStream_t st);
// start LoD rule: the band half-width of a prediction in log1p units and the
// fraction of the Hausdorff terms a distance gap must reach
constexpr float PRED_BAND = 0.15f;
constexpr float START_MARGIN = 0.5f;
void pair_features(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps,
                   int64_t n, float* out, cudaStream_t st, const int64_t* n_live = nullptr);

// Device and pinned-host allocations made by the library (all contexts of
// the process), reported by pj_get_stats as "allocs": lets a caller check
// that an entry point allocated nothing.
extern std::atomic<unsigned long long> g_allocs;
inline void note_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

// count a kernel launch of the library (for the benchmark's launch tally)
inline void count_launch(pj_ctx* ctx, int n = 1) { ctx->launches += (unsigned long long)n; }

// host timing helper
struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

// State of a within join between the issue of its device work and its
// completion (join.cu).
struct WithinTail {
  pj_ctx* ctx;
  const pj_set* R;
  const pj_set* S;
  pj_query q;
  cudaStream_t st;
  double tau;
  bool fp64, learned, spec, graph_ok;
  int64_t n, cap, nn;
  const char* gmode;
  StepLog log;
  unsigned long long launches0;
  Timer tall, tseq;
  double ms_filter;
  bool reran = false;
};

// A within join whose device work may still be in flight when it returns:
// with pend set, a join replayed from a graph returns PJ_PENDING after the
// launch and fills *pend; within_finish then waits for it and completes it.
// Any other join completes before returning.
constexpr pj_status PJ_PENDING = (pj_status)1;
// The context's twin (created on first use); its settings follow ctx's.
pj_ctx* join_twin(pj_ctx* ctx);
// The autotuner's choice stored in `from` for the workload set on `to` (it
// stays set); false when nothing is stored yet.
bool tuned_apply(pj_ctx* from, pj_ctx* to, const pj_set* R, const pj_set* S, const pj_query* q);
pj_status join_within_issue(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                            cudaStream_t st, std::string& stats, WithinTail* pend);
pj_status within_finish(WithinTail& w, pj_result* out, std::string& stats);
pj_status join_within(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                      cudaStream_t st, std::string& stats);

}  // namespace pj
