// Join orchestration on one GPU: MBB filter -> per-LoD [tile build ->
// refine -> decide] from the coarsest LoD (or the autotuned start step) to
// the original surfaces (section 3.1 overview: resolve after each LoD what
// its bounds decide, refine the rest at the next LoD), an FP64 re-decide
// pass for the single-precision path, optional exact distances, and the
// compaction of the result pairs.
#include <algorithm>
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace pj {

// ------------------------------------------------------------------ scan
constexpr int SCAN_T = 512;
constexpr int SCAN_I = 8;
constexpr int SCAN_B = SCAN_T * SCAN_I;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int64_t before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void k_block_sums(const int64_t* in, int64_t n, int64_t* bsum) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_I;
  int64_t v = 0;
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k)
    if (base + k < n) v += in[base + k];
  int64_t tot;
  block_excl_scan(v, sh, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int64_t* in, int64_t n, const int64_t* boff, int64_t nb, int64_t* out) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_I;
  int64_t loc[SCAN_I];
  int64_t v = 0;
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    loc[k] = base + k < n ? in[base + k] : 0;
    v += loc[k];
  }
  int64_t tot;
  int64_t run = block_excl_scan(v, sh, &tot) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    if (base + k < n) out[base + k] = run;
    run += loc[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = boff ? boff[nb] : tot;
}

// Temporary words needed by scan_i64 for n values (all recursion levels).
int64_t scan_tmp_words(int64_t n) {
  int64_t w = 0;
  while (n > SCAN_B) {
    int64_t nb = (n + SCAN_B - 1) / SCAN_B;
    w += 2 * nb + 1;
    n = nb;
  }
  return w;
}

void scan_i64(pj_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, int64_t* tmp) {
  if (n == 0) {
    PJ_CK(cudaMemsetAsync(out, 0, 8, st));
    return;
  }
  int64_t nb = (n + SCAN_B - 1) / SCAN_B;
  if (nb == 1) {
    k_scan_apply<<<1, SCAN_T, 0, st>>>(in, n, nullptr, 0, out);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    return;
  }
  bool own = tmp == nullptr;
  if (own) {
    note_alloc();
    PJ_CK(cudaMallocAsync((void**)&tmp, (size_t)scan_tmp_words(n) * 8, st));
  }
  int64_t* bsum = tmp;
  int64_t* boff = tmp + nb;
  k_block_sums<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, bsum);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, bsum, boff, nb, st, tmp + 2 * nb + 1);
  k_scan_apply<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, boff, nb, out);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  if (own) PJ_CK(cudaFreeAsync(tmp, st));
}

void scan_small_i64(pj_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
  if (n > SCAN_B) throw ApiError{PJ_EINVAL, "scan_small_i64: n above one block"};
  if (n == 0) {
    PJ_CK(cudaMemsetAsync(out, 0, 8, st));
    return;
  }
  k_scan_apply<<<1, SCAN_T, 0, st>>>(in, n, nullptr, 0, out);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// ------------------------------------------------------------------ decide


template <bool F64>
__device__ __forceinline__ double load_bound(const void* a, int64_t p) {
  if (F64) return bits2d(((const unsigned long long*)a)[p]);
  return (double)bits2f(((const unsigned*)a)[p]);
}

// within-tau / intersection decision of the refined pairs (section 3.1:
// ub <= tau -> result, lb > tau -> pruned, else next LoD).  At the original
// surfaces the FP64 bracket is a point; a single-precision bracket that
// still straddles tau sends the pair to the FP64 re-decide pass.
template <bool F64>
__global__ void k_decide_within(int64_t n, uint8_t* status, const uint8_t* lod0, uint8_t want, int step, int full,
                                double tau, const void* lb, const void* ub, const void* mid, double* dlo,
                                double* dhi, double* d, uint8_t* exact, unsigned long long* cnt,
                                const uint8_t* flag, const double* box_lb, const double* anc_ub) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (!(status[p] == want && lod0[p] <= step)) return;
  double l = load_bound<F64>(lb, p), u = load_bound<F64>(ub, p);
  if (flag && flag[p]) {
    // Some units were skipped, and which ones depends on timing: report a
    // bracket that does not (box distance .. threshold / anchor distance),
    // or the exact 0 of a certified crossing.
    if (u <= 0.0) {
      l = 0.0;
      u = 0.0;
    } else {
      l = box_lb[p];
      u = fmin(tau, anc_ub[p]);
    }
  }
  if (want == MAKE_EXACT) {
    dlo[p] = l;
    dhi[p] = u;
    d[p] = u;
    exact[p] = 1;
    status[p] = CONFIRMED;
    return;
  }
  if (u <= tau) {
    status[p] = CONFIRMED;
    dlo[p] = l;
    dhi[p] = u;
    if (full && u == 0.0) {
      exact[p] = 1;
      d[p] = 0.0;
    } else if (full && !(flag && flag[p])) {
      exact[p] = F64 ? 1 : 2;
      d[p] = F64 ? u : load_bound<F64>(mid, p);
    } else {
      exact[p] = 0;
      d[p] = 0.5 * (l + u);
    }
    atomicAdd(&cnt[2], 1ULL);
  } else if (l > tau || (full && F64)) {
    status[p] = REMOVED;
    atomicAdd(&cnt[3], 1ULL);
  } else {
    // still open: keep the tightest upper bound (it lets the next step skip
    // facet pairs that cannot attain the minimum)
    dhi[p] = fmin(dhi[p], u);
    if (full) {
      status[p] = REDECIDE;
      atomicAdd(&cnt[4], 1ULL);
    }
  }
}

void decide_within(pj_ctx* ctx, int64_t n, double tau, const StepSpec& sp, cudaStream_t st) {
  if (n == 0) return;
  int th = 256;
  unsigned g = (unsigned)((n + th - 1) / th);
  auto status = (uint8_t*)ctx->ws[WS_STATUS].p;
  auto lod0 = (const uint8_t*)ctx->ws[WS_LOD0].p;
  const uint8_t* flag = sp.early ? (const uint8_t*)ctx->ws[WS_FLAG].p : nullptr;
  const double* box_lb = (const double*)ctx->ws[WS_BOXLB].p;
  const double* anc_ub = (const double*)ctx->ws[WS_ANCUB].p;
  if (sp.fp64)
    k_decide_within<true><<<g, th, 0, st>>>(n, status, lod0, sp.want, sp.step, sp.full, tau, ctx->ws[WS_LB].p,
                                             ctx->ws[WS_UB].p, ctx->ws[WS_MID].p, (double*)ctx->ws[WS_DLO].p,
                                             (double*)ctx->ws[WS_DHI].p, (double*)ctx->ws[WS_D].p,
                                             (uint8_t*)ctx->ws[WS_EXACT].p, ctx->d_counters, flag, box_lb, anc_ub);
  else
    k_decide_within<false><<<g, th, 0, st>>>(n, status, lod0, sp.want, sp.step, sp.full, tau, ctx->ws[WS_LB].p,
                                              ctx->ws[WS_UB].p, ctx->ws[WS_MID].p, (double*)ctx->ws[WS_DLO].p,
                                              (double*)ctx->ws[WS_DHI].p, (double*)ctx->ws[WS_D].p,
                                              (uint8_t*)ctx->ws[WS_EXACT].p, ctx->d_counters, flag, box_lb, anc_ub);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

__global__ void k_mark_exact(int64_t n, uint8_t* status, const uint8_t* exact) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (status[p] == CONFIRMED && exact[p] != 1) status[p] = MAKE_EXACT;
}

void mark_exact(pj_ctx* ctx, int64_t n, cudaStream_t st) {
  int th = 256;
  k_mark_exact<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, (uint8_t*)ctx->ws[WS_STATUS].p,
                                                             (const uint8_t*)ctx->ws[WS_EXACT].p);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// ------------------------------------------------------------------ results

__global__ void k_flag_status(int64_t n, const uint8_t* status, uint8_t want, int64_t* flag) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) flag[p] = status[p] == want ? 1 : 0;
}

struct ResultPack {
  int32_t* r;
  int32_t* s;
  double* dlo;
  double* dhi;
  double* d;
  uint8_t* exact;
};

__global__ void k_compact(int64_t n, const uint8_t* status, const int64_t* off, const int32_t* pr,
                          const int32_t* ps, const double* dlo, const double* dhi, const double* d,
                          const uint8_t* exact, ResultPack out) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n || status[p] != CONFIRMED) return;
  int64_t w = off[p];
  out.r[w] = pr[p];
  out.s[w] = ps[p];
  out.dlo[w] = dlo[p];
  out.dhi[w] = dhi[p];
  out.d[w] = d[p];
  out.exact[w] = exact[p];
}

struct HostResult {
  void* block = nullptr;
};

// Host arrays for n results inside one block (pageable; the copy from the
// device goes through the context's pinned staging buffer).
void alloc_result(pj_result* res, int64_t n) {
  size_t per = 4 + 4 + 8 + 8 + 8 + 1;
  size_t bytes = std::max<size_t>(64, (size_t)n * per + 64);
  void* blk = malloc(bytes);
  if (!blk) throw ApiError{PJ_ENOMEM, "host allocation of the result failed"};
  char* c = (char*)blk;
  res->n = n;
  res->d_lo = (double*)c;
  c += 8 * n;
  res->d_hi = (double*)c;
  c += 8 * n;
  res->d = (double*)c;
  c += 8 * n;
  res->r = (int32_t*)c;
  c += 4 * n;
  res->s = (int32_t*)c;
  c += 4 * n;
  res->exact = (uint8_t*)c;
  res->priv = blk;
}

static void* stage(pj_ctx* ctx, size_t bytes) {
  if (ctx->h_stage_cap < bytes) {
    if (ctx->h_stage) PJ_CK(cudaFreeHost(ctx->h_stage));
    ctx->h_stage = nullptr;
    size_t cap = std::max(bytes, ctx->h_stage_cap * 2);
    note_alloc();
    PJ_CK(cudaMallocHost(&ctx->h_stage, cap));
    ctx->h_stage_cap = cap;
  }
  return ctx->h_stage;
}

// Status block behind the results in the pinned stage: the error word, the
// join counters and the per-step snapshots, copied in stream order after
// the last kernel so that one synchronization makes all of it readable.
constexpr size_t RES_PER = 4 + 4 + 8 + 8 + 8 + 1;
constexpr size_t STATUS_ERR = 0, STATUS_TOTAL = 8, STATUS_CNT = 64, STATUS_SNAP = 256;
constexpr size_t STATUS_BYTES = STATUS_SNAP + sizeof(long long) * 4 * StepLog::MAX;
static size_t status_at(int64_t n) { return ((size_t)n * RES_PER + 8 + 255) & ~size_t(255); }

void gather_device(pj_ctx* ctx, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int th = 256;
  unsigned g = (unsigned)((n + th - 1) / th);
  auto flag = (int64_t*)ws_get(ctx, WS_TCOUNT, (n + 1) * 8, st);
  auto off = (int64_t*)ws_get(ctx, WS_SCAN, (n + 1) * 8, st);
  auto tmp = (int64_t*)ws_get(ctx, WS_TMP, (scan_tmp_words(n) + 8) * 8, st);
  auto status = (const uint8_t*)ctx->ws[WS_STATUS].p;
  k_flag_status<<<g, th, 0, st>>>(n, status, CONFIRMED, flag);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  scan_i64(ctx, flag, off, n, st, tmp);
  const size_t per = 4 + 4 + 8 + 8 + 8 + 1;
  char* dev = (char*)ws_get(ctx, WS_RES, (size_t)n * per + 64, st);
  ResultPack pk;
  pk.dlo = (double*)dev;
  pk.dhi = pk.dlo + n;
  pk.d = pk.dhi + n;
  pk.r = (int32_t*)(pk.d + n);
  pk.s = pk.r + n;
  pk.exact = (uint8_t*)(pk.s + n);
  k_compact<<<g, th, 0, st>>>(n, status, off, (const int32_t*)ctx->ws[WS_PR].p, (const int32_t*)ctx->ws[WS_PS].p,
                              (const double*)ctx->ws[WS_DLO].p, (const double*)ctx->ws[WS_DHI].p,
                              (const double*)ctx->ws[WS_D].p, (const uint8_t*)ctx->ws[WS_EXACT].p, pk);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  char* h = (char*)stage(ctx, status_at(n) + STATUS_BYTES);
  PJ_CK(cudaMemcpyAsync(h, dev, (size_t)n * per, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaMemcpyAsync(h + (size_t)n * per, off + n, 8, cudaMemcpyDeviceToHost, st));
}

// total (device, may be null): the filter's pair count, when the filter ran
// inside the sequence
void stage_status(pj_ctx* ctx, int64_t n, int steps, cudaStream_t st, const int64_t* total = nullptr) {
  char* h = (char*)stage(ctx, status_at(n) + STATUS_BYTES) + status_at(n);
  PJ_CK(cudaMemcpyAsync(h + STATUS_ERR, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (total) PJ_CK(cudaMemcpyAsync(h + STATUS_TOTAL, total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaMemcpyAsync(h + STATUS_CNT, ctx->d_counters, 15 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        st));
  if (steps > 0)
    PJ_CK(cudaMemcpyAsync(h + STATUS_SNAP, ctx->d_snap, sizeof(long long) * 4 * steps, cudaMemcpyDeviceToHost, st));
}

const char* staged_status(pj_ctx* ctx, int64_t n) { return (const char*)ctx->h_stage + status_at(n); }

int64_t gather_host(pj_ctx* ctx, int64_t n, pj_result* res) {
  if (n == 0) {
    alloc_result(res, 0);
    return 0;
  }
  const size_t per = 4 + 4 + 8 + 8 + 8 + 1;
  const char* h = (const char*)ctx->h_stage;
  int64_t m = 0;
  memcpy(&m, h + (size_t)n * per, 8);
  alloc_result(res, m);
  memcpy(res->d_lo, h, (size_t)m * 8);
  memcpy(res->d_hi, h + (size_t)n * 8, (size_t)m * 8);
  memcpy(res->d, h + (size_t)n * 16, (size_t)m * 8);
  memcpy(res->r, h + (size_t)n * 24, (size_t)m * 4);
  memcpy(res->s, h + (size_t)n * 28, (size_t)m * 4);
  memcpy(res->exact, h + (size_t)n * 32, (size_t)m);
  return m;
}

// Copy the CONFIRMED pairs (in pair order = (r, s) order) to the host: the
// compacted arrays (capacity n) and their count come back in one copy and
// one synchronization.
int64_t gather_results(pj_ctx* ctx, int64_t n, pj_result* res, cudaStream_t st) {
  gather_device(ctx, n, st);
  if (n) PJ_CK(cudaStreamSynchronize(st));
  return gather_host(ctx, n, res);
}

// ------------------------------------------------------------------ driver

void StepLog::add(pj_ctx* ctx, const UnitCount& uc, int event, const StepSpec& sp, cudaStream_t st) {
  if (n >= MAX) return;
  long long* d = ctx->d_snap + 4 * n;
  if (uc.count < 0) PJ_CK(cudaMemcpyAsync(d, uc.dev, 8, cudaMemcpyDeviceToDevice, st));
  PJ_CK(cudaMemcpyAsync(d + 1, ctx->d_counters, 16, cudaMemcpyDeviceToDevice, st));
  // units left after the mask pass (counter 13, written by run_refine)
  masked[n] = uc.count != 0 && sp.full && (!sp.fp64 || sp.cull);
  if (masked[n]) PJ_CK(cudaMemcpyAsync(d + 3, ctx->d_counters + 13, 8, cudaMemcpyDeviceToDevice, st));
  ev[n] = event;
  units[n] = uc.count;
  f64[n] = sp.fp64;
  full[n] = sp.full;
  ++n;
}

std::string StepLog::json(pj_ctx* ctx, double* ms32, double* ms64, int64_t* units_total,
                          const long long* host_snap) const {
  long long snap[MAX * 4];
  if (n && host_snap) memcpy(snap, host_snap, sizeof(long long) * 4 * n);
  else if (n) PJ_CK(cudaMemcpy(snap, ctx->d_snap, sizeof(long long) * 4 * n, cudaMemcpyDeviceToHost));
  std::string out = "[";
  long long prev32 = 0, prev64 = 0;
  *ms32 = *ms64 = 0;
  *units_total = 0;
  for (int i = 0; i < n; ++i) {
    const float kms = refine_ms(ctx, ev[i]);
    (f64[i] ? *ms64 : *ms32) += kms;
    const long long u = units[i] >= 0 ? units[i] : snap[4 * i];
    *units_total += u;
    char buf[256];
    snprintf(buf, sizeof buf,
             "%s{\"step\":%d,\"prec\":\"%s\",\"full\":%d,\"tiles\":%lld,\"tiles_run\":%lld,\"tests\":%lld,"
             "\"refine_ms\":%.4f}",
             i ? "," : "", i, f64[i] ? "fp64" : "fp32", full[i] ? 1 : 0, u, masked[i] ? snap[4 * i + 3] : u,
             (snap[4 * i + 1] - prev32) + (snap[4 * i + 2] - prev64), kms);
    prev32 = snap[4 * i + 1];
    prev64 = snap[4 * i + 2];
    out += buf;
  }
  return out + "]";
}


__global__ void k_lod0_floor(int64_t n, uint8_t* lod0, uint8_t s) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n && lod0[p] < s) lod0[p] = s;
}

// ------------------------------------------------------------------ graphs
// PJ_USE_GRAPH: everything after the filter's one synchronization -- pair
// setup, every LoD step, the FP64 passes, compaction and the result copy --
// is a fixed sequence for a given capacity (the candidate list is padded to
// the next power of two with pairs marked REMOVED, whose work is empty).
// It is captured into a CUDA graph once per key and replayed afterwards;
// the key holds every host-side launch parameter (set shapes and device
// pointers, workspace addresses, query, capacity, kernel choices), so a
// replay issues exactly the launches a direct run would.

static uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
  return h;
}

static std::string graph_key(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, int64_t cap) {
  uint64_t h = 1469598103934665603ULL;
  for (const pj_set* X : {R, S}) {
    h = fnv(h, &X->n, sizeof X->n);
    h = fnv(h, &X->L, sizeof X->L);
    h = fnv(h, &X->mbb, sizeof X->mbb);
    h = fnv(h, &X->anchor, sizeof X->anchor);
    for (int l = 0; l < X->L; ++l) {
      const LodData& d = X->lod[l];
      const void* ptrs[6] = {d.fac, d.foff, d.chunk, d.coff, d.blk, d.boff};
      const int64_t sz[4] = {d.F, d.C, d.B, d.maxF};
      h = fnv(h, ptrs, sizeof ptrs);
      h = fnv(h, sz, sizeof sz);
    }
    // a LoD built on demand reads the chunk's raw arrays inside the sequence
    h = fnv(h, &X->lazy_from, sizeof X->lazy_from);
    h = fnv(h, &X->lazy_raw, sizeof X->lazy_raw);
    h = fnv(h, &X->lazy_state, sizeof X->lazy_state);
    h = fnv(h, &X->lazy_list, sizeof X->lazy_list);
  }
  for (int i = 0; i < WS_COUNT; ++i) {
    h = fnv(h, &ctx->ws[i].p, sizeof(void*));
    h = fnv(h, &ctx->ws[i].cap, sizeof(size_t));
  }
  h = fnv(h, &ctx->h_stage, sizeof(void*));
  h = fnv(h, &ctx->mlp_w, sizeof(void*));   // the proposal's weights are read in place
  h = fnv(h, &ctx->h_stage_cap, sizeof(size_t));
  const int knobs[5] = {ctx->refine_variant, ctx->sched_start, ctx->ctas_per_sm, ctx->refine_split, ctx->refine_tail};
  h = fnv(h, knobs, sizeof knobs);
  char buf[200];
  snprintf(buf, sizeof buf, "%016llx.p%d.t%.17g.x%d.f%u.c%lld", (unsigned long long)h, (int)q->pred, q->tau,
           (int)q->prec, q->flags, (long long)cap);
  return buf;
}

// Graphs kept per context (the oldest is dropped beyond): a streamed R whose
// chunk arrays the caller keeps in device memory gives every chunk its own
// key (the kernels read those arrays in place), so the cache holds a whole
// pass of chunks and replays them on the next join.
constexpr size_t MAX_GRAPHS = 160;

static pj_ctx::GraphEntry* graph_find(pj_ctx* ctx, const std::string& key) {
  for (auto& g : ctx->graphs)
    if (g.key == key) return &g;
  return nullptr;
}

void graphs_clear(pj_ctx* ctx) {
  for (auto& g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
}

static int64_t spec_cap_get(const pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau) {
  for (const auto& e : ctx->spec_caps)
    if (e.nR == R->n && e.LR == R->L && e.sid == S->uid && e.tau == tau) return e.cap;
  return 0;
}

static void spec_cap_set(pj_ctx* ctx, const pj_set* R, const pj_set* S, double tau, int64_t cap) {
  for (auto& e : ctx->spec_caps)
    if (e.nR == R->n && e.LR == R->L && e.sid == S->uid && e.tau == tau) {
      e.cap = cap;
      return;
    }
  if (ctx->spec_caps.size() >= 16) ctx->spec_caps.erase(ctx->spec_caps.begin());
  ctx->spec_caps.push_back(pj_ctx::SpecCap{R->n, R->L, S->uid, tau, cap});
}

static pj_status join_within_once(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q,
                                  pj_result* out, cudaStream_t st, std::string& stats, WithinTail* pend = nullptr);

// The part of a within join after its device work: read the staged status
// (a speculated capacity that did not hold reruns the join unspeculated),
// copy the results out and write the stats.  w.reran is set when the join
// ran again (its results and stats are then the rerun's).
static pj_status within_tail(WithinTail& w, double ms_seq, pj_result* out, std::string& stats) {
  pj_ctx* ctx = w.ctx;
  const pj_set* R = w.R;
  const pj_set* S = w.S;
  const pj_query* q = &w.q;
  cudaStream_t st = w.st;
  const double tau = w.tau;
  const bool fp64 = w.fp64, learned = w.learned, spec = w.spec, graph_ok = w.graph_ok;
  int64_t& n = w.n;
  const int64_t cap = w.cap, nn = w.nn;
  const char* gmode = w.gmode;
  StepLog& log = w.log;
  const unsigned long long launches0 = w.launches0;
  const Timer& tall = w.tall;
  const double ms_filter = w.ms_filter;
  // after the synchronization the error word, the counters and the step
  // snapshots are in the pinned stage (with candidates; else read here)
  int herr = 0;
  unsigned long long cnt[8];
  const long long* snap = nullptr;
  if (nn > 0) {
    const char* h = staged_status(ctx, nn);
    memcpy(&herr, h + STATUS_ERR, sizeof(int));
    memcpy(cnt, h + STATUS_CNT, sizeof cnt);
    snap = (const long long*)(h + STATUS_SNAP);
    if (spec) {
      // the speculated capacity held, and the ranked emit sufficed?
      int64_t total = 0;
      unsigned long long ov = 0;
      memcpy(&total, h + STATUS_TOTAL, sizeof total);
      memcpy(&ov, h + STATUS_CNT + 12 * sizeof(unsigned long long), sizeof ov);
      if (ov != 0 || total > cap) {
        spec_cap_set(ctx, R, S, tau, 0);   // this join runs unspeculated (and sets the capacity again)
        ++ctx->spec_misses;
        w.reran = true;
        return join_within_once(ctx, R, S, q, out, st, stats);
      }
      n = total;
    }
  } else {
    PJ_CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PJ_CK(cudaMemcpyAsync(cnt, ctx->d_counters, sizeof cnt, cudaMemcpyDeviceToHost, st));
    PJ_CK(cudaStreamSynchronize(st));
  }
  // a step whose units overflowed the buffer voids the join (rerun)
  check_units(ctx, herr);
  Timer tg;
  const int64_t m = gather_host(ctx, nn, out);
  double refine_ms_fp32 = 0, refine_ms_fp64 = 0;
  int64_t tiles_total = 0;
  const std::string steps = log.json(ctx, &refine_ms_fp32, &refine_ms_fp64, &tiles_total, snap);
  float graph_ms = 0.f;
  if (!strcmp(gmode, "replay")) PJ_CK(cudaEventElapsedTime(&graph_ms, ctx->ev[60], ctx->ev[61]));
  char buf[1500];
  snprintf(buf, sizeof buf,
           "{\"pred\":\"within\",\"tau\":%.17g,\"prec\":\"%s\",\"mlp\":%d,\"graph\":\"%s\",\"spec\":%d,"
           "\"graph_ms\":%.4f,"
           "\"capacity\":%lld,"
           "\"candidates\":%lld,\"results\":%lld,"
           "\"tests_fp32\":%llu,\"tests_fp64\":%llu,\"tests_culled\":%llu,\"tests_needed\":%llu,\"confirmed\":%llu,"
           "\"removed\":%llu,\"redecide\":%llu,"
           "\"tiles\":%lld,\"ms_filter\":%.3f,\"ms_seq\":%.3f,\"ms_gather\":%.3f,\"ms_total\":%.3f,"
           "\"refine_ms_fp32\":%.4f,\"refine_ms_fp64\":%.4f,\"launches\":%llu,\"steps\":",
           tau, fp64 ? "fp64" : "fp32", learned ? 1 : 0, gmode, spec ? 1 : 0, graph_ms, (long long)nn, (long long)n,
           (long long)m,
           cnt[0],
           cnt[1], cnt[5], cnt[6], cnt[2], cnt[3], cnt[4], (long long)tiles_total,
           ms_filter, ms_seq, tg.ms(), tall.ms(), refine_ms_fp32, refine_ms_fp64, ctx->launches - launches0);
  stats = std::string(buf) + steps + "}";
  JoinSummary& js = ctx->last_sum;
  js.candidates = n;
  js.results = m;
  js.units = tiles_total;
  js.tests32 = cnt[0];
  js.tests64 = cnt[1];
  js.confirmed = cnt[2];
  js.removed = cnt[3];
  js.ms_filter = ms_filter;
  js.ms_total = tall.ms();
  js.refine_ms32 = refine_ms_fp32;
  js.refine_ms64 = refine_ms_fp64;
  js.launches = ctx->launches - launches0;
  js.graph = !strcmp(gmode, "replay") ? 2 : (!strcmp(gmode, "captured") ? 1 : 0);
  js.ms_seq = ms_seq;
  js.graph_ms = graph_ms;
  js.spec = spec ? 1 : 0;
  if (herr & ERR_MBAR_TIMEOUT) return PJ_ETIMEOUT;
  if (herr & ERR_CAPACITY) throw ApiError{PJ_ENOMEM, "refinement units above the unit buffer"};
  if (herr & ERR_BOUNDS) return PJ_EBOUNDS;
  if (herr & ERR_NONFINITE) return PJ_ENONFINITE;   // data of a LoD built on demand
  if (graph_ok && !spec && filter_grid_kept(ctx, R, S, tau)) {
    // the next join of this shape speculates with a quarter of headroom
    int64_t c = 256;
    while (c < n + n / 4) c <<= 1;
    spec_cap_set(ctx, R, S, tau, c);
  }
  return PJ_OK;
}

static pj_status join_within_once(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q,
                                  pj_result* out, cudaStream_t st, std::string& stats, WithinTail* pend) {
  Timer tall;
  const unsigned long long launches0 = ctx->launches;
  const double tau = q->pred == PJ_INTERSECT ? 0.0 : q->tau;
  const bool fp64 = q->prec == PJ_PREC_FP64;
  const bool cull = (q->flags & PJ_TILE_PRUNE) != 0;
  const bool use_mlp = (q->flags & PJ_USE_MLP) != 0;
  if (use_mlp && !ctx->mlp_ready) throw ApiError{PJ_EINVAL, "PJ_USE_MLP needs trained or loaded proposal weights"};
  // the learned per-pair start, unless the autotuner fixed the schedule
  const bool learned = use_mlp && ctx->sched_start < 0;
  // fixed-capacity graph mode: not on the legacy default stream, nor in an
  // autotuning trial (whose steps count their units on the host first).  A
  // replay whose units overflow the buffer of the capture flags the join,
  // which runs again directly with a grown buffer (and a new graph).
  const bool graph_ok = (q->flags & PJ_USE_GRAPH) && st != nullptr && ctx->trial_unit_cap == 0;
  // Speculative mode (graph mode, the filter's grid kept: the chunks of a
  // streamed R after the first): the filter joins the captured sequence,
  // with the capacity of the last join of this shape, so a chunk's join is
  // one graph launch and one synchronization.  A chunk whose pairs exceed
  // that capacity (or need the filter's slow path) runs again unspeculated.
  const int64_t spec_cap = graph_ok && filter_grid_kept(ctx, R, S, tau) ? spec_cap_get(ctx, R, S, tau) : 0;
  const bool spec = spec_cap > 0;
  int* over = (int*)(ctx->d_counters + 12);   // the filter's slow-path / capacity word (zeroed with the counters)
  Timer tf;
  int64_t n = 0;
  if (!spec) {
    PJ_CK(cudaMemsetAsync(ctx->d_counters, 0, 15 * sizeof(unsigned long long), st));
    PJ_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
    n = filter_within(ctx, R, S, tau, st).n_pairs;
  }
  const int Lmax = std::max(R->L, S->L);
  auto deadline_hit = [&]() { return q->timeout_s > 0 && tall.ms() > q->timeout_s * 1000.0; };
  const bool graph = graph_ok && (spec || n > 0);
  int64_t cap = n;
  if (spec) {
    cap = spec_cap;
  } else if (graph) {
    cap = 256;
    while (cap < n) cap <<= 1;
  }
  const int64_t nn = cap;
  const int64_t* n_live_0 = graph ? (const int64_t*)ctx->ws[WS_ROFF].p + R->n : nullptr;   // (reset after a speculative filter)

  // the whole device sequence after the filter (with it, speculatively);
  // false on an expired deadline
  const int64_t* n_live = n_live_0;
  auto enqueue = [&](StepLog& log) -> bool {
    if (spec) {
      PJ_CK(cudaMemsetAsync(ctx->d_counters, 0, 15 * sizeof(unsigned long long), st));
      PJ_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
      filter_within_enqueue(ctx, R, S, tau, cap, over, st);
      n_live = (const int64_t*)ctx->ws[WS_ROFF].p + R->n;   // the filter may have grown its arrays
    }
    setup_pairs(ctx, R, S, nn, tau, true, st, n_live);
    if (learned) start_lod(ctx, R, S, nn, propose(ctx, R, S, nn, st, n_live), tau, st);
    if (ctx->sched_start > 0) {
      // autotuned schedule: no pair is refined before this step
      int th = 256;
      k_lod0_floor<<<(unsigned)((nn + th - 1) / th), th, 0, st>>>(nn, (uint8_t*)ctx->ws[WS_LOD0].p,
                                                                  (uint8_t)ctx->sched_start);
      PJ_CK(cudaGetLastError());
      PJ_COUNT_LAUNCH;
    }
    ctx->ev_used = 0;
    // with a fixed start step (autotuned schedule, no learned start) the
    // steps before it select no pair: they are not enqueued at all
    const int first = ctx->sched_start > 0 ? std::min(ctx->sched_start, Lmax - 1) : 0;
    for (int step = first; step < Lmax; ++step) {
      if (deadline_hit()) return false;
      StepSpec sp;
      sp.rerun_ok = true;
      sp.lodR = std::max(0, step - (Lmax - R->L));
      sp.lodS = std::max(0, step - (Lmax - S->L));
      sp.full = step == Lmax - 1;
      sp.fp64 = fp64;
      sp.cull = cull;
      sp.want = UNDECIDED;
      sp.step = step;
      // early exit (with pruning on): coarse steps only report a bracket, and
      // at full resolution an intersection test's answer is exactly 0
      sp.early = cull && (!sp.full || tau == 0.0);
      init_bounds(ctx, nn, sp, st);
      UnitCount uc = build_tiles(ctx, R, S, nn, sp, st);
      const int ev = run_refine(ctx, R, S, uc, sp, st);
      decide_within(ctx, nn, tau, sp, st);
      log.add(ctx, uc, ev, sp, st);
    }
    if (!fp64) {
      // pairs whose single-precision bracket still straddles tau at full
      // resolution (status REDECIDE) are refined again in double precision;
      // the decision only asks d <= tau, so units farther apart than tau may
      // be skipped
      StepSpec sp;
      sp.rerun_ok = true;
      sp.lodR = R->L - 1;
      sp.lodS = S->L - 1;
      sp.full = true;
      sp.fp64 = true;
      sp.cull = cull;
      sp.want = REDECIDE;
      sp.step = Lmax - 1;
      init_bounds(ctx, nn, sp, st);
      UnitCount uc = build_tiles(ctx, R, S, nn, sp, st);
      const int ev = run_refine(ctx, R, S, uc, sp, st);
      decide_within(ctx, nn, tau, sp, st);
      log.add(ctx, uc, ev, sp, st);
    }
    if (q->flags & PJ_EXACT_DIST) {
      int th = 256;
      k_mark_exact<<<(unsigned)((nn + th - 1) / th), th, 0, st>>>(nn, (uint8_t*)ctx->ws[WS_STATUS].p,
                                                                  (const uint8_t*)ctx->ws[WS_EXACT].p);
      PJ_CK(cudaGetLastError());
      PJ_COUNT_LAUNCH;
      // every result pair has d <= tau, so its closest facet pair lies in a
      // unit within tau: pruned units cannot hold the minimum
      StepSpec sp;
      sp.rerun_ok = true;
      sp.lodR = R->L - 1;
      sp.lodS = S->L - 1;
      sp.full = true;
      sp.fp64 = true;
      sp.cull = cull;
      sp.want = MAKE_EXACT;
      sp.step = Lmax - 1;
      init_bounds(ctx, nn, sp, st);
      UnitCount uc = build_tiles(ctx, R, S, nn, sp, st);
      const int ev = run_refine(ctx, R, S, uc, sp, st);
      decide_within(ctx, nn, tau, sp, st);
      log.add(ctx, uc, ev, sp, st);
    }
    gather_device(ctx, nn, st);
    stage_status(ctx, nn, log.n, st, spec ? n_live : nullptr);
    return true;
  };

  StepLog log;
  const char* gmode = "off";
  double ms_filter = 0;
  bool need_capture = false;
  Timer tseq;
  // a speculative sequence also reads the kept grid: its parameters join the key
  auto key_now = [&]() {
    std::string k = graph_key(ctx, R, S, q, cap);
    if (spec) {
      char b[48];
      snprintf(b, sizeof b, ".spec%016llx", (unsigned long long)fnv(1469598103934665603ULL, ctx->sgrid.grid,
                                                                    sizeof ctx->sgrid.grid));
      k += b;
    }
    return k;
  };
  if (nn > 0) {
    pj_ctx::GraphEntry* ge = graph ? graph_find(ctx, key_now()) : nullptr;
    ms_filter = spec ? 0.0 : tf.ms();
    if (ge) {
      // replay: one launch for the whole sequence
      if (deadline_hit()) return PJ_ETIMEOUT;
      PJ_CK(cudaEventRecord(ctx->ev[60], st));
      PJ_CK(cudaGraphLaunch(ge->exec, st));
      PJ_CK(cudaEventRecord(ctx->ev[61], st));
      ctx->launches += ge->kernels;
      static_cast<StepLogData&>(log) = ge->log;
      gmode = "replay";
      if (pend) {
        // the caller completes it (within_finish) after issuing other work
        *pend = WithinTail{ctx, R, S, *q, st, tau, fp64, learned, spec, graph_ok, n, cap, nn, gmode, log, launches0,
                           tall, tseq, ms_filter};
        return PJ_PENDING;
      }
    } else {
      if (!enqueue(log)) return PJ_ETIMEOUT;
      if (graph) gmode = "captured";
    }
    PJ_CK(cudaStreamSynchronize(st));
    need_capture = graph && !ge;
  } else {
    ms_filter = tf.ms();
  }
  const double ms_seq = tseq.ms();   // the post-filter sequence, issue to completion
  {
    WithinTail w{ctx, R, S, *q, st, tau, fp64, learned, spec, graph_ok, n, cap, nn, gmode, log, launches0, tall,
                 tseq, ms_filter};
    const pj_status rc = within_tail(w, ms_seq, out, stats);
    if (rc != PJ_OK || w.reran) return rc;
  }
  if (need_capture) {
    // the direct run sized every buffer: capture the same sequence now
    // (recorded, not executed) under a key taken after it
    const std::string key = key_now();
    const unsigned long long l0 = ctx->launches;
    StepLog glog;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      try {
        ok = enqueue(glog);
      } catch (...) {
        ok = false;   // not capturable: keep the direct run's results
      }
      if (cudaStreamEndCapture(st, &g) != cudaSuccess) ok = false;
    }
    (void)cudaGetLastError();
    const unsigned long long kernels = ctx->launches - l0;
    ctx->launches = l0;
    if (ok && g) {
      cudaGraphExec_t ex = nullptr;
      if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
        if (ctx->graphs.size() >= MAX_GRAPHS) {
          cudaGraphExecDestroy(ctx->graphs.front().exec);
          ctx->graphs.erase(ctx->graphs.begin());
        }
        pj_ctx::GraphEntry e;
        e.key = key;
        e.exec = ex;
        e.cap = cap;
        e.kernels = kernels;
        e.log = glog;
        ctx->graphs.push_back(e);
      }
      (void)cudaGetLastError();
    }
    if (g) cudaGraphDestroy(g);
  }
  return PJ_OK;
}

// A within / intersection join; reruns (at most three times) when a step's
// refinement units did not fit the unit buffer, which is then grown to the
// count that step needed.
pj_status join_within_issue(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                            cudaStream_t st, std::string& stats, WithinTail* pend) {
  try {
    return join_within_once(ctx, R, S, q, out, st, stats, pend);
  } catch (const UnitsOverflow& e) {
    grow_units(ctx, e.units, st);
    return join_within(ctx, R, S, q, out, st, stats);
  }
}

pj_status within_finish(WithinTail& w, pj_result* out, std::string& stats) {
  PJ_CK(cudaStreamSynchronize(w.st));
  try {
    return within_tail(w, w.tseq.ms(), out, stats);
  } catch (const UnitsOverflow& e) {
    // the replay's units overflowed the buffer of its capture: grow it and
    // run the join again (directly, then captured anew)
    grow_units(w.ctx, e.units, w.st);
    return join_within(w.ctx, w.R, w.S, &w.q, out, w.st, stats);
  }
}

pj_status join_within(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                      cudaStream_t st, std::string& stats) {
  for (int attempt = 0;; ++attempt) {
    try {
      return join_within_once(ctx, R, S, q, out, st, stats);
    } catch (const UnitsOverflow& e) {
      if (attempt >= 3) throw ApiError{PJ_ENOMEM, "refinement units above the unit buffer after resizing"};
      grow_units(ctx, e.units, st);
    }
  }
}

}  // namespace pj
