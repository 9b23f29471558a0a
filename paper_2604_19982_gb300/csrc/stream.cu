// Streamed join: R arrives in chunks, S stays resident (the double-stream
// chunked streaming of section 3.2, Algorithm 3, and the copy / compute
// overlap of section 3.3, Algorithm 5).
//
// A loader thread asks the caller's fill callback for chunk c, checks it,
// and packs its raw arrays (vertices once per distinct host array, vertex
// and face offsets, faces, hd / ph, anchors, and the facet / chunk / block
// offsets computed on the host) into one of two pinned host slots.  Arrays
// the caller already keeps in pinned host memory are not packed: they are
// copied to the device slot directly; arrays in device memory are read in
// place.  The calling thread copies a chunk to the matching device slot
// (one copy per run of packed arrays and one per pinned array) on the
// context's copy stream, builds the chunk's
// facet records and boxes on the build stream once that copy is done (into
// the derived buffers of its slot), and joins the chunk against S with the
// resident-set join.  The copy and the build of chunk c + 1 are issued
// before the join of chunk c starts, so they overlap that join; the loader
// packs chunk c + 2 meanwhile.  Results carry global R ids
// (the ids of chunk c continue those of chunk c - 1).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pj {

pj_status join_within(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                      cudaStream_t st, std::string& stats);
pj_status join_knn(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                   cudaStream_t st, std::string& stats);
pj_status join_autotuned(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                         cudaStream_t st, std::string& stats);
bool tuned_schedule_fixed(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q);

namespace {

constexpr size_t PACK_ALIGN = 256;
size_t pad(size_t x) { return (x + PACK_ALIGN - 1) & ~(PACK_ALIGN - 1); }

// Where the bytes of one array come from: packed into the pinned slot
// (pageable caller memory, or offsets computed here), copied directly from
// the caller's pinned memory, or read in place from device memory.
enum PieceKind { PACK = 0, PINNED = 1, DEVICE = 2 };
struct Piece {
  const void* src;
  size_t off;
  size_t bytes;
  int kind;
};

// The device address of pinned host memory (mapped under unified
// addressing), or nullptr.
const void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int memory_kind(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return PACK;
  }
  return a.type == cudaMemoryTypeDevice ? DEVICE : (a.type == cudaMemoryTypeHost ? PINNED : PACK);
}

// Where each array of one chunk sits inside its packed slot (byte offsets).
struct Plan {
  int index = -1;
  int n = 0;
  int L = 0;
  int64_t first_id = 0;
  int vsrc[PJ_MAX_LODS];           // LoD whose packed vertex array this LoD uses
  size_t o_verts[PJ_MAX_LODS], o_voff[PJ_MAX_LODS], o_faces[PJ_MAX_LODS];
  size_t o_hd[PJ_MAX_LODS], o_ph[PJ_MAX_LODS];
  size_t o_foff[PJ_MAX_LODS], o_coff[PJ_MAX_LODS], o_boff[PJ_MAX_LODS];
  int nfs[PJ_MAX_LODS];
  bool has_hd[PJ_MAX_LODS], has_ph[PJ_MAX_LODS];
  int64_t F[PJ_MAX_LODS], C[PJ_MAX_LODS], B[PJ_MAX_LODS], maxF[PJ_MAX_LODS];
  size_t o_anchor = 0;
  size_t bytes = 0;
  // caller device arrays read in place (nullptr: at their offset in the slot)
  const void* d_verts[PJ_MAX_LODS] = {};
  const void* d_faces[PJ_MAX_LODS] = {};
  const void* d_hd[PJ_MAX_LODS] = {};
  const void* d_ph[PJ_MAX_LODS] = {};
  const void* d_anchor = nullptr;
  std::vector<Piece> pieces;   // what fills the device slot
  size_t bytes_h2d = 0;        // bytes the chunk moves from the host
  size_t bytes_host_read = 0;  // pinned caller arrays read in place (at most this many bytes cross)
};

struct ChunkSlot {
  enum State { FREE, FILLED, COPYING };
  State state = FREE;
  Plan plan;
  cudaEvent_t copied = nullptr;
};

// Check one chunk description (the rules of pj_load_set) and lay it out.
// Host offset arrays are computed into `offs` (kept alive until packed).
// vert_off and face_off must be host memory (read here); verts, faces,
// hd, ph and anchor may lie anywhere.
void plan_chunk(const pj_mesh_set_desc* D, int L_expect, Plan& P, std::vector<Piece>& pieces,
                std::vector<std::vector<int64_t>>& offs, bool host_read) {
  const int n = D->n_objects, L = D->n_lods;
  if (n < 0 || L < 1 || L > PJ_MAX_LODS) throw ApiError{PJ_EINVAL, "chunk: n_objects < 0 or n_lods outside [1, 8]"};
  if (L_expect > 0 && L != L_expect) throw ApiError{PJ_EINVAL, "chunk: n_lods differs from the first chunk"};
  if (n > 0 && !D->anchor) throw ApiError{PJ_EINVAL, "chunk: anchor is NULL"};
  P.n = n;
  P.L = L;
  size_t at = 0;
  P.bytes_host_read = 0;
  // The LoDs between the first (laid out for every object) and the original
  // surfaces (whose vertices give every object's box) are laid out on
  // demand for few objects: their arrays in pinned caller memory are not
  // copied but read in place over the host link by the kernels that lay
  // those objects out.
  const int lazy_from = L >= 2 ? 1 : L;
  auto host_read_lod = [&](int l) { return host_read && l >= lazy_from && l < L - 1; };
  // a caller array (kind from its address) or one computed here (packed);
  // a device array takes no room in the slot and is recorded in *dptr, and
  // so does a pinned one when host_read is set (its device address)
  auto put = [&](const void* src, size_t bytes, bool caller = false, const void** dptr = nullptr,
                 bool host_read = false) {
    const int kind = (caller && bytes) ? memory_kind(src) : PACK;
    if (kind == DEVICE && dptr) {
      *dptr = src;
      return size_t(0);
    }
    if (kind == PINNED && dptr && host_read) {
      const void* dv = device_view(src);
      if (dv) {
        *dptr = dv;
        P.bytes_host_read += bytes;
        return size_t(0);
      }
    }
    const size_t off = at;
    if (bytes) pieces.push_back(Piece{src, off, bytes, kind == DEVICE ? PINNED : kind});
    at = pad(at + bytes);
    return off;
  };
  offs.assign(3 * L, {});
  for (int l = 0; l < L; ++l) {
    if (!D->verts[l] || !D->vert_off[l] || !D->faces[l])
      throw ApiError{PJ_EINVAL, "chunk: verts / vert_off / faces of a LoD is NULL"};
    if (l == L - 1 && (D->hd[l] || D->ph[l])) throw ApiError{PJ_EINVAL, "chunk: hd / ph of the original LoD must be NULL"};
    if (memory_kind(D->vert_off[l]) == DEVICE || (D->face_off[l] && memory_kind(D->face_off[l]) == DEVICE))
      throw ApiError{PJ_EINVAL, "chunk: vert_off / face_off must be host arrays"};
    const int64_t* vo = D->vert_off[l];
    if (n > 0 && vo[0] != 0) throw ApiError{PJ_EINVAL, "chunk: vert_off must start at 0"};
    for (int o = 0; o < n; ++o)
      if (vo[o + 1] < vo[o]) throw ApiError{PJ_EINVAL, "chunk: vert_off not non-decreasing"};
    const int64_t nv = n > 0 ? vo[n] : 0;
    const bool shared = D->face_off[l] == nullptr;
    const int nfs = shared ? D->n_faces_shared[l] : 0;
    if (shared && nfs <= 0 && n > 0) throw ApiError{PJ_EINVAL, "chunk: shared topology needs n_faces_shared > 0"};
    if (!shared && n > 0 && D->face_off[l][0] != 0) throw ApiError{PJ_EINVAL, "chunk: face_off must start at 0"};
    std::vector<int64_t>& fo = offs[3 * l];
    std::vector<int64_t>& co = offs[3 * l + 1];
    std::vector<int64_t>& bo = offs[3 * l + 2];
    fo.assign(n + 1, 0);
    co.assign(n + 1, 0);
    bo.assign(n + 1, 0);
    int64_t maxF = 0;
    for (int o = 0; o < n; ++o) {
      const int64_t c = shared ? nfs : D->face_off[l][o + 1] - D->face_off[l][o];
      if (c < 0) throw ApiError{PJ_EINVAL, "chunk: face_off not non-decreasing"};
      fo[o + 1] = fo[o] + c;
      co[o + 1] = co[o] + (c + CHUNK - 1) / CHUNK;
      bo[o + 1] = bo[o] + (c + BLK - 1) / BLK;
      maxF = std::max(maxF, c);
    }
    if (fo[n] >= (1LL << 31)) throw ApiError{PJ_EINVAL, "chunk: more than 2^31 facets in one LoD"};
    P.F[l] = fo[n];
    P.C[l] = co[n];
    P.B[l] = bo[n];
    P.maxF[l] = maxF;
    P.nfs[l] = nfs;
    P.vsrc[l] = l;
    for (int m = 0; m < l; ++m)
      if (D->verts[m] == D->verts[l] && P.vsrc[m] == m && D->vert_off[m][n] == nv) {
        P.vsrc[l] = m;
        break;
      }
    if (P.vsrc[l] == l) {
      // vertices the first LoD or the original surfaces also use are copied
      const bool own = D->verts[l] != D->verts[0] && D->verts[l] != D->verts[L - 1];
      P.o_verts[l] = put(D->verts[l], (size_t)nv * 12, true, &P.d_verts[l], own && host_read_lod(l));
    } else {
      P.o_verts[l] = P.o_verts[P.vsrc[l]];
      P.d_verts[l] = P.d_verts[P.vsrc[l]];
    }
    P.o_voff[l] = put(vo, (size_t)(n + 1) * 8, true);
    P.o_faces[l] = put(D->faces[l], (size_t)(shared ? nfs : P.F[l]) * 12, true, &P.d_faces[l],
                       !shared && host_read_lod(l));
    P.has_hd[l] = D->hd[l] != nullptr;
    P.has_ph[l] = D->ph[l] != nullptr;
    P.o_hd[l] = P.has_hd[l] ? put(D->hd[l], (size_t)P.F[l] * 4, true, &P.d_hd[l], host_read_lod(l)) : 0;
    P.o_ph[l] = P.has_ph[l] ? put(D->ph[l], (size_t)P.F[l] * 4, true, &P.d_ph[l], host_read_lod(l)) : 0;
    P.o_foff[l] = put(fo.data(), (size_t)(n + 1) * 8);
    P.o_coff[l] = put(co.data(), (size_t)(n + 1) * 8);
    P.o_boff[l] = put(bo.data(), (size_t)(n + 1) * 8);
  }
  P.o_anchor = put(D->anchor, (size_t)n * 12, true, &P.d_anchor);
  P.bytes = at;
  P.bytes_h2d = 0;
  for (const Piece& pc : pieces) P.bytes_h2d += pc.bytes;
}

struct PackJob {
  const unsigned char* src;
  size_t off, bytes;
};

}  // namespace

// Host threads that copy the packed pieces of a chunk into its pinned slot
// (a pageable chunk is hundreds of MB; one thread's memcpy would pace the
// pipeline).  The threads live as long as the context: starting them per
// chunk cost more than packing the few MB of offsets of a chunk whose
// arrays are already pinned or on the device.  One run at a time; the
// calling thread copies too.
class PackPool {
 public:
  explicit PackPool(unsigned n) {
    for (unsigned i = 0; i < n; ++i) th_.emplace_back([this] { work(); });
  }
  ~PackPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  size_t threads() const { return th_.size(); }
  void run(const std::vector<PackJob>& jobs, unsigned char* dst) {
    std::lock_guard<std::mutex> one(run_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      jobs_ = &jobs;
      dst_ = dst;
      next_.store(0);
      busy_ = th_.size();
      ++gen_;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return busy_ == 0; });
    jobs_ = nullptr;
  }

 private:
  void drain() {
    for (;;) {
      const size_t k = next_.fetch_add(1);
      if (k >= jobs_->size()) return;
      const PackJob& j = (*jobs_)[k];
      memcpy(dst_ + j.off, j.src, j.bytes);
    }
  }
  void work() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
      if (stop_) return;
      seen = gen_;
      lk.unlock();
      drain();
      lk.lock();
      if (--busy_ == 0) done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_, run_mu_;
  std::condition_variable cv_, done_;
  const std::vector<PackJob>* jobs_ = nullptr;
  unsigned char* dst_ = nullptr;
  std::atomic<size_t> next_{0};
  size_t busy_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

void destroy_pack_pool(PackPool* p) { delete p; }

namespace {

// Copy the packed pieces into the pinned slot: 1 MB slices over the pool's
// threads, inline when there is a single slice.
void pack_parallel(pj_ctx* ctx, const std::vector<Piece>& pieces, unsigned char* dst, std::vector<PackJob>& jobs) {
  constexpr size_t SLICE = size_t(1) << 20;
  jobs.clear();
  for (const Piece& pc : pieces)
    for (size_t a = 0; pc.kind == PACK && a < pc.bytes; a += SLICE)
      jobs.push_back(PackJob{static_cast<const unsigned char*>(pc.src) + a, pc.off + a, std::min(SLICE, pc.bytes - a)});
  if (jobs.size() <= 1) {
    for (const PackJob& j : jobs) memcpy(dst + j.off, j.src, j.bytes);
    return;
  }
  ctx->pack_pool->run(jobs, dst);   // created before the loaders start
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

pj_status join_streamed(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                        cudaStream_t st, std::string& stats) {
  Timer tall;
  const int N = R->n_chunks;
  ChunkSlot slots[2];
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  pj_status lerr = PJ_OK;
  std::string lmsg;
  double ms_fill = 0, ms_pack = 0, ms_plan = 0, ms_loader_idle = 0;
  int L_first = 0;
  int64_t next_first = 0;
  struct Events {
    cudaEvent_t e[8] = {};
    ~Events() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } evs;
  for (int i = 0; i < 8; ++i)
    PJ_CK(cudaEventCreateWithFlags(&evs.e[i], (i < 2 || i >= 6) ? cudaEventDisableTiming : 0));
  slots[0].copied = evs.e[0];
  slots[1].copied = evs.e[1];
  cudaEvent_t built[2] = {evs.e[6], evs.e[7]};
  // on every exit (also a timeout or an error between chunks) the copy and
  // set-building work still queued for the next chunk finishes before the
  // buffers it writes can be handed to another call
  struct Drain {
    cudaStream_t a, b;
    ~Drain() {
      cudaStreamSynchronize(a);
      cudaStreamSynchronize(b);
    }
  } drain{ctx->copy_stream, ctx->build_stream};
  cudaEvent_t h2d0[2] = {evs.e[2], evs.e[3]}, h2d1[2] = {evs.e[4], evs.e[5]};
  Plan plans[2];   // the calling thread's copy of the plan of each slot in flight
  const int device = ctx->device;

  // ---- loader threads: fill, check, pack.  Two threads, one per slot
  // (chunk c goes to loader c & 1): the fill callbacks are made in chunk
  // order, one at a time (next_fill), while a chunk's layout and packing
  // overlap the next chunk's fill.
  int next_fill = 0;
  double ms_fill_l[2] = {0, 0}, ms_plan_l[2] = {0, 0}, ms_pack_l[2] = {0, 0}, ms_idle_l[2] = {0, 0};
  auto loader_body = [&](int p) {
    cudaSetDevice(device);
    std::vector<Piece> pieces;
    std::vector<PackJob> jobs;
    std::vector<std::vector<int64_t>> offs;
    auto fail_l = [&](pj_status e, const std::string& m) {
      std::lock_guard<std::mutex> lk(mu);
      if (lerr == PJ_OK) {
        lerr = e;
        lmsg = m;
      }
      stop = true;
      cv.notify_all();
    };
    for (int c = p; c < N; c += 2) {
      ChunkSlot& sl = slots[c & 1];
      bool copying;
      auto ti = std::chrono::steady_clock::now();
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || sl.state != ChunkSlot::FILLED; });
        if (stop) return;
        copying = sl.state == ChunkSlot::COPYING;
      }
      // the pinned slot is reused once its previous copy has landed
      const bool copy_ok = !copying || cudaEventSynchronize(sl.copied) == cudaSuccess;
      if (!copy_ok) {
        fail_l(PJ_ECUDA, "loader: waiting for a chunk copy failed");
        return;
      }
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || next_fill == c; });
        if (stop) return;
      }
      ms_idle_l[p] += ms_since(ti);
      pj_mesh_set_desc d;
      memset(&d, 0, sizeof d);
      auto t0 = std::chrono::steady_clock::now();
      const pj_status rc = R->fill(R->user, c, &d);
      ms_fill_l[p] += ms_since(t0);
      {
        std::lock_guard<std::mutex> lk(mu);
        next_fill = c + 1;
      }
      cv.notify_all();
      if (rc != PJ_OK) {
        fail_l(rc == PJ_ECANCELLED ? PJ_ECANCELLED : PJ_ESOURCE,
               "the fill callback returned " + std::to_string((int)rc) + " for chunk " + std::to_string(c));
        return;
      }
      Plan P;
      try {
        auto tp = std::chrono::steady_clock::now();
        pieces.clear();
        plan_chunk(&d, 0, P, pieces, offs, ctx->host_read);
        ms_plan_l[p] += ms_since(tp);
        P.pieces = pieces;
        P.index = c;
        t0 = std::chrono::steady_clock::now();
        void*& hp = ctx->stream_pinned[c & 1];
        size_t& hc = ctx->stream_pinned_cap[c & 1];
        if (hc < P.bytes) {
          if (hp) cudaFreeHost(hp);
          hp = nullptr;
          hc = 0;
          note_alloc();
          if (cudaHostAlloc(&hp, P.bytes, cudaHostAllocDefault) != cudaSuccess)
            throw ApiError{PJ_ENOMEM, "pinned staging allocation failed"};
          hc = P.bytes;
        }
        pack_parallel(ctx, pieces, static_cast<unsigned char*>(hp), jobs);
        ms_pack_l[p] += ms_since(t0);
      } catch (const ApiError& e) {
        fail_l(e.st, e.msg);
        return;
      }
      std::lock_guard<std::mutex> lk(mu);
      sl.plan = P;
      sl.state = ChunkSlot::FILLED;
      cv.notify_all();
    }
  };
  if (!ctx->pack_pool) {
    // all host cores but three: the calling thread drives the GPU, each
    // loader fills a chunk (and copies too); at most 15
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    ctx->pack_pool = new PackPool(std::min(15u, hw > 3 ? hw - 3 : 1u));
  }
  std::thread loader0(loader_body, 0);
  std::thread loader1;
  if (N > 1) loader1 = std::thread(loader_body, 1);
  struct Joiner {
    std::thread& t0;
    std::thread& t1;
    std::mutex& mu;
    std::condition_variable& cv;
    bool& stop;
    ~Joiner() {
      {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
      }
      cv.notify_all();
      if (t0.joinable()) t0.join();
      if (t1.joinable()) t1.join();
    }
  } joiner{loader0, loader1, mu, cv, stop};

  // ---- calling thread: copy, build, join
  int enqueued = 0;   // chunks whose copy has been issued
  double ms_h2d = 0, ms_wait = 0, ms_build = 0, ms_join = 0, ms_issue = 0;
  size_t bytes_h2d = 0, bytes_host_read = 0;
  // issue the copy of chunk c if it is packed (or wait for it when `block`)
  auto enqueue = [&](int c, bool block) -> bool {
    ChunkSlot& sl = slots[c & 1];
    {
      std::unique_lock<std::mutex> lk(mu);
      if (block) {
        auto t0 = std::chrono::steady_clock::now();
        cv.wait(lk, [&] { return stop || (sl.state == ChunkSlot::FILLED && sl.plan.index == c); });
        ms_wait += ms_since(t0);
      }
      if (lerr != PJ_OK) throw ApiError{lerr, lmsg};
      if (!(sl.state == ChunkSlot::FILLED && sl.plan.index == c)) {
        if (stop) throw ApiError{PJ_ECANCELLED, "streamed join stopped"};
        return false;
      }
    }
    // object ids continue the previous chunk's; every chunk has the first
    // chunk's LoD count (chunks are planned in parallel, checked here in order)
    if (c == 0) L_first = sl.plan.L;
    else if (sl.plan.L != L_first) throw ApiError{PJ_EINVAL, "chunk: n_lods differs from the first chunk"};
    sl.plan.first_id = next_first;
    next_first += sl.plan.n;
    if (next_first > R->n_total) throw ApiError{PJ_EINVAL, "the chunks hold more objects than the streamed set"};
    const size_t bytes = sl.plan.bytes;
    unsigned char* dev = (unsigned char*)ws_get(ctx, (c & 1) ? WS_STREAM5 : WS_STREAM4, bytes, ctx->copy_stream);
    const unsigned char* pinned = (const unsigned char*)ctx->stream_pinned[c & 1];
    PJ_CK(cudaEventRecord(h2d0[c & 1], ctx->copy_stream));
    // runs of adjacent packed pieces in one copy each, pinned caller arrays
    // one copy each (pieces are in slot order)
    const std::vector<Piece>& pcs = sl.plan.pieces;
    for (size_t i = 0; i < pcs.size();) {
      if (pcs[i].kind == PINNED) {
        PJ_CK(cudaMemcpyAsync(dev + pcs[i].off, pcs[i].src, pcs[i].bytes, cudaMemcpyDefault, ctx->copy_stream));
        ++i;
        continue;
      }
      size_t j = i + 1;
      while (j < pcs.size() && pcs[j].kind == PACK) ++j;
      const size_t a = pcs[i].off, b = pcs[j - 1].off + pcs[j - 1].bytes;
      PJ_CK(cudaMemcpyAsync(dev + a, pinned + a, b - a, cudaMemcpyHostToDevice, ctx->copy_stream));
      i = j;
    }
    PJ_CK(cudaEventRecord(h2d1[c & 1], ctx->copy_stream));
    PJ_CK(cudaEventRecord(sl.copied, ctx->copy_stream));
    bytes_h2d += sl.plan.bytes_h2d;
    bytes_host_read += sl.plan.bytes_host_read;
    {
      std::lock_guard<std::mutex> lk(mu);
      plans[c & 1] = sl.plan;
      sl.state = ChunkSlot::COPYING;
    }
    cv.notify_all();
    return true;
  };

  // set building of chunk c (its copy issued) on the build stream, into
  // the derived buffers of its slot; the boxes and the error word come back
  // to pinned memory, and built[slot] marks the end
  pj_set views[2];
  int prepared[2] = {-1, -1};
  auto prepare = [&](int c) {
    const int si = c & 1;
    const Plan& P = plans[si];
    unsigned char* dev = (unsigned char*)ctx->ws[si ? WS_STREAM5 : WS_STREAM4].p;
    cudaStream_t bst = ctx->build_stream;
    pj_set& view = views[si];
    view = pj_set();
    view.ctx = ctx;
    view.device = ctx->device;
    view.n = P.n;
    view.L = P.L;
    int64_t fac_n = 0, box_n = 0;
    for (int l = 0; l < P.L; ++l) {
      fac_n += 3 * std::max<int64_t>(1, P.F[l]);
      box_n += 3 * (std::max<int64_t>(1, P.C[l]) + std::max<int64_t>(1, P.B[l]));
    }
    float4* fac = (float4*)ws_get(ctx, si ? WS_STREAM6 : WS_STREAM, fac_n * sizeof(float4), bst);
    float4* box = (float4*)ws_get(ctx, si ? WS_STREAM7 : WS_STREAM2, box_n * sizeof(float4), bst);
    const size_t box_bytes = (size_t)std::max(1, P.n) * 24;
    // the finer LoDs (most of the facets) are laid out on demand, for the
    // objects whose pairs reach a step that uses them; layout of this
    // buffer: boxes, error word, per lazy LoD the objects' states, the
    // list of objects to build and its count
    const int lazy_from = P.L >= 2 ? 1 : P.L;
    const size_t nl = (size_t)(P.L - lazy_from), no = (size_t)std::max(1, P.n);
    const size_t state_bytes = ((nl * no * 4) + 15) & ~size_t(15);
    unsigned char* mb = (unsigned char*)ws_get(ctx, si ? WS_STREAM8 : WS_STREAM3,
                                               box_bytes + 16 + state_bytes + no * 4 + 16, bst);
    view.mbb = (float*)mb;
    int* err = (int*)(mb + box_bytes);
    view.lazy_from = lazy_from;
    view.lazy_state = nl ? (unsigned*)(mb + box_bytes + 16) : nullptr;
    view.lazy_list = (int32_t*)(mb + box_bytes + 16 + state_bytes);
    view.lazy_count = (unsigned*)(mb + box_bytes + 16 + state_bytes + no * 4);
    view.anchor = P.d_anchor ? (float*)P.d_anchor : (float*)(dev + P.o_anchor);
    RawLod raw[PJ_MAX_LODS];
    for (int l = 0; l < P.L; ++l) {
      LodData& ld = view.lod[l];
      ld.F = P.F[l];
      ld.C = P.C[l];
      ld.B = P.B[l];
      ld.maxF = P.maxF[l];
      ld.fac = fac;
      fac += 3 * std::max<int64_t>(1, P.F[l]);
      ld.chunk = box;
      box += 3 * std::max<int64_t>(1, P.C[l]);
      ld.blk = box;
      box += 3 * std::max<int64_t>(1, P.B[l]);
      ld.foff = (int64_t*)(dev + P.o_foff[l]);
      ld.coff = (int64_t*)(dev + P.o_coff[l]);
      ld.boff = (int64_t*)(dev + P.o_boff[l]);
      auto at = [&](const void* d, size_t off) { return d ? d : (const void*)(dev + off); };
      raw[l] = RawLod{(const float*)at(P.d_verts[l], P.o_verts[l]), (const int64_t*)(dev + P.o_voff[l]),
                      (const int32_t*)at(P.d_faces[l], P.o_faces[l]), P.nfs[l],
                      P.has_hd[l] ? (const float*)at(P.d_hd[l], P.o_hd[l]) : nullptr,
                      P.has_ph[l] ? (const float*)at(P.d_ph[l], P.o_ph[l]) : nullptr};
    }
    if (ctx->stream_box_cap[si] < box_bytes + 16) {
      if (ctx->stream_box_pinned[si]) PJ_CK(cudaFreeHost(ctx->stream_box_pinned[si]));
      ctx->stream_box_pinned[si] = nullptr;
      ctx->stream_box_cap[si] = 0;
      note_alloc();
      PJ_CK(cudaHostAlloc(&ctx->stream_box_pinned[si], box_bytes + 16, cudaHostAllocDefault));
      ctx->stream_box_cap[si] = box_bytes + 16;
    }
    for (int l = lazy_from; l < P.L; ++l) view.lazy_raw[l] = raw[l];
    PJ_CK(cudaStreamWaitEvent(bst, slots[si].copied, 0));
    PJ_CK(cudaMemsetAsync(err, 0, sizeof(int), bst));
    if (nl) PJ_CK(cudaMemsetAsync(view.lazy_state, 0, nl * no * 4, bst));
    build_set_kernels(ctx, &view, raw, bst, err, lazy_from);
    // the learned start LoD reads every pair's hd / ph maxima per LoD (at
    // the LoDs laid out on demand, from all objects' hd / ph); not needed
    // when the query has no learned start or the tuned schedule is fixed
    const bool learned = (q->flags & PJ_USE_MLP) && q->pred != PJ_KNN &&
                         !((q->flags & PJ_AUTOTUNE) && tuned_schedule_fixed(ctx, &view, S, q));
    if (learned || q->pred == PJ_KNN)
      for (int l = lazy_from; l < P.L - 1; ++l) chunk_hd_ph(ctx, &view, l, raw[l], bst);
    // the error word back to pinned memory, and the boxes when the host
    // needs them (the k-NN grid spans R's boxes; the within grid is over S)
    if (q->pred == PJ_KNN)
      PJ_CK(cudaMemcpyAsync(ctx->stream_box_pinned[si], mb, box_bytes + sizeof(int), cudaMemcpyDeviceToHost, bst));
    else
      PJ_CK(cudaMemcpyAsync((unsigned char*)ctx->stream_box_pinned[si] + box_bytes, mb + box_bytes, sizeof(int),
                            cudaMemcpyDeviceToHost, bst));
    PJ_CK(cudaEventRecord(built[si], bst));
    prepared[si] = c;
  };

  std::vector<int32_t> rr, ss;
  std::vector<double> dlo, dhi, dd;
  std::vector<uint8_t> ex;
  JoinSummary tot;
  int64_t objects = 0;
  int graph_replays = 0, graph_captures = 0, spec_joins = 0;
  const unsigned long long misses0 = ctx->spec_misses;
  ctx->last_tune.clear();
  // the chunk joins run on the context's greatest-priority stream, after
  // whatever the caller queued on st, so that their many small launches are
  // scheduled ahead of the next chunk's set building
  const cudaStream_t caller = st;
  st = ctx->join_stream;
  struct Rejoin {
    cudaStream_t from, to;
    cudaEvent_t e = nullptr;
    Rejoin(cudaStream_t a, cudaStream_t b) : from(a), to(b) {
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess && cudaEventRecord(e, from) == cudaSuccess)
        cudaStreamWaitEvent(to, e, 0);
    }
    ~Rejoin() {
      // on every exit the caller's stream waits for the chunk joins
      if (e && cudaEventRecord(e, to) == cudaSuccess) cudaStreamWaitEvent(from, e, 0);
      if (e) cudaEventDestroy(e);
    }
  } rejoin(caller, st);
  // Within joins with graph replay take the chunks in turn on two join
  // contexts (ctx and its twin, each with its own workspace and join
  // stream): chunk c's join is issued before chunk c-1's is waited for, so
  // the two overlap on the device, and the next chunk's copy and set
  // building are issued once chunk c-1's slot is free.
  const bool overlap = ctx->chunk_overlap && q->pred != PJ_KNN && (q->flags & PJ_USE_GRAPH) && N > 1;
  pj_ctx* J[2] = {ctx, overlap ? join_twin(ctx) : ctx};
  cudaStream_t JS[2] = {st, overlap ? J[1]->join_stream : st};
  struct KnobSave {   // the tuned choice set on ctx for the chunks is undone on exit
    pj_ctx* c;
    int v, s, k, t;
    ~KnobSave() {
      c->refine_variant = v;
      c->sched_start = s;
      c->refine_split = k;
      c->refine_tail = t;
    }
  } knobs{ctx, ctx->refine_variant, ctx->sched_start, ctx->refine_split, ctx->refine_tail};
  struct Quiesce {   // no chunk join stays in flight past this call
    cudaStream_t a, b;
    ~Quiesce() {
      cudaStreamSynchronize(a);
      if (b != a) cudaStreamSynchronize(b);
    }
  } quiesce{JS[0], JS[1]};
  const unsigned long long twin_misses0 = overlap ? J[1]->spec_misses : 0;
  struct Pending {
    bool on = false;
    WithinTail w;
    pj_result part;
    int64_t first = 0;
    int n = 0;
  } pend;
  // a completed chunk join: totals and results (chunks complete in order)
  auto absorb = [&](const JoinSummary& js, pj_result& part, int64_t first, int nobj) {
    tot.candidates += js.candidates;
    tot.results += js.results;
    tot.units += js.units;
    tot.tests32 += js.tests32;
    tot.tests64 += js.tests64;
    tot.confirmed += js.confirmed;
    tot.removed += js.removed;
    tot.ms_filter += js.ms_filter;
    tot.ms_seq += js.ms_seq;
    tot.graph_ms += js.graph_ms;
    tot.refine_ms32 += js.refine_ms32;
    tot.refine_ms64 += js.refine_ms64;
    tot.launches += js.launches;
    graph_replays += js.graph == 2;
    spec_joins += js.spec;
    graph_captures += js.graph == 1;
    for (int64_t i = 0; i < part.n; ++i) {
      rr.push_back((int32_t)(part.r[i] + first));
      ss.push_back(part.s[i]);
      dlo.push_back(part.d_lo[i]);
      dhi.push_back(part.d_hi[i]);
      dd.push_back(part.d[i]);
      ex.push_back(part.exact[i]);
    }
    free(part.priv);
    part.priv = nullptr;
    objects += nobj;
  };
  std::string st_chunk;
  auto finish_pending = [&]() -> pj_status {
    if (!pend.on) return PJ_OK;
    pend.on = false;
    Timer tj;
    const pj_status rc = within_finish(pend.w, &pend.part, st_chunk);
    ms_join += tj.ms();
    if (rc != PJ_OK) {
      free(pend.part.priv);
      return rc;
    }
    absorb(pend.w.ctx->last_sum, pend.part, pend.first, pend.n);
    return PJ_OK;
  };
  for (int c = 0; c < N; ++c) {
    if (q->timeout_s > 0 && tall.ms() > q->timeout_s * 1000.0) return PJ_ETIMEOUT;
    Timer ti;
    if (enqueued <= c) {
      enqueue(c, true);
      enqueued = c + 1;
    }
    if (prepared[c & 1] != c) prepare(c);
    const Plan P = plans[c & 1];
    // the copy and the set building of the next chunk overlap this chunk's
    // join (with two joins in flight: issued below, once the slot is free)
    if (!overlap && c + 1 < N && enqueued == c + 1 && enqueue(c + 1, false)) {
      enqueued = c + 2;
      prepare(c + 1);
    }
    ms_issue += ti.ms();
    Timer tb;
    PJ_CK(cudaEventSynchronize(built[c & 1]));
    pj_set& view = views[c & 1];
    const size_t box_bytes = (size_t)std::max(1, P.n) * 24;
    int herr = 0;
    memcpy(&herr, (const unsigned char*)ctx->stream_box_pinned[c & 1] + box_bytes, sizeof(int));
    if (herr & ERR_BOUNDS)
      throw ApiError{PJ_EBOUNDS, "chunk " + std::to_string(c) + ": a face index lies outside its object's vertices"};
    if (herr & ERR_NONFINITE)
      throw ApiError{PJ_ENONFINITE, "chunk " + std::to_string(c) + ": non-finite vertex, anchor, hd or ph"};
    if (q->pred == PJ_KNN) {
      const float* hb = (const float*)ctx->stream_box_pinned[c & 1];
      view.mbb_h.assign(hb, hb + (size_t)P.n * 6);
    }
    pj_ctx* Jc = J[c & 1];
    cudaStream_t sc = JS[c & 1];
    PJ_CK(cudaStreamWaitEvent(sc, built[c & 1], 0));
    ms_build += tb.ms();
    float h2d = 0;
    if (cudaEventElapsedTime(&h2d, h2d0[c & 1], h2d1[c & 1]) == cudaSuccess) ms_h2d += h2d;
    // the join of this chunk against S
    pj_query qc = *q;
    if (q->timeout_s > 0) qc.timeout_s = std::max(1e-3, q->timeout_s - tall.ms() / 1000.0);
    pj_result part;
    memset(&part, 0, sizeof part);
    WithinTail w;
    Timer tj;
    pj_status rc;
    if (overlap && (!(q->flags & PJ_AUTOTUNE) || tuned_apply(ctx, Jc, &view, S, &qc))) {
      rc = join_within_issue(Jc, &view, S, &qc, &part, sc, st_chunk, &w);
    } else {
      rc = (q->flags & PJ_AUTOTUNE) ? join_autotuned(Jc, &view, S, &qc, &part, sc, st_chunk)
           : q->pred == PJ_KNN      ? join_knn(Jc, &view, S, &qc, &part, sc, st_chunk)
                                    : join_within(Jc, &view, S, &qc, &part, sc, st_chunk);
    }
    ms_join += tj.ms();
    if (rc != PJ_OK && rc != PJ_PENDING) {
      free(part.priv);
      if (Jc != ctx) ctx->last_error = Jc->last_error;
      return rc;
    }
    // chunk c-1 completes first (in order), then this one or it stays pending
    const pj_status rp = finish_pending();
    if (rp != PJ_OK) {
      free(part.priv);
      return rp;
    }
    if (rc == PJ_PENDING) {
      pend.on = true;
      pend.w = w;
      pend.part = part;
      pend.first = P.first_id;
      pend.n = P.n;
    } else {
      absorb(Jc->last_sum, part, P.first_id, P.n);
    }
    if (overlap) {
      Timer ti2;
      if (c + 1 < N && enqueued == c + 1 && enqueue(c + 1, false)) {
        enqueued = c + 2;
        prepare(c + 1);
      }
      ms_issue += ti2.ms();
    }
  }
  {
    const pj_status rp = finish_pending();
    if (rp != PJ_OK) return rp;
  }
  if (objects != R->n_total)
    throw ApiError{PJ_ESOURCE, "the chunks hold " + std::to_string(objects) + " objects, the streamed set " +
                                   std::to_string(R->n_total)};
  const int64_t m = (int64_t)rr.size();
  alloc_result(out, m);
  if (m) {
    memcpy(out->r, rr.data(), m * 4);
    memcpy(out->s, ss.data(), m * 4);
    memcpy(out->d_lo, dlo.data(), m * 8);
    memcpy(out->d_hi, dhi.data(), m * 8);
    memcpy(out->d, dd.data(), m * 8);
    memcpy(out->exact, ex.data(), m);
  }
  const double ms_total = tall.ms();
  ms_fill = ms_fill_l[0] + ms_fill_l[1];
  ms_plan = ms_plan_l[0] + ms_plan_l[1];
  ms_pack = ms_pack_l[0] + ms_pack_l[1];
  ms_loader_idle = ms_idle_l[0] + ms_idle_l[1];
  char buf[2048];
  snprintf(buf, sizeof buf,
           "{\"pred\":\"%s\",\"streamed\":1,\"chunks\":%d,\"objects\":%lld,\"candidates\":%lld,\"results\":%lld,"
           "\"tests_fp32\":%llu,\"tests_fp64\":%llu,\"confirmed\":%llu,\"removed\":%llu,\"tiles\":%lld,"
           "\"bytes_h2d\":%zu,\"bytes_host_read_max\":%zu,\"ms_h2d\":%.3f,\"h2d_gbs\":%.2f,\"ms_fill\":%.3f,\"ms_plan\":%.3f,"
           "\"ms_pack\":%.3f,\"ms_loader_idle\":%.3f,"
           "\"ms_wait_loader\":%.3f,\"ms_issue\":%.3f,\"ms_build\":%.3f,\"ms_join\":%.3f,\"ms_filter\":%.3f,"
           "\"ms_seq\":%.3f,\"graph_ms\":%.3f,\"refine_ms_fp32\":%.4f,\"refine_ms_fp64\":%.4f,\"ms_total\":%.3f,\"launches\":%llu,"
           "\"graph_replays\":%d,\"graph_captures\":%d,\"spec_joins\":%d,\"spec_misses\":%llu",
           q->pred == PJ_KNN ? "knn" : "within", N, (long long)objects, (long long)tot.candidates, (long long)m,
           tot.tests32, tot.tests64, tot.confirmed, tot.removed, (long long)tot.units, bytes_h2d, bytes_host_read, ms_h2d,
           ms_h2d > 0 ? bytes_h2d / (ms_h2d * 1e6) : 0.0, ms_fill, ms_plan, ms_pack, ms_loader_idle, ms_wait, ms_issue, ms_build, ms_join, tot.ms_filter, tot.ms_seq, tot.graph_ms,
           tot.refine_ms32,
           tot.refine_ms64, ms_total, tot.launches, graph_replays, graph_captures, spec_joins,
           ctx->spec_misses - misses0 + (overlap ? J[1]->spec_misses - twin_misses0 : 0));
  // the autotuner's choice for the chunks (tuned on the first, reused after)
  stats = std::string(buf) + (ctx->last_tune.empty() ? "" : ",\"autotune\":" + ctx->last_tune) + "}";
  tot.results = m;
  tot.ms_total = ms_total;
  ctx->last_sum = tot;
  return PJ_OK;
}

}  // namespace pj
