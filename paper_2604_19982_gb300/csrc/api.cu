// C ABI of the join library (declared in include/pj.h): contexts, device
// resident mesh sets and the entry points.  No exception crosses the ABI.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "tritri.cuh"

namespace pj {

pj_status join_within(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                      cudaStream_t st, std::string& stats);
pj_status join_knn(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                   cudaStream_t st, std::string& stats);
pj_status join_autotuned(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                         cudaStream_t st, std::string& stats);
pj_status join_streamed(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out,
                        cudaStream_t st, std::string& stats);
void alloc_result(pj_result* res, int64_t n);
pj_status mlp_train_impl(pj_ctx* ctx, const float* feats, const float* target, int64_t n, int epochs,
                         uint64_t seed);
void mlp_ensure(pj_ctx* ctx);

std::atomic<unsigned long long> g_allocs{0};

void* ws_get(pj_ctx* ctx, int slot, size_t bytes, cudaStream_t st) {
  (void)st;
  DevBuf& b = ctx->ws[slot];
  if (bytes == 0) bytes = 1;
  if (b.cap < bytes) {
    if (b.p) PJ_CK(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
    size_t cap = std::max(bytes, b.cap + b.cap / 2);
    note_alloc();
    PJ_CK(cudaMalloc(&b.p, cap));
    b.cap = cap;
  }
  return b.p;
}

// ------------------------------------------------------------------ load

__device__ __forceinline__ int64_t upper_obj(const int64_t* off, int n, int64_t f) {
  // largest o with off[o] <= f (off non-decreasing, off[0] = 0)
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= f) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One 32-facet block, one warp: each lane expands one facet into its
// record (v0, hd), (v1, ph), (v2, 0); the warp reduces the block's box, max
// hd / ph, max edge length and min facet sine from registers, so the
// records are written once and never read back.
__device__ __forceinline__ void expand_block(int64_t bi, int64_t o, const float* verts, const int64_t* voff,
                                             const int32_t* faces, const int64_t* foff, const int64_t* boff,
                                             int nf_shared, const float* hd, const float* ph, float4* fac,
                                             float4* blk, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t f = foff[o] + (bi - boff[o]) * BLK + lane;
  const bool act = f < foff[o + 1];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  float mhd = 0.f, mph = 0.f, medge = 0.f, smin = 1.f;
  if (act) {
    const int64_t row = nf_shared > 0 ? f - o * nf_shared : f;
    const int64_t v0 = voff[o], nv = voff[o + 1] - v0;
    float x[3][3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int id = faces[3 * row + k];
      if (id < 0 || id >= nv) {
        ok = false;
        id = 0;
      }
      const float* v = verts + 3 * (v0 + id);
      x[k][0] = v[0];
      x[k][1] = v[1];
      x[k][2] = v[2];
    }
    const float h = hd ? hd[f] : 0.f, p = ph ? ph[f] : 0.f;
    bool fin = isfinite(h) && isfinite(p) && h >= 0.f && p >= 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) fin = fin && isfinite(x[k][0]) && isfinite(x[k][1]) && isfinite(x[k][2]);
    if (!ok) set_err(err, ERR_BOUNDS);
    if (!fin) set_err(err, ERR_NONFINITE);
    fac[3 * f + 0] = make_float4(x[0][0], x[0][1], x[0][2], h);
    fac[3 * f + 1] = make_float4(x[1][0], x[1][1], x[1][2], p);
    fac[3 * f + 2] = make_float4(x[2][0], x[2][1], x[2][2], 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(x[0][k], fminf(x[1][k], x[2][k]));
      hi[k] = fmaxf(x[0][k], fmaxf(x[1][k], x[2][k]));
    }
    mhd = h;
    mph = p;
    float e0 = 0, e1 = 0, e2 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e0 += (x[1][k] - x[0][k]) * (x[1][k] - x[0][k]);
      e1 += (x[2][k] - x[1][k]) * (x[2][k] - x[1][k]);
      e2 += (x[0][k] - x[2][k]) * (x[0][k] - x[2][k]);
    }
    medge = sqrtf(fmaxf(e0, fmaxf(e1, e2))) * 1.0001f;
    smin = facet_sin<float>(x[0], x[1], x[2]) * 0.999f;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = warp_min(lo[k]);
    hi[k] = -warp_min(-hi[k]);
  }
  mhd = -warp_min(-mhd);
  mph = -warp_min(-mph);
  medge = -warp_min(-medge);
  smin = warp_min(smin);
  if (lane == 0) {
    blk[3 * bi + 0] = make_float4(lo[0], lo[1], lo[2], mhd);
    blk[3 * bi + 1] = make_float4(hi[0], hi[1], hi[2], mph);
    blk[3 * bi + 2] = make_float4(medge, smin, 0.f, 0.f);
  }
}

// One warp per block of every object (blocks of an object with shared
// topology are found by division, others by a search of the offsets).
__global__ void k_expand_blocks(int64_t B, int n, const float* verts, const int64_t* voff, const int32_t* faces,
                                const int64_t* foff, const int64_t* boff, int nf_shared, const float* hd,
                                const float* ph, float4* fac, float4* blk, int* err) {
  const int64_t bi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (bi >= B) return;
  const int64_t bpo = nf_shared > 0 ? (nf_shared + BLK - 1) / BLK : 0;
  const int64_t o = bpo ? bi / bpo : upper_obj(boff, n, bi);
  expand_block(bi, o, verts, voff, faces, foff, boff, nf_shared, hd, ph, fac, blk, err);
}

// One 256-facet chunk: the reduction of its (up to 8) blocks.
__device__ __forceinline__ void chunk_from_blocks(int64_t c, int64_t o, const int64_t* coff, const int64_t* boff,
                                                  const float4* blk, float4* chunk) {
  const int64_t b0 = boff[o] + (c - coff[o]) * (CHUNK / BLK), b1 = min(b0 + CHUNK / BLK, boff[o + 1]);
  float4 lo = blk[3 * b0], hi = blk[3 * b0 + 1], ex = blk[3 * b0 + 2];
  for (int64_t b = b0 + 1; b < b1; ++b) {
    const float4 l = blk[3 * b], h = blk[3 * b + 1], e = blk[3 * b + 2];
    lo = make_float4(fminf(lo.x, l.x), fminf(lo.y, l.y), fminf(lo.z, l.z), fmaxf(lo.w, l.w));
    hi = make_float4(fmaxf(hi.x, h.x), fmaxf(hi.y, h.y), fmaxf(hi.z, h.z), fmaxf(hi.w, h.w));
    ex = make_float4(fmaxf(ex.x, e.x), fminf(ex.y, e.y), 0.f, 0.f);
  }
  chunk[3 * c + 0] = lo;
  chunk[3 * c + 1] = hi;
  chunk[3 * c + 2] = ex;
}

__global__ void k_chunks_from_blocks(int64_t C, int n, const int64_t* coff, const int64_t* boff, const float4* blk,
                                     float4* chunk) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= C) return;
  chunk_from_blocks(c, upper_obj(coff, n, c), coff, boff, blk, chunk);
}

// one warp per object: box of its original-surface vertices
__global__ void k_mbb(int n, const float* verts, const int64_t* voff, const float* anchor, float* mbb, int* err) {
  int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (o >= n) return;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool fin = true;
  for (int64_t v = voff[o] + lane; v < voff[o + 1]; v += 32)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float x = verts[3 * v + k];
      fin = fin && isfinite(x);
      lo[k] = fminf(lo[k], x);
      hi[k] = fmaxf(hi[k], x);
    }
  if (!fin) set_err(err, ERR_NONFINITE);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = warp_min(lo[k]);
    hi[k] = -warp_min(-hi[k]);
  }
  if (lane == 0) {
    for (int k = 0; k < 3; ++k) {
      mbb[6 * o + k] = lo[k];
      mbb[6 * o + 3 + k] = hi[k];
      if (!isfinite(anchor[3 * o + k])) set_err(err, ERR_NONFINITE);
    }
  }
}

void free_set_storage(pj_set* s) {
  for (int l = 0; l < PJ_MAX_LODS; ++l) {
    cudaFree(s->lod[l].fac);
    cudaFree(s->lod[l].foff);
    cudaFree(s->lod[l].chunk);
    cudaFree(s->lod[l].coff);
    cudaFree(s->lod[l].blk);
    cudaFree(s->lod[l].boff);
    s->lod[l] = LodData();
  }
  cudaFree(s->mbb);
  cudaFree(s->anchor);
  s->mbb = s->anchor = nullptr;
  free_voxels(s);
}

// Set storage and load temporaries are stream-ordered allocations from the
// device's memory pool (no device-wide synchronization per buffer).
template <class T>
static T* upload(const T* h, size_t count, cudaStream_t st) {
  T* d = nullptr;
  note_alloc();
  PJ_CK(cudaMallocAsync((void**)&d, std::max<size_t>(1, count) * sizeof(T), st));
  if (count) PJ_CK(cudaMemcpyAsync(d, h, count * sizeof(T), cudaMemcpyHostToDevice, st));
  return d;
}

// With the "zero_copy" context option: the device address of a host array
// that lives in pinned, mapped host memory (the build kernels then read it
// over the host link directly, with no staging copy), else nullptr.
static const void* pinned_view(const pj_ctx* ctx, const void* p) {
  if (!ctx->zero_copy || !p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Lay a described set out on the device (see pj_load_set).
void build_set_kernels(pj_ctx* ctx, pj_set* s, const RawLod* raw, cudaStream_t st, int* err, int lod_end) {
  const int n = s->n, L = s->L;
  if (!err) err = ctx->d_err;
  int th = 256;
  for (int l = 0; l < (lod_end < 0 ? L : lod_end); ++l) {
    LodData& ld = s->lod[l];
    if (ld.F == 0) continue;
    k_expand_blocks<<<(unsigned)((ld.B * 32 + th - 1) / th), th, 0, st>>>(
        ld.B, n, raw[l].verts, raw[l].voff, raw[l].faces, ld.foff, ld.boff, raw[l].nfs, raw[l].hd, raw[l].ph, ld.fac,
        ld.blk, err);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    k_chunks_from_blocks<<<(unsigned)((ld.C + th - 1) / th), th, 0, st>>>(ld.C, n, ld.coff, ld.boff, ld.blk,
                                                                         ld.chunk);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
  if (n > 0) {
    k_mbb<<<(unsigned)(((int64_t)n * 32 + th - 1) / th), th, 0, st>>>(n, raw[L - 1].verts, raw[L - 1].voff, s->anchor,
                                                                       s->mbb, err);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
  }
}

// Objects of R that the selected pairs of a step need at a lazily built
// LoD and that are not built yet: state 0 -> 1, appended to the list.
__global__ void k_lazy_mark(int64_t n, const int32_t* pr, const uint8_t* status, const uint8_t* lod0, uint8_t want,
                            int step, unsigned* state, int32_t* list, unsigned* count) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n || status[p] != want || lod0[p] > step) return;
  const int r = pr[p];
  if (state[r] == 0 && atomicCAS(&state[r], 0u, 1u) == 0u) list[atomicAdd(count, 1u)] = r;
}

// The listed objects' blocks: warp w takes block (w mod maxb) of listed
// object (w / maxb) (warps past an object's blocks return).
__global__ void k_expand_listed(const int32_t* list, const unsigned* count, int64_t maxb, const float* verts,
                                const int64_t* voff, const int32_t* faces, const int64_t* foff,
                                const int64_t* boff, int nf_shared, const float* hd, const float* ph, float4* fac,
                                float4* blk, int* err) {
  const int64_t total = (int64_t)(*count) * maxb;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
    const int o = list[w / maxb];
    const int64_t bi = boff[o] + w % maxb;
    if (bi >= boff[o + 1]) continue;   // warp-uniform
    expand_block(bi, o, verts, voff, faces, foff, boff, nf_shared, hd, ph, fac, blk, err);
  }
}

// The listed objects' chunk boxes from their blocks: thread t takes chunk
// (t mod maxc) of listed object (t / maxc).
__global__ void k_chunks_listed(const int32_t* list, const unsigned* count, int64_t maxc, const int64_t* coff,
                                const int64_t* boff, const float4* blk, float4* chunk) {
  const int64_t total = (int64_t)(*count) * maxc;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += nt) {
    const int o = list[t / maxc];
    const int64_t c = coff[o] + t % maxc;
    if (c < coff[o + 1]) chunk_from_blocks(c, o, coff, boff, blk, chunk);
  }
}

void ensure_lod(pj_ctx* ctx, const pj_set* R, int lod, int64_t n_pairs, const int32_t* pr, const uint8_t* status,
                const uint8_t* lod0, uint8_t want, int step, cudaStream_t st) {
  if (lod < R->lazy_from || n_pairs == 0 || R->n == 0) return;
  const LodData& ld = R->lod[lod];
  const RawLod& raw = R->lazy_raw[lod];
  unsigned* state = R->lazy_state + (size_t)(lod - R->lazy_from) * R->n;
  const int th = 256;
  PJ_CK(cudaMemsetAsync(R->lazy_count, 0, sizeof(unsigned), st));
  k_lazy_mark<<<(unsigned)((n_pairs + th - 1) / th), th, 0, st>>>(n_pairs, pr, status, lod0, want, step, state,
                                                                    R->lazy_list, R->lazy_count);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  if (ld.F == 0) return;
  const int64_t maxb = std::max<int64_t>(1, (ld.maxF + BLK - 1) / BLK);
  const int64_t maxc = std::max<int64_t>(1, (ld.maxF + CHUNK - 1) / CHUNK);
  const unsigned grid = (unsigned)std::min<int64_t>(std::max<int64_t>(1, ((int64_t)R->n * maxb * 32 + th - 1) / th),
                                                    (int64_t)ctx->sm_count * 16);
  k_expand_listed<<<grid, th, 0, st>>>(R->lazy_list, R->lazy_count, maxb, raw.verts, raw.voff, raw.faces, ld.foff,
                                       ld.boff, raw.nfs, raw.hd, raw.ph, ld.fac, ld.blk, ctx->d_err);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
  const unsigned gc = (unsigned)std::min<int64_t>(std::max<int64_t>(1, ((int64_t)R->n * maxc + th - 1) / th),
                                                  (int64_t)ctx->sm_count * 8);
  k_chunks_listed<<<gc, th, 0, st>>>(R->lazy_list, R->lazy_count, maxc, ld.coff, ld.boff, ld.blk, ld.chunk);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

// One thread per chunk: the maxima of hd and ph over its facets.
// Max hd / ph of each 256-facet chunk: one warp per object walks its
// chunks (no search for the owning object), the lanes read a chunk's
// facets in consecutive runs and reduce by shuffles.
__global__ void k_chunk_hd_ph(int n, const int64_t* coff, const int64_t* foff, const float* hd, const float* ph,
                              float4* chunk) {
  const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= n) return;   // warp-uniform
  const int64_t fo = foff[o], fe = foff[o + 1];
  for (int64_t c = coff[o]; c < coff[o + 1]; ++c) {
    const int64_t f0 = fo + (c - coff[o]) * CHUNK, f1 = min(f0 + CHUNK, fe);
    float mh = 0.f, mp = 0.f;
    for (int64_t f = f0 + lane; f < f1; f += 32) {
      if (hd) mh = fmaxf(mh, hd[f]);
      if (ph) mp = fmaxf(mp, ph[f]);
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
      mh = fmaxf(mh, __shfl_xor_sync(0xffffffffu, mh, k));
      mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, k));
    }
    if (lane == 0) {
      chunk[3 * c].w = mh;
      chunk[3 * c + 1].w = mp;
    }
  }
}

void chunk_hd_ph(pj_ctx* ctx, pj_set* s, int l, const RawLod& raw, cudaStream_t st) {
  const LodData& ld = s->lod[l];
  if (ld.C == 0 || s->n == 0) return;
  const int th = 256;
  k_chunk_hd_ph<<<(unsigned)(((int64_t)s->n * 32 + th - 1) / th), th, 0, st>>>(s->n, ld.coff, ld.foff, raw.hd,
                                                                                raw.ph, ld.chunk);
  PJ_CK(cudaGetLastError());
  PJ_COUNT_LAUNCH;
}

pj_status load_set_impl(pj_ctx* ctx, const pj_mesh_set_desc* D, pj_set* s, cudaStream_t st) {
  const int n = D->n_objects, L = D->n_lods;
  if (n < 0 || L < 1 || L > PJ_MAX_LODS) throw ApiError{PJ_EINVAL, "n_objects < 0 or n_lods outside [1, 8]"};
  if (n > 0 && !D->anchor) throw ApiError{PJ_EINVAL, "anchor is NULL"};
  s->n = n;
  s->L = L;
  std::map<const void*, float*> vcache;
  struct Temps {
    std::vector<void*> v;
    cudaStream_t st;
    void push_back(void* p) { v.push_back(p); }
    ~Temps() {
      for (void* p : v) cudaFreeAsync(p, st);
    }
  } temps{{}, st};
  PJ_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  RawLod raw[PJ_MAX_LODS];
  for (int l = 0; l < L; ++l) {
    if (!D->verts[l] || !D->vert_off[l] || !D->faces[l])
      throw ApiError{PJ_EINVAL, "verts / vert_off / faces of a LoD is NULL"};
    if (l == L - 1 && (D->hd[l] || D->ph[l]))
      throw ApiError{PJ_EINVAL, "hd / ph of the original LoD must be NULL (zero)"};
    const int64_t* vo = D->vert_off[l];
    if (n > 0 && vo[0] != 0) throw ApiError{PJ_EINVAL, "vert_off must start at 0"};
    for (int o = 0; o < n; ++o)
      if (vo[o + 1] < vo[o]) throw ApiError{PJ_EINVAL, "vert_off not non-decreasing"};
    const int64_t nv = n > 0 ? vo[n] : 0;
    LodData& ld = s->lod[l];
    ld.foff_h.assign(n + 1, 0);
    const bool shared = D->face_off[l] == nullptr;
    const int nfs = shared ? D->n_faces_shared[l] : 0;
    if (shared && nfs <= 0 && n > 0) throw ApiError{PJ_EINVAL, "shared topology needs n_faces_shared > 0"};
    for (int o = 0; o < n; ++o) {
      int64_t cnt = shared ? nfs : D->face_off[l][o + 1] - D->face_off[l][o];
      if (cnt < 0) throw ApiError{PJ_EINVAL, "face_off not non-decreasing"};
      ld.foff_h[o + 1] = ld.foff_h[o] + cnt;
    }
    if (!shared && n > 0 && D->face_off[l][0] != 0) throw ApiError{PJ_EINVAL, "face_off must start at 0"};
    ld.F = ld.foff_h[n];
    if (ld.F >= (1LL << 31)) throw ApiError{PJ_EINVAL, "more than 2^31 facets in one LoD"};
    ld.maxF = 0;
    ld.coff_h.assign(n + 1, 0);
    for (int o = 0; o < n; ++o) {
      int64_t fo = ld.foff_h[o + 1] - ld.foff_h[o];
      ld.maxF = std::max(ld.maxF, fo);
      ld.coff_h[o + 1] = ld.coff_h[o] + (fo + CHUNK - 1) / CHUNK;
    }
    ld.C = ld.coff_h[n];
    ld.boff_h.assign(n + 1, 0);
    for (int o = 0; o < n; ++o) {
      int64_t fo = ld.foff_h[o + 1] - ld.foff_h[o];
      ld.boff_h[o + 1] = ld.boff_h[o] + (fo + BLK - 1) / BLK;
    }
    ld.B = ld.boff_h[n];
    // uploads (or, for pinned arrays with zero_copy, their device views)
    float* dv;
    auto it = vcache.find(D->verts[l]);
    if (it != vcache.end()) {
      dv = it->second;
    } else if (const void* pv = pinned_view(ctx, D->verts[l])) {
      dv = (float*)pv;
      vcache[D->verts[l]] = dv;
    } else {
      dv = upload(D->verts[l], (size_t)nv * 3, st);
      temps.push_back(dv);
      vcache[D->verts[l]] = dv;
    }
    int64_t* dvo = (int64_t*)pinned_view(ctx, vo);
    if (!dvo) {
      dvo = upload(vo, (size_t)n + 1, st);
      temps.push_back(dvo);
    }
    size_t nrows = shared ? (size_t)nfs : (size_t)ld.F;
    int32_t* dfa = (int32_t*)pinned_view(ctx, D->faces[l]);
    if (!dfa) {
      dfa = upload(D->faces[l], nrows * 3, st);
      temps.push_back(dfa);
    }
    ld.foff = upload(ld.foff_h.data(), (size_t)n + 1, st);
    ld.coff = upload(ld.coff_h.data(), (size_t)n + 1, st);
    ld.boff = upload(ld.boff_h.data(), (size_t)n + 1, st);
    float* dhd = nullptr;
    float* dph = nullptr;
    if (D->hd[l] && !(dhd = (float*)pinned_view(ctx, D->hd[l]))) {
      dhd = upload(D->hd[l], (size_t)ld.F, st);
      temps.push_back(dhd);
    }
    if (D->ph[l] && !(dph = (float*)pinned_view(ctx, D->ph[l]))) {
      dph = upload(D->ph[l], (size_t)ld.F, st);
      temps.push_back(dph);
    }
    note_alloc();
    PJ_CK(cudaMallocAsync((void**)&ld.fac, std::max<int64_t>(1, 3 * ld.F) * sizeof(float4), st));
    note_alloc();
    PJ_CK(cudaMallocAsync((void**)&ld.chunk, std::max<int64_t>(1, 3 * ld.C) * sizeof(float4), st));
    note_alloc();
    PJ_CK(cudaMallocAsync((void**)&ld.blk, std::max<int64_t>(1, 3 * ld.B) * sizeof(float4), st));
    raw[l] = RawLod{dv, dvo, dfa, nfs, dhd, dph};
  }
  note_alloc();
  PJ_CK(cudaMallocAsync((void**)&s->mbb, std::max(1, n) * 6 * sizeof(float), st));
  s->anchor = upload(D->anchor, (size_t)n * 3, st);
  build_set_kernels(ctx, s, raw, st);
  if (ctx->voxelize) voxelize_set(ctx, s, raw[0].verts, raw[0].voff, st);
  s->mbb_h.resize((size_t)n * 6);
  if (n > 0) PJ_CK(cudaMemcpyAsync(s->mbb_h.data(), s->mbb, (size_t)n * 6 * 4, cudaMemcpyDeviceToHost, st));
  int herr = 0;
  PJ_CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  for (void* p : temps.v) PJ_CK(cudaFreeAsync(p, st));
  temps.v.clear();
  PJ_CK(cudaStreamSynchronize(st));
  if (herr & ERR_BOUNDS) throw ApiError{PJ_EBOUNDS, "a face index lies outside its object's vertices"};
  if (herr & ERR_NONFINITE) throw ApiError{PJ_ENONFINITE, "non-finite vertex, anchor, hd or ph (or negative hd/ph)"};
  return PJ_OK;
}

static std::string json_str(const char* js, const char* key) {
  if (!js) return "";
  std::string s(js), k = std::string("\"") + key + "\"";
  size_t p = s.find(k);
  if (p == std::string::npos) return "";
  p = s.find(':', p + k.size());
  if (p == std::string::npos) return "";
  ++p;
  while (p < s.size() && (s[p] == ' ' || s[p] == '\t')) ++p;
  if (p < s.size() && s[p] == '"') {
    size_t e = s.find('"', p + 1);
    return e == std::string::npos ? "" : s.substr(p + 1, e - p - 1);
  }
  size_t e = p;
  while (e < s.size() && s[e] != ',' && s[e] != '}') ++e;
  return s.substr(p, e - p);
}

pj_ctx* join_twin(pj_ctx* ctx) {
  if (!ctx->twin) {
    pj_ctx* t = new pj_ctx();
    t->device = ctx->device;
    t->sm_count = ctx->sm_count;
    t->cc_major = ctx->cc_major;
    t->cc_minor = ctx->cc_minor;
    try {
      PJ_CK(cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking));
      int lo = 0, hi = 0;
      PJ_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      PJ_CK(cudaStreamCreateWithPriority(&t->join_stream, cudaStreamNonBlocking, hi));
      note_alloc();
      PJ_CK(cudaMalloc((void**)&t->d_err, sizeof(int)));
      note_alloc();
      PJ_CK(cudaMalloc((void**)&t->d_counters, 16 * sizeof(unsigned long long)));
      PJ_CK(cudaMemset(t->d_err, 0, sizeof(int)));
      PJ_CK(cudaMemset(t->d_counters, 0, 16 * sizeof(unsigned long long)));
      for (auto& e : t->ev) PJ_CK(cudaEventCreate(&e));
      note_alloc();
      PJ_CK(cudaMalloc((void**)&t->d_snap, 64 * 4 * sizeof(long long)));
    } catch (...) {
      pj_destroy(t);
      throw;
    }
    t->borrowed_mlp = true;
    ctx->twin = t;
  }
  pj_ctx* t = ctx->twin;
  t->ctas_per_sm = ctx->ctas_per_sm;
  t->refine_variant = ctx->refine_variant;
  t->variant_fixed = ctx->variant_fixed;
  t->refine_split = ctx->refine_split;
  t->refine_tail = ctx->refine_tail;
  t->split_fixed = ctx->split_fixed;
  t->sched_start = ctx->sched_start;
  t->unit_budget = ctx->unit_budget;
  t->mlp_w = ctx->mlp_w;
  t->mlp_ready = ctx->mlp_ready;
  t->tuned = ctx->tuned;
  return t;
}

}  // namespace pj

using namespace pj;

static pj_status fail(pj_ctx* ctx, pj_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

#define PJ_API_TRY try {
#define PJ_API_CATCH(ctx)                                                                         \
  }                                                                                               \
  catch (const pj::CudaError& e) {                                                                \
    std::string m = std::string(e.what) + ": " + cudaGetErrorString(e.e);                         \
    return fail(ctx, e.e == cudaErrorMemoryAllocation ? PJ_ENOMEM : PJ_ECUDA, m);                 \
  }                                                                                               \
  catch (const pj::ApiError& e) {                                                                 \
    return fail(ctx, e.st, e.msg);                                                                \
  }                                                                                               \
  catch (const std::bad_alloc&) {                                                                 \
    return fail(ctx, PJ_ENOMEM, "host allocation failed");                                        \
  }                                                                                               \
  catch (...) {                                                                                   \
    return fail(ctx, PJ_EINVAL, "unexpected internal error");                                     \
  }

extern "C" {

const char* pj_status_str(pj_status s) {
  switch (s) {
    case PJ_OK: return "PJ_OK";
    case PJ_EINVAL: return "PJ_EINVAL";
    case PJ_ENOMEM: return "PJ_ENOMEM";
    case PJ_ECUDA: return "PJ_ECUDA";
    case PJ_ETIMEOUT: return "PJ_ETIMEOUT";
    case PJ_ENONFINITE: return "PJ_ENONFINITE";
    case PJ_EBOUNDS: return "PJ_EBOUNDS";
    case PJ_ECANCELLED: return "PJ_ECANCELLED";
    case PJ_ESOURCE: return "PJ_ESOURCE";
  }
  return "unknown";
}

const char* pj_last_error(const pj_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

pj_status pj_create(pj_ctx** out, int device, const char* options_json) {
  if (!out) return PJ_EINVAL;
  *out = nullptr;
  pj_ctx* ctx = new (std::nothrow) pj_ctx();
  if (!ctx) return PJ_ENOMEM;
  PJ_API_TRY
  int ndev = 0;
  PJ_CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) throw ApiError{PJ_EINVAL, "no such CUDA device"};
  PJ_CK(cudaSetDevice(device));
  cudaDeviceProp prop;
  PJ_CK(cudaGetDeviceProperties(&prop, device));
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  ctx->cc_major = prop.major;
  ctx->cc_minor = prop.minor;
  if (!(prop.major == 10 && prop.minor == 3))
    throw ApiError{PJ_ECUDA, "this library is built for sm_103a (GB300); device is sm_" +
                                 std::to_string(prop.major) + std::to_string(prop.minor)};
  PJ_CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
  {
    // keep freed pool memory for the next set instead of returning it
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    (void)cudaGetLastError();
  }
  PJ_CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  PJ_CK(cudaStreamCreateWithFlags(&ctx->build_stream, cudaStreamNonBlocking));
  {
    int lo = 0, hi = 0;
    PJ_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    PJ_CK(cudaStreamCreateWithPriority(&ctx->join_stream, cudaStreamNonBlocking, hi));
  }
  note_alloc();
  PJ_CK(cudaMalloc((void**)&ctx->d_err, sizeof(int)));
  note_alloc();
  PJ_CK(cudaMalloc((void**)&ctx->d_counters, 16 * sizeof(unsigned long long)));
  PJ_CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
  PJ_CK(cudaMemset(ctx->d_counters, 0, 16 * sizeof(unsigned long long)));
  for (auto& e : ctx->ev) PJ_CK(cudaEventCreate(&e));
  note_alloc();
  PJ_CK(cudaMalloc((void**)&ctx->d_snap, 64 * 4 * sizeof(long long)));
  std::string v = json_str(options_json, "persistent_ctas_per_sm");
  if (!v.empty()) ctx->ctas_per_sm = std::max(0, atoi(v.c_str()));
  v = json_str(options_json, "refine_variant");
  if (!v.empty()) {
    const int rv = atoi(v.c_str());
    if (rv != 1 && rv != 2) {
      pj_destroy(ctx);
      return PJ_EINVAL;
    }
    ctx->refine_variant = rv;
    ctx->variant_fixed = true;
  }
  v = json_str(options_json, "refine_split");
  if (!v.empty()) {
    const int k = atoi(v.c_str());
    if (k != 1 && k != 2 && k != 4 && k != 8) {
      pj_destroy(ctx);
      return PJ_EINVAL;
    }
    ctx->refine_split = k;
    ctx->split_fixed = true;
  }
  v = json_str(options_json, "host_read");
  if (!v.empty()) ctx->host_read = atoi(v.c_str()) != 0;
  v = json_str(options_json, "chunk_overlap");
  if (!v.empty()) ctx->chunk_overlap = atoi(v.c_str()) != 0;
  v = json_str(options_json, "voxels");
  if (!v.empty()) ctx->voxelize = atoi(v.c_str()) != 0;
  v = json_str(options_json, "zero_copy");
  if (!v.empty()) ctx->zero_copy = atoi(v.c_str()) != 0;
  v = json_str(options_json, "refine_tail");
  if (!v.empty()) {
    const int t = atoi(v.c_str());
    if (t < 0 || t > 64) {
      pj_destroy(ctx);
      return PJ_EINVAL;
    }
    ctx->refine_tail = t;
    ctx->split_fixed = true;
  }
  v = json_str(options_json, "unit_budget_mb");
  if (!v.empty()) {
    const long long mb = atoll(v.c_str());
    if (mb < 1 || mb > (1LL << 20)) {
      pj_destroy(ctx);
      return PJ_EINVAL;
    }
    ctx->unit_budget = (size_t)mb << 20;
  }
  ctx->autotune_cache = json_str(options_json, "autotune_cache");
  *out = ctx;
  return PJ_OK;
  }
  catch (const pj::CudaError& e) {
    pj_status st = PJ_ECUDA;
    delete ctx;
    (void)e;
    return st;
  }
  catch (const pj::ApiError& e) {
    delete ctx;
    return e.st;
  }
  catch (...) {
    delete ctx;
    return PJ_ECUDA;
  }
}

void pj_destroy(pj_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->twin) {
    pj_destroy(ctx->twin);
    ctx->twin = nullptr;
  }
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  graphs_clear(ctx);
  destroy_pack_pool(ctx->pack_pool);
  for (auto& b : ctx->ws) cudaFree(b.p);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_counters);
  if (!ctx->borrowed_mlp) cudaFree(ctx->mlp_w);
  cudaFree(ctx->d_snap);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  for (void* hp : ctx->stream_pinned)
    if (hp) cudaFreeHost(hp);
  for (void* hp : ctx->stream_box_pinned)
    if (hp) cudaFreeHost(hp);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->build_stream) cudaStreamDestroy(ctx->build_stream);
  if (ctx->join_stream) cudaStreamDestroy(ctx->join_stream);
  delete ctx;
}

pj_status pj_load_set(pj_ctx* ctx, const pj_mesh_set_desc* desc, pj_set** out) {
  if (!ctx || !desc || !out) return PJ_EINVAL;
  *out = nullptr;
  pj_set* s = new (std::nothrow) pj_set();
  if (!s) return fail(ctx, PJ_ENOMEM, "host allocation failed");
  s->ctx = ctx;
  s->device = ctx->device;
  try {
    PJ_CK(cudaSetDevice(ctx->device));
    (void)cudaGetLastError();  // drop a stale non-sticky error of an unrelated call
    load_set_impl(ctx, desc, s, ctx->stream);
    static std::atomic<uint64_t> next_uid{1};
    s->uid = next_uid.fetch_add(1);
    *out = s;
    return PJ_OK;
  } catch (const pj::CudaError& e) {
    free_set_storage(s);
    delete s;
    return fail(ctx, e.e == cudaErrorMemoryAllocation ? PJ_ENOMEM : PJ_ECUDA,
                std::string(e.what) + ": " + cudaGetErrorString(e.e));
  } catch (const pj::ApiError& e) {
    free_set_storage(s);
    delete s;
    return fail(ctx, e.st, e.msg);
  } catch (...) {
    free_set_storage(s);
    delete s;
    return fail(ctx, PJ_ENOMEM, "host allocation failed");
  }
}

pj_status pj_load_set_streamed(pj_ctx* ctx, int64_t n_objects, int n_chunks, pj_fill_fn fill, void* user,
                               pj_set** out) {
  if (!ctx || !out || !fill || n_objects < 0 || n_chunks < 1) return fail(ctx, PJ_EINVAL, "bad streamed set");
  pj_set* s = new (std::nothrow) pj_set();
  if (!s) return fail(ctx, PJ_ENOMEM, "host allocation failed");
  s->ctx = ctx;
  s->device = ctx->device;
  s->streamed = true;
  s->n_total = n_objects;
  s->n_chunks = n_chunks;
  s->fill = fill;
  s->user = user;
  *out = s;
  return PJ_OK;
}

void pj_free_set(pj_set* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  free_set_storage(s);
  delete s;
}

pj_status pj_join_async(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, void* cuda_stream,
                        pj_result* out) {
  if (!ctx || !R || !S || !q || !out) return fail(ctx, PJ_EINVAL, "null argument");
  memset(out, 0, sizeof(*out));
  if (S->streamed) return fail(ctx, PJ_EINVAL, "only R may be a streamed set");
  if (q->pred == PJ_WITHIN && !(q->tau >= 0.0 && std::isfinite(q->tau)))
    return fail(ctx, PJ_EINVAL, "tau must be finite and >= 0");
  if (q->pred == PJ_KNN && q->k < 1) return fail(ctx, PJ_EINVAL, "k must be >= 1");
  if (q->pred != PJ_WITHIN && q->pred != PJ_INTERSECT && q->pred != PJ_KNN)
    return fail(ctx, PJ_EINVAL, "unknown predicate");
  if (q->prec != PJ_PREC_FP64 && q->prec != PJ_PREC_FP32_REDECIDE) return fail(ctx, PJ_EINVAL, "unknown precision");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  PJ_API_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  (void)cudaGetLastError();
  std::string stats;
  pj_status rc;
  if (R->streamed) rc = join_streamed(ctx, R, S, q, out, st, stats);
  else if (q->flags & PJ_AUTOTUNE) rc = join_autotuned(ctx, R, S, q, out, st, stats);
  else if (q->pred == PJ_KNN) rc = join_knn(ctx, R, S, q, out, st, stats);
  else rc = join_within(ctx, R, S, q, out, st, stats);
  ctx->stats = stats;
  if (rc != PJ_OK) {
    if (out->priv) pj_result_free(out);
    if (ctx->last_error.empty() || rc == PJ_ETIMEOUT)
      ctx->last_error = rc == PJ_ETIMEOUT ? "deadline expired or a device wait hit its limit" : pj_status_str(rc);
  }
  return rc;
  PJ_API_CATCH(ctx)
}

pj_status pj_join(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out) {
  return pj_join_async(ctx, R, S, q, nullptr, out);
}

void pj_result_free(pj_result* res) {
  if (!res) return;
  free(res->priv);
  memset(res, 0, sizeof(*res));
}

pj_status pj_get_stats(const pj_ctx* ctx, char* buf, size_t cap) {
  if (!ctx || !buf || cap == 0) return PJ_EINVAL;
  // the last join's record plus the library's allocation count and the
  // context's workspace bytes at the time of the call
  std::string s = ctx->stats.empty() ? std::string("{}") : ctx->stats;
  size_t ws = 0;
  for (const auto& b : ctx->ws) ws += b.cap;
  const size_t close = s.rfind('}');
  if (close != std::string::npos) {
    const bool empty = s.find_first_not_of(" \n\t{", 0) == close;
    s.insert(close, std::string(empty ? "" : ", ") + "\"allocs\": " + std::to_string(g_allocs.load()) +
                        ", \"ws_bytes\": " + std::to_string(ws));
  }
  if (s.size() + 1 > cap) return PJ_EINVAL;
  memcpy(buf, s.c_str(), s.size() + 1);
  return PJ_OK;
}

pj_status pj_tri_dist(pj_ctx* ctx, const float* P, const float* Q, int64_t n, pj_precision prec, double* out,
                      double* err_out, void* cuda_stream) {
  if (!ctx || n < 0 || (n > 0 && (!P || !Q || !out))) return fail(ctx, PJ_EINVAL, "bad tri_dist arguments");
  PJ_API_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  (void)cudaGetLastError();
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  tri_dist_batch(ctx, P, Q, n, prec == PJ_PREC_FP64, out, err_out, st);
  PJ_CK(cudaStreamSynchronize(st));
  return PJ_OK;
  PJ_API_CATCH(ctx)
}

pj_status pj_pair_bounds(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps,
                         int64_t n, int lod, pj_precision prec, double* lb, double* ub) {
  if (!ctx || !R || !S || n < 0 || (n > 0 && (!pr || !ps || !lb || !ub)))
    return fail(ctx, PJ_EINVAL, "bad pair_bounds arguments");
  if (R->streamed || S->streamed) return fail(ctx, PJ_EINVAL, "streamed sets are not addressable");
  if (lod < 0 || lod >= R->L || lod >= S->L) return fail(ctx, PJ_EINVAL, "lod out of range");
  for (int64_t i = 0; i < n; ++i)
    if (pr[i] < 0 || pr[i] >= R->n || ps[i] < 0 || ps[i] >= S->n) return fail(ctx, PJ_EBOUNDS, "pair id out of range");
  if (n == 0) return PJ_OK;
  PJ_API_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  (void)cudaGetLastError();
  cudaStream_t st = ctx->stream;
  auto dpr = (int32_t*)ws_get(ctx, WS_PR, n * 4, st);
  auto dps = (int32_t*)ws_get(ctx, WS_PS, n * 4, st);
  PJ_CK(cudaMemcpyAsync(dpr, pr, n * 4, cudaMemcpyHostToDevice, st));
  PJ_CK(cudaMemcpyAsync(dps, ps, n * 4, cudaMemcpyHostToDevice, st));
  PJ_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  setup_pairs(ctx, R, S, n, 0.0, false, st);
  StepSpec sp;
  sp.lodR = lod;
  sp.lodS = lod;
  sp.full = (lod == R->L - 1) && (lod == S->L - 1);
  sp.fp64 = prec == PJ_PREC_FP64;
  sp.cull = false;
  sp.want = UNDECIDED;
  sp.step = 0;
  sp.exact_cross = true;
  init_bounds(ctx, n, sp, st);
  UnitCount nt = build_tiles(ctx, R, S, n, sp, st);
  run_refine(ctx, R, S, nt, sp, st);
  std::vector<unsigned char> blo(n * 8), bub(n * 8);
  PJ_CK(cudaMemcpyAsync(blo.data(), ctx->ws[WS_LB].p, n * (sp.fp64 ? 8 : 4), cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaMemcpyAsync(bub.data(), ctx->ws[WS_UB].p, n * (sp.fp64 ? 8 : 4), cudaMemcpyDeviceToHost, st));
  int herr = 0;
  PJ_CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  if (herr & ERR_MBAR_TIMEOUT) return fail(ctx, PJ_ETIMEOUT, "a device wait hit its limit");
  for (int64_t i = 0; i < n; ++i) {
    if (sp.fp64) {
      double a, b;
      memcpy(&a, &blo[8 * i], 8);
      memcpy(&b, &bub[8 * i], 8);
      lb[i] = a;
      ub[i] = b;
    } else {
      float a, b;
      memcpy(&a, &blo[4 * i], 4);
      memcpy(&b, &bub[4 * i], 4);
      lb[i] = a;
      ub[i] = b;
    }
  }
  return PJ_OK;
  PJ_API_CATCH(ctx)
}

pj_status pj_voxel_count(const pj_set* set, int64_t* n_voxels) {
  if (!set || !n_voxels) return PJ_EINVAL;
  if (!set->voxels) return PJ_EINVAL;
  *n_voxels = set->V;
  return PJ_OK;
}

pj_status pj_voxels_read(pj_ctx* ctx, const pj_set* set, int64_t* voxel_off, double* centre, float* box,
                         float* anchor) {
  if (!ctx || !set) return fail(ctx, PJ_EINVAL, "bad voxels_read arguments");
  if (!set->voxels) return fail(ctx, PJ_EINVAL, "the set was loaded without voxels (context option \"voxels\")");
  PJ_API_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  if (voxel_off) memcpy(voxel_off, set->vox_off_h.data(), ((size_t)set->n + 1) * 8);
  const size_t V = (size_t)set->V;
  if (centre && V) PJ_CK(cudaMemcpyAsync(centre, set->vox_centre, V * 3 * 8, cudaMemcpyDeviceToHost, st));
  if (box && V) PJ_CK(cudaMemcpyAsync(box, set->vox_box, V * 6 * 4, cudaMemcpyDeviceToHost, st));
  if (anchor && V) PJ_CK(cudaMemcpyAsync(anchor, set->vox_anchor, V * 3 * 4, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  return PJ_OK;
  PJ_API_CATCH(ctx)
}

pj_status pj_voxel_labels_read(pj_ctx* ctx, const pj_set* set, int lod, int32_t* label) {
  if (!ctx || !set || !label) return fail(ctx, PJ_EINVAL, "bad voxel_labels_read arguments");
  if (!set->voxels) return fail(ctx, PJ_EINVAL, "the set was loaded without voxels (context option \"voxels\")");
  if (lod < 0 || lod >= set->L) return fail(ctx, PJ_EINVAL, "lod out of range");
  PJ_API_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const size_t F = (size_t)set->lod[lod].F;
  if (F) PJ_CK(cudaMemcpyAsync(label, set->vox_label[lod], F * 4, cudaMemcpyDeviceToHost, st));
  PJ_CK(cudaStreamSynchronize(st));
  return PJ_OK;
  PJ_API_CATCH(ctx)
}

pj_status pj_voxel_filter(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps,
                          int64_t n, double tau, pj_precision prec, double* op_lb, double* op_ub, uint8_t* status, int64_t* vp_off,
                          double* vp_lb, double* vp_ub, int64_t vp_cap, int64_t* kept_off, int32_t* kept,
                          int64_t* n_kept, void* cuda_stream) {
  if (!ctx || !R || !S || n < 0 || vp_cap < 0 || !n_kept || !vp_off || !kept_off)
    return fail(ctx, PJ_EINVAL, "bad voxel_filter arguments");
  if (n > 0 && (!pr || !ps || !op_lb || !op_ub || !status)) return fail(ctx, PJ_EINVAL, "bad voxel_filter arguments");
  if (vp_cap > 0 && (!vp_lb || !vp_ub || !kept)) return fail(ctx, PJ_EINVAL, "bad voxel_filter arguments");
  if (!R->voxels || !S->voxels)
    return fail(ctx, PJ_EINVAL, "a set was loaded without voxels (context option \"voxels\")");
  if (n >= (1LL << 31)) return fail(ctx, PJ_EINVAL, "more than 2^31 object pairs");
  if (prec != PJ_PREC_FP64 && prec != PJ_PREC_FP32_REDECIDE) return fail(ctx, PJ_EINVAL, "unknown precision");
  PJ_API_TRY
  PJ_CK(cudaSetDevice(ctx->device));
  (void)cudaGetLastError();
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  voxel_filter(ctx, R, S, pr, ps, n, tau, prec == PJ_PREC_FP64, op_lb, op_ub, status, vp_off, vp_lb, vp_ub, vp_cap,
               kept_off, kept,
               n_kept, st);
  return PJ_OK;
  PJ_API_CATCH(ctx)
}

}  // extern "C"
