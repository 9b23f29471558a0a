/*
 * pj.h -- C ABI of the GB300 (sm_103a) polyhedral spatial join library.
 *
 * Problem statement (3DPipe, arXiv 2604.19982, section 3): for every object r
 * of a set R, find the objects s of a set S with
 *   - intersection:     d(r, s) = 0,
 *   - within-tau:       d(r, s) <= tau,
 *   - k nearest (k-NN): the k smallest d(r, s), ties broken by the id of s,
 * where d is the minimum Euclidean distance between the two triangle
 * surfaces (section 2.1).  Objects carry levels of detail (LoDs) with
 * per-facet Hausdorff bounds hd / ph (section 2.1, Eq. 1 and Eq. 2) so that
 * pairs can be decided at a coarse LoD; the answer is always the one of the
 * original (finest) surfaces.
 *
 * Conventions
 *   - Every call returns pj_status (0 = PJ_OK, < 0 error).  Outputs are valid
 *     only on PJ_OK.  On error, pj_last_error(ctx) describes it; the context
 *     stays usable unless the status is PJ_ECUDA with a sticky CUDA error.
 *   - No C++ exception crosses this boundary.  A context is used by one host
 *     thread at a time.
 *   - "host" pointers are ordinary (pageable or pinned) CPU memory, "device"
 *     pointers are CUDA global memory of the context's device.  The library
 *     never frees caller memory and copies what it keeps.
 *   - All arithmetic of the join runs in this library's CUDA kernels; there is
 *     no CPU fallback: without a usable GPU, pj_create fails with PJ_ECUDA.
 */
#ifndef PJ_H
#define PJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PJ_OK = 0,
  PJ_EINVAL = -1,      /* bad argument (null pointer, size, predicate, ...) */
  PJ_ENOMEM = -2,      /* device or pinned-host allocation failed           */
  PJ_ECUDA = -3,       /* CUDA runtime error (message in pj_last_error)     */
  PJ_ETIMEOUT = -4,    /* query deadline (pj_query.timeout_s) expired, or a
                          device-side wait hit its iteration limit          */
  PJ_ENONFINITE = -5,  /* a vertex, hd or ph value is NaN or infinite       */
  PJ_EBOUNDS = -6,     /* an index is out of range (face -> vertex, ...)    */
  PJ_ECANCELLED = -7,  /* a streaming source asked to stop                  */
  PJ_ESOURCE = -8      /* a streaming source callback reported an error     */
} pj_status;

typedef enum { PJ_WITHIN = 0, PJ_INTERSECT = 1, PJ_KNN = 2 } pj_predicate;

/* Arithmetic of the triangle-distance tests.
 *   PJ_PREC_FP64: every test in double precision (the plain path).
 *   PJ_PREC_FP32_REDECIDE: tests in single precision with a forward error
 *     bound per tile; a pair whose single-precision bracket straddles the
 *     decision threshold at full resolution is re-decided in double
 *     precision, so decisions equal those of the FP64 path. */
typedef enum { PJ_PREC_FP64 = 0, PJ_PREC_FP32_REDECIDE = 1 } pj_precision;

/* pj_query.flags */
enum {
  PJ_EXACT_DIST = 1,   /* refine every result pair to its exact FP64 distance  */
  PJ_USE_MLP = 2,      /* learned proposal: order k-NN work, pick start LoD    */
  PJ_USE_GRAPH = 4,    /* replay the per-LoD launch sequence from a CUDA graph */
  PJ_AUTOTUNE = 8,     /* time the FP32 refinement variant (tests per lane) and
                          the LoD start step, then the unit tile (32 r facets
                          x 32, 16 or 8 s facets), on the first join of a
                          workload, keep the fastest (cached per context and
                          in "autotune_cache"; the choices and the timed
                          trials are in the join's stats under "autotune") */
  PJ_TILE_PRUNE = 16   /* skip facet tiles/blocks that cannot change a decision */
};

typedef struct pj_ctx pj_ctx; /* opaque, library-owned */
typedef struct pj_set pj_set; /* opaque, library-owned, device resident */

#define PJ_MAX_LODS 8

/* A set of closed triangle meshes with n_lods levels of detail (LoD 0 =
 * coarsest, n_lods-1 = original surface).  All pointers are HOST memory,
 * read during pj_load_set only.
 *   verts[l]     float32 [nv_l][3]; several LoDs may pass the same array.
 *   vert_off[l]  int64 [n_objects + 1]: object o owns vertices
 *                vert_off[l][o] .. vert_off[l][o+1]-1 of verts[l].
 *   faces[l]     int32 [..][3] object-local vertex ids.  With face_off[l]
 *                non-NULL (int64 [n_objects + 1]) object o owns face rows
 *                face_off[l][o] .. face_off[l][o+1]-1; with face_off[l] NULL
 *                all objects share the n_faces_shared[l] rows of faces[l].
 *   hd[l], ph[l] float32, one per face of the LoD in object order (rows of
 *                object 0, then object 1, ...): facet-level Hausdorff bound
 *                hd(f', P) and proxy Hausdorff bound ph(P, f') (section 2.1),
 *                already rounded up.  NULL means 0 (required at the last LoD).
 *   anchor       float32 [n_objects][3]: a point of each original surface
 *                (its distance to another anchor bounds d from above,
 *                section 2.1 "Object and Voxel Centers").
 * Errors: PJ_EINVAL for inconsistent sizes, PJ_EBOUNDS for a face index
 * outside its object's vertices, PJ_ENONFINITE for NaN/Inf data. */
typedef struct {
  int32_t n_objects;
  int32_t n_lods;
  const float* verts[PJ_MAX_LODS];
  const int64_t* vert_off[PJ_MAX_LODS];
  const int32_t* faces[PJ_MAX_LODS];
  const int64_t* face_off[PJ_MAX_LODS];
  int32_t n_faces_shared[PJ_MAX_LODS];
  const float* hd[PJ_MAX_LODS];
  const float* ph[PJ_MAX_LODS];
  const float* anchor;
} pj_mesh_set_desc;

/* One join.  pred PJ_INTERSECT ignores tau (uses 0); PJ_KNN uses k >= 1.
 * timeout_s <= 0 means no deadline. */
typedef struct {
  pj_predicate pred;
  double tau;
  int32_t k;
  pj_precision prec;
  uint32_t flags;
  double timeout_s;
} pj_query;

/* Result pairs, library-owned host memory (free with pj_result_free); the
 * device-to-host copy goes through the context's pinned staging buffer.
 * within/intersection: ordered by (r, s).  k-NN: for each r in order,
 * min(k, |S|) entries ordered by (d, s).
 *   d_lo <= d(r, s) <= d_hi always holds; d is the best estimate.
 *   exact[i] = 1: d_lo = d = d_hi is the FP64 full-resolution distance;
 *   exact[i] = 2: d is a single-precision full-resolution distance and
 *                 [d_lo, d_hi] its forward error bracket;
 *   exact[i] = 0: decided from a coarse LoD or from the anchor bound, only
 *                 the bracket is known (set PJ_EXACT_DIST to refine). */
typedef struct {
  int64_t n;
  int32_t* r;
  int32_t* s;
  double* d_lo;
  double* d_hi;
  double* d;
  uint8_t* exact;
  void* priv; /* library use */
} pj_result;

/* Create a context on CUDA device `device`.  options_json may be NULL or a
 * JSON object with optional keys "persistent_ctas_per_sm" (int, 0 = from
 * occupancy), "refine_variant" (1, the default: scalar single-precision
 * refinement, one triangle test per lane and instruction; 2: packed FP32x2
 * refinement, two tests per lane and instruction; anything else gives
 * PJ_EINVAL; when given, PJ_AUTOTUNE keeps it and tunes the schedule only),
 * "refine_split" (1 (default), 2, 4 or 8: the last units of a
 * refinement launch are handed out as that many parts over their s facets,
 * 1 = never; anything else gives PJ_EINVAL; parts restart the facet-ball
 * culling bound, so splitting pays only when launches are tail-bound),
 * "refine_tail" (0..64, default 2: how many units per resident warp are
 * split; when either of the two is given, PJ_AUTOTUNE keeps them and does
 * not tune the tile), "zero_copy" (0, the default, or 1: pj_load_set reads the arrays
 * that live in pinned, mapped host memory in place over the host link
 * instead of staging them, other arrays are copied as usual),
 * "unit_budget_mb" (1 .. 2^20, default 512: the refinement-unit buffer is
 * sized for a step's worst case when that fits this budget; otherwise units
 * are emitted into the buffer as it is, and a join whose units overflowed
 * it grows the buffer to the count needed and runs again), "chunk_overlap"
 * (1, the default, or 0: a streamed within-tau / intersection join with
 * PJ_USE_GRAPH takes its chunks in turn on the context and a second,
 * internal join context with its own workspace and stream, so that one
 * chunk's join is issued before the previous one is waited for),
 * "host_read" (1, the default, or 0: copy the middle-LoD arrays of streamed
 * chunks in pinned host memory like the others instead of reading them in
 * place), "voxels" (0, the default, or 1: pj_load_set also voxelizes every
 * object it loads, see pj_voxel_count; joins do not read the voxels) and
 * "autotune_cache" (path string).  The options change scheduling only,
 * never a result.  Fails with PJ_ECUDA when the device is not compute
 * capability 10.3 (GB300). */
pj_status pj_create(pj_ctx** out, int device, const char* options_json);
void pj_destroy(pj_ctx* ctx);

/* Copy a mesh set to the device and lay it out for refinement: per LoD,
 * de-indexed facets (three float4: vertex xyz + hd, vertex xyz + ph, vertex
 * xyz + 0), per-object facet offsets, per-256-facet chunk boxes, and per
 * object its original-surface box and anchor.  Synchronous. */
pj_status pj_load_set(pj_ctx* ctx, const pj_mesh_set_desc* desc, pj_set** out);

/* A set streamed in n_chunks pieces during pj_join (R side only).  For each
 * chunk the library calls fill(user, chunk, &desc) from one of its two
 * loader threads, in chunk order and never two calls at once; the
 * callback fills desc with that chunk's objects.  Object ids of chunk c
 * continue those of chunk c-1.  A fill returning PJ_ECANCELLED stops the
 * join with that status; any other non-zero value gives PJ_ESOURCE.
 * Where the arrays may live, and for how long:
 *   - pageable host memory: packed into the library's pinned staging, so it
 *     must stay valid until fill is called for chunk c + 2 (chunk c + 1 may
 *     be filled while chunk c is still being packed) or the join ends;
 *   - pinned host memory (cudaHostAlloc / cudaHostRegister): copied to the
 *     device directly, without packing (the link-bound path); the hd, ph,
 *     per-object faces and own vertex arrays of the LoDs between the first
 *     and the last are not copied but read in place over the host link, for
 *     the objects whose pairs reach those LoDs; so it must stay valid and
 *     unchanged until pj_join returns;
 *   - device memory (verts, faces, hd, ph, anchor only): read in place by
 *     the set-building kernels, likewise until pj_join returns.
 * vert_off and face_off are always host memory (read by the host, with the
 * lifetime of pageable arrays; PJ_EINVAL otherwise). */
typedef pj_status (*pj_fill_fn)(void* user, int chunk, pj_mesh_set_desc* out);
pj_status pj_load_set_streamed(pj_ctx* ctx, int64_t n_objects, int n_chunks, pj_fill_fn fill,
                               void* user, pj_set** out);
void pj_free_set(pj_set* set);

/* Join R against S.  Synchronous; results in *out (caller-allocated struct,
 * library-allocated arrays). */
pj_status pj_join(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, pj_result* out);

/* Same as pj_join but every device operation is issued on `cuda_stream`
 * (a cudaStream_t of the context's device, NULL = the context's stream); the
 * call returns once the results are on the host, synchronizing only that
 * stream. */
pj_status pj_join_async(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q,
                        void* cuda_stream, pj_result* out);
void pj_result_free(pj_result* res);

/* Counters and timings of the last join as a JSON object (candidates, pairs
 * decided per LoD, tiles, triangle tests scheduled/executed per precision,
 * re-decided pairs, bytes copied, milliseconds per stage).  Among them:
 * "tests_fp32" / "tests_fp64" (facet-pair tests executed), "tests_culled"
 * (facet pairs skipped by the facet-ball tests), "tests_needed" (executed
 * tests that the testing lane's own ball test asked for; the others ran
 * because another lane of the warp needed the same s facet), and per step
 * in "steps": "tiles" (units built) and "tiles_run" (units left after the
 * full-resolution mask pass).  A join with a streamed R adds per-stage
 * times summed over its chunks ("ms_fill", "ms_pack", "ms_wait_loader",
 * "ms_build", "ms_join", "ms_filter", "ms_h2d"), "bytes_h2d" (copied to
 * the device), "bytes_host_read_max" (pinned caller arrays read in place;
 * at most this many bytes cross the link), "graph_replays" /
 * "graph_captures" and, with PJ_AUTOTUNE, the tuned choice under
 * "autotune".  Also, at the time of the call: "allocs", the
 * number of device and pinned-host allocations the library has made in this
 * process (all contexts), and "ws_bytes", the context's workspace bytes.
 * Fails with PJ_EINVAL when cap is too small. */
pj_status pj_get_stats(const pj_ctx* ctx, char* json_buf, size_t cap);

/* ------------------------------------------------------------------ *
 * Learned proposal (optional): a 16 -> 64 -> 64 -> 1 ReLU MLP in bf16 on
 * the tensor cores predicting log(1 + d) of a pair from box and coarse-LoD
 * features.  It only orders k-NN refinement and picks the starting LoD; it
 * never changes a result.
 * ------------------------------------------------------------------ */

/* With PJ_USE_MLP a join first predicts y = log(1 + d) for every candidate
 * pair.  k-NN: each step's first wave (the k candidates of every r refined
 * before the rest, section 3.4) is picked by smallest prediction at the
 * coarsest step, by bracket midpoint after that.  within-tau / intersection:
 * a pair starts at the coarsest step whose per-object Hausdorff terms w_l
 * (max hd + max ph of r plus those of s at that LoD) satisfy
 * max |x - tau| >= 0.5 * w_l over x in [expm1(y - 0.15), expm1(y + 0.15)],
 * else at full resolution.  The join fails with PJ_EINVAL if no weights
 * were trained, fitted or loaded. */

/* Fit the proposal to a workload: run q's candidate filter on R x S, take a
 * seeded sample of at most max_pairs candidates, label them with their
 * full-resolution distances (the refinement kernel), and train fresh weights
 * for `epochs` passes (Adam, mini-batches of 2048) on 90 % of them.  *rmse
 * (may be NULL) receives the prediction error in log(1 + d) on the other
 * 10 %.  PJ_EINVAL if q is malformed, max_pairs < 16, or the filter yields
 * fewer than 16 candidates. */
pj_status pj_mlp_fit(pj_ctx* ctx, const pj_set* R, const pj_set* S, const pj_query* q, int64_t max_pairs,
                     int epochs, uint64_t seed, double* rmse);

/* Train on n examples: feats HOST float32 [n][16], target HOST float32 [n]
 * (log(1 + d)).  Adam over shuffled mini-batches of 2048, `epochs` passes,
 * shuffled with `seed`; forward and backward run in the library's kernels.
 * Continues from the current weights (He-initialized from `seed` if none). */
pj_status pj_mlp_train(pj_ctx* ctx, const float* feats, const float* target, int64_t n, int epochs,
                       uint64_t seed);
pj_status pj_mlp_save(const pj_ctx* ctx, const char* path);
pj_status pj_mlp_load(pj_ctx* ctx, const char* path);

/* Weights as float32 HOST arrays (W1 [64][16], b1 [64], W2 [64][64], b2 [64],
 * W3 [64], b3 [1]); set copies in, get copies out. */
pj_status pj_mlp_set_weights(pj_ctx* ctx, const float* w1, const float* b1, const float* w2,
                             const float* b2, const float* w3, const float* b3);
pj_status pj_mlp_get_weights(const pj_ctx* ctx, float* w1, float* b1, float* w2, float* b2, float* w3,
                             float* b3);

/* Forward pass on DEVICE buffers: feats float32 [n][16] -> out float32 [n]. */
pj_status pj_mlp_forward(pj_ctx* ctx, const float* feats, int64_t n, float* out, void* cuda_stream);

/* One forward+backward pass on DEVICE buffers with the current weights:
 * loss = mean over n of (out - target)^2 / 2; gradients written to DEVICE
 * float32 buffers of the shapes above (any may be NULL).  loss is a DEVICE
 * float32 scalar. */
pj_status pj_mlp_grad(pj_ctx* ctx, const float* feats, const float* target, int64_t n, float* loss,
                      float* g_w1, float* g_b1, float* g_w2, float* g_b2, float* g_w3, float* g_b3,
                      void* cuda_stream);

/* Features of candidate pairs (the MLP input), DEVICE out float32 [n][16]
 * for host pair lists pr/ps. */
pj_status pj_pair_features(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr,
                           const int32_t* ps, int64_t n, float* out_dev);

/* ------------------------------------------------------------------ *
 * Kernel-level entry points (the building blocks of pj_join, exposed for
 * verification).
 * ------------------------------------------------------------------ */

/* Triangle-triangle minimum distance (section 2.2 plus the meeting test) of
 * n independent pairs: P, Q DEVICE float32 [n][9] (three xyz vertices),
 * out DEVICE double [n].  prec selects the FP64 or the FP32 kernel; with
 * FP32, err_out (DEVICE double [n], may be NULL) receives the forward error
 * bound used by the FP32 path for that pair. */
pj_status pj_tri_dist(pj_ctx* ctx, const float* P, const float* Q, int64_t n, pj_precision prec,
                      double* out, double* err_out, void* cuda_stream);

/* Eq. 1 / Eq. 2 bounds of explicit object pairs at one LoD, every facet pair
 * evaluated (no pruning): pr, ps HOST int32 [n] (ids in R and S), lod in
 * [0, n_lods) of both sets, lb/ub HOST double [n].  With FP32 the returned
 * bracket includes the forward error bound. */
pj_status pj_pair_bounds(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr,
                         const int32_t* ps, int64_t n, int lod, pj_precision prec, double* lb, double* ub);

/* pj_pair_bounds for callers that cannot allocate device memory: the same
 * bounds, computed without any cudaMalloc / cudaFree (nor any allocating
 * library call).  Meant for code embedded in a host application that owns
 * and budgets every device allocation itself (a database engine's or a
 * renderer's memory manager) and forbids libraries from allocating, and for
 * latency-critical loops that cannot afford the device-wide synchronization
 * cudaMalloc / cudaFree imply.  The paper has no counterpart; it is a
 * property of this library's interface.
 *   pr, ps   DEVICE int32 [n] object ids in R and S (ids out of range give
 *            PJ_EBOUNDS before any bound is computed);
 *   lb, ub   DEVICE double [n] outputs, as for pj_pair_bounds;
 *   cuda_stream  stream to work on (NULL = the context's stream); the call
 *            returns when the results are written.
 * Scratch: one fixed array of about 2.4 MB in the library's device code,
 * held by every GPU that loads the library until the process exits.  Its
 * device address is looked up on the first call on each device (with that
 * device current).  Sizes beyond it are rejected with PJ_EINVAL:
 * n <= PJ_STATIC_MAX_PAIRS, and n x (blocks of the largest R object) x
 * (blocks of the largest S object) at `lod` <= PJ_STATIC_MAX_TILES with a
 * block of 32 facets.  All calls share the array; it keeps the previous
 * call's contents (the call clears what must start at zero), and calls that
 * overlap on the GPU -- on two streams or from two host threads -- race on
 * it and must be serialized by the caller. */
#define PJ_STATIC_MAX_PAIRS 4096
#define PJ_STATIC_MAX_TILES 32768
pj_status pj_pair_bounds_static(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr,
                                const int32_t* ps, int64_t n, int lod, pj_precision prec, double* lb,
                                double* ub, void* cuda_stream);

/* ---- Voxels and voxel-pair filtering (section 2.1; section 3.2,
 * Algorithms 1 and 2) ----
 * With the context option "voxels": 1, pj_load_set clusters the facets of
 * every object into voxels:
 *   - k = round(F / 50) voxels (2 % of the object's original facets F,
 *     halves rounded up), at least 1 and at most the coarsest LoD's facet
 *     count; an object without coarsest facets has none;
 *   - k-means over the centroids ((v0 + v1) + v2) / 3 of the coarsest LoD's
 *     facets with two centroid updates (a centre without members stays),
 *     started from the coarsest vertex array's entries at the positions
 *     floor((2j + 1) V / 2k), V its vertex count;
 *   - every facet of every LoD belongs to the voxel whose final centre is
 *     nearest to its centroid (the lowest index on ties), one partition
 *     for all LoDs;
 *   - a voxel's box bounds its original-LoD facets, its anchor is the
 *     vertex of those facets nearest to the box centre (the first in facet
 *     and corner order among equals).
 * All in double precision, with every sum and product rounded in the
 * order written (no fused multiply-add).  Sets streamed with
 * pj_load_set_streamed are not voxelized.  Objects with more than
 * PJ_VOXEL_MAX voxels (over about 102,400 original facets) make pj_load_set
 * fail with PJ_EINVAL. */
#define PJ_VOXEL_MAX 2048

/* Voxels of all objects of a set (PJ_EINVAL when it has none). */
pj_status pj_voxel_count(const pj_set* set, int64_t* n_voxels);

/* Copies of a set's voxels to HOST buffers, each may be NULL:
 *   voxel_off [n_objects + 1]  object o owns voxels voxel_off[o] ..
 *                              voxel_off[o + 1] - 1 (object-local index
 *                              v - voxel_off[o]);
 *   centre    [n_voxels][3]    final k-means centres (double);
 *   box       [n_voxels][6]    lo.xyz, hi.xyz (+inf / -inf for a voxel with
 *                              no original facet);
 *   anchor    [n_voxels][3]    the anchor vertex (NaN for such a voxel).
 * Synchronous. */
pj_status pj_voxels_read(pj_ctx* ctx, const pj_set* set, int64_t* voxel_off, double* centre, float* box,
                         float* anchor);

/* The object-local voxel of every facet of LoD `lod` (HOST int32 [facets of
 * that LoD], in the set's facet order; -1 for objects without voxels).
 * Synchronous. */
pj_status pj_voxel_labels_read(pj_ctx* ctx, const pj_set* set, int lod, int32_t* label);

/* Voxel-pair filtering of n object pairs (pr[p] in R, ps[p] in S), both
 * sets voxelized.  Every array is a caller-allocated DEVICE buffer:
 *   pr, ps       int32 [n]        the object pairs (an id outside its set
 *                                 gives PJ_EBOUNDS, with every output
 *                                 undefined);
 *   op_lb, op_ub double [n]       Algorithm 1's object-pair bounds: the
 *                                 minima over the pair's voxel pairs of
 *                                 lb = MINDIST of the two voxel boxes and
 *                                 ub = distance of the two voxel anchors
 *                                 (+inf when either object has no voxel);
 *   status       uint8 [n]        with tau >= 0: 1 a result (op_ub <= tau),
 *                                 2 pruned (op_lb > tau), 0 undecided;
 *                                 with tau < 0 every pair is undecided
 *                                 (the k-NN use);
 *   vp_off       int64 [n + 1]    offsets of each pair's n_r x n_s voxel
 *                                 pairs in vp_lb / vp_ub (op2vpOffsets);
 *   vp_lb, vp_ub double [vp_cap]  every voxel pair's bounds, pair p's block
 *                                 row-major (t = i n_s + j, i the voxel of
 *                                 pr[p], j of ps[p]);
 *   kept_off     int64 [n + 1]    offsets of each pair's surviving voxel
 *                                 pairs (Algorithm 2: those of undecided
 *                                 pairs with lb <= op_ub);
 *   kept         int32 [vp_cap][2] the survivors (i, j), row-major order.
 * n_kept (HOST) receives kept_off[n].  vp_cap below the sum of n_r x n_s
 * gives PJ_EINVAL (nothing past vp_cap is written).  prec PJ_PREC_FP64:
 * the distances in double precision, rounded to nearest in the order of
 * the voxel data above; PJ_PREC_FP32_REDECIDE: in single precision rounded
 * outward (lb rounded down, ub up, step by step), so every bound still
 * holds and the decisions and survivors are those of the exact bounds
 * except where a bound lies within rounding (about 1e-6 relative) of the
 * value it is compared with, where the pair stays undecided or the voxel
 * pair is kept (the outputs stay double arrays).  Works
 * on cuda_stream (NULL = the context's stream) and returns when the
 * results are written; pj_get_stats then reports the pair and voxel-pair
 * counts and each step's device time. */
pj_status pj_voxel_filter(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr, const int32_t* ps,
                          int64_t n, double tau, pj_precision prec, double* op_lb, double* op_ub, uint8_t* status, int64_t* vp_off,
                          double* vp_lb, double* vp_ub, int64_t vp_cap, int64_t* kept_off, int32_t* kept,
                          int64_t* n_kept, void* cuda_stream);

/* ---- Out-of-core chunks: a streamed set read from chunk files ----
 * The paper streams R from host memory (section 3.2, Algorithm 3) and leaves
 * facets kept on disk to future work.  A chunk file holds one chunk exactly
 * as a pj_mesh_set_desc describes it: a 1,024-byte little-endian header
 * (magic "PJCHUNK1", version 1, counts and the byte offset of every array)
 * followed by the arrays at 64-byte aligned offsets.  A chunk source reads
 * such files on a thread of its own, ahead of the join, and is the fill
 * callback of pj_load_set_streamed:
 *
 *   pj_chunk_source* src;  pj_chunk_source_open(paths, n, 2, &src);
 *   pj_chunk_source_info(src, &n_objects, NULL, NULL);
 *   pj_load_set_streamed(ctx, n_objects, n, pj_chunk_source_fill, src, &R);
 *   ... pj_join(ctx, R, S, ...) ...   (any number of joins)
 *   pj_free_set(R);  pj_chunk_source_close(src);
 *
 * None of these calls touches the GPU. */
typedef struct pj_chunk_source pj_chunk_source; /* opaque */

/* Write the chunk described by desc (HOST arrays, as for pj_load_set) to
 * path, through a temporary file "<path>.part" renamed into place when
 * complete.  PJ_EINVAL for an inconsistent desc, PJ_ESOURCE for an I/O
 * error (the file is then left absent). */
pj_status pj_chunk_file_write(const char* path, const pj_mesh_set_desc* desc);

/* Open n_chunks chunk files (paths[c] is chunk c; every file with the same
 * LoD count) and start the reader thread.  The headers are read and checked
 * here (PJ_ESOURCE: a file cannot be opened; PJ_EINVAL: not a chunk file,
 * an offset outside the file, or LoD counts that differ).  The source keeps
 * readahead + 2 chunk buffers in host memory (readahead 0..16): while the
 * join lays out chunk c the reader loads chunks up to c + readahead.  The
 * buffers are pageable memory, so the library packs them into its pinned
 * staging as for any pageable chunk. */
pj_status pj_chunk_source_open(const char* const* paths, int n_chunks, int readahead, pj_chunk_source** out);

/* Total objects, chunk count and LoD count of an open source (each output
 * may be NULL). */
pj_status pj_chunk_source_info(const pj_chunk_source* src, int64_t* n_objects, int* n_chunks, int* n_lods);

/* The pj_fill_fn of a source (user = the source): waits for chunk `chunk`
 * and points out's arrays into its buffer, valid until the chunk two after
 * it is asked for (the pageable-array contract of pj_load_set_streamed).
 * Chunks are asked for in order; a request that does not follow the
 * previous one (the next join's chunk 0) restarts the reader there.
 * PJ_ESOURCE when the file can no longer be read or its header changed
 * since pj_chunk_source_open. */
pj_status pj_chunk_source_fill(void* src, int chunk, pj_mesh_set_desc* out);

/* JSON statistics of a source: chunks_read, bytes_read, ms_read (time the
 * reader spent in reads), read_gbs, ms_fill_wait (time fills waited for the
 * reader: I/O the join did not hide), restarts, buffers. */
pj_status pj_chunk_source_stats(pj_chunk_source* src, char* json_buf, size_t cap);

/* Stop the reader and free the buffers; no set streamed from the source may
 * be joined afterwards. */
void pj_chunk_source_close(pj_chunk_source* src);

/* Measured fused-multiply-add throughput of the device (independent FMA
 * chains on every SM), GFLOP/s with an FMA counted as 2 operations: the
 * arithmetic peak the refinement kernels are compared against (their work
 * is scalar ALU arithmetic, not a tensor-core contraction).  fp64 = 0 for
 * single, 1 for double precision. */
pj_status pj_fma_peak(pj_ctx* ctx, int fp64, double* gflops);

const char* pj_last_error(const pj_ctx* ctx);
const char* pj_status_str(pj_status s);

#ifdef __cplusplus
}
#endif
#endif /* PJ_H */
