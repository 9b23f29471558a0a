/*
 * Plain FP64 CPU oracle for the polyhedral spatial join (3DPipe, arXiv
 * 2604.19982).  TEST INFRASTRUCTURE ONLY: it is loaded by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the library.
 * It shares no code with the CUDA path.
 *
 * What it computes, and where the paper defines it:
 *   - d(P1, P2) = min over surface points of |p1 - p2|           (section 2.1)
 *   - intersection: d = 0; within-tau: d <= tau; k-NN: the k objects of S
 *     closest to r, ties broken by object id                       (section 3)
 *   - LoD bounds: ub = min_{f1,f2} d(f1,f2) + hd1 + hd2 (Eq. 1),
 *                 lb = min_{f1,f2} d(f1,f2) - ph1 - ph2 (Eq. 2)
 *   - triangle-triangle distance: 0 when the triangles meet, otherwise the
 *     smallest of the six vertex-to-triangle and nine edge-to-edge distances
 *     (section 2.2, "Triangle-Triangle Distance Computation"); the meeting
 *     test is added because an edge piercing the other triangle's interior
 *     is not among those fifteen cases.
 *
 * Everything is brute force over full-resolution facet pairs in double
 * precision; each distance is sqrt(dot(p - q, p - q)) of the two closest
 * points.  Compile with -ffp-contract=off.  Threads: one work item per object
 * r of R (pthreads, dynamic counter).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ vec3 */

typedef struct { double x, y, z; } v3;

static v3 mk(const double* p) { v3 r = {p[0], p[1], p[2]}; return r; }
static v3 sub(v3 a, v3 b) { v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static v3 add(v3 a, v3 b) { v3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static v3 scl(v3 a, double s) { v3 r = {a.x * s, a.y * s, a.z * s}; return r; }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
  v3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
  return r;
}
static double dist(v3 a, v3 b) { v3 d = sub(a, b); return sqrt(dot(d, d)); }
static double clamp01(double t) { return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }

/* ------------------------------------------------------- closest points */

/* closest point of segment [a, b] to point p */
static v3 seg_point(v3 a, v3 b, v3 p) {
  v3 ab = sub(b, a);
  double len2 = dot(ab, ab);
  if (len2 <= 0.0) return a;
  double t = clamp01(dot(sub(p, a), ab) / len2);
  return add(a, scl(ab, t));
}

/* closest point of triangle (a, b, c) to p: the projection onto the plane
 * when it falls inside the triangle, else the nearest of the three edges'
 * closest points.  A zero-area triangle has no interior case. */
static v3 tri_point(v3 a, v3 b, v3 c, v3 p) {
  v3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
  double g00 = dot(ab, ab), g01 = dot(ab, ac), g11 = dot(ac, ac);
  double r0 = dot(ap, ab), r1 = dot(ap, ac);
  double det = g00 * g11 - g01 * g01;
  if (det > 0.0) {
    /* solve [g00 g01; g01 g11] [u v]^T = [r0 r1]^T for p's projection
     * a + u ab + v ac */
    double u = (r0 * g11 - r1 * g01) / det;
    double v = (g00 * r1 - g01 * r0) / det;
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0)
      return add(a, add(scl(ab, u), scl(ac, v)));
  }
  v3 best = seg_point(a, b, p);
  double bd = dist(best, p);
  v3 q = seg_point(b, c, p);
  double qd = dist(q, p);
  if (qd < bd) { best = q; bd = qd; }
  q = seg_point(c, a, p);
  qd = dist(q, p);
  if (qd < bd) best = q;
  return best;
}

/* closest points of segments [p0, p1] and [q0, q1]: the stationary point of
 * |p(s) - q(t)|^2 when it exists inside [0,1]^2, else the best of the four
 * boundary cases s=0, s=1, t=0, t=1 (each a point-to-segment problem). */
static void seg_seg(v3 p0, v3 p1, v3 q0, v3 q1, v3* cp, v3* cq) {
  v3 u = sub(p1, p0), v = sub(q1, q0), w = sub(p0, q0);
  double a = dot(u, u), b = dot(u, v), c = dot(v, v), d = dot(u, w), e = dot(v, w);
  double det = a * c - b * b;
  double best = INFINITY;
  if (det > 0.0) {
    /* d/ds: a s - b t + d = 0 ; d/dt: -b s + c t - e = 0 */
    double s = (b * e - c * d) / det;
    double t = (a * e - b * d) / det;
    if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
      *cp = add(p0, scl(u, s));
      *cq = add(q0, scl(v, t));
      best = dist(*cp, *cq);
    }
  }
  v3 x, y;
  double dd;
  y = seg_point(q0, q1, p0); dd = dist(p0, y);
  if (dd < best) { best = dd; *cp = p0; *cq = y; }
  y = seg_point(q0, q1, p1); dd = dist(p1, y);
  if (dd < best) { best = dd; *cp = p1; *cq = y; }
  x = seg_point(p0, p1, q0); dd = dist(x, q0);
  if (dd < best) { best = dd; *cp = x; *cq = q0; }
  x = seg_point(p0, p1, q1); dd = dist(x, q1);
  if (dd < best) { best = dd; *cp = x; *cq = q1; }
}

/* signed volume of tetrahedron (a, b, c, d), times 6, with a bound on its
 * rounding error: the first-order error of the three differences, the cross
 * product and the dot product is below 8 u times the "permanent" (the same
 * expression with every product taken in absolute value), u = 2^-53; twice
 * that is used.  A sign is trusted only when |value| exceeds the bound. */
static double orient(v3 a, v3 b, v3 c, v3 d, double* err) {
  v3 x = sub(b, a), y = sub(c, a), z = sub(d, a);
  double cx = y.y * z.z - y.z * z.y, cy = y.z * z.x - y.x * z.z, cz = y.x * z.y - y.y * z.x;
  double px = fabs(y.y * z.z) + fabs(y.z * z.y), py = fabs(y.z * z.x) + fabs(y.x * z.z),
         pz = fabs(y.x * z.y) + fabs(y.y * z.x);
  double perm = fabs(x.x) * px + fabs(x.y) * py + fabs(x.z) * pz;
  *err = 16.0 * ldexp(1.0, -53) * perm;
  return x.x * cx + x.y * cy + x.z * cz;
}

static int sure_pos(double v, double e) { return v > e; }
static int sure_neg(double v, double e) { return v < -e; }

/* Does segment [a, b] cross triangle (t0, t1, t2)?  A crossing is claimed
 * only when every sign involved is certain: the endpoints lie strictly on
 * opposite sides of the plane and the line passes strictly inside all three
 * edges.  Touching, coplanar and near-degenerate configurations are left to
 * the vertex/edge distances, which are exact there up to rounding.  If yes,
 * *x is the crossing point. */
static int seg_crosses_tri(v3 a, v3 b, v3 t0, v3 t1, v3 t2, v3* x) {
  double ea, eb, e1, e2, e3;
  double sa = orient(t0, t1, t2, a, &ea), sb = orient(t0, t1, t2, b, &eb);
  int opposite = (sure_pos(sa, ea) && sure_neg(sb, eb)) || (sure_neg(sa, ea) && sure_pos(sb, eb));
  if (!opposite) return 0;
  double o1 = orient(a, b, t0, t1, &e1), o2 = orient(a, b, t1, t2, &e2), o3 = orient(a, b, t2, t0, &e3);
  int pos = sure_pos(o1, e1) && sure_pos(o2, e2) && sure_pos(o3, e3);
  int neg = sure_neg(o1, e1) && sure_neg(o2, e2) && sure_neg(o3, e3);
  if (!pos && !neg) return 0;
  double t = sa / (sa - sb);
  *x = add(a, scl(sub(b, a), t));
  return 1;
}

/* Triangle-triangle distance.  P and Q are 9 doubles (3 vertices).  If cp is
 * not NULL it receives the closest point on P then on Q. */
double or_tri_dist(const double* P, const double* Q, double* cp) {
  v3 p[3] = {mk(P), mk(P + 3), mk(P + 6)};
  v3 q[3] = {mk(Q), mk(Q + 3), mk(Q + 6)};
  v3 bp = p[0], bq = q[0], x, y;
  for (int i = 0; i < 3; ++i) {
    if (seg_crosses_tri(p[i], p[(i + 1) % 3], q[0], q[1], q[2], &x) ||
        seg_crosses_tri(q[i], q[(i + 1) % 3], p[0], p[1], p[2], &x)) {
      if (cp) { cp[0] = cp[3] = x.x; cp[1] = cp[4] = x.y; cp[2] = cp[5] = x.z; }
      return 0.0;
    }
  }
  double best = INFINITY, d;
  for (int i = 0; i < 3; ++i) {
    y = tri_point(q[0], q[1], q[2], p[i]);
    d = dist(p[i], y);
    if (d < best) { best = d; bp = p[i]; bq = y; }
    x = tri_point(p[0], p[1], p[2], q[i]);
    d = dist(x, q[i]);
    if (d < best) { best = d; bp = x; bq = q[i]; }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      seg_seg(p[i], p[(i + 1) % 3], q[j], q[(j + 1) % 3], &x, &y);
      d = dist(x, y);
      if (d < best) { best = d; bp = x; bq = y; }
    }
  if (cp) { cp[0] = bp.x; cp[1] = bp.y; cp[2] = bp.z; cp[3] = bq.x; cp[4] = bq.y; cp[5] = bq.z; }
  return best;
}

/* point to triangle distance (used by the Hausdorff checks in the tests) */
double or_point_tri_dist(const double* p, const double* T) {
  v3 x = mk(p);
  return dist(x, tri_point(mk(T), mk(T + 3), mk(T + 6), x));
}

static void load_tri(const float* t, double* out) {
  for (int k = 0; k < 9; ++k) out[k] = (double)t[k];
}

/* distance from point p to a triangle soup of nf facets (float32 [nf][9]) */
double or_point_mesh_dist(const double* p, const float* tri, int64_t nf) {
  double best = INFINITY, T[9];
  for (int64_t i = 0; i < nf; ++i) {
    load_tri(tri + 9 * i, T);
    double d = or_point_tri_dist(p, T);
    if (d < best) best = d;
  }
  return best;
}

/* d(A, B): brute force over all facet pairs (float32 [n][9] soups) */
double or_obj_dist(const float* A, int64_t na, const float* B, int64_t nb) {
  double best = INFINITY, P[9], Q[9];
  for (int64_t i = 0; i < na; ++i) {
    load_tri(A + 9 * i, P);
    for (int64_t j = 0; j < nb; ++j) {
      load_tri(B + 9 * j, Q);
      double d = or_tri_dist(P, Q, NULL);
      if (d < best) best = d;
      if (best == 0.0) return 0.0;
    }
  }
  return best;
}

/* Eq. 1 / Eq. 2 bounds of one object pair at one LoD. */
void or_lod_bounds(const float* A, const float* hdA, const float* phA, int64_t na,
                   const float* B, const float* hdB, const float* phB, int64_t nb,
                   double* lb, double* ub) {
  double lo = INFINITY, hi = INFINITY, P[9], Q[9];
  for (int64_t i = 0; i < na; ++i) {
    load_tri(A + 9 * i, P);
    for (int64_t j = 0; j < nb; ++j) {
      load_tri(B + 9 * j, Q);
      double d = or_tri_dist(P, Q, NULL);
      double l = d - (double)phA[i] - (double)phB[j];
      double u = d + (double)hdA[i] + (double)hdB[j];
      if (l < lo) lo = l;
      if (u < hi) hi = u;
    }
  }
  *lb = lo;
  *ub = hi;
}

/* ------------------------------------------------------------------ sets */

typedef struct {
  int64_t n;          /* objects */
  const float* tri;   /* full-resolution triangles, float32 [nf_total][9] */
  const int64_t* off; /* [n + 1] facet offsets */
} or_set;

static void set_mbb(const or_set* s, int64_t o, double* lo, double* hi) {
  lo[0] = lo[1] = lo[2] = INFINITY;
  hi[0] = hi[1] = hi[2] = -INFINITY;
  for (int64_t f = s->off[o]; f < s->off[o + 1]; ++f)
    for (int v = 0; v < 3; ++v)
      for (int k = 0; k < 3; ++k) {
        double x = s->tri[9 * f + 3 * v + k];
        if (x < lo[k]) lo[k] = x;
        if (x > hi[k]) hi[k] = x;
      }
}

/* minimum distance between two boxes (an exact lower bound of d, since each
 * surface lies inside its box) */
static double box_mindist(const double* alo, const double* ahi, const double* blo, const double* bhi) {
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    double g = 0.0;
    if (blo[k] > ahi[k]) g = blo[k] - ahi[k];
    else if (alo[k] > bhi[k]) g = alo[k] - bhi[k];
    s += g * g;
  }
  return sqrt(s);
}

static double set_dist(const or_set* R, int64_t r, const or_set* S, int64_t s) {
  return or_obj_dist(R->tri + 9 * R->off[r], R->off[r + 1] - R->off[r],
                     S->tri + 9 * S->off[s], S->off[s + 1] - S->off[s]);
}

/* per-r result buffers */
typedef struct {
  int64_t n, cap;
  int32_t* s;
  double* d;
} hits;

static void hits_push(hits* h, int32_t s, double d) {
  if (h->n == h->cap) {
    h->cap = h->cap ? 2 * h->cap : 16;
    h->s = (int32_t*)realloc(h->s, (size_t)h->cap * sizeof(int32_t));
    h->d = (double*)realloc(h->d, (size_t)h->cap * sizeof(double));
  }
  h->s[h->n] = s;
  h->d[h->n] = d;
  h->n++;
}

/* S boxes sorted by min x, for the sweep */
typedef struct {
  double lo[3], hi[3];
  int32_t id;
} sbox;

static int cmp_sbox(const void* a, const void* b) {
  const sbox* x = (const sbox*)a;
  const sbox* y = (const sbox*)b;
  if (x->lo[0] < y->lo[0]) return -1;
  if (x->lo[0] > y->lo[0]) return 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

typedef struct {
  const or_set *R, *S;
  double tau;
  int k;
  int prune;
  const int64_t* rlist; /* objects of R to evaluate */
  int64_t nr;
  sbox* boxes;          /* S boxes sorted by lo.x */
  double max_ext_x;     /* largest x extent among S boxes */
  hits* out;            /* [nr] */
  int64_t next;         /* work counter */
  pthread_mutex_t mu;
} job;

static int64_t take(job* j) {
  pthread_mutex_lock(&j->mu);
  int64_t i = j->next++;
  pthread_mutex_unlock(&j->mu);
  return i;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* lower bound index of first box with lo.x >= v */
static int64_t lower_x(const sbox* b, int64_t n, double v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) / 2;
    if (b[m].lo[0] < v) lo = m + 1; else hi = m;
  }
  return lo;
}

static void* within_worker(void* arg) {
  job* j = (job*)arg;
  int64_t nS = j->S->n;
  int32_t* cand = (int32_t*)malloc((size_t)(nS > 0 ? nS : 1) * sizeof(int32_t));
  double rlo[3], rhi[3];
  /* a box farther than tau by more than this relative slack is pruned; the
   * slack keeps pairs whose MBB distance rounds across tau */
  const double slack = 1e-9;
  for (;;) {
    int64_t i = take(j);
    if (i >= j->nr) break;
    int64_t r = j->rlist[i];
    int64_t nc = 0;
    if (!j->prune) {
      for (int64_t s = 0; s < nS; ++s) cand[nc++] = (int32_t)s;
    } else {
      set_mbb(j->R, r, rlo, rhi);
      int64_t a = lower_x(j->boxes, nS, rlo[0] - j->tau - j->max_ext_x - 1.0);
      int64_t b = lower_x(j->boxes, nS, rhi[0] + j->tau * (1.0 + slack) + 1e-300);
      for (int64_t q = a; q < nS && q <= b; ++q) {
        const sbox* sb = &j->boxes[q];
        if (sb->lo[0] > rhi[0] + j->tau * (1.0 + slack)) break;
        if (box_mindist(rlo, rhi, sb->lo, sb->hi) <= j->tau * (1.0 + slack)) cand[nc++] = sb->id;
      }
      qsort(cand, (size_t)nc, sizeof(int32_t), cmp_i32);
    }
    for (int64_t c = 0; c < nc; ++c) {
      double d = set_dist(j->R, r, j->S, cand[c]);
      if (d <= j->tau) hits_push(&j->out[i], cand[c], d);
    }
  }
  free(cand);
  return NULL;
}

typedef struct {
  double key;
  int32_t id;
} kd;

static int cmp_kd(const void* a, const void* b) {
  const kd* x = (const kd*)a;
  const kd* y = (const kd*)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* k-NN for one r: visit S by increasing box distance, keep the best k by
 * (d, id), stop once the next box distance exceeds the k-th distance. */
static void* knn_worker(void* arg) {
  job* j = (job*)arg;
  int64_t nS = j->S->n;
  kd* order = (kd*)malloc((size_t)(nS > 0 ? nS : 1) * sizeof(kd));
  kd* top = (kd*)malloc((size_t)(j->k + 1) * sizeof(kd));
  double rlo[3], rhi[3];
  for (;;) {
    int64_t i = take(j);
    if (i >= j->nr) break;
    int64_t r = j->rlist[i];
    set_mbb(j->R, r, rlo, rhi);
    for (int64_t q = 0; q < nS; ++q) {
      order[q].key = box_mindist(rlo, rhi, j->boxes[q].lo, j->boxes[q].hi);
      order[q].id = j->boxes[q].id;
    }
    qsort(order, (size_t)nS, sizeof(kd), cmp_kd);
    int nt = 0;
    for (int64_t q = 0; q < nS; ++q) {
      if (nt == j->k && order[q].key > top[nt - 1].key) break;
      kd c = {set_dist(j->R, r, j->S, order[q].id), order[q].id};
      /* insert into the sorted top list */
      int pos = nt;
      while (pos > 0 && cmp_kd(&c, &top[pos - 1]) < 0) {
        if (pos < j->k) top[pos] = top[pos - 1];
        --pos;
      }
      if (pos < j->k) {
        top[pos] = c;
        if (nt < j->k) ++nt;
      }
    }
    for (int t = 0; t < nt; ++t) hits_push(&j->out[i], top[t].id, top[t].key);
  }
  free(order);
  free(top);
  return NULL;
}

static void prepare_boxes(job* j) {
  int64_t nS = j->S->n;
  j->boxes = (sbox*)malloc((size_t)(nS > 0 ? nS : 1) * sizeof(sbox));
  j->max_ext_x = 0.0;
  for (int64_t s = 0; s < nS; ++s) {
    set_mbb(j->S, s, j->boxes[s].lo, j->boxes[s].hi);
    j->boxes[s].id = (int32_t)s;
    double e = j->boxes[s].hi[0] - j->boxes[s].lo[0];
    if (e > j->max_ext_x) j->max_ext_x = e;
  }
  qsort(j->boxes, (size_t)nS, sizeof(sbox), cmp_sbox);
}

static void run(job* j, void* (*fn)(void*), int threads) {
  if (threads < 1) threads = 1;
  pthread_t* th = (pthread_t*)malloc((size_t)threads * sizeof(pthread_t));
  for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, fn, j);
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  free(th);
}

/* Join driver.  pred 0 = within tau (intersection is tau = 0), 1 = k-NN.
 * rlist/nr select the objects of R to evaluate (NULL = all, in order).
 * Results go to freshly malloc'ed arrays handed back through *out_*:
 * per evaluated r (in rlist order) its hits, within: sorted by s, k-NN:
 * sorted by (d, s).  *out_cnt[i] is the hit count of rlist[i].
 * Release them with or_free. */
int64_t or_join(int64_t nR, const float* triR, const int64_t* offR,
                int64_t nS, const float* triS, const int64_t* offS,
                int pred, double tau, int k, int prune,
                const int64_t* rlist, int64_t nr, int threads,
                int32_t** out_s, double** out_d, int64_t** out_cnt) {
  or_set R = {nR, triR, offR}, S = {nS, triS, offS};
  job j;
  memset(&j, 0, sizeof(j));
  j.R = &R;
  j.S = &S;
  j.tau = tau;
  j.k = k;
  j.prune = prune;
  int64_t* all = NULL;
  if (!rlist) {
    all = (int64_t*)malloc((size_t)(nR > 0 ? nR : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nR; ++i) all[i] = i;
    rlist = all;
    nr = nR;
  }
  j.rlist = rlist;
  j.nr = nr;
  j.out = (hits*)calloc((size_t)(nr > 0 ? nr : 1), sizeof(hits));
  pthread_mutex_init(&j.mu, NULL);
  prepare_boxes(&j);
  if (pred == 1 && k > 0) run(&j, knn_worker, threads);
  else if (pred == 0) run(&j, within_worker, threads);
  int64_t total = 0;
  for (int64_t i = 0; i < nr; ++i) total += j.out[i].n;
  *out_s = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  *out_d = (double*)malloc((size_t)(total > 0 ? total : 1) * sizeof(double));
  *out_cnt = (int64_t*)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
  int64_t w = 0;
  for (int64_t i = 0; i < nr; ++i) {
    (*out_cnt)[i] = j.out[i].n;
    for (int64_t h = 0; h < j.out[i].n; ++h) {
      (*out_s)[w] = j.out[i].s[h];
      (*out_d)[w] = j.out[i].d[h];
      ++w;
    }
    free(j.out[i].s);
    free(j.out[i].d);
  }
  free(j.out);
  free(j.boxes);
  free(all);
  pthread_mutex_destroy(&j.mu);
  return total;
}

void or_free(void* p) { free(p); }

/* ---------------------------------------------------- pair-list helpers */

typedef struct {
  const float *A, *B;
  const int64_t *offA, *offB;
  const float *hdA, *phA, *hdB, *phB; /* NULL => exact distance only */
  const int32_t *pr, *ps;
  int64_t n;
  double *lb, *ub;
  int64_t next;
  pthread_mutex_t mu;
} pjob;

static void* pair_worker(void* arg) {
  pjob* j = (pjob*)arg;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    int64_t i = j->next++;
    pthread_mutex_unlock(&j->mu);
    if (i >= j->n) break;
    int64_t r = j->pr[i], s = j->ps[i];
    int64_t a0 = j->offA[r], a1 = j->offA[r + 1], b0 = j->offB[s], b1 = j->offB[s + 1];
    if (j->hdA) {
      or_lod_bounds(j->A + 9 * a0, j->hdA + a0, j->phA + a0, a1 - a0,
                    j->B + 9 * b0, j->hdB + b0, j->phB + b0, b1 - b0, &j->lb[i], &j->ub[i]);
    } else {
      double d = or_obj_dist(j->A + 9 * a0, a1 - a0, j->B + 9 * b0, b1 - b0);
      j->lb[i] = j->ub[i] = d;
    }
  }
  return NULL;
}

/* Distances (hd == NULL) or Eq. 1/2 bounds of an explicit list of pairs. */
void or_pairs(const float* A, const int64_t* offA, const float* hdA, const float* phA,
              const float* B, const int64_t* offB, const float* hdB, const float* phB,
              const int32_t* pr, const int32_t* ps, int64_t n, int threads,
              double* lb, double* ub) {
  pjob j;
  memset(&j, 0, sizeof(j));
  j.A = A; j.B = B; j.offA = offA; j.offB = offB;
  j.hdA = hdA; j.phA = phA; j.hdB = hdB; j.phB = phB;
  j.pr = pr; j.ps = ps; j.n = n; j.lb = lb; j.ub = ub;
  pthread_mutex_init(&j.mu, NULL);
  if (threads < 1) threads = 1;
  pthread_t* th = (pthread_t*)malloc((size_t)threads * sizeof(pthread_t));
  for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, pair_worker, &j);
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&j.mu);
}

/* batch of independent triangle pairs (tests): P, Q double [n][9] */
void or_tri_dist_batch(const double* P, const double* Q, int64_t n, double* d, double* cp) {
  for (int64_t i = 0; i < n; ++i) d[i] = or_tri_dist(P + 9 * i, Q + 9 * i, cp ? cp + 6 * i : NULL);
}
