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

/* ------------------------------------------------------ exact signs */

/* Exact integer arithmetic for the orientation signs.  Every finite double
 * is m * 2^e with an integer m, |m| < 2^53.  With E the smallest such e over
 * the inputs of one predicate, every input is the integer m * 2^(e - E)
 * times 2^E, and the determinants below (homogeneous of degree 3 or 2 in
 * the coordinates) have the sign of the same expressions evaluated on those
 * integers.  Integers are sign and magnitude, 32-bit limbs, least
 * significant first; 224 limbs hold the largest case (inputs up to 2^2099
 * after scaling, products of three differences, sums of six of them). */
#define BN_LIMBS 224
typedef struct {
  int neg;
  int n; /* limbs in use; 0 is zero */
  uint32_t d[BN_LIMBS];
} bn;

static void bn_zero(bn* x) { x->neg = 0; x->n = 0; }

static void bn_trim(bn* x) {
  while (x->n > 0 && x->d[x->n - 1] == 0) x->n--;
  if (x->n == 0) x->neg = 0;
}

/* x = sign * mag * 2^shift, mag < 2^64 */
static void bn_set(bn* x, int neg, uint64_t mag, int shift) {
  bn_zero(x);
  if (mag == 0) return;
  int w = shift / 32, b = shift % 32;
  for (int i = 0; i < w; ++i) x->d[i] = 0;
  /* mag << b spans at most three limbs */
  uint64_t lo = mag << b;
  uint64_t hi = b ? mag >> (64 - b) : 0;
  x->d[w] = (uint32_t)lo;
  x->d[w + 1] = (uint32_t)(lo >> 32);
  x->d[w + 2] = (uint32_t)hi;
  x->n = w + 3;
  x->neg = neg;
  bn_trim(x);
}

static int bn_cmp_mag(const bn* a, const bn* b) {
  if (a->n != b->n) return a->n < b->n ? -1 : 1;
  for (int i = a->n - 1; i >= 0; --i)
    if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
  return 0;
}

/* r = |a| + |b| (r may alias neither) */
static void bn_add_mag(bn* r, const bn* a, const bn* b) {
  int n = a->n > b->n ? a->n : b->n;
  uint64_t carry = 0;
  for (int i = 0; i < n; ++i) {
    uint64_t s = carry + (i < a->n ? a->d[i] : 0) + (i < b->n ? b->d[i] : 0);
    r->d[i] = (uint32_t)s;
    carry = s >> 32;
  }
  r->n = n;
  if (carry) r->d[r->n++] = (uint32_t)carry;
}

/* r = |a| - |b| for |a| >= |b| */
static void bn_sub_mag(bn* r, const bn* a, const bn* b) {
  int64_t borrow = 0;
  for (int i = 0; i < a->n; ++i) {
    int64_t s = (int64_t)a->d[i] - (i < b->n ? b->d[i] : 0) - borrow;
    borrow = s < 0;
    r->d[i] = (uint32_t)(s + (borrow ? ((int64_t)1 << 32) : 0));
  }
  r->n = a->n;
}

/* r = a + (flip ? -b : b) */
static void bn_addsub(bn* r, const bn* a, const bn* b, int flip) {
  int bneg = b->n ? (b->neg ^ flip) : 0;
  if (a->neg == bneg) {
    bn_add_mag(r, a, b);
    r->neg = a->neg;
  } else if (bn_cmp_mag(a, b) >= 0) {
    bn_sub_mag(r, a, b);
    r->neg = a->neg;
  } else {
    bn_sub_mag(r, b, a);
    r->neg = bneg;
  }
  bn_trim(r);
}

/* r = a * b (schoolbook) */
static void bn_mul(bn* r, const bn* a, const bn* b) {
  bn_zero(r);
  if (a->n == 0 || b->n == 0) return;
  int n = a->n + b->n;
  for (int i = 0; i < n; ++i) r->d[i] = 0;
  for (int i = 0; i < a->n; ++i) {
    uint64_t carry = 0;
    for (int j = 0; j < b->n; ++j) {
      uint64_t t = (uint64_t)a->d[i] * b->d[j] + r->d[i + j] + carry;
      r->d[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    r->d[i + b->n] = (uint32_t)carry;
  }
  r->n = n;
  r->neg = a->neg ^ b->neg;
  bn_trim(r);
}

static int bn_sign(const bn* x) { return x->n == 0 ? 0 : (x->neg ? -1 : 1); }

/* The inputs v[0..k) as integers over a common power of two. */
static void to_ints(const double* v, int k, bn* out) {
  int E = 1 << 30;
  int ex[12];
  int64_t m[12];
  for (int i = 0; i < k; ++i) {
    int e = 0;
    double f = frexp(v[i], &e); /* v = f 2^e, 1/2 <= |f| < 1 */
    m[i] = (int64_t)ldexp(f, 53);
    ex[i] = e - 53;
    if (m[i] != 0 && ex[i] < E) E = ex[i];
  }
  for (int i = 0; i < k; ++i) {
    if (m[i] == 0) bn_zero(&out[i]);
    else bn_set(&out[i], m[i] < 0, (uint64_t)(m[i] < 0 ? -m[i] : m[i]), ex[i] - E);
  }
}

/* exact sign of (b - a) . ((c - a) x (d - a)) */
static int orient3d_exact(v3 a, v3 b, v3 c, v3 d) {
  double v[12] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, d.x, d.y, d.z};
  bn I[12], x[3], y[3], z[3], t1, t2, m, acc, acc2;
  to_ints(v, 12, I);
  for (int k = 0; k < 3; ++k) {
    bn_addsub(&x[k], &I[3 + k], &I[k], 1);
    bn_addsub(&y[k], &I[6 + k], &I[k], 1);
    bn_addsub(&z[k], &I[9 + k], &I[k], 1);
  }
  bn_zero(&acc);
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    /* component k of y x z: y[k1] z[k2] - y[k2] z[k1] */
    bn_mul(&t1, &y[k1], &z[k2]);
    bn_mul(&t2, &y[k2], &z[k1]);
    bn_addsub(&m, &t1, &t2, 1);
    bn_mul(&t1, &x[k], &m);
    bn_addsub(&acc2, &acc, &t1, 0);
    acc = acc2;
  }
  return bn_sign(&acc);
}

/* exact sign of (b - a) x (c - a) in the plane (2-D points) */
static int orient2d_exact(const double* a, const double* b, const double* c) {
  double v[6] = {a[0], a[1], b[0], b[1], c[0], c[1]};
  bn I[6], bx, by, cx, cy, t1, t2, r;
  to_ints(v, 6, I);
  bn_addsub(&bx, &I[2], &I[0], 1);
  bn_addsub(&by, &I[3], &I[1], 1);
  bn_addsub(&cx, &I[4], &I[0], 1);
  bn_addsub(&cy, &I[5], &I[1], 1);
  bn_mul(&t1, &bx, &cy);
  bn_mul(&t2, &by, &cx);
  bn_addsub(&r, &t1, &t2, 1);
  return bn_sign(&r);
}

/* Orientation signs: a double-precision evaluation whose sign is taken
 * when it clears an error bound, else the exact integer evaluation.  The
 * first-order error of the rounded differences, products and sums is below
 * 8 u times the permanent (the same expression over absolute values),
 * u = 2^-53, for orient3d and below 4 u of it for orient2d; twice that is
 * used.  Outside a safe range of magnitudes (underflow, overflow) the exact
 * path decides. */
static int orient3d(v3 a, v3 b, v3 c, v3 d) {
  v3 x = sub(b, a), y = sub(c, a), z = sub(d, a);
  double cx = y.y * z.z - y.z * z.y, cy = y.z * z.x - y.x * z.z, cz = y.x * z.y - y.y * z.x;
  double px = fabs(y.y * z.z) + fabs(y.z * z.y), py = fabs(y.z * z.x) + fabs(y.x * z.z),
         pz = fabs(y.x * z.y) + fabs(y.y * z.x);
  double perm = fabs(x.x) * px + fabs(x.y) * py + fabs(x.z) * pz;
  double det = x.x * cx + x.y * cy + x.z * cz;
  if (perm > 1e-250 && perm < 1e250) {
    double err = 16.0 * ldexp(1.0, -53) * perm;
    if (det > err) return 1;
    if (det < -err) return -1;
  }
  return orient3d_exact(a, b, c, d);
}

static int orient2d(const double* a, const double* b, const double* c) {
  double bx = b[0] - a[0], by = b[1] - a[1], cx = c[0] - a[0], cy = c[1] - a[1];
  double det = bx * cy - by * cx;
  double perm = fabs(bx * cy) + fabs(by * cx);
  if (perm > 1e-250 && perm < 1e250) {
    double err = 8.0 * ldexp(1.0, -53) * perm;
    if (det > err) return 1;
    if (det < -err) return -1;
  }
  return orient2d_exact(a, b, c);
}

/* ------------------------------------------------ exact meeting test */

/* 2-D projection of p that drops coordinate k */
static void proj(v3 p, int k, double* o) {
  double c[3] = {p.x, p.y, p.z};
  o[0] = c[k == 0 ? 1 : 0];
  o[1] = c[k == 2 ? 1 : 2];
}

/* x collinear with segment [p, q] (2-D): is it inside the segment's box? */
static int within_box2(const double* p, const double* q, const double* x) {
  for (int i = 0; i < 2; ++i) {
    double lo = p[i] < q[i] ? p[i] : q[i], hi = p[i] < q[i] ? q[i] : p[i];
    if (x[i] < lo || x[i] > hi) return 0;
  }
  return 1;
}

/* Do the closed 2-D segments [a, b] and [c, d] share a point?  (Either may
 * be a single point.) */
static int segs_meet2(const double* a, const double* b, const double* c, const double* d) {
  int s1 = orient2d(c, d, a), s2 = orient2d(c, d, b);
  int s3 = orient2d(a, b, c), s4 = orient2d(a, b, d);
  if (s1 * s2 < 0 && s3 * s4 < 0) return 1;
  if (s1 == 0 && within_box2(c, d, a)) return 1;
  if (s2 == 0 && within_box2(c, d, b)) return 1;
  if (s3 == 0 && within_box2(a, b, c)) return 1;
  if (s4 == 0 && within_box2(a, b, d)) return 1;
  return 0;
}

/* Do the closed 3-D segments [a, b] and [c, d] share a point?  They must be
 * coplanar; then they meet iff their projections onto all three coordinate
 * planes meet (one of those projections is one-to-one on a plane holding
 * them, and a common point of the segments projects to a common point of
 * every projection). */
static int segs_meet3(v3 a, v3 b, v3 c, v3 d) {
  if (orient3d(a, b, c, d) != 0) return 0;
  for (int k = 0; k < 3; ++k) {
    double A[2], B[2], Cc[2], D[2];
    proj(a, k, A);
    proj(b, k, B);
    proj(c, k, Cc);
    proj(d, k, D);
    if (!segs_meet2(A, B, Cc, D)) return 0;
  }
  return 1;
}

/* p in the closed 2-D triangle (t0, t1, t2) of orientation o != 0 */
static int in_tri2(const double* p, const double* t0, const double* t1, const double* t2, int o) {
  return orient2d(t0, t1, p) * o >= 0 && orient2d(t1, t2, p) * o >= 0 && orient2d(t2, t0, p) * o >= 0;
}

/* Does the closed segment [a, b] share a point with the closed triangle
 * (t0, t1, t2)?  All decisions are exact signs.  *strict is set when the
 * segment crosses the triangle's plane at one point strictly between its
 * endpoints (then *x is that point, up to rounding). */
static int seg_meets_tri(v3 a, v3 b, v3 t0, v3 t1, v3 t2, int* strict, v3* x) {
  *strict = 0;
  int sa = orient3d(t0, t1, t2, a), sb = orient3d(t0, t1, t2, b);
  if (sa * sb > 0) return 0; /* both ends strictly on one side */
  if (sa != 0 && sb != 0) {
    /* the segment crosses the (well-defined) plane at one interior point;
     * it lies in the closed triangle iff the line passes no edge on the
     * wrong side */
    int o1 = orient3d(a, b, t0, t1), o2 = orient3d(a, b, t1, t2), o3 = orient3d(a, b, t2, t0);
    int pos = o1 > 0 || o2 > 0 || o3 > 0, neg = o1 < 0 || o2 < 0 || o3 < 0;
    if (pos && neg) return 0;
    double ha = fabs(dot(sub(a, t0), cross(sub(t1, t0), sub(t2, t0))));
    double hb = fabs(dot(sub(b, t0), cross(sub(t1, t0), sub(t2, t0))));
    double t = ha + hb > 0.0 ? ha / (ha + hb) : 0.5;
    *x = add(a, scl(sub(b, a), t));
    *strict = 1;
    return 1;
  }
  /* a coordinate plane onto which the triangle projects with non-zero area */
  int k = -1, o = 0;
  double T0[2], T1[2], T2[2];
  for (int kk = 0; kk < 3 && k < 0; ++kk) {
    proj(t0, kk, T0);
    proj(t1, kk, T1);
    proj(t2, kk, T2);
    o = orient2d(T0, T1, T2);
    if (o != 0) k = kk;
  }
  if (k < 0) /* collinear or coincident vertices: the triangle is its edges */
    return segs_meet3(a, b, t0, t1) || segs_meet3(a, b, t1, t2) || segs_meet3(a, b, t2, t0);
  double A[2], B[2];
  proj(a, k, A);
  proj(b, k, B);
  if (sa == 0 && sb == 0) /* the segment lies in the triangle's plane */
    return in_tri2(A, T0, T1, T2, o) || in_tri2(B, T0, T1, T2, o) || segs_meet2(A, B, T0, T1) ||
           segs_meet2(A, B, T1, T2) || segs_meet2(A, B, T2, T0);
  /* exactly one end lies in the plane */
  return in_tri2(sa == 0 ? A : B, T0, T1, T2, o);
}

/* Do the closed triangles P and Q share a point?  (*strict: 0, or 1 / 2 when
 * an edge of P / of Q crosses the other's plane inside the other, at *x.)
 * Two closed triangles meet
 * iff an edge of one meets the other: in the non-coplanar case their common
 * part is a segment of the planes' common line whose ends lie on edges; in
 * the coplanar case the boundaries cross or one triangle holds the other,
 * with its vertices. */
static int tri_meet(const v3* p, const v3* q, int* strict, v3* x) {
  int any = 0;
  *strict = 0;
  for (int side = 0; side < 2; ++side) {
    const v3* A = side ? q : p;
    const v3* B = side ? p : q;
    for (int i = 0; i < 3; ++i) {
      int s = 0;
      v3 y;
      if (seg_meets_tri(A[i], A[(i + 1) % 3], B[0], B[1], B[2], &s, &y)) {
        any = 1;
        if (s) {
          *strict = 1 + side; /* 1: an edge of P crosses Q; 2: of Q crosses P */
          *x = y;
          return 1;
        }
      }
    }
  }
  return any;
}

int or_tri_meet(const double* P, const double* Q) {
  v3 p[3] = {mk(P), mk(P + 3), mk(P + 6)};
  v3 q[3] = {mk(Q), mk(Q + 3), mk(Q + 6)};
  int s;
  v3 x;
  return tri_meet(p, q, &s, &x);
}

/* signs for the tests: exact (integers only) and filtered */
int or_orient3d_exact(const double* a, const double* b, const double* c, const double* d) {
  return orient3d_exact(mk(a), mk(b), mk(c), mk(d));
}
int or_orient3d(const double* a, const double* b, const double* c, const double* d) {
  return orient3d(mk(a), mk(b), mk(c), mk(d));
}
int or_orient2d_exact(const double* a, const double* b, const double* c) { return orient2d_exact(a, b, c); }

/* Triangle-triangle distance.  P and Q are 9 doubles (3 vertices).  If cp is
 * not NULL it receives the closest point on P then on Q.  The distance is 0
 * exactly when the closed triangles meet (decided by exact signs); else it
 * is the smallest of the fifteen candidates, which is positive for exact
 * values: where rounding makes it 0, the smallest positive double stands
 * in, so that 0 always means "meet". */
double or_tri_dist(const double* P, const double* Q, double* cp) {
  v3 p[3] = {mk(P), mk(P + 3), mk(P + 6)};
  v3 q[3] = {mk(Q), mk(Q + 3), mk(Q + 6)};
  v3 bp = p[0], bq = q[0], x, y, cx = p[0];
  int strict = 0;
  int meet = tri_meet(p, q, &strict, &cx);
  if (meet && !cp) return 0.0;
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
  if (meet && strict) {
    /* a common point: the crossing point (on the crossing edge), and its
     * nearest point on the crossed triangle; kept when it beats the
     * candidates' points (which it does unless the crossing is nearly
     * tangential, where a candidate is nearly 0) */
    x = strict == 1 ? cx : tri_point(p[0], p[1], p[2], cx);
    y = strict == 2 ? cx : tri_point(q[0], q[1], q[2], cx);
    if (dist(x, y) < best) { bp = x; bq = y; }
  }
  if (cp) { cp[0] = bp.x; cp[1] = bp.y; cp[2] = bp.z; cp[3] = bq.x; cp[4] = bq.y; cp[5] = bq.z; }
  if (meet) return 0.0;
  return best > 0.0 ? best : ldexp(1.0, -1074);
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
      /* boxes sorted by lo.x: from the first that can reach r's box to the
       * last whose lo.x is still within tau of its hi.x (equal lo.x values
       * all included) */
      int64_t a = lower_x(j->boxes, nS, rlo[0] - j->tau - j->max_ext_x - 1.0);
      for (int64_t q = a; q < nS; ++q) {
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
