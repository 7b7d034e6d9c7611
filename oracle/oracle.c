/* CPU ORACLE for the stackless triangulation ray walk -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and
 * its reference arm) may load this library.  The product path never does: it
 * has no CPU fallback.  Nothing here is shared with the CUDA path; the two only
 * read the same seeded inputs.
 *
 * What it computes (Frederickx & Dutre, arXiv 2112.05570):
 *   - closest hit of a ray with the scene segments, by brute force over all
 *     segments: the plain definition of the query the walk answers (Sec. 5.1);
 *   - the walk itself, step by step as Sec. 5.1 states it: in the current
 *     triangle find the edge the ray leaves through; a constrained edge is the
 *     hit, a hull edge a miss, otherwise continue in the neighbour.  One step =
 *     one exit-edge determination (Sec. 5.4);
 *   - the step count by brute force (1 + interior edges crossed before the hit);
 *   - point location by scanning all triangles (Sec. 5.2's start triangle);
 *   - triangulation invariants and the Cauchy-Crofton line statistic that ties
 *     edge length to traversal cost (Sec. 1.4).
 *
 * Degeneracy rule (the paper does not fix one; Sec. 5.1 only asks for
 * consistent predicates).  With k = 2^22 * d (exact integers), the side of a
 * point v is s(v) = L if k.x*(v.y-o.y) - k.y*(v.x-o.x) >= 0, else R: a point on
 * the ray's line counts as left, i.e. the ray is shifted infinitesimally to its
 * right.  A segment (a,b) is hit iff s(a) != s(b) and its exact parameter t > 0.
 * Equal t (a common endpoint on the ray's line) is broken by the order in which
 * the shifted ray meets the segments: smaller (k.u)/|k x u| first, u = far
 * endpoint - common point.
 *
 * All hit / step decisions are exact integer arithmetic (int64, int128); t is
 * reported as the fp32 rounding of num/den computed in fp64 (both exact in fp64).
 * parity pinned: see tests/test_oracle.py (brute force vs walk vs step count,
 * golden worked examples, Crofton identity, planted mutations).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define ORC_SIDE_L 1
#define ORC_SIDE_R 0

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0 /* >0 plants a known mistake; used only by the pin tests */
#endif

/* ------------------------------------------------------------------ predicates */
/* k.x*(v.y-o.y) - k.y*(v.x-o.x), exact: |k| <= 2^22, |v-o| <= 2^21 */
static int64_t side_value(int64_t kx, int64_t ky, int64_t ox, int64_t oy, int64_t vx, int64_t vy) {
#if ORACLE_MUTANT == 1
  return kx * (vy - oy) + ky * (vx - ox); /* planted: wrong sign */
#else
  return kx * (vy - oy) - ky * (vx - ox);
#endif
}
static int side(int64_t kx, int64_t ky, int64_t ox, int64_t oy, int64_t vx, int64_t vy) {
#if ORACLE_MUTANT == 2
  return side_value(kx, ky, ox, oy, vx, vy) > 0 ? ORC_SIDE_L : ORC_SIDE_R; /* planted: on-line = right */
#else
  return side_value(kx, ky, ox, oy, vx, vy) >= 0 ? ORC_SIDE_L : ORC_SIDE_R;
#endif
}

static int64_t orient3(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy) {
  return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

/* Direction components must be multiples of 2^-22 with magnitude <= 1. */
static int dir_to_int(float d, int64_t* k) {
  double s = (double)d * 4194304.0;
  if (!(s >= -4194304.0 && s <= 4194304.0)) return 0;
  if (s != floor(s)) return 0;
  *k = (int64_t)s;
  return 1;
}

/* Parameter of the crossing of the ray's line with the line through (a,b):
 * o + t d with t = cross(b-a, a-o) / cross(b-a, d).  With d = k / 2^22,
 * t = 2^22 * num / den, num = cross(b-a, a-o), den = cross(b-a, k). */
typedef struct {
  int64_t num, den; /* den > 0 after normalisation */
} ratio;

static ratio seg_param(int64_t kx, int64_t ky, int64_t ox, int64_t oy, int64_t ax, int64_t ay, int64_t bx,
                       int64_t by) {
  ratio r;
  int64_t ex = bx - ax, ey = by - ay;
  r.num = ex * (ay - oy) - ey * (ax - ox);
  r.den = ex * ky - ey * kx;
  if (r.den < 0) {
    r.num = -r.num;
    r.den = -r.den;
  }
  return r;
}

static int ratio_cmp(ratio a, ratio b) { /* sign of a - b, denominators > 0 */
  i128 l = (i128)a.num * b.den, r = (i128)b.num * a.den;
  return (l > r) - (l < r);
}

static float ratio_to_t(ratio r) {
  double q = (double)r.num / (double)r.den; /* both exact in fp64 */
  return (float)(q * 4194304.0);
}

/* Tie order at a common point v on the ray's line: for a far point w on the
 * right, key = (k.u) / |k x u| with u = w - v; the shifted ray meets smaller
 * keys first.  Returns sign(key(u1) - key(u2)). */
static int tie_cmp(int64_t kx, int64_t ky, int64_t u1x, int64_t u1y, int64_t u2x, int64_t u2y) {
  i128 d1 = (i128)kx * u1x + (i128)ky * u1y, d2 = (i128)kx * u2x + (i128)ky * u2y;
  i128 c1 = (i128)kx * u1y - (i128)ky * u1x, c2 = (i128)kx * u2y - (i128)ky * u2x;
  if (c1 < 0) c1 = -c1;
  if (c2 < 0) c2 = -c2;
  /* compare d1/c1 with d2/c2 (c > 0): products up to 2^43 * 2^43 */
  i128 l = d1 * c2, r = d2 * c1;
  return (l > r) - (l < r);
}

/* ------------------------------------------------------------------ threading */
typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct {
  range_fn fn;
  void* ctx;
  int64_t lo, hi;
} job;
static void* job_run(void* p) {
  job* j = (job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}
static void run_parallel(range_fn fn, void* ctx, int64_t n, int n_threads) {
  if (n_threads <= 1 || n < 256) {
    fn(ctx, 0, n);
    return;
  }
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  job jobs[256];
  int64_t chunk = (n + n_threads - 1) / n_threads;
  int used = 0;
  for (int k = 0; k < n_threads; ++k) {
    int64_t lo = (int64_t)k * chunk, hi = lo + chunk < n ? lo + chunk : n;
    if (lo >= hi) break;
    jobs[k].fn = fn;
    jobs[k].ctx = ctx;
    jobs[k].lo = lo;
    jobs[k].hi = hi;
    pthread_create(&th[k], NULL, job_run, &jobs[k]);
    ++used;
  }
  for (int k = 0; k < used; ++k) pthread_join(th[k], NULL);
}

/* ------------------------------------------------------------------ brute force */
typedef struct {
  int64_t n_seg;
  const int32_t* seg; /* 4 per segment: x0 y0 x1 y1 */
  const int32_t *ox, *oy;
  const float *dx, *dy;
  int32_t* hit;
  float* t;
} bf_ctx;

/* The closest segment under the degeneracy rule; returns -1 for none.  */
static int32_t closest_segment(const int32_t* seg, int64_t n_seg, int64_t ox, int64_t oy, int64_t kx, int64_t ky,
                               ratio* best_t) {
  int32_t best = -1;
  ratio bt = {0, 1};
  int64_t bux = 0, buy = 0;
  for (int64_t s = 0; s < n_seg; ++s) {
    int64_t ax = seg[4 * s], ay = seg[4 * s + 1], bx = seg[4 * s + 2], by = seg[4 * s + 3];
    int sa = side(kx, ky, ox, oy, ax, ay), sb = side(kx, ky, ox, oy, bx, by);
    if (sa == sb) continue;
    ratio r = seg_param(kx, ky, ox, oy, ax, ay, bx, by);
#if ORACLE_MUTANT != 3 /* planted (3): accepts hits behind the origin */
    if (r.num <= 0) continue;
#endif
    /* far endpoint on the right, seen from the crossing point */
    int64_t wx = sa == ORC_SIDE_R ? ax : bx, wy = sa == ORC_SIDE_R ? ay : by;
    if (best < 0) {
      best = (int32_t)s;
      bt = r;
      bux = wx;
      buy = wy;
      continue;
    }
    int c = ratio_cmp(r, bt);
    if (c < 0) {
      best = (int32_t)s;
      bt = r;
      bux = wx;
      buy = wy;
    } else if (c == 0) {
      /* same crossing point: it is a common endpoint v on the ray's line
         (disjoint segments meet nowhere else); v is the endpoint of s that is
         not w.  Compare the right-hand far endpoints seen from v. */
      int64_t pvx, pvy;
      pvx = (wx == ax && wy == ay) ? bx : ax;
      pvy = (wx == ax && wy == ay) ? by : ay;
      if (tie_cmp(kx, ky, wx - pvx, wy - pvy, bux - pvx, buy - pvy) < 0) {
        best = (int32_t)s;
        bt = r;
        bux = wx;
        buy = wy;
      }
    }
  }
  *best_t = bt;
  return best;
}

static void bf_range(void* p, int64_t lo, int64_t hi) {
  bf_ctx* c = (bf_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    int64_t kx, ky;
    if (!dir_to_int(c->dx[i], &kx) || !dir_to_int(c->dy[i], &ky) || (kx == 0 && ky == 0)) {
      c->hit[i] = -1;
      c->t[i] = NAN;
      continue;
    }
    ratio bt;
    int32_t s = closest_segment(c->seg, c->n_seg, c->ox[i], c->oy[i], kx, ky, &bt);
    c->hit[i] = s;
    c->t[i] = s >= 0 ? ratio_to_t(bt) : INFINITY;
  }
}

/* Closest hit by scanning every segment.  hit = segment id or -1 (miss or an
 * invalid direction); t = fp32 hit parameter, +inf on a miss, NaN if invalid. */
int oracle_closest_bruteforce(int64_t n_seg, const int32_t* seg, int64_t n, const int32_t* ox, const int32_t* oy,
                              const float* dx, const float* dy, int32_t* hit, float* t, int32_t n_threads) {
  bf_ctx c = {n_seg, seg, ox, oy, dx, dy, hit, t};
  run_parallel(bf_range, &c, n, n_threads);
  return 0;
}

/* ------------------------------------------------------------------ the walk */
typedef struct {
  int64_t n_tri;
  const int32_t *vx, *vy, *tri_v, *tri_nb, *tri_seg;
  const int32_t *ox, *oy;
  const float *dx, *dy;
  const int32_t* start;
  int32_t *hit, *steps, *last_tri;
  float* t;
  int64_t max_steps;
  int32_t through; /* 1: cross constrained edges as if unconstrained (Crofton test) */
} walk_ctx;

static int strictly_inside(const walk_ctx* c, int64_t tri, int64_t px, int64_t py) {
  for (int i = 0; i < 3; ++i) {
    int32_t a = c->tri_v[3 * tri + (i + 1) % 3], b = c->tri_v[3 * tri + (i + 2) % 3];
    if (orient3(c->vx[a], c->vy[a], c->vx[b], c->vy[b], px, py) <= 0) return 0;
  }
  return 1;
}

static void walk_range(void* p, int64_t lo, int64_t hi) {
  walk_ctx* c = (walk_ctx*)p;
  for (int64_t r = lo; r < hi; ++r) {
    int64_t kx, ky, ox = c->ox[r], oy = c->oy[r];
    int64_t T = c->start[r];
    c->hit[r] = -1;
    c->t[r] = NAN;
    c->steps[r] = -1;
    if (c->last_tri) c->last_tri[r] = -1;
    if (!dir_to_int(c->dx[r], &kx) || !dir_to_int(c->dy[r], &ky) || (kx == 0 && ky == 0)) continue;
    if (T < 0 || T >= c->n_tri || !strictly_inside(c, T, ox, oy)) continue;
    int64_t steps = 0;
    for (;;) {
      ++steps;
      if (steps > c->max_steps) {
        c->steps[r] = -2;
        break;
      }
      /* exit edge: the CCW edge (a -> b) with s(a) = R and s(b) = L */
      int e = -1;
      for (int i = 0; i < 3; ++i) {
        int32_t a = c->tri_v[3 * T + (i + 1) % 3], b = c->tri_v[3 * T + (i + 2) % 3];
        int sa = side(kx, ky, ox, oy, c->vx[a], c->vy[a]);
        int sb = side(kx, ky, ox, oy, c->vx[b], c->vy[b]);
#if ORACLE_MUTANT == 4
        if (sa == ORC_SIDE_L && sb == ORC_SIDE_R) { /* planted: takes the entry edge */
#else
        if (sa == ORC_SIDE_R && sb == ORC_SIDE_L) {
#endif
          e = i;
          break;
        }
      }
      if (e < 0) { /* cannot happen for a strictly interior origin */
        c->steps[r] = -3;
        break;
      }
      int32_t seg = c->tri_seg[3 * T + e];
      int32_t nb = c->tri_nb[3 * T + e];
      if (seg >= 0 && !c->through) {
        int32_t a = c->tri_v[3 * T + (e + 1) % 3], b = c->tri_v[3 * T + (e + 2) % 3];
        ratio q = seg_param(kx, ky, ox, oy, c->vx[a], c->vy[a], c->vx[b], c->vy[b]);
        c->hit[r] = seg;
        c->t[r] = ratio_to_t(q);
        c->steps[r] = (int32_t)steps;
        if (c->last_tri) c->last_tri[r] = (int32_t)T;
        break;
      }
      if (nb < 0) {
        c->hit[r] = -1;
        c->t[r] = INFINITY;
        c->steps[r] = (int32_t)steps;
        if (c->last_tri) c->last_tri[r] = (int32_t)T;
        break;
      }
      T = nb;
    }
  }
}

/* The walk of Sec. 5.1 from the given start triangles.  steps = triangles
 * visited including the start one; -1 = invalid ray (direction off the 2^-22
 * grid, zero direction, start triangle not strictly containing the origin);
 * -2 = more than max_steps steps.  last_tri (optional) = final triangle. */
int oracle_walk(int64_t n_tri, const int32_t* vx, const int32_t* vy, const int32_t* tri_v, const int32_t* tri_nb,
                const int32_t* tri_seg, int64_t n, const int32_t* ox, const int32_t* oy, const float* dx,
                const float* dy, const int32_t* start, int32_t* hit, float* t, int32_t* steps, int32_t* last_tri,
                int64_t max_steps, int32_t through, int32_t n_threads) {
  walk_ctx c = {n_tri, vx, vy, tri_v, tri_nb, tri_seg, ox, oy, dx, dy, start, hit, steps, last_tri, t,
                max_steps, through};
  run_parallel(walk_range, &c, n, n_threads);
  return 0;
}

/* ------------------------------------------------------------------ steps by brute force */
typedef struct {
  int64_t n_tri, n_seg;
  const int32_t *vx, *vy, *tri_v, *tri_nb, *seg;
  const int32_t *ox, *oy;
  const float *dx, *dy;
  const int32_t* hit;
  int32_t* steps;
} sbf_ctx;

static void sbf_range(void* p, int64_t lo, int64_t hi) {
  sbf_ctx* c = (sbf_ctx*)p;
  for (int64_t r = lo; r < hi; ++r) {
    int64_t kx, ky, ox = c->ox[r], oy = c->oy[r];
    if (!dir_to_int(c->dx[r], &kx) || !dir_to_int(c->dy[r], &ky) || (kx == 0 && ky == 0)) {
      c->steps[r] = -1;
      continue;
    }
    int32_t h = c->hit[r];
    ratio th = {0, 1};
    int64_t hwx = 0, hwy = 0; /* right-hand endpoint of the hit segment */
    if (h >= 0) {
      int64_t ax = c->seg[4 * h], ay = c->seg[4 * h + 1], bx = c->seg[4 * h + 2], by = c->seg[4 * h + 3];
      th = seg_param(kx, ky, ox, oy, ax, ay, bx, by);
      int sa = side(kx, ky, ox, oy, ax, ay);
      hwx = sa == ORC_SIDE_R ? ax : bx;
      hwy = sa == ORC_SIDE_R ? ay : by;
    }
    int64_t count = 0;
    for (int64_t T = 0; T < c->n_tri; ++T)
      for (int i = 0; i < 3; ++i) {
        int32_t nb = c->tri_nb[3 * T + i];
        if (nb < 0 || nb < T) continue; /* interior edges, each once */
        int32_t a = c->tri_v[3 * T + (i + 1) % 3], b = c->tri_v[3 * T + (i + 2) % 3];
        int64_t ax = c->vx[a], ay = c->vy[a], bx = c->vx[b], by = c->vy[b];
        int64_t va = side_value(kx, ky, ox, oy, ax, ay), vb = side_value(kx, ky, ox, oy, bx, by);
        int sa = va >= 0, sb = vb >= 0;
        if (sa == sb) continue;
        ratio q = seg_param(kx, ky, ox, oy, ax, ay, bx, by);
        if (q.num <= 0) continue;
        if (h < 0) {
          ++count;
          continue;
        }
        int cmp = ratio_cmp(q, th);
        if (cmp < 0) {
          ++count;
        } else if (cmp == 0) {
          /* crossing at the hit point: if it is this edge's endpoint on the
             line, order by the shifted ray; otherwise it is the hit edge */
          int64_t px, py, wx, wy;
          if (va == 0) {
            px = ax; py = ay; wx = bx; wy = by;
          } else if (vb == 0) {
            px = bx; py = by; wx = ax; wy = ay;
          } else {
            continue;
          }
          if (tie_cmp(kx, ky, wx - px, wy - py, hwx - px, hwy - py) < 0) ++count;
        }
      }
    c->steps[r] = (int32_t)(1 + count);
  }
}

/* Step count without walking: 1 + the number of interior triangulation edges
 * the (right-shifted) ray crosses before its closest hit `hit` (or before the
 * hull on a miss).  O(n_tri) per ray. */
int oracle_steps_bruteforce(int64_t n_tri, const int32_t* vx, const int32_t* vy, const int32_t* tri_v,
                            const int32_t* tri_nb, int64_t n_seg, const int32_t* seg, int64_t n, const int32_t* ox,
                            const int32_t* oy, const float* dx, const float* dy, const int32_t* hit, int32_t* steps,
                            int32_t n_threads) {
  sbf_ctx c = {n_tri, n_seg, vx, vy, tri_v, tri_nb, seg, ox, oy, dx, dy, hit, steps};
  run_parallel(sbf_range, &c, n, n_threads);
  return 0;
}

/* ------------------------------------------------------------------ point location */
typedef struct {
  int64_t n_tri;
  const int32_t *vx, *vy, *tri_v;
  const int32_t *px, *py;
  int32_t* tri;
} loc_ctx;

static void loc_range(void* p, int64_t lo, int64_t hi) {
  loc_ctx* c = (loc_ctx*)p;
  for (int64_t k = lo; k < hi; ++k) {
    int32_t found = -2;
    for (int64_t T = 0; T < c->n_tri && found == -2; ++T) {
      int zero = 0, neg = 0;
      for (int i = 0; i < 3; ++i) {
        int32_t a = c->tri_v[3 * T + (i + 1) % 3], b = c->tri_v[3 * T + (i + 2) % 3];
        int64_t o = orient3(c->vx[a], c->vy[a], c->vx[b], c->vy[b], c->px[k], c->py[k]);
        if (o < 0) neg = 1;
        if (o == 0) zero = 1;
      }
      if (!neg) found = zero ? -1 : (int32_t)T;
    }
    c->tri[k] = found;
  }
}

/* Triangle whose interior strictly contains each point; -1 = the point lies on
 * an edge or a vertex; -2 = outside every triangle.  O(n_tri) per point. */
int oracle_locate_bruteforce(int64_t n_tri, const int32_t* vx, const int32_t* vy, const int32_t* tri_v, int64_t n,
                             const int32_t* px, const int32_t* py, int32_t* tri, int32_t n_threads) {
  loc_ctx c = {n_tri, vx, vy, tri_v, px, py, tri};
  run_parallel(loc_range, &c, n, n_threads);
  return 0;
}

/* ------------------------------------------------------------------ invariants */
/* Failure bits of oracle_check_triangulation. */
#define ORC_BAD_INDEX 1
#define ORC_NOT_CCW 2
#define ORC_AREA 4
#define ORC_NB_ASYM 8
#define ORC_HULL 16
#define ORC_EULER 32
#define ORC_CONSTRAINT_ASYM 64
#define ORC_COVERAGE 128
#define ORC_NOT_DELAUNAY 256

static int on_square_side(int64_t D, int64_t ax, int64_t ay, int64_t bx, int64_t by) {
  return (ax == 0 && bx == 0) || (ay == 0 && by == 0) || (ax == D && bx == D) || (ay == D && by == D);
}

static int incircle_sign(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy, int64_t dx,
                         int64_t dy) {
  int64_t adx = ax - dx, ady = ay - dy, bdx = bx - dx, bdy = by - dy, cdx = cx - dx, cdy = cy - dy;
  i128 al = (i128)adx * adx + (i128)ady * ady, bl = (i128)bdx * bdx + (i128)bdy * bdy,
       cl = (i128)cdx * cdx + (i128)cdy * cdy;
  i128 det = al * ((i128)bdx * cdy - (i128)bdy * cdx) + bl * ((i128)cdx * ady - (i128)cdy * adx) +
             cl * ((i128)adx * bdy - (i128)ady * bdx);
  return (det > 0) - (det < 0);
}

typedef struct {
  int64_t lo, hi; /* parameter interval along the segment, scaled by |b-a|^2 */
} span;
static int span_cmp(const void* a, const void* b) {
  const span *x = (const span*)a, *y = (const span*)b;
  return (x->lo > y->lo) - (x->lo < y->lo);
}

/* Checks, for a triangulation of the square [0,D]^2:
 *   every index in range; every triangle strictly CCW; sum of doubled areas
 *   = 2 D^2; neighbour symmetry (same two vertices, pointing back); hull edges
 *   (-1) exactly the edges on the square's sides; Euler: T = 2V - h - 2 with h
 *   the vertices on the square's boundary; constrained labels equal on both
 *   sides; every segment covered exactly by collinear constrained edges
 *   carrying its id, and no other constrained edge; if check_delaunay, every
 *   unconstrained interior edge is locally Delaunay (int128 in-circle).
 * Returns the OR of the failure bits (0 = all hold). */
int32_t oracle_check_triangulation(int64_t D, int64_t n_vert, const int32_t* vx, const int32_t* vy, int64_t n_tri,
                                   const int32_t* tri_v, const int32_t* tri_nb, const int32_t* tri_seg,
                                   int64_t n_seg, const int32_t* seg, int32_t check_delaunay) {
  int32_t bad = 0;
  i128 area2 = 0;
  for (int64_t T = 0; T < n_tri; ++T)
    for (int i = 0; i < 3; ++i) {
      int32_t v = tri_v[3 * T + i], nb = tri_nb[3 * T + i], s = tri_seg[3 * T + i];
      if (v < 0 || v >= n_vert || nb < -1 || nb >= n_tri || s < -1 || s >= n_seg) return ORC_BAD_INDEX;
    }
  for (int64_t T = 0; T < n_tri; ++T) {
    const int32_t* t = tri_v + 3 * T;
    int64_t o = orient3(vx[t[0]], vy[t[0]], vx[t[1]], vy[t[1]], vx[t[2]], vy[t[2]]);
    if (o <= 0) bad |= ORC_NOT_CCW;
    area2 += o;
    for (int i = 0; i < 3; ++i) {
      int32_t a = t[(i + 1) % 3], b = t[(i + 2) % 3], nb = tri_nb[3 * T + i];
      if (nb < 0) {
        if (!on_square_side(D, vx[a], vy[a], vx[b], vy[b])) bad |= ORC_HULL;
        if (tri_seg[3 * T + i] >= 0) bad |= ORC_CONSTRAINT_ASYM; /* hull is not scene geometry here */
        continue;
      }
      int j, found = -1;
      for (j = 0; j < 3; ++j) {
        int32_t a2 = tri_v[3 * nb + (j + 1) % 3], b2 = tri_v[3 * nb + (j + 2) % 3];
        if (a2 == b && b2 == a) found = j;
      }
      if (found < 0 || tri_nb[3 * nb + found] != T) {
        bad |= ORC_NB_ASYM;
        continue;
      }
      if (tri_seg[3 * nb + found] != tri_seg[3 * T + i]) bad |= ORC_CONSTRAINT_ASYM;
      if (on_square_side(D, vx[a], vy[a], vx[b], vy[b])) bad |= ORC_HULL;
      if (check_delaunay && tri_seg[3 * T + i] < 0) {
        int32_t s = tri_v[3 * nb + found];
        if (incircle_sign(vx[t[0]], vy[t[0]], vx[t[1]], vy[t[1]], vx[t[2]], vy[t[2]], vx[s], vy[s]) > 0)
          bad |= ORC_NOT_DELAUNAY;
      }
    }
  }
  if (area2 != (i128)2 * D * D) bad |= ORC_AREA;
  /* Euler with all vertices used */
  {
    char* used = (char*)calloc((size_t)n_vert, 1);
    for (int64_t k = 0; k < 3 * n_tri; ++k) used[tri_v[k]] = 1;
    int64_t h = 0, nv = 0;
    for (int64_t v = 0; v < n_vert; ++v) {
      if (!used[v]) continue;
      ++nv;
      if (vx[v] == 0 || vy[v] == 0 || vx[v] == D || vy[v] == D) ++h;
    }
    free(used);
    if (nv != n_vert || n_tri != 2 * nv - h - 2) bad |= ORC_EULER;
  }
  /* coverage: collect constrained edges per segment (each once) */
  {
    int64_t* cnt = (int64_t*)calloc((size_t)n_seg + 1, sizeof(int64_t));
    for (int64_t T = 0; T < n_tri; ++T)
      for (int i = 0; i < 3; ++i) {
        int32_t s = tri_seg[3 * T + i], nb = tri_nb[3 * T + i];
        if (s >= 0 && nb > T) cnt[s]++;
      }
    int64_t* off = (int64_t*)calloc((size_t)n_seg + 1, sizeof(int64_t));
    for (int64_t s = 0; s < n_seg; ++s) off[s + 1] = off[s] + cnt[s];
    span* sp = (span*)malloc(sizeof(span) * (size_t)(off[n_seg] + 1));
    int64_t* fill = (int64_t*)calloc((size_t)n_seg + 1, sizeof(int64_t));
    for (int64_t T = 0; T < n_tri; ++T)
      for (int i = 0; i < 3; ++i) {
        int32_t s = tri_seg[3 * T + i], nb = tri_nb[3 * T + i];
        if (s < 0 || nb <= T) continue;
        int64_t ax = seg[4 * s], ay = seg[4 * s + 1], bx = seg[4 * s + 2], by = seg[4 * s + 3];
        int32_t p = tri_v[3 * T + (i + 1) % 3], q = tri_v[3 * T + (i + 2) % 3];
        if (orient3(ax, ay, bx, by, vx[p], vy[p]) != 0 || orient3(ax, ay, bx, by, vx[q], vy[q]) != 0) {
          bad |= ORC_COVERAGE;
          continue;
        }
        int64_t ex = bx - ax, ey = by - ay;
        int64_t tp = (vx[p] - ax) * ex + (vy[p] - ay) * ey, tq = (vx[q] - ax) * ex + (vy[q] - ay) * ey;
        span z = {tp < tq ? tp : tq, tp < tq ? tq : tp};
        sp[off[s] + fill[s]++] = z;
      }
    for (int64_t s = 0; s < n_seg; ++s) {
      int64_t ex = seg[4 * s + 2] - seg[4 * s], ey = seg[4 * s + 3] - seg[4 * s + 1];
      int64_t L2 = ex * ex + ey * ey;
      int64_t m = fill[s];
      if (m == 0) {
        bad |= ORC_COVERAGE;
        continue;
      }
      qsort(sp + off[s], (size_t)m, sizeof(span), span_cmp);
      int64_t pos = 0;
      for (int64_t k = 0; k < m; ++k) {
        if (sp[off[s] + k].lo != pos) bad |= ORC_COVERAGE;
        pos = sp[off[s] + k].hi;
      }
      if (pos != L2) bad |= ORC_COVERAGE;
    }
    free(cnt);
    free(off);
    free(sp);
    free(fill);
  }
  return bad;
}

/* ------------------------------------------------------------------ Cauchy-Crofton */
/* Total length of the interior (non-hull) edges, fp64. */
double oracle_interior_length(int64_t n_tri, const int32_t* vx, const int32_t* vy, const int32_t* tri_v,
                              const int32_t* tri_nb) {
  double L = 0.0;
  for (int64_t T = 0; T < n_tri; ++T)
    for (int i = 0; i < 3; ++i) {
      int32_t nb = tri_nb[3 * T + i];
      if (nb < 0 || nb < T) continue;
      int32_t a = tri_v[3 * T + (i + 1) % 3], b = tri_v[3 * T + (i + 2) % 3];
      double ex = (double)vx[b] - vx[a], ey = (double)vy[b] - vy[a];
      L += sqrt(ex * ex + ey * ey);
    }
  return L;
}

/* For each line (unit normal (cx, cy), offset p: the points x with n.x = p),
 * count the interior edges whose endpoints lie strictly on opposite sides.
 * Brute force over all edges, fp64 (a random line passes through no vertex). */
int oracle_count_line_crossings(int64_t n_tri, const int32_t* vx, const int32_t* vy, const int32_t* tri_v,
                                const int32_t* tri_nb, int64_t n_lines, const double* cx, const double* cy,
                                const double* p, int32_t* count) {
  for (int64_t l = 0; l < n_lines; ++l) {
    int64_t c = 0;
    for (int64_t T = 0; T < n_tri; ++T)
      for (int i = 0; i < 3; ++i) {
        int32_t nb = tri_nb[3 * T + i];
        if (nb < 0 || nb < T) continue;
        int32_t a = tri_v[3 * T + (i + 1) % 3], b = tri_v[3 * T + (i + 2) % 3];
        double fa = cx[l] * vx[a] + cy[l] * vy[a] - p[l], fb = cx[l] * vx[b] + cy[l] * vy[b] - p[l];
        if ((fa < 0) != (fb < 0)) ++c;
      }
    count[l] = (int32_t)c;
  }
  return 0;
}

int32_t oracle_mutant(void) { return ORACLE_MUTANT; }
