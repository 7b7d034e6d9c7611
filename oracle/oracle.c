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
 *   - paths of secondary rays that start in the final triangle of their
 *     parent's walk (Sec. 5.2), walk-chained and by brute force (see the
 *     section "secondary rays" for the readings);
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
 * golden worked examples, Crofton identity, planted mutations) and
 * tests/test_oracle_bounce.py (secondary rays: brute force vs chained walks,
 * closed forms on parallel and 45-degree mirrors, exact snapped origins,
 * planted mutations).
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

/* ------------------------------------------------------------------ comparison structures (Sec. 5.3) */
/* Parameters along the ray as exact rationals of t / 2^22: a slab parameter
 * (X - o) / k and a segment parameter num / den, denominators positive; a
 * zero denominator stands for +infinity. */
typedef struct {
  int64_t num, den;
} q64;

static int q_cmp(q64 a, q64 b) { /* sign of a - b */
  if (a.den == 0 && b.den == 0) return 0;
  if (a.den == 0) return 1;
  if (b.den == 0) return -1;
  i128 l = (i128)a.num * b.den, r = (i128)b.num * a.den;
  return (l > r) - (l < r);
}

typedef struct {
  int32_t seg;
  ratio t;
  int64_t wx, wy; /* right-hand endpoint of the best segment */
} best_hit;

/* The segment test of the brute force, keeping the closest hit; `limit`
 * (den > 0) bounds the accepted parameter (inclusive). */
static void consider(best_hit* b, const int32_t* q, int32_t sid, int64_t ox, int64_t oy, int64_t kx, int64_t ky,
                     const q64* limit) {
  int64_t ax = q[0], ay = q[1], bx = q[2], by = q[3];
  int sa = side(kx, ky, ox, oy, ax, ay), sb = side(kx, ky, ox, oy, bx, by);
  if (sa == sb) return;
  ratio r = seg_param(kx, ky, ox, oy, ax, ay, bx, by);
  if (r.num <= 0) return;
  if (limit) {
    q64 rq = {r.num, r.den};
    if (q_cmp(rq, *limit) > 0) return;
  }
  int64_t wx = sa == ORC_SIDE_R ? ax : bx, wy = sa == ORC_SIDE_R ? ay : by;
  int64_t vx = sa == ORC_SIDE_R ? bx : ax, vy = sa == ORC_SIDE_R ? by : ay;
  int take = b->seg < 0;
  if (!take) {
    int c = ratio_cmp(r, b->t);
    take = c < 0 || (c == 0 && tie_cmp(kx, ky, wx - vx, wy - vy, b->wx - vx, b->wy - vy) < 0);
  }
  if (take) {
    b->seg = sid;
    b->t = r;
    b->wx = wx;
    b->wy = wy;
  }
}

/* Entry parameter of the ray into a closed box; 0 if it misses the box. */
static int slab(const int32_t* B, int64_t ox, int64_t oy, int64_t kx, int64_t ky, q64* tn) {
  q64 nr = {0, 1}, fr = {0, 0};
  int64_t lo[2] = {B[0], B[1]}, hi[2] = {B[2], B[3]}, o[2] = {ox, oy}, k[2] = {kx, ky};
  for (int a = 0; a < 2; ++a) {
    if (k[a] == 0) {
      if (o[a] < lo[a] || o[a] > hi[a]) return 0;
      continue;
    }
    q64 near = k[a] > 0 ? (q64){lo[a] - o[a], k[a]} : (q64){o[a] - hi[a], -k[a]};
    q64 far = k[a] > 0 ? (q64){hi[a] - o[a], k[a]} : (q64){o[a] - lo[a], -k[a]};
    if (q_cmp(near, nr) > 0) nr = near;
    if (q_cmp(far, fr) < 0) fr = far;
  }
  if (q_cmp(fr, nr) < 0) return 0;
  *tn = nr;
  return 1;
}

typedef struct {
  int32_t n_nodes;
  const int32_t *box, *c0, *c1, *prims, *seg;
  const int32_t *ox, *oy;
  const float *dx, *dy;
  int32_t *hit, *ops;
  float* t;
} bvh_ctx;

static void bvh_range(void* p, int64_t lo, int64_t hi) {
  bvh_ctx* c = (bvh_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    int64_t kx, ky, ox = c->ox[i], oy = c->oy[i];
    if (!dir_to_int(c->dx[i], &kx) || !dir_to_int(c->dy[i], &ky) || (kx == 0 && ky == 0)) {
      c->hit[i] = -1;
      c->t[i] = NAN;
      c->ops[2 * i] = c->ops[2 * i + 1] = -1;
      continue;
    }
    best_hit b = {-1, {0, 1}, 0, 0};
    int32_t n_aabb = 1, n_prim = 0;
    int32_t stack[128];
    q64 st_t[128];
    int sp = 0;
    q64 tn;
    if (slab(c->box, ox, oy, kx, ky, &tn)) {
      stack[sp] = 0;
      st_t[sp++] = tn;
    }
    while (sp > 0) {
      --sp;
      int32_t N = stack[sp];
      q64 bt = {b.t.num, b.t.den};
#if ORACLE_MUTANT != 10 /* planted (10): nodes entered beyond the best hit are still opened */
      if (b.seg >= 0 && q_cmp(st_t[sp], bt) > 0) continue; /* entered beyond the best hit */
#endif
      int32_t c0 = c->c0[N], c1 = c->c1[N];
      if (c0 < 0) { /* leaf: test every segment */
        for (int32_t k = 0; k < c1; ++k) {
          int32_t sid = c->prims[-1 - c0 + k];
          ++n_prim;
          consider(&b, c->seg + 4 * (int64_t)sid, sid, ox, oy, kx, ky, NULL);
        }
        continue;
      }
      q64 t0, t1;
      n_aabb += 2;
      int h0 = slab(c->box + 4 * (int64_t)c0, ox, oy, kx, ky, &t0);
      int h1 = slab(c->box + 4 * (int64_t)c1, ox, oy, kx, ky, &t1);
      bt = (q64){b.t.num, b.t.den};
      if (h0 && b.seg >= 0 && q_cmp(t0, bt) > 0) h0 = 0;
      if (h1 && b.seg >= 0 && q_cmp(t1, bt) > 0) h1 = 0;
      if (h0 && h1) { /* the nearer child is visited first; the left one on equal entry */
#if ORACLE_MUTANT == 11 /* planted: the left child first whatever the entry parameters */
        int left_first = 1;
#else
        int left_first = q_cmp(t0, t1) <= 0;
#endif
        stack[sp] = left_first ? c1 : c0;
        st_t[sp++] = left_first ? t1 : t0;
        stack[sp] = left_first ? c0 : c1;
        st_t[sp++] = left_first ? t0 : t1;
      } else if (h0) {
        stack[sp] = c0;
        st_t[sp++] = t0;
      } else if (h1) {
        stack[sp] = c1;
        st_t[sp++] = t1;
      }
    }
    c->hit[i] = b.seg;
    c->t[i] = b.seg >= 0 ? ratio_to_t(b.t) : INFINITY;
    c->ops[2 * i] = n_aabb;
    c->ops[2 * i + 1] = n_prim;
  }
}

/* BVH traversal (Sec. 5.3.1): from the root, nearer child first, boxes
 * entered beyond the best hit skipped.  ops: AABB tests, segment tests. */
int oracle_bvh_trace(int32_t n_nodes, const int32_t* box, const int32_t* c0, const int32_t* c1, const int32_t* prims,
                     const int32_t* seg, int64_t n, const int32_t* ox, const int32_t* oy, const float* dx,
                     const float* dy, int32_t* hit, float* t, int32_t* ops, int32_t n_threads) {
  bvh_ctx c = {n_nodes, box, c0, c1, prims, seg, ox, oy, dx, dy, hit, ops, t};
  run_parallel(bvh_range, &c, n, n_threads);
  return 0;
}

typedef struct {
  int32_t n_nodes;
  const int32_t *axis, *split, *child, *count, *box, *rope, *refs, *seg;
  const int32_t *ox, *oy;
  const float *dx, *dy;
  int32_t *hit, *ops;
  float* t;
} kd_ctx;

/* The number of ropes of a leaf's face (Sec. 5.3.2: a leaf has one rope per
 * neighbour cell along each of its boundary segments): the leaves on the far
 * side of the face's plane whose boxes share a piece of positive length with
 * the face.  Found by a plain spatial query from the root, independent of the
 * ropes stored in the tree: a node is entered only if its box contains the
 * plane's coordinate and overlaps the face's extent on the other axis (every
 * qualifying leaf lies inside all its ancestors' boxes). */
static int32_t kd_face_neighbours(const kd_ctx* c, int32_t L, int face, int32_t* stack) {
  const int32_t* B = c->box + 4 * (int64_t)L;
  int fa = face / 2, fmax = face & 1;
  int64_t plane = fmax ? B[2 + fa] : B[fa];
  int64_t f0 = B[1 - fa], f1 = B[3 - fa];
  int32_t n = 0, sp = 0; /* stack: room for n_nodes + 1 entries */
  stack[sp++] = 0;
  while (sp > 0) {
    int32_t N = stack[--sp];
    const int32_t* nb = c->box + 4 * (int64_t)N;
    if (nb[fa] > plane || nb[2 + fa] < plane) continue;
    int64_t lo = nb[1 - fa] > f0 ? nb[1 - fa] : f0, hi = nb[3 - fa] < f1 ? nb[3 - fa] : f1;
    if (hi <= lo) continue; /* shares a point at most with the face */
    if (c->axis[N] != 2) {
      stack[sp++] = c->child[N];
      stack[sp++] = c->child[N] + 1;
      continue;
    }
    if (N == L) continue;
    /* a leaf on the far side touches the plane with its near boundary */
    if (fmax ? nb[fa] == plane : nb[2 + fa] == plane) ++n;
  }
  return n;
}

/* Rope search steps of an ideal rope tree over n ropes (Sec. 5.3.2 counts
 * log n steps for a boundary with n ropes): ceil(log2 n), 0 for one rope. */
static int32_t ideal_rope_steps(int32_t n) {
  int32_t s = 0;
#if ORACLE_MUTANT == 9 /* planted: floor(log2 n) */
  while ((2 << s) <= n) ++s;
#else
  while ((1 << s) < n) ++s;
#endif
  return s;
}

static int i32_cmp(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Which child of a split at s on axis a holds a point at coordinate s: the side
 * the ray moves to, or (moving parallel to the plane) the side it is shifted
 * to -- its right, normal (ky, -kx).  1 = the child with coordinates >= s. */
static int plane_side(int a, int64_t kx, int64_t ky) {
  int64_t ka = a == 0 ? kx : ky;
  if (ka != 0) return ka > 0;
  return (a == 0 ? ky : -kx) > 0;
}

static void kd_range(void* p, int64_t lo, int64_t hi) {
  kd_ctx* c = (kd_ctx*)p;
  int32_t cap = 1024, *tested = (int32_t*)malloc(sizeof(int32_t) * cap);
  int32_t* nstack = (int32_t*)malloc(sizeof(int32_t) * ((size_t)c->n_nodes + 1));
  for (int64_t i = lo; i < hi; ++i) {
    int32_t* o = c->ops + 6 * i;
    int64_t kx, ky, ox = c->ox[i], oy = c->oy[i];
    const int32_t* rb = c->box;
    if (!dir_to_int(c->dx[i], &kx) || !dir_to_int(c->dy[i], &ky) || (kx == 0 && ky == 0) || ox < rb[0] ||
        ox > rb[2] || oy < rb[1] || oy > rb[3]) {
      c->hit[i] = -1;
      c->t[i] = NAN;
      for (int q = 0; q < 6; ++q) o[q] = -1;
      continue;
    }
    /* start leaf: descend with the origin (known a priori, not counted) */
    int32_t L = 0;
    while (c->axis[L] != 2) {
      int a = c->axis[L];
      int64_t v = (a == 0 ? ox : oy) - c->split[L];
      L = c->child[L] + ((v > 0 || (v == 0 && plane_side(a, kx, ky))) ? 1 : 0);
    }
    best_hit b = {-1, {0, 1}, 0, 0};
    int32_t leaves = 0, desc = 0, tests = 0, ropes = 0, n_tested = 0;
    for (;;) {
      ++leaves;
      if (leaves > c->n_nodes + 8) {
        b.seg = -1;
        break;
      }
      const int32_t* B = c->box + 4 * (int64_t)L;
      /* exit face and parameter */
      q64 tx = kx > 0 ? (q64){B[2] - ox, kx} : (kx < 0 ? (q64){ox - B[0], -kx} : (q64){0, 0});
      q64 ty = ky > 0 ? (q64){B[3] - oy, ky} : (ky < 0 ? (q64){oy - B[1], -ky} : (q64){0, 0});
      int xface = q_cmp(ty, tx) >= 0; /* a corner exit takes the x face */
      q64 te = xface ? tx : ty;
      int face = xface ? (kx > 0 ? 1 : 0) : (ky > 0 ? 3 : 2);
      int32_t first = c->child[L], cnt = c->count[L];
      for (int32_t q = 0; q < cnt; ++q) {
        int32_t sid = c->refs[first + q];
        ++tests;
        if (n_tested == cap) {
          cap *= 2;
          tested = (int32_t*)realloc(tested, sizeof(int32_t) * cap);
        }
        tested[n_tested++] = sid;
        consider(&b, c->seg + 4 * (int64_t)sid, sid, ox, oy, kx, ky, &te);
      }
#if ORACLE_MUTANT == 8 /* planted: a rope search counted for every leaf, the last one included */
      ropes += ideal_rope_steps(kd_face_neighbours(c, L, face, nstack));
#endif
      if (b.seg >= 0) break;
      int32_t nxt = c->rope[4 * (int64_t)L + face];
      if (nxt < 0) break;
#if ORACLE_MUTANT != 8
      ropes += ideal_rope_steps(kd_face_neighbours(c, L, face, nstack));
#endif
      int fa = face / 2;
      int64_t plane = face == 0 ? B[0] : (face == 1 ? B[2] : (face == 2 ? B[1] : B[3]));
      int32_t N = nxt;
      while (c->axis[N] != 2) {
        int a = c->axis[N];
        int64_t s = c->split[N];
        int right;
        if (a == fa) {
          right = plane > s || (plane == s && plane_side(a, kx, ky));
        } else { /* exit point coordinate o_a + te * k_a compared with s */
          int64_t v = ((a == 0 ? ox : oy) - s) * te.den + te.num * (a == 0 ? kx : ky);
          right = v > 0 || (v == 0 && plane_side(a, kx, ky));
        }
        N = c->child[N] + right;
        ++desc;
      }
      L = N;
    }
    /* ideal mailbox: distinct segments tested */
    qsort(tested, (size_t)n_tested, sizeof(int32_t), i32_cmp);
    int32_t uniq = 0;
    for (int32_t q = 0; q < n_tested; ++q)
      if (q == 0 || tested[q] != tested[q - 1]) ++uniq;
    c->hit[i] = b.seg;
    c->t[i] = b.seg >= 0 ? ratio_to_t(b.t) : INFINITY;
    o[0] = leaves;
    o[1] = desc;
    o[2] = tests;
    o[3] = uniq;
    o[4] = ropes;
    o[5] = 0;
    n_tested = 0;
  }
  free(tested);
  free(nstack);
}

/* Roped kd-tree traversal (Sec. 5.3.2) from the leaf holding the origin.
 * ops per ray: leaves visited, nodes passed in rope descents, segment tests,
 * distinct segments tested (an ideal mailbox), rope search steps of an ideal
 * rope tree (sum over the faces crossed of ceil(log2 of the face's rope
 * count), the count found by kd_face_neighbours), 0. */
int oracle_kd_trace(int32_t n_nodes, const int32_t* axis, const int32_t* split, const int32_t* child,
                    const int32_t* count, const int32_t* box, const int32_t* rope, const int32_t* refs,
                    const int32_t* seg, int64_t n, const int32_t* ox, const int32_t* oy, const float* dx,
                    const float* dy, int32_t* hit, float* t, int32_t* ops, int32_t n_threads) {
  kd_ctx c = {n_nodes, axis, split, child, count, box, rope, refs, seg, ox, oy, dx, dy, hit, ops, t};
  run_parallel(kd_range, &c, n, n_threads);
  return 0;
}

/* ------------------------------------------------------------------ secondary rays */
/* Sec. 5.2: a secondary ray starts where its parent hit the geometry, and the
 * final triangle of the parent's walk is its start triangle.  The paper fixes
 * nothing else; readings used here (and by the GPU path):
 *   - the secondary ray is the mirror image of its parent about the hit
 *     segment;
 *   - its origin is the parent's exact hit point moved onto the hit
 *     constrained edge (a -> b) of the final triangle (a right of the parent
 *     ray, b left of it or on its line): P' = a + (i / 2^32) (b - a) with
 *     i = round(2^32 mu) (halves up) clamped to [1, 2^32 - 1], mu the exact
 *     parameter of the hit point on that edge.  P' lies exactly on the edge,
 *     strictly between its endpoints, so its coordinates are multiples of
 *     2^-32: origins are held as X = 2^32 x, Y = 2^32 y (int64);
 *   - its direction is k' = 2 (k.u) u / |u|^2 - k rounded componentwise to
 *     integers (halves up) and clamped to [-2^22, 2^22], u = b - a; when k'
 *     does not point strictly back to the parent's side of the segment (the
 *     sign of u x k' must be opposite to that of u x k) the path ends;
 *   - or, when the caller gives it, the direction (c, s) in the hit edge's
 *     frame: d' = c u/|u| + s n, n the unit normal of u pointing back to the
 *     parent's side, c and s on the 2^-22 grid with |c|, |s| <= 1 and s > 0
 *     (else the ray is invalid); k' = 2^22 d' rounded componentwise (halves
 *     up, an exact comparison with the square root) and clamped to 2^22, then
 *     the same test;
 *   - every ray of the path, the first included, follows the rules of the
 *     primary rays (side rule, hit, tie order), with the origin in 2^-32
 *     units.  A path of a primary ray has up to 1 + n_bounce rays; it ends at
 *     a miss, an invalid primary ray, a walk limit or a grazing reflection.
 * Records of a path: entry b * n + r for ray b of path r.  steps: as for the
 * walk; -3 = no ray (the path ended before this bounce), with hit -1, t NaN,
 * origin 0 and direction 0. */
#define BNC_NONE (-3)
static const i128 QONE = (i128)1 << 32;

/* 2^32 * (k x (v - P)) = kx (vy 2^32 - Y) - ky (vx 2^32 - X), exact (|.| < 2^76) */
static int side_q(int64_t kx, int64_t ky, int64_t X, int64_t Y, int64_t vx, int64_t vy) {
  i128 v = (i128)kx * ((i128)vy * QONE - Y) - (i128)ky * ((i128)vx * QONE - X);
  return v >= 0 ? ORC_SIDE_L : ORC_SIDE_R;
}

/* t = cross(b - a, a - P) / cross(b - a, d) = 2^22 num / (2^32 den), den > 0 */
typedef struct {
  i128 num;
  i128 den;
} qratio;

static qratio seg_param_q(int64_t kx, int64_t ky, int64_t X, int64_t Y, int64_t ax, int64_t ay, int64_t bx,
                          int64_t by) {
  qratio r;
  int64_t ex = bx - ax, ey = by - ay;
  r.num = (i128)ex * ((i128)ay * QONE - Y) - (i128)ey * ((i128)ax * QONE - X);
  r.den = (i128)ex * ky - (i128)ey * kx;
  if (r.den < 0) {
    r.num = -r.num;
    r.den = -r.den;
  }
  return r;
}

static int qratio_cmp(qratio a, qratio b) { /* |num| < 2^75, den < 2^45: products < 2^120 */
  i128 l = a.num * b.den, r = b.num * a.den;
  return (l > r) - (l < r);
}

static float qratio_to_t(qratio r) { return (float)((double)r.num / (double)r.den * 0x1p-10); }

static i128 floordiv(i128 n, i128 d) { /* d > 0 */
  i128 q = n / d;
  if (n % d != 0 && n < 0) q -= 1;
  return q;
}

/* The origin of the secondary ray on the hit edge (a -> b). */
static void snap_origin(int64_t kx, int64_t ky, int64_t X, int64_t Y, int64_t ax, int64_t ay, int64_t bx,
                        int64_t by, int64_t* X2, int64_t* Y2) {
  int64_t ex = bx - ax, ey = by - ay;
  /* mu = cross(k, P - a) / cross(k, b - a); 2^32 mu = num / den */
  i128 num = (i128)kx * ((i128)Y - (i128)ay * QONE) - (i128)ky * ((i128)X - (i128)ax * QONE);
  i128 den = (i128)kx * ey - (i128)ky * ex;
  if (den < 0) {
    num = -num;
    den = -den;
  }
  i128 i = floordiv(2 * num + den, 2 * den);
  if (i < 1) i = 1;
  if (i > QONE - 1) i = QONE - 1;
#if ORACLE_MUTANT == 6 /* planted: measures the parameter from the wrong endpoint */
  *X2 = (int64_t)((i128)bx * QONE - i * ex);
  *Y2 = (int64_t)((i128)by * QONE - i * ey);
#else
  *X2 = (int64_t)((i128)ax * QONE + i * ex);
  *Y2 = (int64_t)((i128)ay * QONE + i * ey);
#endif
}

/* Mirror direction about u; returns 0 when it does not point strictly back. */
static int reflect_dir(int64_t kx, int64_t ky, int64_t ux, int64_t uy, int64_t* rx, int64_t* ry) {
  const i128 ku = (i128)kx * ux + (i128)ky * uy, uu = (i128)ux * ux + (i128)uy * uy;
#if ORACLE_MUTANT == 5 /* planted: adds the incoming direction instead of subtracting it */
  const i128 nx = 2 * ku * ux + uu * kx, ny = 2 * ku * uy + uu * ky;
#else
  const i128 nx = 2 * ku * ux - uu * kx, ny = 2 * ku * uy - uu * ky;
#endif
  i128 qx = floordiv(2 * nx + uu, 2 * uu), qy = floordiv(2 * ny + uu, 2 * uu);
  const i128 lim = (i128)1 << 22;
  if (qx > lim) qx = lim;
  if (qx < -lim) qx = -lim;
  if (qy > lim) qy = lim;
  if (qy < -lim) qy = -lim;
  *rx = (int64_t)qx;
  *ry = (int64_t)qy;
  const i128 c0 = (i128)ux * ky - (i128)uy * kx, c1 = (i128)ux * qy - (i128)uy * qx;
  return (c0 > 0 && c1 < 0) || (c0 < 0 && c1 > 0);
}

/* is a < b sqrt(m), exactly (m >= 0; |a| < 2^62, |b| sqrt(m) < 2^62) */
static int lt_sqrt(i128 a, i128 b, i128 m) {
  if (b >= 0) return a < 0 || a * a < b * b * m;
  return a < 0 && a * a > b * b * m;
}

/* round(n / sqrt(m)) with halves up: the q with (2q - 1) sqrt(m) <= 2n < (2q + 1) sqrt(m) */
static int64_t round_div_sqrt(int64_t n, int64_t m) {
  int64_t q = (int64_t)floor((double)n / sqrt((double)m) + 0.5);
  while (!lt_sqrt(2 * (i128)n, 2 * (i128)q + 1, m)) ++q;
  while (lt_sqrt(2 * (i128)n, 2 * (i128)q - 1, m)) --q;
  return q;
}

/* The direction (c, s) in the frame of the hit edge u = b - a (a right of the
 * parent ray k, b left): k' = round(2^22 (c u + s n) / |u|) with n = (-u_y, u_x),
 * the normal on the parent's side.  Returns -1 if (c, s) is not a valid frame
 * direction, 0 if k' does not point strictly back, 1 otherwise. */
static int frame_dir(float c, float s, int64_t kx, int64_t ky, int64_t ux, int64_t uy, int64_t* rx, int64_t* ry) {
  int64_t kc, ks;
  if (!dir_to_int(c, &kc) || !dir_to_int(s, &ks) || ks <= 0) return -1;
  const int64_t m = ux * ux + uy * uy;
#if ORACLE_MUTANT == 7 /* planted: the normal on the far side */
  int64_t qx = round_div_sqrt(kc * ux + ks * uy, m), qy = round_div_sqrt(kc * uy - ks * ux, m);
#else
  int64_t qx = round_div_sqrt(kc * ux - ks * uy, m), qy = round_div_sqrt(kc * uy + ks * ux, m);
#endif
  const int64_t lim = (int64_t)1 << 22;
  qx = qx > lim ? lim : (qx < -lim ? -lim : qx);
  qy = qy > lim ? lim : (qy < -lim ? -lim : qy);
  *rx = qx;
  *ry = qy;
  const i128 c0 = (i128)ux * ky - (i128)uy * kx, c1 = (i128)ux * qy - (i128)uy * qx;
  return (c0 > 0 && c1 < 0) || (c0 < 0 && c1 > 0);
}

typedef struct {
  int64_t n_tri, n_seg;
  const int32_t *vx, *vy, *tri_v, *tri_nb, *tri_seg, *seg;
  int64_t n;
  const int32_t *ox, *oy;
  const float *dx, *dy;
  const int32_t* start;
  int32_t n_bounce;
  int32_t *hit, *steps;
  float* t;
  int64_t *org_x, *org_y;
  float *dir_x, *dir_y;
  int64_t max_steps;
  const float* frame; /* optional: (c, s) of ray b >= 1 of path r at 2 ((b - 1) n + r) */
} bounce_ctx;

/* The next ray's direction after ray b of path r hit edge (a -> b) (u): 1 = go on,
 * 0 = the path ends, -1 = ray b + 1 is invalid (a caller's frame direction). */
static int next_dir(const bounce_ctx* c, int b, int64_t r, int64_t kx, int64_t ky, int64_t ux, int64_t uy,
                    int64_t* rx, int64_t* ry) {
  if (!c->frame) return reflect_dir(kx, ky, ux, uy, rx, ry);
  const int64_t k = 2 * ((int64_t)b * c->n + r);
  return frame_dir(c->frame[k], c->frame[k + 1], kx, ky, ux, uy, rx, ry);
}

static void bounce_clear(const bounce_ctx* c, int64_t r) {
  for (int b = 0; b <= c->n_bounce; ++b) {
    int64_t k = (int64_t)b * c->n + r;
    c->hit[k] = -1;
    c->t[k] = NAN;
    if (c->steps) c->steps[k] = BNC_NONE;
    c->org_x[k] = c->org_y[k] = 0;
    c->dir_x[k] = c->dir_y[k] = 0.0f;
  }
}

static void bounce_origin(const bounce_ctx* c, int64_t k, int64_t X, int64_t Y, int64_t kx, int64_t ky) {
  c->org_x[k] = X;
  c->org_y[k] = Y;
  c->dir_x[k] = (float)kx * 0x1p-22f;
  c->dir_y[k] = (float)ky * 0x1p-22f;
}

/* Whether the primary ray r is valid: direction on the grid and non-zero,
 * origin inside the domain's range; its k. */
static int bounce_primary(const bounce_ctx* c, int64_t r, int64_t* kx, int64_t* ky) {
  return dir_to_int(c->dx[r], kx) && dir_to_int(c->dy[r], ky) && (*kx != 0 || *ky != 0) && c->ox[r] >= 0 &&
         c->oy[r] >= 0;
}

/* The walk path: every ray of the path walks from the final triangle of the
 * previous one (Sec. 5.1 in each triangle, the start cell of Sec. 5.2). */
static void bounce_walk_range(void* p, int64_t lo, int64_t hi) {
  const bounce_ctx* c = (const bounce_ctx*)p;
  walk_ctx w; /* only for strictly_inside */
  memset(&w, 0, sizeof w);
  w.vx = c->vx;
  w.vy = c->vy;
  w.tri_v = c->tri_v;
  for (int64_t r = lo; r < hi; ++r) {
    bounce_clear(c, r);
    int64_t kx, ky;
    int64_t T = c->start[r];
    if (!bounce_primary(c, r, &kx, &ky) || T < 0 || T >= c->n_tri || !strictly_inside(&w, T, c->ox[r], c->oy[r])) {
      c->steps[r] = -1;
      continue;
    }
    int64_t X = (int64_t)c->ox[r] << 32, Y = (int64_t)c->oy[r] << 32;
    for (int b = 0; b <= c->n_bounce; ++b) {
      const int64_t k = (int64_t)b * c->n + r;
      bounce_origin(c, k, X, Y, kx, ky);
      int64_t steps = 0;
      int more = 0;
      for (;;) {
        ++steps;
        if (steps > c->max_steps) {
          c->steps[k] = -2;
          break;
        }
        int e = -1;
        for (int i = 0; i < 3; ++i) {
          int32_t a = c->tri_v[3 * T + (i + 1) % 3], bb = c->tri_v[3 * T + (i + 2) % 3];
          if (side_q(kx, ky, X, Y, c->vx[a], c->vy[a]) == ORC_SIDE_R &&
              side_q(kx, ky, X, Y, c->vx[bb], c->vy[bb]) == ORC_SIDE_L) {
            e = i;
            break;
          }
        }
        if (e < 0) { /* cannot happen: the origin is inside T or on its entry edge */
          c->steps[k] = -1;
          break;
        }
        const int32_t seg = c->tri_seg[3 * T + e], nb = c->tri_nb[3 * T + e];
        if (seg >= 0) {
          const int32_t a = c->tri_v[3 * T + (e + 1) % 3], bb = c->tri_v[3 * T + (e + 2) % 3];
          const int64_t ax = c->vx[a], ay = c->vy[a], bx = c->vx[bb], by = c->vy[bb];
          c->hit[k] = seg;
          c->t[k] = qratio_to_t(seg_param_q(kx, ky, X, Y, ax, ay, bx, by));
          c->steps[k] = (int32_t)steps;
          if (b < c->n_bounce) {
            int64_t X2, Y2, kx2, ky2;
            snap_origin(kx, ky, X, Y, ax, ay, bx, by, &X2, &Y2);
            const int nd = next_dir(c, b, r, kx, ky, bx - ax, by - ay, &kx2, &ky2);
            if (nd > 0) {
              X = X2;
              Y = Y2;
              kx = kx2;
              ky = ky2;
              more = 1; /* T stays: the next ray starts in the final triangle */
            } else if (nd < 0) {
              c->steps[(int64_t)(b + 1) * c->n + r] = -1; /* invalid frame direction */
            }
          }
          break;
        }
        if (nb < 0) {
          c->t[k] = INFINITY;
          c->steps[k] = (int32_t)steps;
          break;
        }
        T = nb;
      }
      if (!more) break;
    }
  }
}

/* Closest segment of the ray (P, k), P in 2^-32 units; -1 for none.  As
 * closest_segment, with the exact arithmetic widened. */
static int32_t closest_segment_q(const int32_t* seg, int64_t n_seg, int64_t X, int64_t Y, int64_t kx, int64_t ky,
                                 qratio* best_t) {
  int32_t best = -1;
  qratio bt = {0, 1};
  int64_t bux = 0, buy = 0;
  for (int64_t s = 0; s < n_seg; ++s) {
    int64_t ax = seg[4 * s], ay = seg[4 * s + 1], bx = seg[4 * s + 2], by = seg[4 * s + 3];
    int sa = side_q(kx, ky, X, Y, ax, ay), sb = side_q(kx, ky, X, Y, bx, by);
    if (sa == sb) continue;
    qratio r = seg_param_q(kx, ky, X, Y, ax, ay, bx, by);
    if (r.num <= 0) continue;
    int64_t wx = sa == ORC_SIDE_R ? ax : bx, wy = sa == ORC_SIDE_R ? ay : by;
    int c = best < 0 ? -1 : qratio_cmp(r, bt);
    if (c == 0) {
      int64_t pvx = (wx == ax && wy == ay) ? bx : ax, pvy = (wx == ax && wy == ay) ? by : ay;
      c = tie_cmp(kx, ky, wx - pvx, wy - pvy, bux - pvx, buy - pvy);
    }
    if (c < 0) {
      best = (int32_t)s;
      bt = r;
      bux = wx;
      buy = wy;
    }
  }
  *best_t = bt;
  return best;
}

/* The same paths by brute force: each ray's closest hit over all segments,
 * the hit constrained edge found by scanning every edge labelled with the hit
 * segment (the one whose endpoints lie on opposite sides of the ray). */
static void bounce_bf_range(void* p, int64_t lo, int64_t hi) {
  const bounce_ctx* c = (const bounce_ctx*)p;
  for (int64_t r = lo; r < hi; ++r) {
    bounce_clear(c, r);
    int64_t kx, ky;
    if (!bounce_primary(c, r, &kx, &ky)) continue;
    int64_t X = (int64_t)c->ox[r] << 32, Y = (int64_t)c->oy[r] << 32;
    for (int b = 0; b <= c->n_bounce; ++b) {
      const int64_t k = (int64_t)b * c->n + r;
      bounce_origin(c, k, X, Y, kx, ky);
      qratio bt;
      const int32_t s = closest_segment_q(c->seg, c->n_seg, X, Y, kx, ky, &bt);
      if (s < 0) {
        c->t[k] = INFINITY;
        break;
      }
      c->hit[k] = s;
      c->t[k] = qratio_to_t(bt);
      if (b == c->n_bounce) break;
      int64_t ax = 0, ay = 0, bx = 0, by = 0;
      int found = 0;
      for (int64_t q = 0; q < 3 * c->n_tri && !found; ++q) {
        if (c->tri_seg[q] != s) continue;
        const int64_t T = q / 3, i = q % 3;
        const int32_t u = c->tri_v[3 * T + (i + 1) % 3], v = c->tri_v[3 * T + (i + 2) % 3];
        const int su = side_q(kx, ky, X, Y, c->vx[u], c->vy[u]), sv = side_q(kx, ky, X, Y, c->vx[v], c->vy[v]);
        if (su == sv) continue;
        const int32_t ra = su == ORC_SIDE_R ? u : v, lb = su == ORC_SIDE_R ? v : u;
        ax = c->vx[ra];
        ay = c->vy[ra];
        bx = c->vx[lb];
        by = c->vy[lb];
        found = 1;
      }
      if (!found) break; /* cannot happen for a triangulation that covers the segments */
      int64_t X2, Y2, kx2, ky2;
      snap_origin(kx, ky, X, Y, ax, ay, bx, by, &X2, &Y2);
      if (next_dir(c, b, r, kx, ky, bx - ax, by - ay, &kx2, &ky2) <= 0) break;
      X = X2;
      Y = Y2;
      kx = kx2;
      ky = ky2;
    }
  }
}

/* Mirror paths of n primary rays with up to n_bounce secondary rays each, by
 * walks chained through their final triangles.  Outputs (1 + n_bounce) * n
 * entries, entry b * n + r: hit, t, steps as oracle_walk plus -3 (no ray),
 * origin (2^-32 units) and direction of each ray of the path.  frame
 * (optional): the caller's directions in the hit edges' frames instead of
 * mirror images; an invalid one gives steps -1 at its ray. */
int oracle_bounce_walk(int64_t n_tri, const int32_t* vx, const int32_t* vy, const int32_t* tri_v,
                       const int32_t* tri_nb, const int32_t* tri_seg, int64_t n, const int32_t* ox,
                       const int32_t* oy, const float* dx, const float* dy, const int32_t* start, int32_t n_bounce,
                       int32_t* hit, float* t, int32_t* steps, int64_t* org_x, int64_t* org_y, float* dir_x,
                       float* dir_y, int64_t max_steps, const float* frame, int32_t n_threads) {
  bounce_ctx c = {n_tri, 0, vx, vy, tri_v, tri_nb, tri_seg, NULL, n, ox, oy, dx, dy, start, n_bounce,
                  hit, steps, t, org_x, org_y, dir_x, dir_y, max_steps, frame};
  run_parallel(bounce_walk_range, &c, n, n_threads);
  return 0;
}

/* The same paths by brute force over the segments (no steps). */
int oracle_bounce_bruteforce(int64_t n_tri, const int32_t* vx, const int32_t* vy, const int32_t* tri_v,
                             const int32_t* tri_seg, int64_t n_seg, const int32_t* seg, int64_t n,
                             const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                             int32_t n_bounce, int32_t* hit, float* t, int64_t* org_x, int64_t* org_y,
                             float* dir_x, float* dir_y, const float* frame, int32_t n_threads) {
  bounce_ctx c = {n_tri, n_seg, vx, vy, tri_v, NULL, tri_seg, seg, n, ox, oy, dx, dy, NULL, n_bounce,
                  hit, NULL, t, org_x, org_y, dir_x, dir_y, 0, frame};
  run_parallel(bounce_bf_range, &c, n, n_threads);
  return 0;
}

int32_t oracle_mutant(void) { return ORACLE_MUTANT; }
