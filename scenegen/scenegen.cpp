// Seeded inputs for the constrained-triangulation ray walk: scene segments on the
// integer grid, the constrained Delaunay triangulation (CDT) that contains them,
// a flip-based annealer that lowers its total edge length, and ray batches with
// their start triangles.
//
// This module is the offline CPU prerequisite of the method (Sec. 3.5: an initial
// CDT, Sec. 3.2.7 / 3.3: annealing with edge flips).  It is the ONE module that
// both the CUDA path and the CPU oracle consume, and it contains none of the
// ray-walk / closest-hit arithmetic (Sec. 5.1): it only produces inputs.
//
// Conventions (the domain): vertices are integer points of [0, D]^2 with
// D = 2^20; the four corners of that square are vertices and its boundary is the
// hull of every triangulation.  Triangles are CCW; edge i of a triangle is the
// edge opposite its vertex i.  Neighbour -1 = hull.  tri_seg[3t+i] = scene
// segment id carried by edge i (a constrained edge) or -1.
//
// Exactness: all geometric predicates here are exact (int64 orientation,
// int128 in-circle), so the CDT is built without tolerances.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <climits>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

typedef __int128 i128;

struct Pt {
  int32_t x, y;
};
static inline bool operator==(const Pt& a, const Pt& b) { return a.x == b.x && a.y == b.y; }

// ---------------------------------------------------------------- random numbers
// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014).  One counter-based stream per (seed, stream id).
struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed, uint64_t stream = 0) {
    s = seed;
    uint64_t t = stream * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull;
    s ^= mix(t);
    (void)next();
  }
  static uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  uint64_t next() { return mix(s += 0x9E3779B97F4A7C15ull); }
  double uni() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)
  uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
  double normal() {  // Box-Muller
    double u1 = uni(), u2 = uni();
    if (u1 < 1e-300) u1 = 1e-300;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

// ---------------------------------------------------------------- exact predicates
static inline int64_t orient(const Pt& a, const Pt& b, const Pt& c) {
  return (int64_t)(b.x - a.x) * (int64_t)(c.y - a.y) - (int64_t)(b.y - a.y) * (int64_t)(c.x - a.x);
}
static inline int sgn(int64_t v) { return (v > 0) - (v < 0); }
static inline int sgn128(i128 v) { return (v > 0) - (v < 0); }

// > 0 iff d lies strictly inside the circumcircle of the CCW triangle (a, b, c).
static inline int incircle(const Pt& a, const Pt& b, const Pt& c, const Pt& d) {
  int64_t adx = a.x - d.x, ady = a.y - d.y;
  int64_t bdx = b.x - d.x, bdy = b.y - d.y;
  int64_t cdx = c.x - d.x, cdy = c.y - d.y;
  i128 al = (i128)adx * adx + (i128)ady * ady;
  i128 bl = (i128)bdx * bdx + (i128)bdy * bdy;
  i128 cl = (i128)cdx * cdx + (i128)cdy * cdy;
  i128 det = al * ((i128)bdx * cdy - (i128)bdy * cdx) + bl * ((i128)cdx * ady - (i128)cdy * adx) +
             cl * ((i128)adx * bdy - (i128)ady * bdx);
  return sgn128(det);
}

static inline bool on_closed_box(const Pt& a, const Pt& b, const Pt& p) {
  return std::min(a.x, b.x) <= p.x && p.x <= std::max(a.x, b.x) && std::min(a.y, b.y) <= p.y &&
         p.y <= std::max(a.y, b.y);
}

// Closed segments [a,b] and [c,d] share at least one point.
static bool seg_touch(const Pt& a, const Pt& b, const Pt& c, const Pt& d) {
  int o1 = sgn(orient(a, b, c)), o2 = sgn(orient(a, b, d));
  int o3 = sgn(orient(c, d, a)), o4 = sgn(orient(c, d, b));
  if (o1 * o2 < 0 && o3 * o4 < 0) return true;
  if (o1 == 0 && on_closed_box(a, b, c)) return true;
  if (o2 == 0 && on_closed_box(a, b, d)) return true;
  if (o3 == 0 && on_closed_box(c, d, a)) return true;
  if (o4 == 0 && on_closed_box(c, d, b)) return true;
  return false;
}

static inline int64_t len2(const Pt& a, const Pt& b) {
  int64_t dx = a.x - b.x, dy = a.y - b.y;
  return dx * dx + dy * dy;
}

// ---------------------------------------------------------------- segment soup with a hash grid
struct SegGrid {
  int32_t D;
  int G;
  double cell;
  std::vector<std::vector<int32_t>> cells;
  std::vector<Pt> A, B;
  SegGrid(int32_t D_, double cell_size) : D(D_) {
    G = (int)std::ceil((double)D / cell_size);
    G = std::max(1, std::min(G, 4096));
    cell = (double)D / G + 1e-9;
    cells.assign((size_t)G * G, {});
  }
  void range(const Pt& a, const Pt& b, int& i0, int& i1, int& j0, int& j1) const {
    i0 = std::clamp((int)(std::min(a.x, b.x) / cell), 0, G - 1);
    i1 = std::clamp((int)(std::max(a.x, b.x) / cell), 0, G - 1);
    j0 = std::clamp((int)(std::min(a.y, b.y) / cell), 0, G - 1);
    j1 = std::clamp((int)(std::max(a.y, b.y) / cell), 0, G - 1);
  }
  // true if the closed segment [a,b] shares a point with any stored segment
  bool touches(const Pt& a, const Pt& b) const {
    int i0, i1, j0, j1;
    range(a, b, i0, i1, j0, j1);
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i)
        for (int32_t s : cells[(size_t)j * G + i])
          if (seg_touch(a, b, A[s], B[s])) return true;
    return false;
  }
  void add(const Pt& a, const Pt& b) {
    int id = (int)A.size();
    A.push_back(a);
    B.push_back(b);
    int i0, i1, j0, j1;
    range(a, b, i0, i1, j0, j1);
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) cells[(size_t)j * G + i].push_back(id);
  }
};

static inline int32_t rnd_coord(double v) { return (int32_t)std::llround(v); }

// Random, pairwise disjoint segments (no shared points), lengths uniform in
// [len_lo, len_hi] * D * scale, centres uniform (or from Gaussian clusters),
// endpoints at least `margin`*D from the border.
static int64_t gen_segments(int64_t n, uint64_t seed, int32_t D, double len_lo, double len_hi, double scale,
                            double margin, int n_clusters, double sigma, int32_t* out, int64_t cap) {
  Rng rng(seed, 0x5E6);
  double lmax = len_hi * D * scale;
  SegGrid grid(D, std::max(lmax, (double)D / 4096.0));
  double lo = margin * D, hi = (1.0 - margin) * D;
  std::vector<double> ccx, ccy;
  for (int c = 0; c < n_clusters; ++c) {
    ccx.push_back((0.1 + 0.8 * rng.uni()) * D);
    ccy.push_back((0.1 + 0.8 * rng.uni()) * D);
  }
  int64_t cnt = 0, tries = 0, max_tries = std::max<int64_t>(1000 * n, 100000);
  while (cnt < n && cnt < cap && tries < max_tries) {
    ++tries;
    double cx, cy;
    if (n_clusters > 0) {
      int c = (int)rng.below((uint32_t)n_clusters);
      cx = ccx[c] + sigma * D * rng.normal();
      cy = ccy[c] + sigma * D * rng.normal();
    } else {
      cx = lo + (hi - lo) * rng.uni();
      cy = lo + (hi - lo) * rng.uni();
    }
    double L = D * scale * (len_lo + (len_hi - len_lo) * rng.uni());
    double th = 6.283185307179586 * rng.uni();
    double hx = 0.5 * L * std::cos(th), hy = 0.5 * L * std::sin(th);
    Pt a{rnd_coord(cx - hx), rnd_coord(cy - hy)}, b{rnd_coord(cx + hx), rnd_coord(cy + hy)};
    if (a == b) continue;
    if (a.x < lo || a.x > hi || a.y < lo || a.y > hi || b.x < lo || b.x > hi || b.y < lo || b.y > hi) continue;
    if (grid.touches(a, b)) continue;
    grid.add(a, b);
    out[4 * cnt + 0] = a.x;
    out[4 * cnt + 1] = a.y;
    out[4 * cnt + 2] = b.x;
    out[4 * cnt + 3] = b.y;
    ++cnt;
  }
  return cnt;
}

// Closed regular polygon with m sides around (cx, cy), radius r, phase phi,
// vertices rounded to the grid.  Returns false if rounding collapsed a side.
static bool polygon(double cx, double cy, double r, int m, double phi, std::vector<Pt>& v) {
  v.clear();
  for (int k = 0; k < m; ++k) {
    double a = phi + 6.283185307179586 * k / m;
    v.push_back(Pt{rnd_coord(cx + r * std::cos(a)), rnd_coord(cy + r * std::sin(a))});
  }
  for (int k = 0; k < m; ++k)
    if (v[k] == v[(k + 1) % m]) return false;
  // reject a fold-back from rounding: consecutive sides must not turn by more
  // than 90 degrees (slight clockwise turns from rounding are harmless)
  for (int k = 0; k < m; ++k) {
    const Pt &a = v[k], &b = v[(k + 1) % m], &c = v[(k + 2) % m];
    int64_t dot = (int64_t)(b.x - a.x) * (c.x - b.x) + (int64_t)(b.y - a.y) * (c.y - b.y);
    if (dot <= 0) return false;
  }
  return true;
}

static int64_t emit_polygon(const std::vector<Pt>& v, int32_t* out, int64_t cnt, int64_t cap) {
  int m = (int)v.size();
  for (int k = 0; k < m && cnt < cap; ++k) {
    out[4 * cnt + 0] = v[k].x;
    out[4 * cnt + 1] = v[k].y;
    out[4 * cnt + 2] = v[(k + 1) % m].x;
    out[4 * cnt + 3] = v[(k + 1) % m].y;
    ++cnt;
  }
  return cnt;
}

// ---------------------------------------------------------------- triangulation
struct Tri {
  int32_t v[3];
  int32_t n[3];
  int32_t c[3];
};

struct Triangulation {
  int32_t D = 0;
  std::vector<Pt> P;
  std::vector<Tri> T;
  std::vector<int32_t> vtri;
  int32_t last = 0;
  Rng rng{12345, 7};
  int status = 0;  // 0 ok, <0 error

  static int idx_of(const Tri& t, int v) { return t.v[0] == v ? 0 : (t.v[1] == v ? 1 : (t.v[2] == v ? 2 : -1)); }
  int nb_edge(int u, int t) const {
    const Tri& x = T[u];
    return x.n[0] == t ? 0 : (x.n[1] == t ? 1 : (x.n[2] == t ? 2 : -1));
  }
  void replace_nb(int x, int old_t, int new_t) {
    if (x < 0) return;
    for (int k = 0; k < 3; ++k)
      if (T[x].n[k] == old_t) {
        T[x].n[k] = new_t;
        return;
      }
  }

  void init_square(int32_t D_) {
    D = D_;
    P = {{0, 0}, {D, 0}, {D, D}, {0, D}};
    vtri = {0, 0, 0, 1};
    T.clear();
    T.push_back(Tri{{0, 1, 2}, {-1, 1, -1}, {-1, -1, -1}});
    T.push_back(Tri{{0, 2, 3}, {-1, -1, 0}, {-1, -1, -1}});
    last = 0;
  }

  // Visibility walk with a random first edge (Devillers, Pion & Teillaud,
  // "Walking in a triangulation", 2002); terminates with probability one.
  int locate(const Pt& p, int start, Rng& r) const {
    int t = start;
    for (int64_t guard = 0; guard < 50000000; ++guard) {
      const Tri& tr = T[t];
      int s = (int)r.below(3);
      bool moved = false;
      for (int k = 0; k < 3; ++k) {
        int i = (s + k) % 3;
        if (orient(P[tr.v[(i + 1) % 3]], P[tr.v[(i + 2) % 3]], p) < 0) {
          if (tr.n[i] < 0) return -1;
          t = tr.n[i];
          moved = true;
          break;
        }
      }
      if (!moved) return t;
    }
    return -1;
  }

  void legalize(std::vector<std::pair<int, int>>& st) {
    while (!st.empty()) {
      auto [t, i] = st.back();
      st.pop_back();
      int u = T[t].n[i];
      if (u < 0 || T[t].c[i] >= 0) continue;
      int j = nb_edge(u, t);
      int s = T[u].v[j];
      if (incircle(P[T[t].v[0]], P[T[t].v[1]], P[T[t].v[2]], P[s]) > 0) {
        flip(t, i);
        st.push_back({t, 0});
        st.push_back({u, 0});
      }
    }
  }

  // Flip the edge i of t.  Before: t = (p, q, r), u = (s, r, q) across edge i.
  // After: t = (p, q, s), u = (p, s, r).
  void flip(int t, int i) {
    Tri ot = T[t];
    int p = ot.v[i], q = ot.v[(i + 1) % 3], r = ot.v[(i + 2) % 3];
    int u = ot.n[i];
    Tri ou = T[u];
    int j = nb_edge(u, t);
    int s = ou.v[j];
    int nA = ot.n[(i + 1) % 3], nB = ot.n[(i + 2) % 3];
    int cA = ot.c[(i + 1) % 3], cB = ot.c[(i + 2) % 3];
    int nC = ou.n[(j + 1) % 3], nD = ou.n[(j + 2) % 3];
    int cC = ou.c[(j + 1) % 3], cD = ou.c[(j + 2) % 3];
    T[t] = Tri{{p, q, s}, {nC, u, nB}, {cC, -1, cB}};
    T[u] = Tri{{p, s, r}, {nD, nA, t}, {cD, cA, -1}};
    replace_nb(nA, t, u);
    replace_nb(nC, u, t);
    vtri[p] = t;
    vtri[q] = t;
    vtri[s] = t;
    vtri[r] = u;
  }

  void split_tri(int t, int pi, std::vector<std::pair<int, int>>& st) {
    Tri o = T[t];
    int a = o.v[0], b = o.v[1], c = o.v[2];
    int t1 = (int)T.size(), t2 = t1 + 1;
    T.resize(T.size() + 2);
    T[t] = Tri{{pi, b, c}, {o.n[0], t1, t2}, {o.c[0], -1, -1}};
    T[t1] = Tri{{pi, c, a}, {o.n[1], t2, t}, {o.c[1], -1, -1}};
    T[t2] = Tri{{pi, a, b}, {o.n[2], t, t1}, {o.c[2], -1, -1}};
    replace_nb(o.n[1], t, t1);
    replace_nb(o.n[2], t, t2);
    vtri[pi] = t;
    vtri[b] = t;
    vtri[c] = t;
    vtri[a] = t1;
    st.push_back({t, 0});
    st.push_back({t1, 0});
    st.push_back({t2, 0});
    last = t;
  }

  // p lies on edge i of t (between q and r, apex a); split both sides.
  void split_edge(int t, int i, int pi, std::vector<std::pair<int, int>>& st) {
    Tri ot = T[t];
    int a = ot.v[i], q = ot.v[(i + 1) % 3], r = ot.v[(i + 2) % 3];
    int nq = ot.n[(i + 1) % 3], nr = ot.n[(i + 2) % 3];
    int cs = ot.c[i], cq = ot.c[(i + 1) % 3], cr = ot.c[(i + 2) % 3];
    int u = ot.n[i];
    int t2 = (int)T.size();
    T.push_back(Tri{});
    int u2 = -1;
    if (u >= 0) {
      u2 = (int)T.size();
      T.push_back(Tri{});
    }
    T[t] = Tri{{a, q, pi}, {u2, t2, nr}, {cs, -1, cr}};
    T[t2] = Tri{{a, pi, r}, {u, nq, t}, {cs, cq, -1}};
    replace_nb(nq, t, t2);
    vtri[a] = t;
    vtri[q] = t;
    vtri[pi] = t;
    vtri[r] = t2;
    st.push_back({t, 2});
    st.push_back({t2, 1});
    if (u >= 0) {
      Tri ou = T[u];
      int j = nb_edge(u, t);
      int s = ou.v[j];
      int nur = ou.n[(j + 1) % 3], nuq = ou.n[(j + 2) % 3];
      int cur = ou.c[(j + 1) % 3], cuq = ou.c[(j + 2) % 3];
      T[u] = Tri{{s, r, pi}, {t2, u2, nuq}, {cs, -1, cuq}};
      T[u2] = Tri{{s, pi, q}, {t, nur, u}, {cs, cur, -1}};
      replace_nb(nur, u, u2);
      vtri[s] = u;
      st.push_back({u, 2});
      st.push_back({u2, 1});
    }
    last = t;
  }

  // Insert a point; returns its vertex index (existing index for a duplicate).
  int insert_point(const Pt& p) {
    int t = locate(p, last, rng);
    if (t < 0) {
      status = -2;
      return -1;
    }
    const Tri& tr = T[t];
    int64_t o[3];
    int zeros = 0, zi = -1;
    for (int i = 0; i < 3; ++i) {
      o[i] = orient(P[tr.v[(i + 1) % 3]], P[tr.v[(i + 2) % 3]], p);
      if (o[i] == 0) {
        ++zeros;
        zi = i;
      }
    }
    if (zeros >= 2) {
      for (int k = 0; k < 3; ++k)
        if (P[tr.v[k]] == p) return tr.v[k];
      status = -3;
      return -1;
    }
    int pi = (int)P.size();
    P.push_back(p);
    vtri.push_back(t);
    std::vector<std::pair<int, int>> st;
    if (zeros == 1)
      split_edge(t, zi, pi, st);
    else
      split_tri(t, pi, st);
    legalize(st);
    last = vtri[pi];
    return pi;
  }

  template <class F>
  bool for_fan(int a, F f) const {
    int t0 = vtri[a], t = t0;
    do {
      int k = idx_of(T[t], a);
      if (f(t, k)) return true;
      t = T[t].n[(k + 1) % 3];
    } while (t != t0 && t >= 0);
    if (t < 0) {
      int k0 = idx_of(T[t0], a);
      t = T[t0].n[(k0 + 2) % 3];
      while (t >= 0) {
        int k = idx_of(T[t], a);
        if (f(t, k)) return true;
        t = T[t].n[(k + 2) % 3];
      }
    }
    return false;
  }

  // Edge (a,b): triangle t and its edge index i (edge opposite the third vertex).
  bool find_edge(int a, int b, int& to, int& io) const {
    return for_fan(a, [&](int t, int k) {
      const Tri& x = T[t];
      if (x.v[(k + 1) % 3] == b) {
        to = t;
        io = (k + 2) % 3;
        return true;
      }
      if (x.v[(k + 2) % 3] == b) {
        to = t;
        io = (k + 1) % 3;
        return true;
      }
      return false;
    });
  }

  void mark(int t, int i, int seg) {
    T[t].c[i] = seg;
    int u = T[t].n[i];
    if (u >= 0) T[u].c[nb_edge(u, t)] = seg;
  }

  bool strictly_convex(int t, int i, int& x, int& y) const {
    int u = T[t].n[i];
    if (u < 0) return false;
    x = T[t].v[i];
    y = T[u].v[nb_edge(u, t)];
    int q = T[t].v[(i + 1) % 3], r = T[t].v[(i + 2) % 3];
    return sgn(orient(P[x], P[y], P[q])) * sgn(orient(P[x], P[y], P[r])) < 0;
  }

  // Sloan's edge-flip constraint insertion (Sloan, "A fast algorithm for
  // generating constrained Delaunay triangulations", 1993).
  void insert_segment(int a0, int b0, int seg) {
    std::vector<std::pair<int, int>> work{{a0, b0}};
    int guard = 0;
    while (!work.empty()) {
      if (++guard > 1000000) {
        status = -4;
        return;
      }
      auto [a, b] = work.back();
      work.pop_back();
      int t, i;
      if (a == b) continue;
      if (find_edge(a, b, t, i)) {
        if (T[t].c[i] >= 0 && T[t].c[i] != seg) status = -5;  // overlapping segments
        mark(t, i, seg);
        continue;
      }
      const Pt A = P[a], B = P[b];
      // first triangle of the fan of a that the segment enters
      int ft = -1, fe = -1, onv = -1;
      for_fan(a, [&](int tt, int k) {
        int u = T[tt].v[(k + 1) % 3], w = T[tt].v[(k + 2) % 3];
        int64_t ou = orient(A, B, P[u]), ow = orient(A, B, P[w]);
        for (int z : {u, w}) {
          int64_t oz = (z == u) ? ou : ow;
          if (oz == 0 && z >= 0) {
            int64_t dot = (int64_t)(P[z].x - A.x) * (B.x - A.x) + (int64_t)(P[z].y - A.y) * (B.y - A.y);
            if (dot > 0 && len2(A, P[z]) < len2(A, B)) {
              onv = z;
              return true;
            }
          }
        }
        if (ou < 0 && ow > 0) {
          ft = tt;
          fe = k;
          return true;
        }
        return false;
      });
      if (onv >= 0) {
        work.push_back({onv, b});
        work.push_back({a, onv});
        continue;
      }
      if (ft < 0) {
        status = -6;
        return;
      }
      // walk across the triangles pierced by (a,b), collecting crossed edges
      std::vector<std::pair<int, int>> cross;
      int t_cur = ft, e = fe;
      int u = T[ft].v[(fe + 1) % 3], w = T[ft].v[(fe + 2) % 3];
      bool split = false;
      while (true) {
        if (T[t_cur].c[e] >= 0) {
          status = -7;  // crossing constraints
          return;
        }
        cross.push_back({u, w});
        int nt = T[t_cur].n[e];
        if (nt < 0) {
          status = -8;
          return;
        }
        int j = nb_edge(nt, t_cur);
        int z = T[nt].v[j];
        if (z == b) break;
        int64_t oz = orient(A, B, P[z]);
        if (oz == 0) {
          work.push_back({z, b});
          work.push_back({a, z});
          split = true;
          break;
        }
        // nt = (z, w, u) CCW starting at j
        if (oz < 0) {
          e = (j + 2) % 3;  // exits through (z, w)
          u = z;
        } else {
          e = (j + 1) % 3;  // exits through (u, z)
          w = z;
        }
        t_cur = nt;
      }
      if (split) continue;
      // remove crossings by flips
      std::vector<std::pair<int, int>> fresh;
      size_t head = 0;
      int64_t fguard = 0;
      while (head < cross.size()) {
        if (++fguard > 50000000) {
          status = -9;
          return;
        }
        auto [p, q] = cross[head++];
        int tt, ii;
        if (!find_edge(p, q, tt, ii)) {
          status = -10;
          return;
        }
        int x, y;
        if (strictly_convex(tt, ii, x, y)) {
          flip(tt, ii);
          int64_t sx = sgn(orient(A, B, P[x])), sy = sgn(orient(A, B, P[y]));
          if (sx * sy < 0)
            cross.push_back({x, y});
          else
            fresh.push_back({x, y});
        } else {
          cross.push_back({p, q});
        }
        if (head > 4096 && head * 2 > cross.size()) {
          cross.erase(cross.begin(), cross.begin() + head);
          head = 0;
        }
      }
      // restore the Delaunay property among the new edges
      bool swapped = true;
      int rounds = 0;
      while (swapped && ++rounds < 10000) {
        swapped = false;
        for (auto& ed : fresh) {
          if ((ed.first == a && ed.second == b) || (ed.first == b && ed.second == a)) continue;
          int tt, ii;
          if (!find_edge(ed.first, ed.second, tt, ii)) continue;
          if (T[tt].c[ii] >= 0) continue;
          int uu = T[tt].n[ii];
          if (uu < 0) continue;
          int s = T[uu].v[nb_edge(uu, tt)];
          if (incircle(P[T[tt].v[0]], P[T[tt].v[1]], P[T[tt].v[2]], P[s]) > 0) {
            int x, y;
            if (!strictly_convex(tt, ii, x, y)) continue;
            flip(tt, ii);
            ed = {x, y};
            swapped = true;
          }
        }
      }
      if (find_edge(a, b, t, i))
        mark(t, i, seg);
      else
        status = -11;
    }
  }

  // Lawson flips on every unconstrained interior edge until all are locally
  // (constrained-)Delaunay.
  void make_delaunay() {
    std::vector<std::pair<int, int>> st;
    for (int t = 0; t < (int)T.size(); ++t)
      for (int i = 0; i < 3; ++i)
        if (T[t].n[i] > t) st.push_back({t, i});
    while (!st.empty()) {
      auto [t, i] = st.back();
      st.pop_back();
      int u = T[t].n[i];
      if (u < 0 || T[t].c[i] >= 0) continue;
      int j = nb_edge(u, t);
      if (j < 0) continue;
      int s = T[u].v[j];
      if (incircle(P[T[t].v[0]], P[T[t].v[1]], P[T[t].v[2]], P[s]) > 0) {
        int x, y;
        if (!strictly_convex(t, i, x, y)) continue;
        flip(t, i);
        for (int k = 0; k < 3; ++k) {
          st.push_back({t, k});
          st.push_back({u, k});
        }
      }
    }
  }

  double total_length(bool interior_only) const;
};

// Hilbert index of (x, y) on a 2^order grid (the classic rotate-and-flip form).
static uint64_t hilbert_d(int order, uint32_t x, uint32_t y) {
  uint64_t d = 0;
  for (uint32_t s = 1u << (order - 1); s > 0; s >>= 1) {
    uint32_t rx = (x & s) > 0, ry = (y & s) > 0;
    d += (uint64_t)s * s * ((3 * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = s - 1 - x;
        y = s - 1 - y;
      }
      std::swap(x, y);
    }
  }
  return d;
}

// Compensated (Kahan) fp32 sum of edge lengths.
struct KahanF {
  float s = 0.f, c = 0.f;
  void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

static inline float edge_len(const Pt& a, const Pt& b) { return std::sqrt((float)len2(a, b)); }

double Triangulation::total_length(bool interior_only) const {
  KahanF k;
  for (int t = 0; t < (int)T.size(); ++t)
    for (int i = 0; i < 3; ++i) {
      int u = T[t].n[i];
      if (u >= 0 && u < t) continue;
      if (u < 0 && interior_only) continue;
      k.add(edge_len(P[T[t].v[(i + 1) % 3]], P[T[t].v[(i + 2) % 3]]));
    }
  return (double)k.s;
}

static Triangulation* build_cdt(int64_t n_seg, const int32_t* seg, int32_t D) {
  auto* tr = new Triangulation();
  tr->init_square(D);
  // unique endpoints, inserted in Hilbert order
  std::vector<Pt> pts;
  pts.reserve(2 * n_seg);
  for (int64_t s = 0; s < n_seg; ++s) {
    pts.push_back(Pt{seg[4 * s + 0], seg[4 * s + 1]});
    pts.push_back(Pt{seg[4 * s + 2], seg[4 * s + 3]});
  }
  for (const Pt& p : pts)
    if (p.x < 0 || p.y < 0 || p.x > D || p.y > D) {
      tr->status = -1;
      return tr;
    }
  std::vector<std::pair<uint64_t, int64_t>> key(pts.size());
  for (size_t k = 0; k < pts.size(); ++k) key[k] = {hilbert_d(21, (uint32_t)pts[k].x, (uint32_t)pts[k].y), (int64_t)k};
  std::sort(key.begin(), key.end());
  std::vector<int32_t> vid(pts.size(), -1);
  std::unordered_map<uint64_t, int32_t> seen;
  seen.reserve(pts.size() * 2);
  tr->P.reserve(pts.size() + 4);
  tr->T.reserve(2 * pts.size() + 8);
  for (auto& kv : key) {
    const Pt& p = pts[kv.second];
    uint64_t h = ((uint64_t)(uint32_t)p.x << 32) | (uint32_t)p.y;
    auto it = seen.find(h);
    if (it != seen.end()) {
      vid[kv.second] = it->second;
      continue;
    }
    int v = tr->insert_point(p);
    if (v < 0) return tr;
    seen[h] = v;
    vid[kv.second] = v;
  }
  for (int64_t s = 0; s < n_seg; ++s) {
    tr->insert_segment(vid[2 * s], vid[2 * s + 1], (int)s);
    if (tr->status < 0) return tr;
  }
  tr->make_delaunay();
  return tr;
}

// ---------------------------------------------------------------- annealing
// Greedy flips to a shorter diagonal until none is left (each flip strictly
// lowers the total length, so this terminates).  Squared lengths are exact.
static int64_t greedy_flips(Triangulation& tr) {
  std::vector<std::pair<int, int>> st;
  for (int t = 0; t < (int)tr.T.size(); ++t)
    for (int i = 0; i < 3; ++i)
      if (tr.T[t].n[i] > t) st.push_back({t, i});
  int64_t flips = 0;
  while (!st.empty()) {
    auto [t, i] = st.back();
    st.pop_back();
    if (tr.T[t].c[i] >= 0 || tr.T[t].n[i] < 0) continue;
    int x, y;
    if (!tr.strictly_convex(t, i, x, y)) continue;
    const Pt& q = tr.P[tr.T[t].v[(i + 1) % 3]];
    const Pt& r = tr.P[tr.T[t].v[(i + 2) % 3]];
    if (len2(tr.P[x], tr.P[y]) < len2(q, r)) {
      int u = tr.T[t].n[i];
      tr.flip(t, i);
      ++flips;
      for (int k = 0; k < 3; ++k) {
        st.push_back({t, k});
        st.push_back({u, k});
      }
    }
  }
  return flips;
}

// Vertex classes for the vertex perturbation (Sec. 3.2.2): 0 fixed (hull
// vertices, segment endpoints, vertices shared by several segments), 1 free
// Steiner vertex (no incident constrained edge: two degrees of freedom), 2
// Steiner vertex inside one segment (its two constrained edges carry the same
// segment and are collinear: the displacement is projected onto the segment,
// Sec. 3.2.1); dir = the segment's primitive lattice step, nb = its two
// neighbours along it.
struct VertexClasses {
  std::vector<int8_t> kind;
  std::vector<Pt> dir;
  std::vector<std::pair<int32_t, int32_t>> nb;
  int64_t movable = 0;
};

static int64_t gcd64(int64_t a, int64_t b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

static void classify_vertices(const Triangulation& tr, VertexClasses& vc) {
  const int nv = (int)tr.P.size();
  vc.kind.assign(nv, 0);
  vc.dir.assign(nv, Pt{0, 0});
  vc.nb.assign(nv, {-1, -1});
  vc.movable = 0;
  std::vector<std::pair<int32_t, int32_t>> ce;  // (other vertex, segment) of incident constrained edges
  for (int v = 0; v < nv; ++v) {
    const Pt& p = tr.P[v];
    if (p.x <= 0 || p.y <= 0 || p.x >= tr.D || p.y >= tr.D) continue;
    ce.clear();
    tr.for_fan(v, [&](int t, int k) {
      const Tri& x = tr.T[t];
      // edge (k+2)%3 joins v and vertex (k+1)%3; each incident edge is seen once this way
      if (x.c[(k + 2) % 3] >= 0) ce.push_back({x.v[(k + 1) % 3], x.c[(k + 2) % 3]});
      return false;
    });
    if (ce.empty()) {
      vc.kind[v] = 1;
      ++vc.movable;
      continue;
    }
    if (ce.size() != 2 || ce[0].second != ce[1].second) continue;
    const Pt &a = tr.P[ce[0].first], &b = tr.P[ce[1].first];
    if (orient(a, b, p) != 0) continue;
    const int64_t dot = (int64_t)(a.x - p.x) * (b.x - p.x) + (int64_t)(a.y - p.y) * (b.y - p.y);
    if (dot >= 0) continue;  // not between its neighbours
    const int64_t dx = (int64_t)b.x - a.x, dy = (int64_t)b.y - a.y, g = gcd64(dx, dy);
    vc.kind[v] = 2;
    vc.dir[v] = Pt{(int32_t)(dx / g), (int32_t)(dy / g)};
    vc.nb[v] = {ce[0].first, ce[1].first};
    ++vc.movable;
  }
}

// Proposes moving vertex v to q: true (and the change of the total edge
// length in *delta) if every triangle of v's star stays strictly CCW.
static bool vertex_move_delta(const Triangulation& tr, int v, const Pt& q, float* delta) {
  const Pt& p = tr.P[v];
  bool ok = true;
  float d = 0.f;
  tr.for_fan(v, [&](int t, int k) {
    const Tri& x = tr.T[t];
    const Pt &a = tr.P[x.v[(k + 1) % 3]], &b = tr.P[x.v[(k + 2) % 3]];
    if (orient(q, a, b) <= 0) {
      ok = false;
      return true;
    }
    d += edge_len(q, a) - edge_len(p, a);  // edge (v, a): once per star triangle
    return false;
  });
  *delta = d;
  return ok;
}

// The vertex perturbation of Sec. 3.2.2, p -> p + lambda eta xi: xi a point
// uniform in the unit disk with its radius multiplied by a Pareto factor
// (pdf alpha / x^(alpha + 1), alpha = 1/2, x > 1: heavy-tailed), eta the
// square root of the area of the vertex's star, lambda adapted to keep the
// acceptance rate near 23 % (its own value per vertex class).  The result is
// rounded to the integer lattice (after projection onto the segment for a
// vertex inside one), which keeps every predicate of the walk exact.
struct VertexMover {
  double lambda[3] = {0.0, 0.1, 0.1};
  int64_t tried[3] = {0, 0, 0}, accepted[3] = {0, 0, 0};

  bool propose(const Triangulation& tr, const VertexClasses& vc, int v, Rng& rng, Pt& q) const {
    const Pt p = tr.P[v];
    double area2 = 0.0;
    tr.for_fan(v, [&](int t, int) {
      const Tri& x = tr.T[t];
      area2 += (double)orient(tr.P[x.v[0]], tr.P[x.v[1]], tr.P[x.v[2]]);
      return false;
    });
    const double eta = std::sqrt(0.5 * area2);
    const double r = std::sqrt(rng.uni()), th = 6.283185307179586 * rng.uni();
    const double pareto = std::pow(1.0 - rng.uni(), -2.0);  // alpha = 1/2
    double ex = lambda[vc.kind[v]] * eta * r * pareto * std::cos(th);
    double ey = lambda[vc.kind[v]] * eta * r * pareto * std::sin(th);
    if (!(std::fabs(ex) < 4.0 * tr.D && std::fabs(ey) < 4.0 * tr.D)) return false;
    if (vc.kind[v] == 1) {
      q = Pt{(int32_t)(p.x + std::llround(ex)), (int32_t)(p.y + std::llround(ey))};
      return q.x > 0 && q.y > 0 && q.x < tr.D && q.y < tr.D && !(q == p);
    }
    // inside a segment: project onto it, whole lattice steps, strictly between its neighbours
    const Pt dir = vc.dir[v];
    const int64_t m = std::llround((ex * dir.x + ey * dir.y) / (double)len2(Pt{0, 0}, dir));
    if (m == 0) return false;
    q = Pt{(int32_t)(p.x + m * dir.x), (int32_t)(p.y + m * dir.y)};
    const Pt &a = tr.P[vc.nb[v].first], &b = tr.P[vc.nb[v].second];
    return (int64_t)(a.x - q.x) * (b.x - q.x) + (int64_t)(a.y - q.y) * (b.y - q.y) < 0;
  }

  // The resampling of Sec. 3.2.4: a new position uniform (by area) in the
  // triangles around the vertex (for a vertex inside a segment: a lattice
  // point uniform between its two neighbours along it), rounded to the lattice.
  bool resample(const Triangulation& tr, const VertexClasses& vc, int v, Rng& rng, Pt& q) const {
    const Pt p = tr.P[v];
    if (vc.kind[v] == 2) {
      const Pt dir = vc.dir[v];
      const Pt &a = tr.P[vc.nb[v].first], &b = tr.P[vc.nb[v].second];
      const int64_t sx = dir.x != 0 ? dir.x : dir.y;
      const int64_t ma = ((int64_t)(dir.x != 0 ? a.x - p.x : a.y - p.y)) / sx;  // a = p + ma dir
      const int64_t mb = ((int64_t)(dir.x != 0 ? b.x - p.x : b.y - p.y)) / sx;
      const int64_t lo = std::min(ma, mb) + 1, hi = std::max(ma, mb) - 1;  // strictly between
      if (hi < lo) return false;
      const int64_t m = lo + (int64_t)(rng.uni() * (double)(hi - lo + 1));
      if (m == 0 || m > hi) return false;
      q = Pt{(int32_t)(p.x + m * dir.x), (int32_t)(p.y + m * dir.y)};
      return true;
    }
    double total = 0.0;
    tr.for_fan(v, [&](int t, int k) {
      const Tri& x = tr.T[t];
      total += (double)orient(p, tr.P[x.v[(k + 1) % 3]], tr.P[x.v[(k + 2) % 3]]);
      return false;
    });
    double pick = rng.uni() * total;
    bool done = false;
    tr.for_fan(v, [&](int t, int k) {
      const Tri& x = tr.T[t];
      const Pt &a = tr.P[x.v[(k + 1) % 3]], &b = tr.P[x.v[(k + 2) % 3]];
      const double w = (double)orient(p, a, b);
      if (pick > w) {
        pick -= w;
        return false;
      }
      double r1 = rng.uni(), r2 = rng.uni();
      if (r1 + r2 > 1.0) {
        r1 = 1.0 - r1;
        r2 = 1.0 - r2;
      }
      q = Pt{(int32_t)std::llround(p.x + r1 * (a.x - p.x) + r2 * (b.x - p.x)),
             (int32_t)std::llround(p.y + r1 * (a.y - p.y) + r2 * (b.y - p.y))};
      done = true;
      return true;
    });
    return done && !(q == p) && q.x > 0 && q.y > 0 && q.x < tr.D && q.y < tr.D;
  }

  void record(int kind, bool acc) {
    ++tried[kind];
    accepted[kind] += acc;
    if (tried[kind] == 256) {  // steer towards 23 % acceptance
      const double rate = (double)accepted[kind] / 256.0;
      lambda[kind] *= std::exp(2.0 * (rate - 0.23));
      lambda[kind] = std::min(10.0, std::max(1e-6, lambda[kind]));
      tried[kind] = accepted[kind] = 0;
    }
  }
};

// Contraction, in the discrete form this exact-lattice build allows (the
// paper contracts fuzzily: vertices first move onto one another under the
// objective of Sec. 2.2, Sec. 3.2.6, and are merged afterwards, Sec. 3.4.1):
// Steiner vertex v is merged into its neighbour u, deleting the two triangles
// on edge (u, v).  A free Steiner vertex may merge into any neighbour, one
// inside a segment only into a neighbour along that segment (so the segment
// stays covered).  Valid iff the links of u and v share exactly the two apexes
// (the topology stays a triangulation) and every triangle of v's star, with v
// replaced by u, stays strictly CCW (exact).  *delta = the change of the total
// edge length.  Triangles and vertices are only marked dead (v[0] = -1,
// vtri = -1); compact_dead renumbers at the end.
static bool collapse_delta(const Triangulation& tr, int v, int u, int& t1, int& t2, float* delta) {
  int i1;
  if (!tr.find_edge(v, u, t1, i1)) return false;
  t2 = tr.T[t1].n[i1];
  if (t2 < 0) return false;
  const int a = tr.T[t1].v[i1], b = tr.T[t2].v[tr.nb_edge(t2, t1)];
  // link condition
  std::vector<int32_t> lv, lu;
  tr.for_fan(v, [&](int t, int k) {
    lv.push_back(tr.T[t].v[(k + 1) % 3]);
    lv.push_back(tr.T[t].v[(k + 2) % 3]);
    return false;
  });
  tr.for_fan(u, [&](int t, int k) {
    lu.push_back(tr.T[t].v[(k + 1) % 3]);
    lu.push_back(tr.T[t].v[(k + 2) % 3]);
    return false;
  });
  std::sort(lv.begin(), lv.end());
  lv.erase(std::unique(lv.begin(), lv.end()), lv.end());
  std::sort(lu.begin(), lu.end());
  lu.erase(std::unique(lu.begin(), lu.end()), lu.end());
  int shared = 0;
  for (int32_t x : lv)
    if (x != u && std::binary_search(lu.begin(), lu.end(), x)) {
      if (x != a && x != b) return false;
      ++shared;
    }
  if (shared != 2) return false;
  const Pt &pv = tr.P[v], &pu = tr.P[u];
  bool ok = true;
  float d = -edge_len(pv, pu);
  tr.for_fan(v, [&](int t, int k) {
    const Tri& x = tr.T[t];
    const int p = x.v[(k + 1) % 3], q = x.v[(k + 2) % 3];
    // edge (v, p) once per star triangle: removed if p is an apex, else moved to u
    d += (p == a || p == b) ? -edge_len(pv, tr.P[p]) : (p == u ? 0.f : edge_len(pu, tr.P[p]) - edge_len(pv, tr.P[p]));
    if (t == t1 || t == t2) return false;
    if (orient(pu, tr.P[p], tr.P[q]) <= 0) {
      ok = false;
      return true;
    }
    return false;
  });
  *delta = d;
  return ok;
}

static void do_collapse(Triangulation& tr, int v, int u, int t1, int t2) {
  // v's star, collected before any neighbour pointer changes
  std::vector<int> star;
  tr.for_fan(v, [&](int t, int) {
    star.push_back(t);
    return false;
  });
  // the outer neighbours of t1 / t2 across their edges at v and at u become
  // neighbours of each other across the merged edge (u, apex)
  for (int t : {t1, t2}) {
    const Tri x = tr.T[t];
    const int kv = Triangulation::idx_of(x, v), ku = Triangulation::idx_of(x, u);
    const int n_v = x.n[ku], n_u = x.n[kv];  // across the edge at v (opposite u) / at u (opposite v)
    const int c_u = x.c[kv];
    if (n_v >= 0) {
      const int e = tr.nb_edge(n_v, t);
      tr.T[n_v].n[e] = n_u;
      tr.T[n_v].c[e] = c_u;
    }
    if (n_u >= 0) {
      const int e = tr.nb_edge(n_u, t);
      tr.T[n_u].n[e] = n_v;
    }
    const int apex = x.v[3 - kv - ku];
    tr.vtri[apex] = n_v >= 0 ? n_v : n_u;
    tr.vtri[u] = n_v >= 0 ? n_v : n_u;
  }
  // every other triangle of v's star takes u in v's place
  for (int t : star) {
    if (t == t1 || t == t2) continue;
    const int k = Triangulation::idx_of(tr.T[t], v);
    tr.T[t].v[k] = u;
    tr.vtri[u] = t;
  }
  tr.T[t1].v[0] = -1;
  tr.T[t2].v[0] = -1;
  tr.vtri[v] = -1;
}

// Drops dead triangles and vertices and renumbers the rest.
static void compact_dead(Triangulation& tr) {
  std::vector<int32_t> tmap(tr.T.size(), -1), vmap(tr.P.size(), -1);
  std::vector<Tri> T2;
  std::vector<Pt> P2;
  for (size_t v = 0; v < tr.P.size(); ++v)
    if (tr.vtri[v] >= 0) {
      vmap[v] = (int32_t)P2.size();
      P2.push_back(tr.P[v]);
    }
  for (size_t t = 0; t < tr.T.size(); ++t)
    if (tr.T[t].v[0] >= 0) {
      tmap[t] = (int32_t)T2.size();
      T2.push_back(tr.T[t]);
    }
  if (T2.size() == tr.T.size()) return;
  std::vector<int32_t> vtri2(P2.size(), 0);
  for (size_t t = 0; t < T2.size(); ++t)
    for (int i = 0; i < 3; ++i) {
      T2[t].v[i] = vmap[T2[t].v[i]];
      if (T2[t].n[i] >= 0) T2[t].n[i] = tmap[T2[t].n[i]];
      vtri2[T2[t].v[i]] = (int32_t)t;
    }
  tr.T.swap(T2);
  tr.P.swap(P2);
  tr.vtri.swap(vtri2);
  tr.last = 0;
}

// Simulated annealing (Sec. 3.1-3.3) over edge flips (Sec. 3.2.7) and, when
// moves > 0, the vertex perturbations of Sec. 3.2.2 and 3.2.4 on Steiner
// vertices (see VertexMover), with Metropolis acceptance and an exponential
// temperature schedule.  The energy is the total edge length; lengths and differences are
// fp32.  A vertex proposal is drawn with probability
// moves * (movable vertices / vertices).
static void anneal_flips(Triangulation& tr, uint64_t seed, double sweeps, double T0, double T1, double moves,
                         double collapse) {
  int64_t n_collapsed = 0;
  Rng rng(seed, 0xA77);
  int64_t n_half = (int64_t)tr.T.size() * 3;
  int64_t K = (int64_t)(sweeps * (double)n_half);
  if (K <= 0) return;
  VertexClasses vc;
  VertexMover mover;
  double p_move = 0.0;
  std::vector<int32_t> movable;
  if (moves > 0) {
    classify_vertices(tr, vc);
    for (int v = 0; v < (int)vc.kind.size(); ++v)
      if (vc.kind[v]) movable.push_back(v);
    p_move = movable.empty() ? 0.0 : moves * (double)movable.size() / (double)tr.P.size();
  }
  double lt0 = std::log(T0), lt1 = std::log(T1);
  for (int64_t k = 0; k < K; ++k) {
    float temp = (float)std::exp(lt0 + (lt1 - lt0) * ((double)k / (double)K));
    if (p_move > 0 && rng.uni() < p_move) {
      const int v = movable[rng.below((uint32_t)movable.size())];
      if (tr.vtri[v] < 0) continue;  // merged away
      Pt q;
      float delta;
      bool acc = false;
      if (collapse > 0 && rng.uni() < collapse) {
        // merge v into a neighbour: any for a free vertex, one along its segment otherwise
        int u = -1;
        if (vc.kind[v] == 2) {
          u = rng.uni() < 0.5 ? vc.nb[v].first : vc.nb[v].second;
        } else {
          int deg = 0;
          tr.for_fan(v, [&](int, int) {
            ++deg;
            return false;
          });
          int pick = (int)rng.below((uint32_t)deg);
          tr.for_fan(v, [&](int t, int kk) {
            if (pick-- == 0) {
              u = tr.T[t].v[(kk + 1) % 3];
              return true;
            }
            return false;
          });
        }
        int t1, t2;
        if (u >= 0 && collapse_delta(tr, v, u, t1, t2, &delta) &&
            (delta <= 0.f || (float)rng.uni() < std::exp(-delta / temp))) {
          if (vc.kind[v] == 2) {
            // the segment neighbours of v now neighbour each other
            const int w = vc.nb[v].first == u ? vc.nb[v].second : vc.nb[v].first;
            for (int x : {u, w})
              if (x >= 0 && vc.kind[x] == 2) {
                if (vc.nb[x].first == v) vc.nb[x].first = (x == u ? w : u);
                if (vc.nb[x].second == v) vc.nb[x].second = (x == u ? w : u);
              }
          }
          do_collapse(tr, v, u, t1, t2);
          vc.kind[v] = 0;
          ++n_collapsed;
        }
        continue;
      }
      // the two vertex strategies share the vertex proposals equally (Sec. 3.3)
      const bool resample = rng.uni() < 0.5;
      const bool proposed = resample ? mover.resample(tr, vc, v, rng, q) : mover.propose(tr, vc, v, rng, q);
      if (proposed && vertex_move_delta(tr, v, q, &delta) &&
          (delta <= 0.f || (float)rng.uni() < std::exp(-delta / temp))) {
        tr.P[v] = q;
        acc = true;
      }
      if (!resample) mover.record(vc.kind[v], acc);  // lambda steers the Sec. 3.2.2 move only
      continue;
    }
    int t = (int)rng.below((uint32_t)tr.T.size());
    int i = (int)rng.below(3);
    if (tr.T[t].v[0] < 0 || tr.T[t].c[i] >= 0 || tr.T[t].n[i] < 0) continue;
    int x, y;
    if (!tr.strictly_convex(t, i, x, y)) continue;
    const Pt& q = tr.P[tr.T[t].v[(i + 1) % 3]];
    const Pt& r = tr.P[tr.T[t].v[(i + 2) % 3]];
    float delta = edge_len(tr.P[x], tr.P[y]) - edge_len(q, r);
    if (delta <= 0.f || (float)rng.uni() < std::exp(-delta / temp)) tr.flip(t, i);
  }
  if (n_collapsed > 0) compact_dead(tr);
}

// ---------------------------------------------------------------- fuzzy objective (Sec. 2.2)
// f = W_contr + mu_angle Pi_angle + mu_len Pi_len in unit-square units (lengths / D):
//   W_contr = sum_e w(e) |e|,  w(e) = P M(P),  P = prod of c(e') over the other edges e' of the
//   (one or two) triangles of e,  c(e') = 1/2 + min(1, |e'| / eps) / 2 for a contractible edge, else 1;
//   M(x) = 0 below 1/4, 4x - 1 on [1/4, 1/2], 1 above (the correction for multiply merged edges).
//   The printed weight is M(P) alone; the text's worked example (an isolated contraction gives the
//   two merging edges 1/2 each, a doubly merged edge 0, and M "not counting" multiply contracted
//   edges) holds for w = P M(P), the reading used here.
//   Pi_angle = sum over the three angles of every triangle of max(0, -1 + delta - cos) / delta
//   (angles near 180 degrees); when polishing (fixed topology, w = 1) max(0, cos - 1 + delta) / delta
//   (angles near 0 degrees) instead.  Pi_len = sum_e max(0, eps0 - |e|) / eps0.
struct FuzzyParams {
  double eps, delta, eps0, mu_angle, mu_len;
  int polish;
};

// Contractibility of edge i of triangle t (Sec. 2.2.2).  By degrees of freedom: a free vertex
// merges into any vertex; two vertices without freedom (segment endpoints and junctions, the
// hull's vertices) never merge; a Steiner vertex inside a segment merges only along its segment
// (the edge is then a constrained edge of that segment).  By planarity: a common neighbour of the
// two endpoints that is not an apex of the edge's triangles (a nontrivial 1-hop connection) forbids
// it unless that neighbour lies within eps of an apex, or an apex lies within eps of both endpoints
// (the whole triangle contracts to one point, so the triangles joining the neighbour to the two
// endpoints through that apex degenerate instead of overlapping: the case of the text's example of
// three contracted edges, which the distance rule alone would forbid).  The conditioning and flat-triangle checks of
// the paper are left to the exact validity test of the actual contraction (exact predicates cannot
// be broken by thin triangles).
static bool fuzzy_contractible(const Triangulation& tr, const VertexClasses& vc, double eps_lattice, int t,
                               int i) {
  const Tri& x = tr.T[t];
  const int p = x.v[(i + 1) % 3], q = x.v[(i + 2) % 3];
  const int kp = vc.kind[p], kq = vc.kind[q];
  if (kp != 1 && kq != 1) {
    if (kp == 0 && kq == 0) return false;
    if (x.c[i] < 0) return false;  // both constrained: only along their own segment
  }
  const int a = x.v[i], n = x.n[i];
  const int b = n >= 0 ? tr.T[n].v[tr.nb_edge(n, t)] : -1;
  int np = 0;
  int nbp[64];
  bool overflow = false;
  tr.for_fan(p, [&](int tt, int k) {
    for (int s = 1; s <= 2; ++s) {
      const int w = tr.T[tt].v[(k + s) % 3];
      bool seen = false;
      for (int j = 0; j < np; ++j) seen |= nbp[j] == w;
      if (!seen) {
        if (np == 64) {
          overflow = true;
          return true;
        }
        nbp[np++] = w;
      }
    }
    return false;
  });
  if (overflow) return false;
  const double e2 = eps_lattice * eps_lattice;
  const Pt &pp = tr.P[p], &pq = tr.P[q];
  const bool a_in = (double)len2(tr.P[a], pp) < e2 && (double)len2(tr.P[a], pq) < e2;
  const bool b_in = b >= 0 && (double)len2(tr.P[b], pp) < e2 && (double)len2(tr.P[b], pq) < e2;
  if (a_in || b_in) return true;
  bool ok = true;
  tr.for_fan(q, [&](int tt, int k) {
    for (int s = 1; s <= 2; ++s) {
      const int w = tr.T[tt].v[(k + s) % 3];
      if (w == p || w == a || w == b) continue;
      bool common = false;
      for (int j = 0; j < np; ++j) common |= nbp[j] == w;
      if (!common) continue;
      const double da = (double)len2(tr.P[w], tr.P[a]), db = b >= 0 ? (double)len2(tr.P[w], tr.P[b]) : 1e300;
      if (da >= e2 && db >= e2) {
        ok = false;
        return true;
      }
    }
    return false;
  });
  return ok;
}

static inline double multi_merge(double x) { return x < 0.25 ? 0.0 : (x <= 0.5 ? 4.0 * x - 1.0 : 1.0); }

static inline double angle_penalty(double c, const FuzzyParams& fp) {
  return fp.polish ? std::max(0.0, c - 1.0 + fp.delta) / fp.delta : std::max(0.0, -1.0 + fp.delta - c) / fp.delta;
}

// The three angle cosines of triangle t.
static void tri_cosines(const Triangulation& tr, int t, double cs[3]) {
  for (int k = 0; k < 3; ++k) {
    const Pt &a = tr.P[tr.T[t].v[k]], &b = tr.P[tr.T[t].v[(k + 1) % 3]], &c = tr.P[tr.T[t].v[(k + 2) % 3]];
    const double ux = (double)b.x - a.x, uy = (double)b.y - a.y, vx = (double)c.x - a.x, vy = (double)c.y - a.y;
    cs[k] = (ux * vx + uy * vy) / std::sqrt((ux * ux + uy * uy) * (vx * vx + vy * vy));
  }
}

// f and its three terms; w_out (optional, 3 per triangle) receives every edge's weight w(e).
static void fuzzy_objective(const Triangulation& tr, const FuzzyParams& fp, double terms[4], double* w_out) {
  VertexClasses vc;
  classify_vertices(tr, vc);
  const size_t nt = tr.T.size();
  const double D = (double)tr.D, eps_lat = fp.eps * D;
  std::vector<double> len(3 * nt), cw(3 * nt);
  for (size_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      const int n = tr.T[t].n[i];
      if (n >= 0 && (size_t)n < t) {  // the other side holds it
        const int j = tr.nb_edge(n, (int)t);
        len[3 * t + i] = len[3 * n + j];
        cw[3 * t + i] = cw[3 * n + j];
        continue;
      }
      const Pt &p = tr.P[tr.T[t].v[(i + 1) % 3]], &q = tr.P[tr.T[t].v[(i + 2) % 3]];
      len[3 * t + i] = std::sqrt((double)len2(p, q)) / D;
      cw[3 * t + i] = (fp.polish || !fuzzy_contractible(tr, vc, eps_lat, (int)t, i))
                          ? 1.0
                          : 0.5 + std::min(1.0, len[3 * t + i] / fp.eps) / 2.0;
    }
  double W = 0, PA = 0, PL = 0;
  for (size_t t = 0; t < nt; ++t) {
    for (int i = 0; i < 3; ++i) {
      const int n = tr.T[t].n[i];
      double P = cw[3 * t + (i + 1) % 3] * cw[3 * t + (i + 2) % 3];
      if (n >= 0) {
        const int j = tr.nb_edge(n, (int)t);
        P *= cw[3 * n + (j + 1) % 3] * cw[3 * n + (j + 2) % 3];
      }
      const double w = fp.polish ? 1.0 : P * multi_merge(P);
      if (w_out) w_out[3 * t + i] = w;
      if (n >= 0 && (size_t)n < t) continue;  // each edge once
      W += w * len[3 * t + i];
      PL += std::max(0.0, fp.eps0 - len[3 * t + i]) / fp.eps0;
    }
    double cs[3];
    tri_cosines(tr, (int)t, cs);
    for (int k = 0; k < 3; ++k) PA += angle_penalty(cs[k], fp);
  }
  terms[0] = W + fp.mu_angle * PA + fp.mu_len * PL;
  terms[1] = W;
  terms[2] = PA;
  terms[3] = PL;
}

// The fuzzy objective over a region: every edge of the given triangles once, with its weight from
// the current state, plus those triangles' angle penalties.  c values are memoised per edge for one
// evaluation.  A proposal's energy change is the region's energy after minus before, for a region
// that holds every edge whose weight the proposal can change (see anneal_fuzzy).
struct FuzzyLocal {
  const Triangulation& tr;
  const VertexClasses& vc;
  const FuzzyParams& fp;
  // open-addressing tables keyed by edge (cleared per evaluation through a generation stamp):
  // the memoised c of an edge, and the edges already summed; each grows (rehashing its live
  // entries) before it is half full, so a probe always ends at a free slot
  int bits;
  uint32_t mask;
  std::vector<uint64_t> key_c, key_s;
  std::vector<uint32_t> gen_c, gen_s;
  std::vector<double> val_c;
  uint32_t gen = 0;
  size_t used_c = 0, used_s = 0;
  int64_t grows = 0;  // table growths so far

  FuzzyLocal(const Triangulation& t, const VertexClasses& v, const FuzzyParams& f, int init_bits = 12)
      : tr(t), vc(v), fp(f), bits(init_bits), mask((1u << init_bits) - 1), key_c((size_t)1 << init_bits),
        key_s((size_t)1 << init_bits), gen_c((size_t)1 << init_bits, 0), gen_s((size_t)1 << init_bits, 0),
        val_c((size_t)1 << init_bits) {}
  uint32_t slot(uint64_t k) const { return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> (64 - bits)); }
  void grow() {
    ++grows;
    std::vector<uint64_t> kc = key_c, ks = key_s;
    std::vector<uint32_t> gc = gen_c, gs = gen_s;
    std::vector<double> vcv = val_c;
    ++bits;
    mask = (1u << bits) - 1;
    key_c.assign((size_t)1 << bits, 0);
    key_s.assign((size_t)1 << bits, 0);
    gen_c.assign((size_t)1 << bits, 0);
    gen_s.assign((size_t)1 << bits, 0);
    val_c.assign((size_t)1 << bits, 0.0);
    for (size_t j = 0; j < kc.size(); ++j)
      if (gc[j] == gen) {
        uint32_t h = slot(kc[j]);
        while (gen_c[h] == gen) h = (h + 1) & mask;
        gen_c[h] = gen;
        key_c[h] = kc[j];
        val_c[h] = vcv[j];
      }
    for (size_t j = 0; j < ks.size(); ++j)
      if (gs[j] == gen) {
        uint32_t h = slot(ks[j]);
        while (gen_s[h] == gen) h = (h + 1) & mask;
        gen_s[h] = gen;
        key_s[h] = ks[j];
      }
  }
  static uint64_t key(int p, int q) {
    return p < q ? ((uint64_t)(uint32_t)p << 32) | (uint32_t)q : ((uint64_t)(uint32_t)q << 32) | (uint32_t)p;
  }
  double len(int t, int i) const {
    const Tri& x = tr.T[t];
    return std::sqrt((double)len2(tr.P[x.v[(i + 1) % 3]], tr.P[x.v[(i + 2) % 3]])) / (double)tr.D;
  }
  double c(int t, int i) {
    if (fp.polish) return 1.0;
    const Tri& x = tr.T[t];
    const uint64_t k = key(x.v[(i + 1) % 3], x.v[(i + 2) % 3]);
    uint32_t h = slot(k);
    while (gen_c[h] == gen) {
      if (key_c[h] == k) return val_c[h];
      h = (h + 1) & mask;
    }
    const double v = fuzzy_contractible(tr, vc, fp.eps * (double)tr.D, t, i)
                         ? 0.5 + std::min(1.0, len(t, i) / fp.eps) / 2.0
                         : 1.0;
    if (2 * (used_c + 1) > key_c.size()) {
      grow();
      h = slot(k);
      while (gen_c[h] == gen) h = (h + 1) & mask;
    }
    ++used_c;
    gen_c[h] = gen;
    key_c[h] = k;
    val_c[h] = v;
    return v;
  }
  // whether edge k was summed already in this evaluation (and mark it)
  bool seen_before(uint64_t k) {
    uint32_t h = slot(k);
    while (gen_s[h] == gen) {
      if (key_s[h] == k) return true;
      h = (h + 1) & mask;
    }
    if (2 * (used_s + 1) > key_s.size()) {
      grow();
      h = slot(k);
      while (gen_s[h] == gen) h = (h + 1) & mask;
    }
    ++used_s;
    gen_s[h] = gen;
    key_s[h] = k;
    return false;
  }
  double w(int t, int i) {
    if (fp.polish) return 1.0;
    double P = c(t, (i + 1) % 3) * c(t, (i + 2) % 3);
    const int n = tr.T[t].n[i];
    if (n >= 0) {
      const int j = tr.nb_edge(n, t);
      P *= c(n, (j + 1) % 3) * c(n, (j + 2) % 3);
    }
    return P * multi_merge(P);
  }
  double energy(const std::vector<int>& tris) {
    if (++gen == 0) {  // the stamp wrapped: clear the tables
      std::fill(gen_c.begin(), gen_c.end(), 0);
      std::fill(gen_s.begin(), gen_s.end(), 0);
      gen = 1;
    }
    used_c = used_s = 0;
    double E = 0.0;
    for (int t : tris)
      for (int i = 0; i < 3; ++i) {
        const Tri& x = tr.T[t];
        const uint64_t k = key(x.v[(i + 1) % 3], x.v[(i + 2) % 3]);
        if (seen_before(k)) continue;
        const double l = len(t, i);
        E += w(t, i) * l + fp.mu_len * std::max(0.0, fp.eps0 - l) / fp.eps0;
      }
    for (int t : tris) {
      double cs[3];
      tri_cosines(tr, t, cs);
      for (int k = 0; k < 3; ++k) E += fp.mu_angle * angle_penalty(cs[k], fp);
    }
    return E;
  }
};

static void add_star(const Triangulation& tr, int v, std::vector<int>& out) {
  tr.for_fan(v, [&](int t, int) {
    out.push_back(t);
    return false;
  });
}
static void sort_unique(std::vector<int>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

// "Contraction to a neighbour" (Sec. 3.2): v is resampled within distance eps of a random neighbour u
// (a Steiner vertex inside a segment: along the segment, towards itself, from a segment neighbour).
static bool propose_to_neighbour(const Triangulation& tr, const VertexClasses& vc, int v, double eps_lat, Rng& rng,
                                 Pt& q) {
  if (vc.kind[v] == 2) {
    const int u = rng.uni() < 0.5 ? vc.nb[v].first : vc.nb[v].second;
    const Pt &pu = tr.P[u], &pv = tr.P[v], dir = vc.dir[v];
    const int64_t sx = dir.x != 0 ? dir.x : dir.y;
    const int64_t mv = ((int64_t)(dir.x != 0 ? pv.x - pu.x : pv.y - pu.y)) / sx;  // v = u + mv dir
    const int64_t other = vc.nb[v].first == u ? vc.nb[v].second : vc.nb[v].first;
    const Pt& pw = tr.P[other];
    const int64_t mw = ((int64_t)(dir.x != 0 ? pw.x - pu.x : pw.y - pu.y)) / sx;  // w = u + mw dir
    const double step = std::sqrt((double)dir.x * dir.x + (double)dir.y * dir.y);
    const int64_t reach = std::max<int64_t>(1, (int64_t)(eps_lat / step));
    const int64_t sgn_w = mw > 0 ? 1 : -1;
    const int64_t lim = std::min<int64_t>(reach, std::llabs(mw) - 1);
    if (lim < 1) return false;
    const int64_t m = sgn_w * (1 + (int64_t)(rng.uni() * (double)lim));
    if (m == mv) return false;
    q = Pt{(int32_t)(pu.x + m * dir.x), (int32_t)(pu.y + m * dir.y)};
    return true;
  }
  int deg = 0;
  tr.for_fan(v, [&](int, int) {
    ++deg;
    return false;
  });
  int pick = (int)rng.below((uint32_t)deg), u = -1;
  tr.for_fan(v, [&](int t, int k) {
    if (pick-- == 0) {
      u = tr.T[t].v[(k + 1) % 3];
      return true;
    }
    return false;
  });
  if (u < 0) return false;
  const double r = eps_lat * std::sqrt(rng.uni()), a = 6.283185307179586 * rng.uni();
  const Pt& pu = tr.P[u];
  q = Pt{(int32_t)std::llround(pu.x + r * std::cos(a)), (int32_t)std::llround(pu.y + r * std::sin(a))};
  return q.x > 0 && q.y > 0 && q.x < tr.D && q.y < tr.D && !(q == tr.P[v]);
}

// Whether vertex v (at position q) has a neighbour closer than r (lattice units).
static bool has_neighbour_within(const Triangulation& tr, int v, const Pt& q, double r) {
  const double r2 = r * r;
  return tr.for_fan(v, [&](int t, int k) { return (double)len2(q, tr.P[tr.T[t].v[(k + 1) % 3]]) < r2; });
}

// Sec. 3.2.2's second variant: 2 % of the movable vertices (at least one, at most 64) each get the
// vertex perturbation, decided together.  Fills group / newpos; false when no vertex got a move.
static bool propose_many(const Triangulation& tr, const VertexClasses& vc, const std::vector<int32_t>& movable,
                         VertexMover& mover, Rng& rng, std::vector<int>& group, std::vector<Pt>& newpos) {
  const size_t m = std::min<size_t>(64, std::max<size_t>(1, (size_t)std::llround(0.02 * (double)movable.size())));
  for (size_t g = 0; g < m; ++g) {
    const int u = movable[rng.below((uint32_t)movable.size())];
    if (std::find(group.begin(), group.end(), u) != group.end()) continue;
    Pt pu;
    if (!mover.propose(tr, vc, u, rng, pu)) continue;
    group.push_back(u);
    newpos.push_back(pu);
  }
  return !group.empty();
}

// The region of a move of `group`: the triangles of the stars of the moved vertices and of their
// neighbours (every edge whose weight the move can change lies in it).
static void group_region(const Triangulation& tr, const std::vector<int>& group, std::vector<int>& region) {
  region.clear();
  for (int u : group) {
    add_star(tr, u, region);
    tr.for_fan(u, [&](int t, int kk) {
      add_star(tr, tr.T[t].v[(kk + 1) % 3], region);
      return false;
    });
  }
  sort_unique(region);
}

// Simulated annealing on the fuzzy objective f (Sec. 2.2, 3.1-3.3): T and eps decrease
// exponentially together (T0 -> T1, eps_a -> eps_b, unit-square units); proposals are edge flips
// and, in equal shares, the vertex perturbation (Sec. 3.2.2), the perturbation of a group of
// contracted vertices (Sec. 3.2.3: the free vertices within d ~ U[eps/2, 5 eps] of a central one move
// together by one heavy-tailed step scaled by the root of their stars' area), the resampling within
// the neighbouring triangles (Sec. 3.2.4), the swap of a contracted edge (Sec. 3.2.5: a vertex with a
// neighbour closer than l ~ U[0.2 eps, 2 eps] resampled in the disk of radius l about a random
// neighbour) and the contraction to a neighbour (Sec. 3.2.6: an uncontracted vertex resampled within
// eps of a random neighbour, a contracted one by the resampling of Sec. 3.2.4 kept only if it leaves
// every neighbour), and, in 2 % of the vertex proposals, the perturbation of 2 % of the movable
// vertices at once (Sec. 3.2.2's second variant, one Metropolis decision),
// with Metropolis acceptance on the exact change of f over a region that holds every edge whose
// weight the proposal can change: for a vertex move the triangles of the stars of the vertex and of
// its neighbours (lengths and contractibility distances change at the vertex; an edge's weight reads
// the c of the edges of its own triangles); for a flip the stars of the quadrilateral's four vertices
// (their neighbour sets change, hence the 1-hop test of every edge at them).
static void anneal_fuzzy(Triangulation& tr, uint64_t seed, double sweeps, double T0, double T1, double eps_a,
                         double eps_b, double moves) {
  Rng rng(seed, 0xF022);
  VertexClasses vc;
  classify_vertices(tr, vc);
  std::vector<int32_t> movable;
  for (int v = 0; v < (int)vc.kind.size(); ++v)
    if (vc.kind[v]) movable.push_back(v);
  const double p_move = movable.empty() ? 0.0 : moves * (double)movable.size() / (double)tr.P.size();
  FuzzyParams fp{eps_a, 1.0 + std::cos(179.0 * 3.14159265358979323846 / 180.0), 1e-10, 1.0, 10.0, 0};
  FuzzyLocal loc(tr, vc, fp);
  VertexMover mover;
  const int64_t K = (int64_t)(sweeps * (double)tr.T.size() * 3.0);
  const double lt0 = std::log(T0), lt1 = std::log(T1), le0 = std::log(eps_a), le1 = std::log(eps_b);
  std::vector<int> region, group;
  std::vector<Pt> newpos, oldpos;
  for (int64_t k = 0; k < K; ++k) {
    const double fr = (double)k / (double)K;
    const double temp = std::exp(lt0 + (lt1 - lt0) * fr);
    fp.eps = std::exp(le0 + (le1 - le0) * fr);
    if (p_move > 0 && rng.uni() < p_move) {
      const int v = movable[rng.below((uint32_t)movable.size())];
      const double eps_lat = fp.eps * (double)tr.D;
      // 3.2.2, 3.2.3, 3.2.4, 3.2.5, 3.2.6 in equal shares; 3.2.2 on 2 % of the vertices at once
      // in 2 % of the proposals (each costs as much as up to 64 single moves)
      const int kind = rng.uni() < 0.02 ? 5 : (int)rng.below(5);
      // the vertices that move and their new positions
      group.clear();
      newpos.clear();
      bool ok = false;
      Pt q;
      if (kind == 0) {
        ok = mover.propose(tr, vc, v, rng, q);
      } else if (kind == 2) {
        ok = mover.resample(tr, vc, v, rng, q);
      } else if (kind == 3) {
        const double l = eps_lat * (0.2 + 1.8 * rng.uni());
        if (vc.kind[v] == 1 && has_neighbour_within(tr, v, tr.P[v], l)) ok = propose_to_neighbour(tr, vc, v, l, rng, q);
      } else if (kind == 4) {
        // contract an uncontracted vertex onto a random neighbour (within eps of it), or uncontract a
        // contracted one by the resampling of Sec. 3.2.4, kept only if it leaves every neighbour
        if (!has_neighbour_within(tr, v, tr.P[v], eps_lat))
          ok = propose_to_neighbour(tr, vc, v, eps_lat, rng, q) && has_neighbour_within(tr, v, q, eps_lat);
        else
          ok = mover.resample(tr, vc, v, rng, q) && !has_neighbour_within(tr, v, q, eps_lat);
      } else if (kind == 5) {
        ok = propose_many(tr, vc, movable, mover, rng, group, newpos);
      } else if (vc.kind[v] == 1) {
        // the group: free vertices within d of v, found through the triangulation's edges
        const double d = eps_lat * (0.5 + 4.5 * rng.uni()), d2 = d * d;
        group.push_back(v);
        for (size_t g = 0; g < group.size() && group.size() < 64; ++g)
          tr.for_fan(group[g], [&](int t, int kk) {
            const int u = tr.T[t].v[(kk + 1) % 3];
            if (vc.kind[u] == 1 && (double)len2(tr.P[u], tr.P[v]) <= d2 &&
                std::find(group.begin(), group.end(), u) == group.end())
              group.push_back(u);
            return false;
          });
        region.clear();
        for (int u : group) add_star(tr, u, region);
        sort_unique(region);
        double area2 = 0.0;
        for (int t : region) area2 += (double)orient(tr.P[tr.T[t].v[0]], tr.P[tr.T[t].v[1]], tr.P[tr.T[t].v[2]]);
        const double eta = std::sqrt(0.5 * area2), r = std::sqrt(rng.uni()), th = 6.283185307179586 * rng.uni();
        const double step = mover.lambda[1] * eta * r * std::pow(1.0 - rng.uni(), -2.0);
        const int64_t sx = std::llround(step * std::cos(th)), sy = std::llround(step * std::sin(th));
        ok = (sx != 0 || sy != 0) && std::llabs(sx) < tr.D && std::llabs(sy) < tr.D;
        for (int u : group) {
          const Pt pu{(int32_t)(tr.P[u].x + sx), (int32_t)(tr.P[u].y + sy)};
          ok = ok && pu.x > 0 && pu.y > 0 && pu.x < tr.D && pu.y < tr.D;
          newpos.push_back(pu);
        }
      }
      if (group.empty() && ok) {
        group.push_back(v);
        newpos.push_back(q);
      }
      bool acc = false;
      if (ok) {
        group_region(tr, group, region);
        const double e0 = loc.energy(region);
        oldpos.clear();
        for (size_t g = 0; g < group.size(); ++g) {
          oldpos.push_back(tr.P[group[g]]);
          tr.P[group[g]] = newpos[g];
        }
        // every triangle around a moved vertex stays strictly CCW
        bool valid = true;
        for (int u : group)
          valid = valid && !tr.for_fan(u, [&](int t, int) {
            return orient(tr.P[tr.T[t].v[0]], tr.P[tr.T[t].v[1]], tr.P[tr.T[t].v[2]]) <= 0;
          });
        if (valid) {
          const double dlt = loc.energy(region) - e0;
          acc = dlt <= 0.0 || rng.uni() < std::exp(-dlt / temp);
        }
        if (!acc)
          for (size_t g = 0; g < group.size(); ++g) tr.P[group[g]] = oldpos[g];
      }
      if (kind == 0) mover.record(vc.kind[v], acc);
      continue;
    }
    const int t = (int)rng.below((uint32_t)tr.T.size()), i = (int)rng.below(3);
    if (tr.T[t].c[i] >= 0 || tr.T[t].n[i] < 0) continue;
    int x, y;
    if (!tr.strictly_convex(t, i, x, y)) continue;
    const int qv = tr.T[t].v[(i + 1) % 3], rv = tr.T[t].v[(i + 2) % 3];
    region.clear();
    for (int w : {qv, rv, x, y}) add_star(tr, w, region);
    sort_unique(region);
    const double e0 = loc.energy(region);
    tr.flip(t, i);
    const double d = loc.energy(region) - e0;
    if (d <= 0.0 || rng.uni() < std::exp(-d / temp)) continue;
    int t2, i2;
    if (tr.find_edge(x, y, t2, i2)) tr.flip(t2, i2);  // undo: the quadrilateral's other diagonal
  }
}

// Turns the fuzzy topology into a true one (Sec. 3.4): while some contractible edge is shorter than
// eps (unit-square units), the shortest is contracted by a discrete collapse of its less constrained
// endpoint into the other (a free vertex into anything, a segment's Steiner vertex along its segment;
// both directions tried for two free vertices); an edge whose collapse would fold the triangulation is
// skipped (temporarily incontractible).  Returns the number of contractions.
static int64_t contract_short_edges(Triangulation& tr, double eps) {
  int64_t done = 0;
  const double eps_lat = eps * (double)tr.D;
  for (int round = 0; round < 64; ++round) {
    VertexClasses vc;
    classify_vertices(tr, vc);
    std::vector<std::pair<double, std::pair<int, int>>> cand;
    for (int t = 0; t < (int)tr.T.size(); ++t) {
      if (tr.T[t].v[0] < 0) continue;
      for (int i = 0; i < 3; ++i) {
        const int n = tr.T[t].n[i];
        if (n >= 0 && n < t) continue;
        const Tri& x = tr.T[t];
        const int p = x.v[(i + 1) % 3], q = x.v[(i + 2) % 3];
        const double l = std::sqrt((double)len2(tr.P[p], tr.P[q]));
        if (l >= eps_lat || !fuzzy_contractible(tr, vc, eps_lat, t, i)) continue;
        cand.push_back({l, {p, q}});
      }
    }
    if (cand.empty()) break;
    std::sort(cand.begin(), cand.end());
    std::vector<char> touched(tr.P.size(), 0);
    int64_t this_round = 0;
    for (const auto& cd : cand) {
      const int p = cd.second.first, q = cd.second.second;
      if (touched[p] || touched[q] || tr.vtri[p] < 0 || tr.vtri[q] < 0) continue;
      // the vertex that moves: the one with more freedom
      int order[2][2] = {{p, q}, {q, p}};
      int n_try = 0;
      const int kp = vc.kind[p], kq = vc.kind[q];
      int tries[2][2];
      if (kp == 1 && kq == 1) {
        tries[0][0] = p, tries[0][1] = q, tries[1][0] = q, tries[1][1] = p;
        n_try = 2;
      } else if (kp == 1 || (kp == 2 && kq == 0)) {
        tries[0][0] = p, tries[0][1] = q;
        n_try = 1;
      } else if (kq == 1 || (kq == 2 && kp == 0)) {
        tries[0][0] = q, tries[0][1] = p;
        n_try = 1;
      } else if (kp == 2 && kq == 2) {
        tries[0][0] = p, tries[0][1] = q, tries[1][0] = q, tries[1][1] = p;
        n_try = 2;
      }
      (void)order;
      for (int k = 0; k < n_try; ++k) {
        const int v = tries[k][0], u = tries[k][1];
        int t1, t2;
        float dl;
        if (!collapse_delta(tr, v, u, t1, t2, &dl)) continue;
        // mark the neighbourhood: its classification is stale until the next round
        tr.for_fan(v, [&](int t, int kk) {
          for (int s = 0; s < 3; ++s) touched[tr.T[t].v[s]] = 1;
          (void)kk;
          return false;
        });
        do_collapse(tr, v, u, t1, t2);
        ++this_round;
        break;
      }
    }
    done += this_round;
    if (this_round == 0) break;
    compact_dead(tr);  // the next round classifies every vertex: none may be dead
  }
  return done;
}

// ---------------------------------------------------------------- rays
struct SeedGrid {
  int G = 1;
  double cell = 1;
  std::vector<int32_t> tri;
};

static void build_seed_grid(const Triangulation& tr, SeedGrid& sg) {
  int64_t nt = (int64_t)tr.T.size();
  sg.G = std::max(1, std::min(1024, (int)std::sqrt((double)nt / 4.0)));
  sg.cell = (double)tr.D / sg.G;
  sg.tri.assign((size_t)sg.G * sg.G, 0);
  Rng r(99, 1);
  int last = 0;
  for (int j = 0; j < sg.G; ++j)
    for (int ii = 0; ii < sg.G; ++ii) {
      int i = (j & 1) ? sg.G - 1 - ii : ii;  // boustrophedon keeps walks short
      Pt c{(int32_t)((i + 0.5) * sg.cell), (int32_t)((j + 0.5) * sg.cell)};
      int t = tr.locate(c, last, r);
      if (t < 0) t = last;
      sg.tri[(size_t)j * sg.G + i] = t;
      last = t;
    }
}

// Locate p; returns the triangle containing p strictly inside, or -1 if p lies
// on an edge or a vertex.
static int locate_strict(const Triangulation& tr, const SeedGrid& sg, const Pt& p, Rng& r) {
  int i = std::clamp((int)(p.x / sg.cell), 0, sg.G - 1), j = std::clamp((int)(p.y / sg.cell), 0, sg.G - 1);
  int t = tr.locate(p, sg.tri[(size_t)j * sg.G + i], r);
  if (t < 0) return -1;
  const Tri& x = tr.T[t];
  for (int e = 0; e < 3; ++e)
    if (orient(tr.P[x.v[(e + 1) % 3]], tr.P[x.v[(e + 2) % 3]], p) == 0) return -1;
  return t;
}

static inline float dir_on_grid(double c) {
  // round to a multiple of 2^-22 (exact in fp32)
  return (float)(std::nearbyint(c * 4194304.0) / 4194304.0);
}

template <class F>
static void parallel_for(int64_t n, int n_threads, F f) {
  if (n_threads <= 1 || n < 4096) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + n_threads - 1) / n_threads;
  for (int k = 0; k < n_threads; ++k) {
    int64_t lo = k * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([=]() { f(lo, hi); });
  }
  for (auto& x : th) x.join();
}

// ---------------------------------------------------------------- quality refinement (Sec. 3.5.1)
// The paper starts from a quality CDT (Shewchuk's Triangle) whose minimum-angle
// and maximum-area bounds are chosen, by brute force, to give the shortest
// total edge length.  This is a Delaunay refinement of our own on the integer
// grid: a triangle is bad if its smallest angle is below min_angle or its area
// above max_area; its circumcentre, rounded to the grid, is inserted; a
// constrained edge whose diametral circle holds that point is split at its
// midpoint instead, when the midpoint is a lattice point (otherwise the
// triangle is left as it is).  Insertions are capped.  Circumcentres are
// constructed in fp64 and rounded; every predicate stays exact.
static double smallest_angle_cos(const Pt& a, const Pt& b, const Pt& c) {
  const double la = (double)len2(b, c), lb = (double)len2(c, a), lc = (double)len2(a, b);
  // the smallest angle is opposite the shortest side
  double s, u, v;
  if (la <= lb && la <= lc) {
    s = la; u = lb; v = lc;
  } else if (lb <= la && lb <= lc) {
    s = lb; u = la; v = lc;
  } else {
    s = lc; u = la; v = lb;
  }
  return (u + v - s) / (2.0 * std::sqrt(u * v));
}

static bool circumcentre(const Pt& a, const Pt& b, const Pt& c, Pt& out) {
  const double bx = (double)b.x - a.x, by = (double)b.y - a.y, cx = (double)c.x - a.x, cy = (double)c.y - a.y;
  const double d = 2.0 * (bx * cy - by * cx);
  if (d == 0.0) return false;
  const double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
  const double ux = (cy * b2 - by * c2) / d, uy = (bx * c2 - cx * b2) / d;
  const double X = a.x + ux, Y = a.y + uy;
  if (!(X > -1e12 && X < 1e12 && Y > -1e12 && Y < 1e12)) return false;
  out = Pt{(int32_t)std::llround(X), (int32_t)std::llround(Y)};
  return true;
}

static int64_t refine(Triangulation& tr, double min_angle_deg, double max_area, int64_t max_insert) {
  const double cos_min = min_angle_deg > 0 ? std::cos(min_angle_deg * 3.141592653589793 / 180.0) : 2.0;
  const int32_t D = tr.D;
  auto bad = [&](int t) {
    const Tri& x = tr.T[t];
    const Pt &a = tr.P[x.v[0]], &b = tr.P[x.v[1]], &c = tr.P[x.v[2]];
    if (max_area > 0 && 0.5 * (double)orient(a, b, c) > max_area) return true;
    if (cos_min < 1.5 && smallest_angle_cos(a, b, c) > cos_min) return true;
    return false;
  };
  auto key = [&](int t) {
    int v[3] = {tr.T[t].v[0], tr.T[t].v[1], tr.T[t].v[2]};
    std::sort(v, v + 3);
    return ((uint64_t)(uint32_t)v[0] * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)(uint32_t)v[1] << 21) ^ (uint64_t)v[2];
  };
  std::unordered_map<uint64_t, char> tried;
  std::vector<int> work;
  for (int t = 0; t < (int)tr.T.size(); ++t) work.push_back(t);
  int64_t inserted = 0;
  auto push_fan = [&](int v) {
    tr.for_fan(v, [&](int t, int) {
      work.push_back(t);
      return false;
    });
  };
  while (!work.empty() && inserted < max_insert && tr.status == 0) {
    const int t = work.back();
    work.pop_back();
    if (t >= (int)tr.T.size() || !bad(t)) continue;
    const uint64_t k = key(t);
    if (tried.count(k)) continue;
    tried[k] = 1;
    const Tri x = tr.T[t];
    Pt c;
    if (!circumcentre(tr.P[x.v[0]], tr.P[x.v[1]], tr.P[x.v[2]], c)) continue;
    if (c.x <= 0 || c.y <= 0 || c.x >= D || c.y >= D) continue;  // the hull is not split
    const int loc = tr.locate(c, t, tr.rng);
    if (loc < 0) continue;
    // a constrained edge of the containing triangle that c encroaches is split
    // at its midpoint (a lattice point) instead
    bool handled = false;
    for (int e = 0; e < 3 && !handled; ++e) {
      if (tr.T[loc].c[e] < 0) continue;
      const Pt& p = tr.P[tr.T[loc].v[(e + 1) % 3]];
      const Pt& q = tr.P[tr.T[loc].v[(e + 2) % 3]];
      const int64_t dot = (int64_t)(p.x - c.x) * (q.x - c.x) + (int64_t)(p.y - c.y) * (q.y - c.y);
      if (dot > 0) continue;
      handled = true;
      if (((p.x + q.x) & 1) || ((p.y + q.y) & 1)) break;  // no lattice midpoint: leave it
      const Pt m{(p.x + q.x) / 2, (p.y + q.y) / 2};
      tr.last = loc;
      const size_t nv = tr.P.size();
      const int v = tr.insert_point(m);
      if (v >= 0 && (size_t)v >= nv) {
        ++inserted;
        push_fan(v);
      }
    }
    if (handled) continue;
    tr.last = loc;
    const size_t nv = tr.P.size();
    const int v = tr.insert_point(c);
    if (v >= 0 && (size_t)v >= nv) {
      ++inserted;
      push_fan(v);
    }
  }
  return inserted;
}

// ---------------------------------------------------------------- BVH (Sec. 5.3.1)
// Greedy top-down 2D SAH ("perimeter heuristic"): for both axes, sort the
// segments by centroid and try every split k; cost(split) = 2 alpha +
// (P_L N_L + P_R N_R) / P (alpha = cost of an AABB test relative to a segment
// test, P = box perimeter); stop when that is not below the leaf cost N.
struct BvhBuild {
  const int32_t* seg;
  float alpha;
  int max_depth = 60;
  std::vector<int32_t> box, c0, c1, prims;

  void seg_box(int s, int32_t b[4]) const {
    const int32_t* q = seg + 4 * s;
    b[0] = std::min(q[0], q[2]);
    b[1] = std::min(q[1], q[3]);
    b[2] = std::max(q[0], q[2]);
    b[3] = std::max(q[1], q[3]);
  }
  static float perim(const int32_t b[4]) { return 2.0f * ((float)(b[2] - b[0]) + (float)(b[3] - b[1])); }
  static void grow(int32_t b[4], const int32_t o[4]) {
    b[0] = std::min(b[0], o[0]);
    b[1] = std::min(b[1], o[1]);
    b[2] = std::max(b[2], o[2]);
    b[3] = std::max(b[3], o[3]);
  }
  int build(std::vector<int32_t>& ids, int lo, int hi, int depth) {
    const int node = (int)c0.size();
    c0.push_back(0);
    c1.push_back(0);
    int32_t nb[4] = {INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN};
    for (int k = lo; k < hi; ++k) {
      int32_t b[4];
      seg_box(ids[k], b);
      grow(nb, b);
    }
    for (int q = 0; q < 4; ++q) box.push_back(nb[q]);
    const int n = hi - lo;
    const float P = perim(nb);
    float best = (float)n;
    int best_axis = -1, best_k = 0;
    if (n > 1 && depth < max_depth && P > 0.f) {
      std::vector<float> left(n);
      for (int axis = 0; axis < 2; ++axis) {
        std::sort(ids.begin() + lo, ids.begin() + hi, [&](int a, int b) {
          const int64_t ca = (int64_t)seg[4 * a + axis] + seg[4 * a + 2 + axis];
          const int64_t cb = (int64_t)seg[4 * b + axis] + seg[4 * b + 2 + axis];
          return ca < cb || (ca == cb && a < b);
        });
        int32_t acc[4] = {INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN};
        for (int k = 0; k < n; ++k) {
          int32_t b[4];
          seg_box(ids[lo + k], b);
          grow(acc, b);
          left[k] = perim(acc);
        }
        int32_t rb[4] = {INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN};
        for (int k = n - 1; k >= 1; --k) {
          int32_t b[4];
          seg_box(ids[lo + k], b);
          grow(rb, b);
          const float cost = 2.0f * alpha + (left[k - 1] * (float)k + perim(rb) * (float)(n - k)) / P;
          if (cost < best) {
            best = cost;
            best_axis = axis;
            best_k = k;
          }
        }
      }
    }
    if (best_axis < 0) {
      c0[node] = -1 - (int32_t)prims.size();
      c1[node] = n;
      for (int k = lo; k < hi; ++k) prims.push_back(ids[k]);
      return node;
    }
    const int axis = best_axis;
    std::sort(ids.begin() + lo, ids.begin() + hi, [&](int a, int b) {
      const int64_t ca = (int64_t)seg[4 * a + axis] + seg[4 * a + 2 + axis];
      const int64_t cb = (int64_t)seg[4 * b + axis] + seg[4 * b + 2 + axis];
      return ca < cb || (ca == cb && a < b);
    });
    const int l = build(ids, lo, lo + best_k, depth + 1);
    const int r = build(ids, lo + best_k, hi, depth + 1);
    c0[node] = l;
    c1[node] = r;
    return node;
  }
};

// ---------------------------------------------------------------- roped kd-tree (Sec. 5.3.2)
// Greedy top-down 2D SAH; candidate planes at every segment-endpoint
// coordinate strictly inside the node (both axes); cost(split) = lambda +
// (P_L N_L + P_R N_R) / P, leaf when not below N.  A segment belongs to every
// node whose closed box it touches.  Leaves get ropes (one per face) to the
// deepest node that contains the whole region across that face, and the count
// of leaves adjacent across the face (for the paper's ideal log2 rope cost).
static bool seg_hits_box(const int32_t* q, int64_t x0, int64_t y0, int64_t x1, int64_t y1) {
  const int64_t ax = q[0], ay = q[1], bx = q[2], by = q[3];
  if (std::max(ax, bx) < x0 || std::min(ax, bx) > x1 || std::max(ay, by) < y0 || std::min(ay, by) > y1) return false;
  if ((ax >= x0 && ax <= x1 && ay >= y0 && ay <= y1) || (bx >= x0 && bx <= x1 && by >= y0 && by <= y1)) return true;
  const int64_t cx[4] = {x0, x1, x1, x0}, cy[4] = {y0, y0, y1, y1};
  int pos = 0, neg = 0;
  for (int k = 0; k < 4; ++k) {
    const int64_t o = (bx - ax) * (cy[k] - ay) - (by - ay) * (cx[k] - ax);
    if (o > 0) ++pos;
    if (o < 0) ++neg;
  }
  return !(pos == 4 || neg == 4);
}

struct KdBuild {
  const int32_t* seg;
  float lambda;
  int max_depth = 40;
  std::vector<int32_t> axis, split, child, count, box, rope, rope_log2, refs;

  int new_node(const int64_t b[4]) {
    const int id = (int)axis.size();
    axis.push_back(2);
    split.push_back(0);
    child.push_back(-1);
    count.push_back(0);
    for (int k = 0; k < 4; ++k) box.push_back((int32_t)b[k]);
    for (int k = 0; k < 4; ++k) rope.push_back(-1);
    for (int k = 0; k < 4; ++k) rope_log2.push_back(0);
    return id;
  }

  void build(int node, std::vector<int32_t>& ids, int depth) {
    const int64_t b[4] = {box[4 * node], box[4 * node + 1], box[4 * node + 2], box[4 * node + 3]};
    const int n = (int)ids.size();
    const float P = 2.0f * ((float)(b[2] - b[0]) + (float)(b[3] - b[1]));
    float best = (float)n;
    int best_axis = -1;
    int64_t best_s = 0;
    if (n > 0 && depth < max_depth && P > 0.f) {
      std::vector<int64_t> lo(n), hi(n), cand;
      for (int a = 0; a < 2; ++a) {
        cand.clear();
        for (int k = 0; k < n; ++k) {
          const int32_t* q = seg + 4 * ids[k];
          const int64_t e0 = q[a], e1 = q[2 + a];
          lo[k] = std::max(std::min(e0, e1), b[a]);
          hi[k] = std::min(std::max(e0, e1), b[2 + a]);
          if (e0 > b[a] && e0 < b[2 + a]) cand.push_back(e0);
          if (e1 > b[a] && e1 < b[2 + a]) cand.push_back(e1);
        }
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        std::vector<int64_t> ls = lo, hs = hi;
        std::sort(ls.begin(), ls.end());
        std::sort(hs.begin(), hs.end());
        const float ext_other = (float)(b[3 - a] - b[1 - a]);
        for (int64_t sp : cand) {
          const int nl = (int)(std::lower_bound(ls.begin(), ls.end(), sp) - ls.begin());       // lo < sp
          const int nr = n - (int)(std::upper_bound(hs.begin(), hs.end(), sp) - hs.begin());  // hi > sp
          const float pl = 2.0f * ((float)(sp - b[a]) + ext_other);
          const float pr = 2.0f * ((float)(b[2 + a] - sp) + ext_other);
          const float cost = lambda + (pl * (float)nl + pr * (float)nr) / P;
          if (cost < best) {
            best = cost;
            best_axis = a;
            best_s = sp;
          }
        }
      }
    }
    if (best_axis < 0) {
      axis[node] = 2;
      child[node] = (int32_t)refs.size();
      count[node] = n;
      for (int32_t s : ids) refs.push_back(s);
      return;
    }
    int64_t lb[4] = {b[0], b[1], b[2], b[3]}, rb[4] = {b[0], b[1], b[2], b[3]};
    lb[2 + best_axis] = best_s;
    rb[best_axis] = best_s;
    std::vector<int32_t> lids, rids;
    for (int32_t s : ids) {
      if (seg_hits_box(seg + 4 * s, lb[0], lb[1], lb[2], lb[3])) lids.push_back(s);
      if (seg_hits_box(seg + 4 * s, rb[0], rb[1], rb[2], rb[3])) rids.push_back(s);
    }
    ids.clear();
    ids.shrink_to_fit();
    const int l = new_node(lb);
    const int r = new_node(rb);
    axis[node] = best_axis;
    split[node] = (int32_t)best_s;
    child[node] = l;
    (void)r;  // right child = left + 1
    build(l, lids, depth + 1);
    build(r, rids, depth + 1);
  }

  // faces: 0 x-min, 1 x-max, 2 y-min, 3 y-max
  void ropes(int node, const int32_t in[4]) {
    if (axis[node] == 2) {
      for (int f = 0; f < 4; ++f) {
        int32_t r = optimise(node, f, in[f]);
        rope[4 * node + f] = r;
        int cnt = r < 0 ? 0 : adjacent_leaves(node, f, r);
        int lg = 0;
        while ((1 << lg) < cnt) ++lg;
        rope_log2[4 * node + f] = lg;
      }
      return;
    }
    const int a = axis[node], l = child[node], r = l + 1;
    int32_t rl[4] = {in[0], in[1], in[2], in[3]}, rr[4] = {in[0], in[1], in[2], in[3]};
    rl[2 * a + 1] = r;  // left child's max face on the split axis
    rr[2 * a] = l;      // right child's min face
    ropes(l, rl);
    ropes(r, rr);
  }
  int32_t optimise(int leaf, int f, int32_t N) const {
    if (N < 0) return N;
    const int fa = f / 2;  // axis normal to the face
    const bool fmax = (f & 1) != 0;
    const int32_t* lb = &box[4 * leaf];
    const int32_t plane = fmax ? lb[2 + fa] : lb[fa];
    const int32_t f0 = lb[1 - fa], f1 = lb[3 - fa];  // face extent on the other axis
    while (axis[N] != 2) {
      const int a = axis[N];
      const int32_t sp = split[N];
      const int l = child[N];
      if (a == fa) {
        if (fmax)
          N = (sp > plane) ? l : l + 1;
        else
          N = (sp >= plane) ? l : l + 1;
      } else {
        if (sp <= f0)
          N = l + 1;
        else if (sp >= f1)
          N = l;
        else
          break;
      }
    }
    return N;
  }
  int adjacent_leaves(int leaf, int f, int32_t N) const {
    const int fa = f / 2;
    const bool fmax = (f & 1) != 0;
    const int32_t* lb = &box[4 * leaf];
    const int32_t plane = fmax ? lb[2 + fa] : lb[fa];
    const int32_t f0 = lb[1 - fa], f1 = lb[3 - fa];
    int cnt = 0;
    std::vector<int32_t> st{N};
    while (!st.empty()) {
      const int32_t x = st.back();
      st.pop_back();
      const int32_t* xb = &box[4 * x];
      const int32_t o0 = std::max(f0, xb[1 - fa]), o1 = std::min(f1, xb[3 - fa]);
      if (o1 <= o0) continue;  // touches the face in a point at most
      // the node must reach the face's plane: cells beyond a split on the
      // face's own axis are not adjacent across the face
      if (fmax ? xb[fa] != plane : xb[2 + fa] != plane) continue;
      if (axis[x] == 2) {
        ++cnt;
      } else {
        st.push_back(child[x]);
        st.push_back(child[x] + 1);
      }
    }
    return std::max(1, cnt);
  }
};

}  // namespace

// =============================================================== C ABI
extern "C" {

// Config-1 style random disjoint segments.  Lengths are uniform in
// [len_lo, len_hi]*D*scale; returns the number written (<= n).
int64_t sg_gen_random_segments(int64_t n, uint64_t seed, int32_t D, double len_lo, double len_hi, double scale,
                               double margin, int32_t* out, int64_t cap) {
  return gen_segments(n, seed, D, len_lo, len_hi, scale, margin, 0, 0.0, out, cap);
}

// Random disjoint segments whose centres come from n_clusters Gaussian clusters
// of standard deviation sigma*D.
int64_t sg_gen_clustered(int64_t n, uint64_t seed, int32_t D, double len_lo, double len_hi, double scale,
                         int32_t n_clusters, double sigma, int32_t* out, int64_t cap) {
  return gen_segments(n, seed, D, len_lo, len_hi, scale, 0.01, n_clusters, sigma, out, cap);
}

// The `lines' scenes of Sec. 4.2: n pairwise-disjoint segments of one length,
// min(0.95, factor * 0.95 / sqrt(n)) * D, centres uniform, endpoints at least
// margin * D from the border; orientation 0 = uniform in [0, pi), 1 = mostly
// vertical (90 degrees + a normal spread), 2 = mostly diagonal (45 degrees +
// a normal spread), spread in degrees.  Dense scenes may hold fewer than n:
// returns the number written.
int64_t sg_gen_lines(int64_t n, uint64_t seed, int32_t D, double factor, int32_t orientation, double spread_deg,
                     double margin, int32_t* out, int64_t cap) {
  Rng rng(seed, 0x11E5);
  const double L = std::min(0.95, factor * 0.95 / std::sqrt((double)std::max<int64_t>(1, n))) * D;
  SegGrid grid(D, std::max(L, (double)D / 4096.0));
  const double lo = margin * D, hi = (1.0 - margin) * D;
  const double deg = 3.141592653589793 / 180.0;
  int64_t cnt = 0, tries = 0;
  const int64_t max_tries = std::max<int64_t>(2000 * n, 100000);
  while (cnt < n && cnt < cap && tries < max_tries) {
    ++tries;
    double th;
    if (orientation == 1)
      th = (90.0 + spread_deg * rng.normal()) * deg;
    else if (orientation == 2)
      th = (45.0 + spread_deg * rng.normal()) * deg;
    else
      th = 3.141592653589793 * rng.uni();
    const double hx = 0.5 * L * std::cos(th), hy = 0.5 * L * std::sin(th);
    const double cx = lo + std::fabs(hx) + (hi - lo - 2 * std::fabs(hx)) * rng.uni();
    const double cy = lo + std::fabs(hy) + (hi - lo - 2 * std::fabs(hy)) * rng.uni();
    Pt a{rnd_coord(cx - hx), rnd_coord(cy - hy)}, b{rnd_coord(cx + hx), rnd_coord(cy + hy)};
    if (a == b) continue;
    if (a.x < lo || a.x > hi || a.y < lo || a.y > hi || b.x < lo || b.x > hi || b.y < lo || b.y > hi) continue;
    if (grid.touches(a, b)) continue;
    grid.add(a, b);
    out[4 * cnt + 0] = a.x;
    out[4 * cnt + 1] = a.y;
    out[4 * cnt + 2] = b.x;
    out[4 * cnt + 3] = b.y;
    ++cnt;
  }
  return cnt;
}

// Disjoint polygonal circles with sides uniform in [min_sides, max_sides],
// until about n_target segments.  Fill: the discs cover about 30% of the domain.
int64_t sg_gen_circles(int64_t n_target, uint64_t seed, int32_t D, int32_t min_sides, int32_t max_sides,
                       int32_t* out, int64_t cap) {
  Rng rng(seed, 0xC1C);
  double mean_sides = 0.5 * (min_sides + max_sides);
  double k_est = std::max(1.0, (double)n_target / mean_sides);
  double r_mean = D * std::sqrt(0.30 / (3.141592653589793 * k_est));
  std::vector<double> cx, cy, cr;
  std::vector<Pt> poly;
  int64_t cnt = 0;
  int64_t tries = 0;
  while (cnt < n_target && tries < 2000000) {
    ++tries;
    int m = min_sides + (int)rng.below((uint32_t)(max_sides - min_sides + 1));
    if (cnt + m > cap) break;
    double r = r_mean * (0.6 + 0.8 * rng.uni());
    double minr = 16.0 * m / 6.283185307179586;  // side >= 16 grid units
    if (tries > 200000) r *= 0.5;
    if (r < minr) r = minr;
    double x = r + 0.01 * D + (D - 2 * r - 0.02 * D) * rng.uni();
    double y = r + 0.01 * D + (D - 2 * r - 0.02 * D) * rng.uni();
    if (x - r < 0.01 * D || y - r < 0.01 * D || x + r > 0.99 * D || y + r > 0.99 * D) continue;
    bool ok = true;
    for (size_t k = 0; k < cx.size() && ok; ++k) {
      double dd = std::hypot(x - cx[k], y - cy[k]);
      if (dd < (r + cr[k]) * 1.02 + 4.0) ok = false;
    }
    if (!ok) continue;
    if (!polygon(x, y, r, m, 6.283185307179586 * rng.uni(), poly)) continue;
    cx.push_back(x);
    cy.push_back(y);
    cr.push_back(r);
    cnt = emit_polygon(poly, out, cnt, cap);
  }
  return cnt;
}

// Regular lattice of disjoint dashes (length 0.7 * pitch), horizontal and
// vertical in a checkerboard, rotated by theta_deg about the domain centre and
// clipped to the domain; about n_target dashes.
int64_t sg_gen_dash_grid(int64_t n_target, double theta_deg, int32_t D, int32_t* out, int64_t cap) {
  double side = std::sqrt((double)n_target);
  double pitch = 0.96 * D / side;
  double th = theta_deg * 3.141592653589793 / 180.0;
  double c = std::cos(th), s = std::sin(th);
  double h = 0.35 * pitch, lo = 0.01 * D, hi = 0.99 * D;
  int64_t cnt = 0;
  int R = (int)std::ceil(side * 0.75) + 2;
  for (int j = -R; j <= R; ++j)
    for (int i = -R; i <= R; ++i) {
      double lx = (i + 0.5) * pitch, ly = (j + 0.5) * pitch;
      bool horiz = ((i + j) & 1) == 0;
      double ax = lx - (horiz ? h : 0), ay = ly - (horiz ? 0 : h);
      double bx = lx + (horiz ? h : 0), by = ly + (horiz ? 0 : h);
      double X0 = 0.5 * D + c * ax - s * ay, Y0 = 0.5 * D + s * ax + c * ay;
      double X1 = 0.5 * D + c * bx - s * by, Y1 = 0.5 * D + s * bx + c * by;
      if (X0 < lo || X0 > hi || Y0 < lo || Y0 > hi || X1 < lo || X1 > hi || Y1 < lo || Y1 > hi) continue;
      if (cnt >= cap) return cnt;
      out[4 * cnt + 0] = rnd_coord(X0);
      out[4 * cnt + 1] = rnd_coord(Y0);
      out[4 * cnt + 2] = rnd_coord(X1);
      out[4 * cnt + 3] = rnd_coord(Y1);
      ++cnt;
    }
  return cnt;
}

// A ring of M polygonal circles in a fixed domain, n_target sides in total.
int64_t sg_gen_ring_of_circles(int64_t n_target, int32_t D, int32_t* out, int64_t cap) {
  int M = std::max(8, (int)std::lround(std::sqrt((double)n_target) / 4.0));
  int m = (int)std::max<int64_t>(3, n_target / M);
  // ring radius R and circle radius rc = 0.95 pi R / M (neighbours never touch),
  // with R + rc = 0.49 D so every circle stays inside the domain
  double R = 0.49 * D / (1.0 + 0.95 * 3.141592653589793 / M);
  double rc = 0.95 * 3.141592653589793 * R / M;
  std::vector<Pt> poly;
  int64_t cnt = 0;
  for (int k = 0; k < M; ++k) {
    double a = 6.283185307179586 * k / M;
    if (!polygon(0.5 * D + R * std::cos(a), 0.5 * D + R * std::sin(a), rc, m, 0.1 * k, poly)) return -1;
    cnt = emit_polygon(poly, out, cnt, cap);
  }
  return cnt;
}

// Constrained Delaunay triangulation of the segments (4 int32 per segment:
// x0 y0 x1 y1) inside the square [0,D]^2.  Segment s becomes constrained edges
// labelled s.  *status < 0 on failure (crossing or overlapping segments, point
// outside the domain).
void* sg_cdt_build(int64_t n_seg, const int32_t* seg, int32_t D, int32_t* status) {
  Triangulation* t = build_cdt(n_seg, seg, D);
  *status = t->status;
  return t;
}

// Import an arbitrary triangulation (same array conventions as the export).
void* sg_tri_import(int32_t D, int64_t n_vert, const int32_t* vx, const int32_t* vy, int64_t n_tri,
                    const int32_t* tri_v, const int32_t* tri_nb, const int32_t* tri_seg) {
  auto* tr = new Triangulation();
  tr->D = D;
  tr->P.resize(n_vert);
  tr->vtri.assign(n_vert, 0);
  for (int64_t v = 0; v < n_vert; ++v) tr->P[v] = Pt{vx[v], vy[v]};
  tr->T.resize(n_tri);
  for (int64_t t = 0; t < n_tri; ++t)
    for (int k = 0; k < 3; ++k) {
      tr->T[t].v[k] = tri_v[3 * t + k];
      tr->T[t].n[k] = tri_nb[3 * t + k];
      tr->T[t].c[k] = tri_seg[3 * t + k];
      tr->vtri[tri_v[3 * t + k]] = (int32_t)t;
    }
  return tr;
}

void* sg_tri_copy(void* h) { return new Triangulation(*(Triangulation*)h); }

void sg_tri_free(void* h) { delete (Triangulation*)h; }

int32_t sg_tri_status(void* h) { return ((Triangulation*)h)->status; }

void sg_tri_sizes(void* h, int64_t* n_vert, int64_t* n_tri) {
  auto* t = (Triangulation*)h;
  *n_vert = (int64_t)t->P.size();
  *n_tri = (int64_t)t->T.size();
}

void sg_tri_export(void* h, int32_t* vx, int32_t* vy, int32_t* tri_v, int32_t* tri_nb, int32_t* tri_seg) {
  auto* t = (Triangulation*)h;
  for (size_t v = 0; v < t->P.size(); ++v) {
    vx[v] = t->P[v].x;
    vy[v] = t->P[v].y;
  }
  for (size_t k = 0; k < t->T.size(); ++k)
    for (int i = 0; i < 3; ++i) {
      tri_v[3 * k + i] = t->T[k].v[i];
      tri_nb[3 * k + i] = t->T[k].n[i];
      tri_seg[3 * k + i] = t->T[k].c[i];
    }
}

// Total edge length (fp32, compensated sum); interior_only skips hull edges.
float sg_tri_length(void* h, int32_t interior_only) {
  return (float)((Triangulation*)h)->total_length(interior_only != 0);
}

// Anneal in place: greedy flips, then simulated annealing (over flips, and
// vertex perturbations with weight `moves`, see anneal_flips) from temperature
// T0 to T1 (grid units) for `sweeps` proposals per half-edge, then greedy
// flips again.  Keeps whichever of (greedy-only, annealed) is shorter.
// Returns the number of greedy flips of the kept result.
// The fuzzy objective of Sec. 2.2 (see fuzzy_objective): terms = {f, W_contr, Pi_angle, Pi_len};
// w (optional, 3 per triangle) = each edge's weight.
void sg_fuzzy_objective(void* h, double eps, double delta, double eps0, double mu_angle, double mu_len,
                        int32_t polish, double* terms, double* w) {
  FuzzyParams fp{eps, delta, eps0, mu_angle, mu_len, polish};
  fuzzy_objective(*(Triangulation*)h, fp, terms, w);
}

// Fuzzy annealing (anneal_fuzzy) followed by the contraction of edges shorter than eps_b
// (contract_short_edges); returns the number of contractions.
int64_t sg_anneal_fuzzy(void* h, uint64_t seed, double sweeps, double T0, double T1, double eps_a, double eps_b,
                        double moves) {
  auto* tr = (Triangulation*)h;
  anneal_fuzzy(*tr, seed, sweeps, T0, T1, eps_a, eps_b, moves);
  return contract_short_edges(*tr, eps_b);
}

// Contraction alone (contract_short_edges).
int64_t sg_contract_short_edges(void* h, double eps) { return contract_short_edges(*(Triangulation*)h, eps); }

// Check of the fuzzy annealer's local energy change (for tests): n multi-vertex perturbations
// (propose_many) on a copy of the triangulation at contraction length eps, the region tables
// starting at 2^init_bits slots; for every proposal that keeps the triangulation valid, the
// region's energy change (what the annealer decides on) is compared with the change of the whole
// fuzzy objective.  Half of the proposals are kept, so the state moves.  lambda = the vertex
// move's step factor (the annealer adapts it; small steps keep most proposals valid).  Returns the
// number of proposals compared; *max_err = the largest |local - whole| difference, *grows = table
// growths.
int64_t sg_fuzzy_check_group_deltas(void* h, uint64_t seed, int64_t n, double eps, int32_t init_bits,
                                    double lambda, double* max_err, int64_t* grows) {
  Triangulation tr = *(Triangulation*)h;
  Rng rng(seed, 0xC4EC);
  VertexClasses vc;
  classify_vertices(tr, vc);
  std::vector<int32_t> movable;
  for (int v = 0; v < (int)vc.kind.size(); ++v)
    if (vc.kind[v]) movable.push_back(v);
  FuzzyParams fp{eps, 1.0 + std::cos(179.0 * 3.14159265358979323846 / 180.0), 1e-10, 1.0, 10.0, 0};
  FuzzyLocal loc(tr, vc, fp, init_bits);
  VertexMover mover;
  mover.lambda[1] = mover.lambda[2] = lambda;
  std::vector<int> group, region;
  std::vector<Pt> newpos, oldpos;
  double worst = 0.0, f0[4], f1[4];
  int64_t compared = 0;
  for (int64_t k = 0; k < n && !movable.empty(); ++k) {
    group.clear();
    newpos.clear();
    if (!propose_many(tr, vc, movable, mover, rng, group, newpos)) continue;
    group_region(tr, group, region);
    const double e0 = loc.energy(region);
    fuzzy_objective(tr, fp, f0, nullptr);
    oldpos.clear();
    for (size_t g = 0; g < group.size(); ++g) {
      oldpos.push_back(tr.P[group[g]]);
      tr.P[group[g]] = newpos[g];
    }
    bool valid = true;
    for (int u : group)
      valid = valid && !tr.for_fan(u, [&](int t, int) {
        return orient(tr.P[tr.T[t].v[0]], tr.P[tr.T[t].v[1]], tr.P[tr.T[t].v[2]]) <= 0;
      });
    if (valid) {
      const double local = loc.energy(region) - e0;
      fuzzy_objective(tr, fp, f1, nullptr);
      worst = std::max(worst, std::fabs(local - (f1[0] - f0[0])));
      ++compared;
    }
    if (!valid || rng.uni() < 0.5)
      for (size_t g = 0; g < group.size(); ++g) tr.P[group[g]] = oldpos[g];
  }
  *max_err = worst;
  *grows = loc.grows;
  return compared;
}

int64_t sg_anneal(void* h, uint64_t seed, double sweeps, double T0, double T1, double moves, double collapse) {
  auto* tr = (Triangulation*)h;
  Triangulation g = *tr;
  int64_t f0 = greedy_flips(g);
  float lg = (float)g.total_length(false);
  anneal_flips(*tr, seed, sweeps, T0, T1, moves, collapse);
  int64_t f1 = greedy_flips(*tr);
  float la = (float)tr->total_length(false);
  if (la > lg) {
    *tr = g;
    return f0;
  }
  return f1;
}

// n isotropic rays: origins uniform on the integer grid strictly inside a
// triangle (rejection of points on edges and vertices), directions uniform in
// angle with components rounded to multiples of 2^-22; start = the triangle
// containing the origin (export numbering).  Ray k depends only on (seed, k).
int64_t sg_rays_isotropic(void* h, int64_t n, uint64_t seed, int32_t* ox, int32_t* oy, float* dx, float* dy,
                          int32_t* start, int32_t n_threads) {
  auto* tr = (Triangulation*)h;
  SeedGrid sg;
  build_seed_grid(*tr, sg);
  int32_t D = tr->D;
  parallel_for(n, n_threads, [&](int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi; ++k) {
      Rng r(seed, (uint64_t)k);
      while (true) {
        Pt p{1 + (int32_t)r.below((uint32_t)(D - 1)), 1 + (int32_t)r.below((uint32_t)(D - 1))};
        int t = locate_strict(*tr, sg, p, r);
        if (t < 0) continue;
        double th = 6.283185307179586 * r.uni();
        ox[k] = p.x;
        oy[k] = p.y;
        dx[k] = dir_on_grid(std::cos(th));
        dy[k] = dir_on_grid(std::sin(th));
        start[k] = t;
        break;
      }
    }
  });
  return n;
}

// Pinhole fans: n_eyes eye points (uniform, strictly inside a triangle), each
// with rays_per_eye rays evenly spaced over fov_deg around a uniform central
// direction.  Ray k belongs to eye k / rays_per_eye.
int64_t sg_rays_pinhole(void* h, int64_t n_eyes, int64_t rays_per_eye, double fov_deg, uint64_t seed,
                        int32_t* ox, int32_t* oy, float* dx, float* dy, int32_t* start, int32_t n_threads) {
  auto* tr = (Triangulation*)h;
  SeedGrid sg;
  build_seed_grid(*tr, sg);
  int32_t D = tr->D;
  double fov = fov_deg * 3.141592653589793 / 180.0;
  parallel_for(n_eyes, n_threads, [&](int64_t lo, int64_t hi) {
    for (int64_t e = lo; e < hi; ++e) {
      Rng r(seed, (uint64_t)e);
      Pt p;
      int t;
      while (true) {
        p = Pt{1 + (int32_t)r.below((uint32_t)(D - 1)), 1 + (int32_t)r.below((uint32_t)(D - 1))};
        t = locate_strict(*tr, sg, p, r);
        if (t >= 0) break;
      }
      double phi = 6.283185307179586 * r.uni();
      for (int64_t j = 0; j < rays_per_eye; ++j) {
        int64_t k = e * rays_per_eye + j;
        double th = phi - 0.5 * fov + fov * ((double)j + 0.5) / (double)rays_per_eye;
        ox[k] = p.x;
        oy[k] = p.y;
        dx[k] = dir_on_grid(std::cos(th));
        dy[k] = dir_on_grid(std::sin(th));
        start[k] = t;
      }
    }
  });
  return n_eyes * rays_per_eye;
}

}  // extern "C"

// ---------------------------------------------------------------- baselines
extern "C" {

// SAH BVH over the segments (4 int32 each).  alpha = AABB-test cost relative to a
// segment test.  Returns a handle; sizes via sg_bvh_sizes, arrays via sg_bvh_export.
void* sg_bvh_build(int64_t n_seg, const int32_t* seg, float alpha) {
  auto* b = new BvhBuild();
  b->seg = seg;
  b->alpha = alpha;
  std::vector<int32_t> ids(n_seg);
  for (int64_t k = 0; k < n_seg; ++k) ids[k] = (int32_t)k;
  if (n_seg > 0)
    b->build(ids, 0, (int)n_seg, 0);
  else {
    b->c0.push_back(-1);
    b->c1.push_back(0);
    for (int q = 0; q < 4; ++q) b->box.push_back(0);
  }
  b->seg = nullptr;
  return b;
}
void sg_bvh_sizes(void* h, int64_t* n_nodes, int64_t* n_prims) {
  auto* b = (BvhBuild*)h;
  *n_nodes = (int64_t)b->c0.size();
  *n_prims = (int64_t)b->prims.size();
}
void sg_bvh_export(void* h, int32_t* box, int32_t* c0, int32_t* c1, int32_t* prims) {
  auto* b = (BvhBuild*)h;
  std::copy(b->box.begin(), b->box.end(), box);
  std::copy(b->c0.begin(), b->c0.end(), c0);
  std::copy(b->c1.begin(), b->c1.end(), c1);
  std::copy(b->prims.begin(), b->prims.end(), prims);
}
void sg_bvh_free(void* h) { delete (BvhBuild*)h; }

// Roped SAH kd-tree over the segments inside [0, D]^2.  lambda = traversal cost
// relative to a segment test.
void* sg_kd_build(int64_t n_seg, const int32_t* seg, int32_t D, float lambda, int32_t max_depth) {
  auto* k = new KdBuild();
  k->seg = seg;
  k->lambda = lambda;
  k->max_depth = max_depth;
  const int64_t root_box[4] = {0, 0, D, D};
  const int root = k->new_node(root_box);
  std::vector<int32_t> ids;
  for (int64_t s = 0; s < n_seg; ++s)
    if (seg_hits_box(seg + 4 * s, 0, 0, D, D)) ids.push_back((int32_t)s);
  k->build(root, ids, 0);
  const int32_t none[4] = {-1, -1, -1, -1};
  k->ropes(root, none);
  k->seg = nullptr;
  return k;
}
void sg_kd_sizes(void* h, int64_t* n_nodes, int64_t* n_refs) {
  auto* k = (KdBuild*)h;
  *n_nodes = (int64_t)k->axis.size();
  *n_refs = (int64_t)k->refs.size();
}
void sg_kd_export(void* h, int32_t* axis, int32_t* split, int32_t* child, int32_t* count, int32_t* box,
                  int32_t* rope, int32_t* rope_log2, int32_t* refs) {
  auto* k = (KdBuild*)h;
  std::copy(k->axis.begin(), k->axis.end(), axis);
  std::copy(k->split.begin(), k->split.end(), split);
  std::copy(k->child.begin(), k->child.end(), child);
  std::copy(k->count.begin(), k->count.end(), count);
  std::copy(k->box.begin(), k->box.end(), box);
  std::copy(k->rope.begin(), k->rope.end(), rope);
  std::copy(k->rope_log2.begin(), k->rope_log2.end(), rope_log2);
  std::copy(k->refs.begin(), k->refs.end(), refs);
}
void sg_kd_free(void* h) { delete (KdBuild*)h; }

}  // extern "C"

extern "C" {

// Quality refinement of a CDT in place (see refine above): min_angle_deg (0 =
// none), max_area (0 = none, grid units^2), at most max_insert new vertices.
// Returns the number of vertices inserted, or -1 on a construction failure.
// The 1 -> 4 subdivision of Sec. 3.5.2, on the lattice: the midpoint of every
// interior edge that has a lattice midpoint is inserted (a constrained edge's
// midpoint splits it, keeping its segment), then the triangulation is made
// constrained-Delaunay again by flips; hull edges are not split.  The
// optimiser then moves, flips and contracts the new vertices (Sec. 3.5.3).
// Returns the number of vertices inserted.
int64_t sg_subdivide(void* h) {
  auto* tr = (Triangulation*)h;
  std::vector<Pt> mids;
  for (int t = 0; t < (int)tr->T.size(); ++t)
    for (int i = 0; i < 3; ++i) {
      const int u = tr->T[t].n[i];
      if (u < t) continue;  // each interior edge once; hull edges (u < 0) skipped
      const Pt& p = tr->P[tr->T[t].v[(i + 1) % 3]];
      const Pt& q = tr->P[tr->T[t].v[(i + 2) % 3]];
      if (((p.x + q.x) & 1) || ((p.y + q.y) & 1)) continue;
      mids.push_back(Pt{(p.x + q.x) / 2, (p.y + q.y) / 2});
    }
  int64_t inserted = 0;
  for (const Pt& m : mids) {
    const size_t nv = tr->P.size();
    const int v = tr->insert_point(m);
    if (tr->status < 0) return -1;
    if (v >= 0 && (size_t)v >= nv) ++inserted;
  }
  return inserted;
}

int64_t sg_refine(void* h, double min_angle_deg, double max_area, int64_t max_insert) {
  auto* tr = (Triangulation*)h;
  int64_t n = refine(*tr, min_angle_deg, max_area, max_insert);
  return tr->status < 0 ? -1 : n;
}

// The optimally refined CDT (Sec. 3.5.1): refine copies of the CDT with every
// (angle, area) pair of the given grids, in parallel, and keep the one with
// the shortest total edge length (the unrefined CDT competes too).  Writes the
// chosen pair to *best_angle / *best_area; returns a new handle.
void* sg_refine_optimal(void* h, const double* angles, int32_t n_angles, const double* areas, int32_t n_areas,
                        int64_t max_insert, int32_t n_threads, double* best_angle, double* best_area) {
  auto* base = (Triangulation*)h;
  struct Cand {
    double a, A;
    Triangulation* tr = nullptr;
    float len = 0.f;
  };
  std::vector<Cand> cands;
  cands.push_back(Cand{0.0, 0.0});
  for (int i = 0; i < n_angles; ++i)
    for (int j = 0; j < n_areas; ++j)
      if (angles[i] > 0 || areas[j] > 0) cands.push_back(Cand{angles[i], areas[j]});
  std::vector<std::thread> th;
  std::atomic<size_t> next{0};
  const int nt = std::max(1, std::min<int>(n_threads, (int)cands.size()));
  for (int w = 0; w < nt; ++w)
    th.emplace_back([&]() {
      while (true) {
        const size_t k = next.fetch_add(1);
        if (k >= cands.size()) break;
        auto* tr = new Triangulation(*base);
        if (cands[k].a > 0 || cands[k].A > 0) refine(*tr, cands[k].a, cands[k].A, max_insert);
        cands[k].tr = tr;
        cands[k].len = tr->status < 0 ? 3.4e38f : (float)tr->total_length(false);
      }
    });
  for (auto& x : th) x.join();
  size_t best = 0;
  for (size_t k = 1; k < cands.size(); ++k)
    if (cands[k].len < cands[best].len) best = k;
  for (size_t k = 0; k < cands.size(); ++k)
    if (k != best) delete cands[k].tr;
  *best_angle = cands[best].a;
  *best_area = cands[best].A;
  return cands[best].tr;
}

}  // extern "C"
