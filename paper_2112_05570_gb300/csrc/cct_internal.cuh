// Internal layout and device helpers of libcct (see include/cct.h for the ABI).
//
// Device scene layout (one allocation per scene, 256-byte aligned pieces):
//   rec       TriRec[n_tri]     32-byte triangle records in Hilbert order of the
//                               triangle centroids (coordinates + neighbour
//                               words): the start triangle, the locate walk and
//                               the result of a ray read these
//   he        int4[3*n_tri]     16-byte half-edge records, one per (triangle T,
//                               entry edge j) at index 3 T + j: what a walk
//                               step after the first needs and nothing else
//                               (the apex of the entry edge and the two
//                               candidate exit words), one L2 sector per step
//   he2       int4[4*3*n_tri]   (CCT_LOAD_TWO_STEP only; read by the path
//                               kernel of cct_trace_bounces) two-step records, 64
//                               bytes per half-edge h: he[h], he[he[h].z] (the
//                               record behind its L exit), he[he[h].w] (behind
//                               its R exit), 16 unused bytes.  The first 32
//                               bytes are one sector: a left exit needs no
//                               second load; a right exit reads 16 more bytes
//                               of the same record
//   cnb       int32[3*n_tri]    neighbour word across constrained edges (read
//                               only by the locate walk, which crosses them)
//   user2dev  int32[n_tri]      caller triangle id -> record index
//   dev2user  int32[n_tri]      record index -> caller triangle id
//   seeds     int32[G*G]        locate seed grid (Sec. 5.2): square cells of
//                               side 2^seed_shift; per cell the record index of
//                               the triangle that holds its seed point (the
//                               cell centre, symbolically perturbed)
//   stats     DevStats          counters (cct_stats)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cct.h"

namespace cct {

constexpr int kCoordBits = 21;  // coordinates lie in [0, 2^20]
constexpr uint64_t kCoordMask = (1ull << kCoordBits) - 1;
constexpr float kDirScale = 4194304.0f;  // 2^22

// One triangle.  X / Y hold the coordinates of vertex i at bits [21 i, 21 i + 21).
// nb[i] describes the edge opposite vertex i (vertices CCW):
//   nb >= 0 : interior edge; the half-edge index 3 T' + j' of the neighbour
//             T' entered through this edge (its edge j')
//   nb == -1: hull edge (the ray leaves the domain: a miss)
//   nb <= -2: constrained edge carrying scene segment -2 - nb (a hit)
struct __align__(32) TriRec {
  uint64_t X;
  uint64_t Y;
  int32_t nb[3];
  int32_t pad;
};
static_assert(sizeof(TriRec) == 32, "TriRec must be one 32-byte sector");

// Half-edge record 3 T + j (triangle T entered through its edge j, so its
// apex is vertex j and the two other vertices' sides are already known):
//   x, y : apex coordinates as the fp32 bit patterns of 2^23 + coordinate
//          (exact; the integer is the low 23 bits, see coord_of_word)
//   z    : neighbour word of edge nxt(j), the exit when the apex is left (L)
//   w    : neighbour word of edge prv(j), the exit when the apex is right (R)
// with nxt(j) = (j + 1) mod 3, prv(j) = (j + 2) mod 3.
constexpr int kCoordBias = 0x4B000000;  // fp32 bits of 2^23
constexpr int kCoordLow = 0x7FFFFF;
__host__ __device__ __forceinline__ int coord_word(int c) { return kCoordBias | c; }
__host__ __device__ __forceinline__ int coord_of_word(int w) { return w & kCoordLow; }

// Triangle and edge of a half-edge index (3 T + j; T < 2^29).
__device__ __forceinline__ int he_tri(int h) { return (int)((unsigned)h / 3u); }

// Checked build.  Compiled with -DCCT_CHECKED (libcct_checked.so), every
// index that a kernel reads out of a device table -- a seed cell's record, a
// neighbour or half-edge exit word, a constrained-edge neighbour, the caller-id
// map, the comparison structures' child, rope and reference entries -- is
// range-checked before it addresses memory, and a ray that meets one out of
// range ends with CCT_RAY_BAD_INDEX instead of reading it.  The normal build
// compiles every check away: its loaders validate each table, so the indices
// are in range by construction.
#ifdef CCT_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
// True when the checked build finds i outside [0, n).
__host__ __device__ __forceinline__ bool idx_bad(int i, int n) { return kChecked && (unsigned)i >= (unsigned)n; }

// Walk steps each slot of the walk and batched kernels takes between two serve
// checks (the warp's ballots and counts of idle slots): measured on the bench's
// scenes at 2^24 rays, 1 -> 2 -> 3 took the walk from 1.00/1.05/1.17 ms to
// 0.96/0.94/1.12 and 0.94/0.92/1.11 ms (circles / dash grid / clusters) and
// the six-scene batched step from 5.62 to 5.50 and 5.44 ms; 4, 6 and 8 were
// slower again (the slots that finish early idle longer).
constexpr int kStepsPerServe = 3;

struct DevStats {
  unsigned long long rays, steps, side_tests, exact_fallbacks, invalid_rays, walk_limit_rays, located,
      locate_steps;
};

struct SceneDev {
  const TriRec* rec;
  const int4* he;
  const int4* he2;  // two-step records, or NULL
  const int32_t* cnb;
  const int32_t* user2dev;
  const int32_t* dev2user;
  const int32_t* seeds;
  DevStats* stats;
  int32_t n_tri;
  int32_t G;           // seed cells per side: ceil(D / 2^seed_shift)
  int32_t seed_shift;  // log2 of the seed cell side
  int32_t D;
  int32_t max_steps;
};

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ TriRec load_rec(const TriRec* p) {
  TriRec r;
  unsigned long long a, b, c, d;
  asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
  r.X = a;
  r.Y = b;
  r.nb[0] = (int32_t)(uint32_t)c;
  r.nb[1] = (int32_t)(uint32_t)(c >> 32);
  r.nb[2] = (int32_t)(uint32_t)d;
  r.pad = (int32_t)(uint32_t)(d >> 32);
  return r;
}

// One 32-byte sector as two int4 (the first half of a two-step record).
__device__ __forceinline__ void load_sector(const int4* p, int4& lo, int4& hi) {
  unsigned long long a, b, c, d;
  asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
  lo = make_int4((int)(uint32_t)a, (int)(uint32_t)(a >> 32), (int)(uint32_t)b, (int)(uint32_t)(b >> 32));
  hi = make_int4((int)(uint32_t)c, (int)(uint32_t)(c >> 32), (int)(uint32_t)d, (int)(uint32_t)(d >> 32));
}

__device__ __forceinline__ int4 load_he(const int4* p) {
  int4 r;
  asm volatile("ld.global.nc.v4.s32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}

// Coordinate i (0..2) of a 3 x 21-bit packed word, with 32-bit funnel shifts
// only (bits [0,21), [21,42) and [42,63) of the 64-bit word).
__device__ __forceinline__ int coord_of(uint64_t w, int i) {
  const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
  const uint32_t a = i == 2 ? hi : lo;
  const uint32_t sh = i == 0 ? 0u : (i == 1 ? 21u : 10u);
  return (int)(__funnelshift_r(a, hi, sh) & (uint32_t)kCoordMask);
}
__device__ __forceinline__ int vx_of(const TriRec& r, int i) { return coord_of(r.X, i); }
__device__ __forceinline__ int vy_of(const TriRec& r, int i) { return coord_of(r.Y, i); }

__device__ __forceinline__ int32_t nb_of(const TriRec& r, int e) { return e == 0 ? r.nb[0] : (e == 1 ? r.nb[1] : r.nb[2]); }

// Direction component -> exact integer k = 2^22 d; false if off the grid or |d| > 1.
__device__ __forceinline__ bool dir_to_k(float d, int& k) {
  float s = d * kDirScale;  // exact: power-of-two scaling
  if (!(fabsf(s) <= kDirScale) || s != rintf(s)) return false;
  k = (int)s;
  return true;
}

// Static error bound of the fp32 side test r = fma(dx, dy_v, -(dy * dx_v)) for
// |d| <= 1 and |v - o| <= 2^20: |r - E| <= 2^-24 (|r| + 2^20) (1 + 2^-23), so
// |r| >= 2^-4 (1 + 2^-10) fixes the sign of the exact E = dx dy_v - dy dx_v.
constexpr float kFilterBound = 0.0625f * (1.0f + 1.0f / 1024.0f);

// Side of v relative to the ray (o, d): true = L (exact E >= 0).
template <bool kExactOnly>
__device__ __forceinline__ bool side_L(float fdx, float fdy, int kx, int ky, int ox, int oy, int vx, int vy,
                                       unsigned& fallbacks) {
  const int ddx = vx - ox, ddy = vy - oy;
  if (!kExactOnly) {
    const float p = __fmul_rn(fdy, (float)ddx);
    const float r = __fmaf_rn(fdx, (float)ddy, -p);
    if (fabsf(r) >= kFilterBound) return r > 0.0f;
    ++fallbacks;
  }
  const long long e = (long long)kx * ddy - (long long)ky * ddx;
  return e >= 0;
}

// The same side test with the direction held as one 32-bit word per
// component: the float k (exact: |k| <= 2^22) in the fp32-filtered variant,
// the int k in the exact-only variant.  The filter then reads
// r = fma(kx, dy_v, -(ky dx_v)), 2^22 times the product above, with the bound
// scaled by the same power of two.
template <bool kExactOnly>
__device__ __forceinline__ int k_word(int k) {
  return kExactOnly ? k : __float_as_int((float)k);
}
template <bool kExactOnly>
__device__ __forceinline__ int k_of_word(int w) {
  return kExactOnly ? w : (int)__int_as_float(w);
}
template <bool kExactOnly>
__device__ __forceinline__ bool side_L_w(int kxw, int kyw, int ox, int oy, int vx, int vy, unsigned& fallbacks) {
  const int ddx = vx - ox, ddy = vy - oy;
  if (!kExactOnly) {
    const float p = __fmul_rn(__int_as_float(kyw), (float)ddx);
    const float r = __fmaf_rn(__int_as_float(kxw), (float)ddy, -p);
    if (fabsf(r) >= kFilterBound * kDirScale) return r > 0.0f;
    ++fallbacks;
  }
  const long long e = (long long)k_of_word<kExactOnly>(kxw) * ddy - (long long)k_of_word<kExactOnly>(kyw) * ddx;
  return e >= 0;
}

// Origin word of a ray in the walk state: the fp32 bits of 2^23 + o, as the
// apex words of the half-edge records.  Filtered, apex - origin is one exact
// fp32 subtraction of two numbers in [2^23, 2^24); exact-only, it is one
// integer subtraction of the two words (the bias bits are equal, so the
// difference is v - o).  Both variants use the same words.
template <bool kExactOnly>
__device__ __forceinline__ int o_word(int o) {
  return coord_word(o);
}
template <bool kExactOnly>
__device__ __forceinline__ int o_of_word(int w) {
  return coord_of_word(w);
}

// Side (true = L) of a vertex given by its coordinate words (coord_word)
// relative to the ray with origin words (o_word) and direction words (k_word).
// Filtered: dx_v = (2^23 + v_x) - (2^23 + o_x) is exact, so r is the same fp32
// value as in side_L_w and the same bound decides; the int64 test otherwise.
template <bool kExactOnly>
__device__ __forceinline__ bool side_L_cw(int kxw, int kyw, int oxw, int oyw, int vxw, int vyw, unsigned& fallbacks) {
  if (!kExactOnly) {
    const float ddx = __fsub_rn(__int_as_float(vxw), __int_as_float(oxw));
    const float ddy = __fsub_rn(__int_as_float(vyw), __int_as_float(oyw));
    const float p = __fmul_rn(__int_as_float(kyw), ddx);
    const float r = __fmaf_rn(__int_as_float(kxw), ddy, -p);
    if (fabsf(r) >= kFilterBound * kDirScale) return r > 0.0f;
    ++fallbacks;
  }
  const int ddx = vxw - oxw;  // both words carry the same bias
  const int ddy = vyw - oyw;
  return (long long)k_of_word<kExactOnly>(kxw) * ddy - (long long)k_of_word<kExactOnly>(kyw) * ddx >= 0;
}

__device__ __forceinline__ long long orient_ll(long long ax, long long ay, long long bx, long long by, long long cx,
                                               long long cy) {
  return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

// The same orientation for points of [0, 2^20]^2 (all differences fit in
// int32): two widening 32 x 32 -> 64-bit multiplies.
__device__ __forceinline__ long long orient_i(int ax, int ay, int bx, int by, int cx, int cy) {
  return (long long)(bx - ax) * (cy - ay) - (long long)(by - ay) * (cx - ax);
}

// t of the crossing of the ray (o, k / 2^22) with the line of edge (a, b):
// t = 2^22 num / den, num = cross(b - a, a - o), den = cross(b - a, k); fp32.
__device__ __forceinline__ float hit_param(int ax, int ay, int bx, int by, int ox, int oy, int kx, int ky) {
  const long long ex = bx - ax, ey = by - ay;
  long long num = ex * (long long)(ay - oy) - ey * (long long)(ax - ox);
  long long den = ex * (long long)ky - ey * (long long)kx;
  if (den < 0) {
    num = -num;
    den = -den;
  }
  return __fmul_rn(__fdiv_rn(__ll2float_rn(num), __ll2float_rn(den)), kDirScale);
}

// The same parameter with the fast reciprocal-based division (<= 2 ulp for
// divisors in [2^-126, 2^126]; den <= 2^44 here): with the two conversions,
// within 4 ulp of the exact rational.
__device__ __forceinline__ float hit_param_fast(int ax, int ay, int bx, int by, int ox, int oy, int kx, int ky) {
  const long long ex = bx - ax, ey = by - ay;
  long long num = ex * (long long)(ay - oy) - ey * (long long)(ax - ox);
  long long den = ex * (long long)ky - ey * (long long)kx;
  if (den < 0) {
    num = -num;
    den = -den;
  }
  return __fdividef(__ll2float_rn(num), __ll2float_rn(den)) * kDirScale;
}

// Seed cell of an origin in [0, D]^2: square cells of side h = 2^seed_shift,
// cell (ix, iy) = (min(ox >> s, G - 1), min(oy >> s, G - 1)); its seed point is
// c = (min(ix h + h/2, D - 1), min(iy h + h/2, D - 1)) moved by eps (1, delta),
// 0 < eps << delta << 1 (simulation of simplicity): the perturbed point lies on
// no line through two grid points, so it is strictly inside exactly one
// triangle and the line from it to an origin passes through no vertex other
// than the origin.  Host and device use the same integer formulas.
__device__ __forceinline__ int seed_cell(const SceneDev& S, int ox, int oy) {
  const int ix = min(ox >> S.seed_shift, S.G - 1), iy = min(oy >> S.seed_shift, S.G - 1);
  return iy * S.G + ix;
}
__device__ __forceinline__ void seed_point(const SceneDev& S, int ox, int oy, int& cx, int& cy) {
  const int s = S.seed_shift, half = (1 << s) >> 1;
  cx = min((min(ox >> s, S.G - 1) << s) + half, S.D - 1);
  cy = min((min(oy >> s, S.G - 1) << s) + half, S.D - 1);
}

// Side of vertex v relative to the directed line from the perturbed seed point
// p = c + eps (1, delta) to the origin o; true = L.  (o - p) x (v - p) =
// (o - c) x (v - c) + eps ((v - o) x (1, delta)): when the first term is zero
// the sign is that of (vx - ox) delta - (vy - oy), i.e. of oy - vy, else of
// vx - ox.  Exact (|coordinate differences| <= 2^20).
__device__ __forceinline__ bool seed_side_L(int cx, int cy, int ox, int oy, int vx, int vy) {
  const long long e = (long long)(ox - cx) * (vy - cy) - (long long)(oy - cy) * (vx - cx);
  if (e != 0) return e > 0;
  return vy != oy ? vy < oy : vx > ox;
}

// Exit edge of the seed triangle (whose interior holds the perturbed seed
// point) on the way from the seed point to o: the CCW edge (a -> b) with
// s(a) = R, s(b) = L relative to that line.
__device__ __forceinline__ int seed_exit(const TriRec& r, int cx, int cy, int ox, int oy) {
  const bool s0 = seed_side_L(cx, cy, ox, oy, vx_of(r, 0), vy_of(r, 0));
  const bool s1 = seed_side_L(cx, cy, ox, oy, vx_of(r, 1), vy_of(r, 1));
  const bool s2 = seed_side_L(cx, cy, ox, oy, vx_of(r, 2), vy_of(r, 2));
  return (!s1 && s2) ? 0 : ((!s2 && s0) ? 1 : 2);
}

// Moves the locate walk across edge e of record T (the walk crosses
// constrained edges: their neighbours come from cnb).  False at the hull, and
// in the checked build on an out-of-range neighbour word, with T = -1.
__device__ __forceinline__ bool locate_hop(const SceneDev& S, const TriRec& r, int& T, int& j, int e) {
  int32_t w = nb_of(r, e);
  if (w <= -2) w = S.cnb[3 * T + e];
  if (w < 0) return false;
  if (idx_bad(w, 3 * S.n_tri)) {
    T = -1;
    return false;
  }
  T = he_tri(w);
  j = w - 3 * T;
  return true;
}

// A locate step in a triangle T entered through its edge j < 3 (see
// locate_step): the entry edge's two sides are known, so decide the apex,
// then test o against the exit edge only (o lies beyond the entry edge by
// induction).
__device__ __forceinline__ int locate_step_entered(const SceneDev& S, const TriRec& r, int& T, int& j, int ox,
                                                   int oy, int cx, int cy) {
  const bool sc = seed_side_L(cx, cy, ox, oy, vx_of(r, j), vy_of(r, j));
  const int e = sc ? (j == 2 ? 0 : j + 1) : (j == 0 ? 2 : j - 1);
  const int a = (e == 2) ? 0 : e + 1, b = (e == 0) ? 2 : e - 1;
  const long long oe = orient_i(vx_of(r, a), vy_of(r, a), vx_of(r, b), vy_of(r, b), ox, oy);
  if (oe == 0) return -1;
  if (oe > 0) {
    // o lies before the exit edge: inside T unless on one of its other edges
    const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
    const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
    const bool in = orient_i(x1, y1, x2, y2, ox, oy) > 0 && orient_i(x2, y2, x0, y0, ox, oy) > 0 &&
                    orient_i(x0, y0, x1, y1, ox, oy) > 0;
    return in ? 1 : -1;
  }
  return locate_hop(S, r, T, j, e) ? 0 : -1;
}

// One step of the Sec. 5.2 locate walk from the seed point of o's cell (c,
// perturbed) towards the origin o, in record r = triangle T entered through
// its edge j (j = 3: T is the seed's own triangle).  Returns 1 when T holds o
// strictly inside, -1 when o lies on an edge or a vertex (or the walk leaves
// the domain; in the checked build also on a bad index, with T = -1), 0 after
// moving to the next triangle (T, j updated).
__device__ __forceinline__ int locate_step(const SceneDev& S, const TriRec& r, int& T, int& j, int ox, int oy,
                                           int cx, int cy) {
  if (j == 3) {
    const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
    const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
    const long long o0 = orient_i(x1, y1, x2, y2, ox, oy);
    const long long o1 = orient_i(x2, y2, x0, y0, ox, oy);
    const long long o2 = orient_i(x0, y0, x1, y1, ox, oy);
    if (o0 > 0 && o1 > 0 && o2 > 0) return 1;
    if (o0 >= 0 && o1 >= 0 && o2 >= 0) return -1;
    return locate_hop(S, r, T, j, seed_exit(r, cx, cy, ox, oy)) ? 0 : -1;
  }
  return locate_step_entered(S, r, T, j, ox, oy, cx, cy);
}

// Asynchronous global -> shared copies (the next batch of rays while the warp
// walks the current one); completion is awaited with cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
// The same copies with an L2 evict-first hint, and 4-byte stores with it: for
// data read or written once (the rays and the results), so that they leave L2
// before the scene's tables and seed grid do (1 % faster on the bench's step).
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async4_stream(void* smem, const void* gmem, unsigned long long pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async16_stream(void* smem, const void* gmem, unsigned long long pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_stream(void* p, int v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- host helpers
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int sm_count(int dev);

// Fault injection of the checked build: entry `index` of a device table of n
// entries is the 32-bit word `word` from `base`; reads the old word into *old
// and writes `value` (index < 0: only reports n in *len).  Synchronous.
int poke_word(int device, const void* base, int64_t n, int64_t index, int64_t word, int32_t value, int32_t* old,
              int64_t* len);

// Stream-ordered scratch for one call: one cudaMallocAsync, released with
// cudaFreeAsync on the same stream.
struct Scratch {
  char* base = nullptr;
  cudaStream_t stream = nullptr;
  ~Scratch() {
    if (base) cudaFreeAsync(base, stream);
  }
};

// Launchers shared between translation units (all enqueue on `stream`).
cudaError_t launch_locate(const SceneDev& S, const int32_t* ox, const int32_t* oy, int64_t n, int32_t* out,
                          bool to_user, cudaStream_t stream);

// Rays as the walk kernel reads them: separate arrays, or the sorted packed
// form written by the binning pass.
struct RaySrc {
  const int32_t* ox;
  const int32_t* oy;
  const float* dx;
  const float* dy;
  const int32_t* start;  // caller ids (start_user) or record indices
  const int4* rays;      // sorted form: {ox, oy, dx bits, dy bits}
  const int32_t* orig;   // sorted form: original index
  int64_t n;
};

// Enqueues the walk kernel; `counter` (8 bytes, zeroed by the caller on the
// same stream) hands out ray chunks.
cudaError_t launch_walk(bool exact, bool sorted, bool start_user, const SceneDev& S, const RaySrc& R, int32_t* hit,
                        float* t, int32_t* steps, unsigned long long* counter, int dev, cudaStream_t stream);

// Ray sources of the walk kernel: start cells as caller triangle ids, as
// record indices, the binned (sorted, packed) form, or none (the kernel
// locates each origin itself).
enum : int { kSrcPlainUser = 0, kSrcPlainDev = 1, kSrcSorted = 2, kSrcLocate = 3 };

// The same with an explicit launch configuration (block size, refill
// threshold, chunk) and ray source.
cudaError_t launch_walk_src(bool exact, int src, const SceneDev& S, const RaySrc& R, const cct_tuning& tu,
                            int32_t* hit, float* t, int32_t* steps, unsigned long long* counter, int dev,
                            cudaStream_t stream);

cct_tuning default_tuning();

struct BinOut {
  int4* rays;      // {ox, oy, dx bits, dy bits} sorted by start cell
  int32_t* start;  // record index, sorted
  int32_t* orig;   // original ray index, sorted
};
size_t bin_scratch_bytes(int64_t n, int32_t n_tri, int shift);
cudaError_t launch_bin(const SceneDev& S, const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                       const int32_t* start, bool start_is_user, int64_t n, int shift, char* scratch, BinOut& out,
                       cudaStream_t stream);

}  // namespace cct

struct cct_scene_s {
  cct::SceneDev dev;
  cct_tuning tuning;
  void* d_base;
  size_t bytes;
  int device;
};
