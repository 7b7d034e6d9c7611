// Mirror paths: secondary rays chained through the triangulation (Sec. 5.2:
// "the final triangle in the traversal of the original ray is the starting
// triangle for traversal of the secondary ray").
//
// A path starts as a primary ray (lattice origin, start triangle given or
// located) and continues with up to n_bounce secondary rays, each the mirror
// image of its parent about the hit segment (or takes the caller's direction
// in the frame of the hit edge).  A secondary ray starts on the
// hit constrained edge (a -> b) of its parent's final triangle T, at
// P' = a + (i / 2^32) (b - a) with i = round(2^32 mu) (halves up) clamped to
// [1, 2^32 - 1], mu the exact parameter of the hit point on that edge; it
// enters T through that edge, i.e. at half-edge 3 T + e, so it needs no
// locate and cannot hit the segment it leaves.  Its direction is
// k' = round(2 (k.u) u / |u|^2 - k) (halves up, clamped to 2^22), u = b - a;
// the path ends when k' does not point strictly back to the parent's side.
//
// Origins are held as X = 2^32 x, Y = 2^32 y (int64).  The side of a vertex v
// relative to the ray (P, k) is L iff 2^32 (k x (v - P)) >= 0, i.e. iff
//     A(v) = kx vy - ky vx  >=  ch = ceil((kx Y - ky X) / 2^32)
// (A(v) is an integer): one exact int64 product pair and a compare per step,
// with ch computed once per ray of the path.  For a primary ray ch is
// kx oy - ky ox and the test is the walk kernel's.  No fp32 filter is needed.
// The snapped parameter and the mirror direction are exact quotients whose
// remainders are small: they are found in int64 arithmetic modulo 2^64 from
// fp32 estimates (floordiv_mod); only t's numerator is formed in 128 bits.
//
// One path per lane.  A lane whose ray left its triangle through a hull or
// constrained edge waits (pending) until kBounceServeMin lanes of the warp are
// pending or idle; the warp then finishes all pending rays in one pass (the
// hit parameter, the next origin and direction: a few hundred integer
// instructions that would otherwise run while the other lanes wait) and
// refills idle lanes from chunks of a global work counter.  A lane keeps its
// path across bounces: the next ray continues from 3 T + e in registers.
#include <algorithm>

#include "bounce_arith.cuh"
#include "cct_internal.cuh"

namespace cct {

namespace {

constexpr int kBounceThreads = 256;
// A warp serves (finishes pending rays, refills idle lanes) once this many of
// its lanes are pending or idle (3.4x faster than serving every finished ray
// at once).  On the six bench scenes' two-step records, 2^22 mirror paths of
// 8 bounces: 16, 20, 24, 28, 32 took 19.8, 18.6, 17.2, 16.6, 18.8 ms in all;
// at 28 the dash grids run 5-6 % faster than at 24, circles and clusters 1
// and 5 % slower.
constexpr int kBounceServeMin = 28;

typedef __int128 i128;

struct BounceArgs {
  const int32_t* ox;
  const int32_t* oy;
  const float* dx;
  const float* dy;
  const int32_t* start;  // caller ids (start_user) or record indices
  int32_t start_user;
  int32_t n;         // rays of this launch
  int32_t n_bounce;  // secondary rays per path at most
  int64_t n_total;   // rays of the call: entry b * n_total + off + i
  int64_t off;
  int32_t* hit;
  float* t;
  int32_t* steps;
  const float* frame;  // optional: (c, s) of ray b >= 1 of path i at 2 ((b - 1) n_total + off + i)
  int64_t* org_x;     // optional outputs (NULL: not written)
  int64_t* org_y;
  float* dir_x;
  float* dir_y;
  int32_t chunk;
};

// |v| as fp32 within 2^-23 relative (two correctly rounded halves).
__device__ __forceinline__ float i128_to_float(i128 v) {
  const bool neg = v < 0;
  const unsigned __int128 m = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
  const float f = hi ? __fmaf_rn(__ull2float_rn(hi), 18446744073709551616.0f, __ull2float_rn(lo)) : __ull2float_rn(lo);
  return neg ? -f : f;
}

// Mirror paths: four blocks per SM (64 registers, no spills), 1.07-1.17x faster
// than the compiler's 76 registers at three blocks (more warps to hide the
// gathers).  kFrame: the secondary directions come from A.frame; a separate
// instantiation keeps the mirror paths free of that code's register pressure
// (4-5 % faster), and it runs at three blocks (80 registers): at four it
// spilled and ran 1.14-1.28x slower.
// kTwo: the walk reads the scene's two-step records (CCT_LOAD_TWO_STEP): after
// an L exit the next triangle's record is already in the loaded sector, after
// an R exit 16 more bytes of the same record; two triangles per iteration.  A
// lane walks one path, so its chain of dependent loads bounds it: the records
// halve the chain's length after an L exit (7-12 % faster on the bench's
// scenes).  Steps per serve check do not pay here (1, 2, 3, 4: the serve
// check is one ballot).
template <bool kFrame, bool kTwo>
__global__ void __launch_bounds__(kBounceThreads, kFrame ? 3 : 4) bounce_kernel(SceneDev S, BounceArgs A,
                                                                unsigned long long* __restrict__ counter) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int4* __restrict__ he_tab = S.he;
  const int4* __restrict__ he2_tab = S.he2;
  const int max_steps = S.max_steps;
  const int n_he = 3 * S.n_tri;  // half-edge records (the checked build's bound)
  const int nb_max = A.n_bounce;

  // the lane's path
  bool act = false, pend = false;
  int fT = 0, fe = 0, fw = 0;  // a pending ray: final triangle, exit edge, its neighbour word
  int id = 0, b = 0, ns = 0, h = 0, kx = 0, ky = 0;
  long long ch = 0, X = 0, Y = 0;
  // counters
  unsigned long long c_rays = 0, c_steps = 0, c_sides = 0, c_inv = 0, c_lim = 0;
  int pool_next = 0, pool_end = 0;
  bool exhausted = false;

  auto record = [&](int bb, int32_t hv, float tv, int32_t st, bool with_ray) {
    const long long k = (long long)bb * A.n_total + A.off + id;
    A.hit[k] = hv;
    A.t[k] = tv;
    A.steps[k] = st;
    if (A.org_x) A.org_x[k] = with_ray ? X : 0;
    if (A.org_y) A.org_y[k] = with_ray ? Y : 0;
    if (A.dir_x) A.dir_x[k] = with_ray ? __fmul_rn((float)kx, 1.0f / kDirScale) : 0.0f;
    if (A.dir_y) A.dir_y[k] = with_ray ? __fmul_rn((float)ky, 1.0f / kDirScale) : 0.0f;
  };
  // no ray at bounces bb .. n_bounce
  auto end_path = [&](int bb) {
    const float nan = __int_as_float(0x7fc00000);
    for (int q = bb; q <= nb_max; ++q) record(q, -1, nan, CCT_RAY_NONE, false);
    act = false;
  };
  // The ray of bounce b left its final triangle T through edge e, whose
  // neighbour word is w (< 0): a miss, or a hit that may start the next ray.
  auto finish = [&](int T, int e, int32_t w) {
    c_steps += (unsigned)ns;
    c_sides += (unsigned)ns + (b == 0 ? 2u : 0u);  // one side per triangle, three in a primary's first
    if (w == -1) {
      record(b, -1, __int_as_float(0x7f800000), ns, true);
      end_path(b + 1);
      return;
    }
    const TriRec r = load_rec(S.rec + T);
    const int ia = (e == 2) ? 0 : e + 1, ib = (e == 0) ? 2 : e - 1;
    const long long ax = vx_of(r, ia), ay = vy_of(r, ia), bx = vx_of(r, ib), by = vy_of(r, ib);
    const long long ex = bx - ax, ey = by - ay;
    const long long Rx = X - (ax << 32), Ry = Y - (ay << 32);  // P - a in units of 2^-32
    // t = cross(e, a - P) / cross(e, d) = 2^22 num / (2^32 den)
    i128 num = (i128)ey * Rx - (i128)ex * Ry;
    long long den = ex * ky - ey * kx;
    if (den < 0) {
      num = -num;
      den = -den;
    }
    const float tv = __fmul_rn(__fdiv_rn(i128_to_float(num), __ll2float_rn(den)), 1.0f / 1024.0f);
    record(b, -2 - w, tv, ns, true);
    if (b == nb_max) {
      act = false;
      return;
    }
    // the next origin on the edge; the mirror direction, or the caller's in the edge's frame
    const long long i = bounce::snap_param(kx, ky, Rx, Ry, ex, ey);
    int k2x, k2y;
    bool back;
    if (kFrame) {
      const long long fi = 2 * ((long long)b * A.n_total + A.off + id);
      int kc, ks;
      if (!dir_to_k(A.frame[fi], kc) || !dir_to_k(A.frame[fi + 1], ks) || ks <= 0) {
        record(b + 1, -1, __int_as_float(0x7fc00000), CCT_RAY_INVALID, false);  // an invalid secondary ray
        end_path(b + 2);
        ++c_inv;
        ++c_rays;
        return;
      }
      back = bounce::frame_dir(kc, ks, kx, ky, ex, ey, k2x, k2y);
    } else {
      back = bounce::mirror_dir(kx, ky, ex, ey, k2x, k2y);
    }
    if (!back) {
      end_path(b + 1);
      return;
    }
    X = (ax << 32) + i * ex;
    Y = (ay << 32) + i * ey;
    kx = k2x;
    ky = k2y;
    ch = bounce::ceil_cross_q(kx, ky, X, Y);
    ++b;
    ns = 0;
    h = 3 * T + e;  // enter T again through the hit edge
    act = true;
    ++c_rays;
  };
  // A new path: the primary ray `gi` (index within this launch).
  auto start_path = [&](int gi) {
    id = gi;
    b = 0;
    ++c_rays;
    const int ox = A.ox[gi], oy = A.oy[gi];
    int T0 = A.start ? A.start[gi] : -1;
    bool ok = dir_to_k(A.dx[gi], kx) && dir_to_k(A.dy[gi], ky) && (kx | ky) != 0 && ox >= 0 && oy >= 0 &&
              ox <= S.D && oy <= S.D && T0 >= 0 && T0 < S.n_tri;
    bool bad = false;  // the checked build met an out-of-range table index
    if (ok && A.start_user) {
      T0 = S.user2dev[T0];
      if (idx_bad(T0, S.n_tri)) {
        ok = false;
        bad = true;
      }
    }
    TriRec r;
    if (ok) {
      r = load_rec(S.rec + T0);
      const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
      const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
      ok = orient_i(x1, y1, x2, y2, ox, oy) > 0 && orient_i(x2, y2, x0, y0, ox, oy) > 0 &&
           orient_i(x0, y0, x1, y1, ox, oy) > 0;
    }
    if (!ok) {
      ++c_inv;
      kx = ky = 0;
      record(0, -1, __int_as_float(0x7fc00000), bad ? CCT_RAY_BAD_INDEX : CCT_RAY_INVALID, false);
      end_path(1);
      return;
    }
    X = (long long)ox << 32;
    Y = (long long)oy << 32;
    ch = (long long)kx * oy - (long long)ky * ox;
    // first triangle (Sec. 5.1): all three sides; leave through the CCW edge
    // (a -> b) with s(a) = R, s(b) = L
    const bool s0 = (long long)kx * vy_of(r, 0) - (long long)ky * vx_of(r, 0) >= ch;
    const bool s1 = (long long)kx * vy_of(r, 1) - (long long)ky * vx_of(r, 1) >= ch;
    const bool s2 = (long long)kx * vy_of(r, 2) - (long long)ky * vx_of(r, 2) >= ch;
    const int e = (!s1 && s2) ? 0 : ((!s2 && s0) ? 1 : 2);
    const int32_t w = nb_of(r, e);
    ns = 1;
    act = true;
    if (w >= 0 && idx_bad(w, n_he)) {
      c_sides += 2u;
      record(0, -1, __int_as_float(0x7fc00000), CCT_RAY_BAD_INDEX, true);
      end_path(1);
    } else if (w >= 0) {
      h = w;
    } else {
      finish(T0, e, w);
    }
  };

  while (true) {
    const unsigned busy = __ballot_sync(FULL, act);
    if (32 - __popc(busy) >= kBounceServeMin || busy == 0u) {
      // ---------------------------------------------------------- serve: finish pending rays, refill idle lanes
      if (pend) {
        pend = false;
        finish(fT, fe, fw);
      }
      const unsigned idle = __ballot_sync(FULL, !act);
      if (idle != 0u && !exhausted) {
        const int need = __popc(idle), rank = __popc(idle & lt);
        const int avail = pool_end - pool_next;
        int gi = -1;
        if (!act && rank < avail) gi = pool_next + rank;
        if (avail >= need) {
          pool_next += need;
        } else {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(counter, (unsigned long long)A.chunk);
          base = __shfl_sync(FULL, base, 0);
          if (base >= (unsigned long long)A.n) {
            exhausted = true;
            pool_next = pool_end;
          } else {
            pool_next = (int)base;
            pool_end = (int)min(base + (unsigned long long)A.chunk, (unsigned long long)A.n);
            const int j = pool_next + (rank - avail);
            if (!act && rank >= avail && j < pool_end) gi = j;
            pool_next = min(pool_end, pool_next + (need - avail));
          }
        }
        if (gi >= 0) start_path(gi);
      }
      if (!__any_sync(FULL, act)) {
        if (exhausted) break;  // nothing is pending after a serve
        continue;
      }
    }
    // ------------------------------------------------------------ one step per walking lane
    if (act) {
      auto side = [&](const int4& q) {
        return (long long)kx * coord_of_word(q.y) - (long long)ky * coord_of_word(q.x) >= ch;
      };
      bool sc;
      int32_t w;
      if (kTwo) {
        int4 al, ah;
        load_sector(he2_tab + 4 * h, al, ah);
        sc = side(al);
        ++ns;
        w = sc ? al.z : al.w;
        if (w >= 0 && ns < max_steps && !idx_bad(w, n_he)) {
          const int4 q = sc ? ah : load_he(he2_tab + 4 * h + 2);
          h = w;
          sc = side(q);
          ++ns;
          w = sc ? q.z : q.w;
        }
      } else {
        const int4 q = load_he(he_tab + h);
        sc = side(q);
        ++ns;
        w = sc ? q.z : q.w;
      }
      if (w >= 0 && ns < max_steps && !idx_bad(w, n_he)) {
        h = w;
      } else if (w >= 0 && idx_bad(w, n_he)) {
        c_sides += (unsigned)ns + (b == 0 ? 2u : 0u);
        record(b, -1, __int_as_float(0x7fc00000), CCT_RAY_BAD_INDEX, true);
        end_path(b + 1);
      } else if (w >= 0) {
        ++c_lim;
        c_sides += (unsigned)ns + (b == 0 ? 2u : 0u);
        record(b, -1, __int_as_float(0x7fc00000), CCT_RAY_WALK_LIMIT, true);
        end_path(b + 1);
      } else {
        fT = he_tri(h);
        const int j = h - 3 * fT;
        fe = sc ? (j == 2 ? 0 : j + 1) : (j == 0 ? 2 : j - 1);
        fw = w;
        act = false;
        pend = true;
      }
    }
  }
  // ------------------------------------------------------------ counters: one atomic per warp and counter
  const unsigned long long w_rays = warp_sum(c_rays), w_steps = warp_sum(c_steps), w_sides = warp_sum(c_sides);
  const unsigned long long w_inv = warp_sum(c_inv), w_lim = warp_sum(c_lim);
  if (lane == 0) {
    if (w_rays) atomicAdd(&S.stats->rays, w_rays);
    if (w_steps) atomicAdd(&S.stats->steps, w_steps);
    if (w_sides) atomicAdd(&S.stats->side_tests, w_sides);
    if (w_inv) atomicAdd(&S.stats->invalid_rays, w_inv);
    if (w_lim) atomicAdd(&S.stats->walk_limit_rays, w_lim);
  }
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

}  // namespace cct

using namespace cct;

extern "C" int cct_trace_bounces(cct_scene scene, const int32_t* ox, const int32_t* oy, const float* dx,
                                 const float* dy, const int32_t* start, int64_t n, int32_t n_bounce,
                                 const float* frame, int32_t* hit,
                                 float* t, int32_t* steps, int64_t* org_x, int64_t* org_y, float* dir_x,
                                 float* dir_y, uint32_t flags, void* stream_v) {
  if (!scene || n < 0 || n_bounce < 0 || n_bounce > CCT_MAX_BOUNCES ||
      (flags & ~(CCT_TRACE_EXACT_ONLY | CCT_TRACE_ONE_STEP)) != 0)
    return CCT_ERR_INVALID_ARGUMENT;
  if (n == 0) return CCT_OK;
  if (!ox || !oy || !dx || !dy || !hit || !t || !steps) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(scene->device);
  cudaStream_t stream = (cudaStream_t)stream_v;
  const SceneDev& S = scene->dev;
  const cct_tuning& tu = scene->tuning;
  constexpr int64_t kMaxLaunch = 1ll << 30;  // in-kernel ray indices stay in 32 bits
  const int64_t n_max = std::min<int64_t>(n, kMaxLaunch);
  const size_t total = 256 + (start ? 0 : al256(sizeof(int32_t) * (size_t)n_max));
  Scratch sc;
  sc.stream = stream;
  if (cudaMallocAsync((void**)&sc.base, total, stream) != cudaSuccess) {
    cudaGetLastError();
    sc.base = nullptr;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  unsigned long long* counter = (unsigned long long*)sc.base;
  // the two-step records whenever the scene has them (7-12 % faster on every bench scene, long
  // walks included), unless the call asks for the 16-byte records
  const bool two = S.he2 && (flags & CCT_TRACE_ONE_STEP) == 0;
  auto kern = frame ? (two ? bounce_kernel<true, true> : bounce_kernel<true, false>)
                    : (two ? bounce_kernel<false, true> : bounce_kernel<false, false>);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBounceThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  for (int64_t off = 0; off < n; off += kMaxLaunch) {
    const int64_t m = std::min<int64_t>(kMaxLaunch, n - off);
    if (cudaMemsetAsync(counter, 0, 8, stream) != cudaSuccess) return CCT_ERR_CUDA;
    const int32_t* st = start ? start + off : nullptr;
    bool st_user = true;
    if (!start) {
      int32_t* sbuf = (int32_t*)(sc.base + 256);
      if (launch_locate(S, ox + off, oy + off, m, sbuf, false, stream) != cudaSuccess) return CCT_ERR_CUDA;
      st = sbuf;
      st_user = false;
    }
    BounceArgs A{ox + off, oy + off, dx + off, dy + off, st, st_user ? 1 : 0, (int32_t)m, n_bounce, n, off,
                 hit, t, steps, frame, org_x, org_y, dir_x, dir_y, std::max(32, tu.chunk)};
    const long long want = (m + kBounceThreads - 1) / kBounceThreads;
    long long grid = std::min<long long>((long long)sm_count(scene->device) * per_sm, want);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kBounceThreads, 0, stream>>>(S, A, counter);
    if (cudaGetLastError() != cudaSuccess) return CCT_ERR_CUDA;
  }
  return CCT_OK;
}
