// The stackless walk (Sec. 5.1) and cct_trace.
//
// Per ray: in the start triangle leave through the CCW edge (a -> b) with
// s(a) = R, s(b) = L (two side tests: the origin lies strictly inside, so the
// three vertices are not all on one side).  Across an
// interior edge the neighbour shares the two decided vertices, so each later
// step decides only the new apex c: s(c) = L -> leave through (R-vertex, c),
// else through (c, L-vertex) -- the two remaining candidates of Sec. 7.2.  A
// constrained edge ends the walk with a hit (t from the edge's line), a hull
// edge with a miss.  Step count = triangles visited (Sec. 5.4).
//
// GPU mapping.  Everything done once per ray is done 32 rays at a time, by
// the whole warp, so the per-ray work never runs with most lanes masked off;
// the steps after the first run on two walk slots per lane:
//   prepare  the warp takes 32 ray indices (from its chunk of a global work
//            counter; the rays themselves were copied into shared memory
//            while the warp walked), finds their start triangles (given, or
//            by the Sec. 5.2 locate walk from the seed point of their grid
//            cell) and takes the first step on the 32-byte triangle records;
//            the resulting walk states go on the warp's `ready` stack;
//   walk     each active slot takes one apex step per loop iteration: one
//            dependent 16-byte half-edge load (apex + the two candidate exit
//            words), one side test, one select.  A lane's two slots hold two
//            independent rays, so their loads are in flight together;
//   serve    once `refill_min` of the warp's 64 slots are idle, finished
//            slots park their final state on the `parked` stack and idle
//            slots pop `ready` states (a prepare first when too few are left);
//   flush    32 parked rays at a time: reload the final triangle record,
//            compute hit id and t, write the results.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "cct_internal.cuh"

namespace cct {

// rare per-warp counters (shared memory)
enum : int { kCntRays = 0, kCntInvalid, kCntLocated, kCntLocSteps, kRareCounters };

constexpr int kWalkMaxThreads = 512;

struct WalkParams {
  int refill_min;  // serve idle slots once this many (of the warp's 64) are idle, or the whole warp is
  int chunk;       // ray indices a warp takes from the global counter at once
};

// Per-warp stacks in shared memory.  `ready` holds rays whose first
// triangle is behind them (the state after the first step: the half-edge of
// the second triangle); `parked` holds finished rays waiting for their
// results.  Entries are 16- and 8-byte words, so a push or a pop is two
// accesses.  The whole structure stays near 4 KB per warp: more shared memory
// per SM shrinks the L1 that holds the record loads in flight (measured
// slower).
constexpr int kStack = 64;
template <int kPfRows>
struct WarpStacks {
  int4 r_a[kStack];    // ready: ox word, oy word, kx word, ky word
  int2 r_b[kStack];    // ready: half-edge index, ray index
  int4 d_a[kStack];    // parked: ox word, oy word, kx word, ky word
  int2 d_b[kStack];    // parked: ray index, final record << 2 | exit edge
  int d_st[kStack];    // parked: steps or status
  int pf[kPfRows][32];  // the next batch's ray inputs, copied in while the warp walks (see prefetch)
  unsigned cnt[kRareCounters];
  unsigned long long steps, sides;  // step and side-test counts of the warp's finished rays
};
// rows of the prefetch buffer: ox, oy, dx, dy (+ start) (+ original index)
template <int kSrc>
__host__ __device__ constexpr int pf_rows() {
  return kSrc == kSrcSorted ? 6 : (kSrc == kSrcLocate ? 4 : 5);
}

// One walk slot: a ray past its first triangle.  ox, oy: origin words
// (o_word); kx, ky: direction words (k_word); h: the half-edge to enter next
// while walking, final record << 2 | exit edge once finished; ns: triangles
// visited (or a CCT_RAY_* status); id: ray index.
struct Slot {
  int ox, oy, kx, ky, h, ns, id;
  bool act;  // walking
  bool dn;   // finished, not yet parked
};

// kStage: the block first copies the scene's half-edge table into shared
// memory (after its warps' stacks) and the walk steps read it there: for
// tables small enough to share the SM with the stacks (CCT_TRACE_STAGE).
template <bool kExact, int kSrc, bool kStage>
__global__ void __launch_bounds__(kWalkMaxThreads) walk_kernel(SceneDev S, RaySrc R, WalkParams P,
                                                               int32_t* __restrict__ hit_out,
                                                               float* __restrict__ t_out,
                                                               int32_t* __restrict__ steps_out,
                                                               unsigned long long* __restrict__ counter) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr bool kLocate = (kSrc == kSrcLocate);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Stacks = WarpStacks<pf_rows<kSrc>()>;
  Stacks& W = reinterpret_cast<Stacks*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int n = (int)R.n;
  const int4* __restrict__ he_tab = S.he;
  int4* const sm_he = reinterpret_cast<int4*>(smem_raw + sizeof(Stacks) * (blockDim.x >> 5));
  if (kStage) {
    for (int k = threadIdx.x; k < 3 * S.n_tri; k += blockDim.x) sm_he[k] = load_he(S.he + k);
    __syncthreads();
  }
  const int max_steps = S.max_steps;
  const int n_he = 3 * S.n_tri;     // half-edge records (the checked build's bound)
  int pool_next = 0, pool_end = 0;  // the warp's current range of ray indices
  int pf_base = 0, pf_end = 0;      // the batch in `pf` ([pf_base, pf_end)); pf_base < 0: none left
  int n_ready = 0, n_done = 0;      // stack depths (warp-uniform)
  bool exhausted = false;
  unsigned n_fb = 0, n_lim = 0;  // this lane's int64 fallbacks and walk-limit rays

  Slot sl[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) sl[s] = Slot{0, 0, 0, 0, 0, 0, 0, false, false};
  if (lane < kRareCounters) W.cnt[lane] = 0;
  if (lane == 0) W.steps = W.sides = 0;
  __syncwarp();

  // Results of the parked rays [top - m, top): lane l completes entry top - m + l
  // (the final triangle record is reloaded).  Also counts their steps and
  // their side tests after the first triangle.
  auto flush = [&](int m, int top) {
    __syncwarp();
    unsigned f_steps = 0, f_sides = 0;
    if (lane < m) {
      const int k = top - m + lane;
      const int2 b = W.d_b[k];
      const int id = b.x, te = b.y;
      int st = W.d_st[k];
      int32_t h = -1;
      float tv = __int_as_float(0x7fc00000);  // NaN: invalid ray or step limit
      if (st > 0) {
        f_steps = (unsigned)st;
        f_sides = (unsigned)st - 1u;
        const TriRec r = load_rec(S.rec + (te >> 2));
        const int e = te & 3;
        const int32_t w = nb_of(r, e);
        if (w >= 0 && idx_bad(w, n_he)) {
          st = CCT_RAY_BAD_INDEX;  // the exit word of the final triangle is out of range
        } else if (w <= -2) {
          h = -2 - w;
          const int a = (e == 2) ? 0 : e + 1, b = (e == 0) ? 2 : e - 1;
          const int4 o = W.d_a[k];
          tv = hit_param_fast(vx_of(r, a), vy_of(r, a), vx_of(r, b), vy_of(r, b), o_of_word<kExact>(o.x),
                              o_of_word<kExact>(o.y), k_of_word<kExact>(o.z), k_of_word<kExact>(o.w));
        } else {
          tv = __int_as_float(0x7f800000);  // +inf: left through the hull
        }
      } else if (st == CCT_RAY_WALK_LIMIT) {
        f_sides = (unsigned)S.max_steps - 1u;
      }
      const unsigned long long pol = l2_evict_first();
      st_stream(hit_out + id, h, pol);
      st_stream(t_out + id, __float_as_int(tv), pol);
      st_stream(steps_out + id, st, pol);
    }
    f_steps = __reduce_add_sync(FULL, f_steps);
    f_sides = __reduce_add_sync(FULL, f_sides);
    if (lane == 0) {
      W.steps += f_steps;
      W.sides += f_sides;
    }
    __syncwarp();
  };

  // Starts the copies of the next (up to) 32 rays of the warp's pool into
  // `pf` (a new chunk from the global counter when the pool is empty).
  auto prefetch = [&]() {
    if (pool_next >= pool_end) {
      int base = 0;
      if (lane == 0) base = (int)atomicAdd(counter, (unsigned long long)P.chunk);
      base = __shfl_sync(FULL, base, 0);
      if (base >= n) {
        pf_base = -1;
        return;
      }
      pool_next = base;
      pool_end = min(base + P.chunk, n);
    }
    pf_base = pool_next;
    pf_end = min(pool_next + 32, pool_end);
    pool_next = pf_end;
    const int i = pf_base + lane;
    if (i < pf_end) {
      const unsigned long long pol = l2_evict_first();
      if (kSrc == kSrcSorted) {
        cp_async16_stream(&W.pf[0][4 * lane], R.rays + i, pol);  // rows 0..3 hold 32 int4
        cp_async4_stream(&W.pf[4][lane], R.start + i, pol);
        cp_async4_stream(&W.pf[5][lane], R.orig + i, pol);
      } else {
        cp_async4_stream(&W.pf[0][lane], R.ox + i, pol);
        cp_async4_stream(&W.pf[1][lane], R.oy + i, pol);
        cp_async4_stream(&W.pf[2][lane], R.dx + i, pol);
        cp_async4_stream(&W.pf[3][lane], R.dy + i, pol);
        if (!kLocate) cp_async4_stream(&W.pf[4][lane], R.start + i, pol);
      }
    }
    cp_async_commit();
  };

  // Takes the prefetched rays (up to 32), starts the copies of the next
  // batch, finds their start triangles (given, or by the Sec. 5.2 locate walk
  // from the seed point of their cell) and takes their first step; pushes
  // them on `ready`, or on `parked` when they end in the first triangle or
  // are invalid.  The whole warp works on 32 rays at once.
  auto prepare = [&]() {
    if (pf_base < 0) {
      exhausted = true;
      return;
    }
    cp_async_wait_all();
    const int i = pf_base + lane;
    const bool v = i < pf_end;
    int pox = 0, poy = 0, pkx = 0, pky = 0, pid = i, T0 = -1;  // pkx, pky: direction words
    float pdx = 0.f, pdy = 0.f;
    if (v) {
      if (kSrc == kSrcSorted) {
        const int4 rr = *reinterpret_cast<const int4*>(&W.pf[0][4 * lane]);
        pox = rr.x;
        poy = rr.y;
        pdx = __int_as_float(rr.z);
        pdy = __int_as_float(rr.w);
        T0 = W.pf[4][lane];
        pid = W.pf[5][lane];
      } else {
        pox = W.pf[0][lane];
        poy = W.pf[1][lane];
        pdx = __int_as_float(W.pf[2][lane]);
        pdy = __int_as_float(W.pf[3][lane]);
        if (!kLocate) T0 = W.pf[4][lane];
      }
    }
    __syncwarp();
    prefetch();  // the next batch arrives while this one is prepared and walked
    bool ok = false, bad = false;  // bad: the checked build met an out-of-range table index
    if (v) {
      if (kSrc == kSrcPlainUser) {
        if (T0 >= 0 && T0 < S.n_tri) {
          T0 = S.user2dev[T0];
          bad = idx_bad(T0, S.n_tri);
        } else {
          T0 = -1;
        }
      } else if (kChecked && kSrc != kSrcLocate) {
        bad = T0 == CCT_RAY_BAD_INDEX;  // marked by the locate kernel or the binning pass
      }
      // origins outside the domain lie in no triangle; rejecting them here
      // keeps every coordinate difference of the walk within int32
      ok = dir_to_k(pdx, pkx) && dir_to_k(pdy, pky) && (pkx | pky) != 0 && pox >= 0 && poy >= 0 && pox <= S.D &&
           poy <= S.D;
      pkx = k_word<kExact>(pkx);
      pky = k_word<kExact>(pky);
      if (kLocate) {
        if (ok) {
          T0 = S.seeds[seed_cell(S, pox, poy)];
          if (idx_bad(T0, S.n_tri)) {
            ok = false;
            bad = true;
          }
        }
      } else {
        ok = ok && !bad && T0 >= 0 && T0 < S.n_tri;
      }
    }
    const unsigned m_loc = kLocate ? __ballot_sync(FULL, ok) : 0u;
    TriRec r;
    if (ok) r = load_rec(S.rec + T0);
    int lsteps = 0;
    if (kLocate) {
      // the seed triangle holds the (perturbed) seed point; walk from there
      // towards the origin until the current triangle holds it
      int jj = 3;
      bool locating = false;
      if (ok) {
        lsteps = 1;
        const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
        const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
        const long long o0 = orient_i(x1, y1, x2, y2, pox, poy), o1 = orient_i(x2, y2, x0, y0, pox, poy);
        const long long o2 = orient_i(x0, y0, x1, y1, pox, poy);
        if (o0 < 0 || o1 < 0 || o2 < 0) {
          int cx, cy;
          seed_point(S, pox, poy, cx, cy);
          locating = locate_hop(S, r, T0, jj, seed_exit(r, cx, cy, pox, poy));
          ok = locating;
          if (kChecked && T0 < 0) bad = true;
        } else if (o0 == 0 || o1 == 0 || o2 == 0) {
          ok = false;  // origin on an edge or a vertex: not a valid ray origin
        }
      }
      while (__any_sync(FULL, locating)) {
        if (locating) {
          r = load_rec(S.rec + T0);
          ++lsteps;
          int cx, cy;
          seed_point(S, pox, poy, cx, cy);
          const int res = locate_step_entered(S, r, T0, jj, pox, poy, cx, cy);
          if (res != 0 || lsteps > S.max_steps) {
            locating = false;
            ok = res > 0;
            if (kChecked && T0 < 0) bad = true;
          }
        }
      }
    }
    // first step (Sec. 5.1): leave the start triangle through the CCW edge
    // (a -> b) with s(a) = R, s(b) = L
    const int oxw = o_word<kExact>(pox), oyw = o_word<kExact>(poy);
    int e = 0;
    int32_t w = -1;
    if (ok) {
      const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
      const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
      if (!kLocate)
        ok = orient_i(x1, y1, x2, y2, pox, poy) > 0 && orient_i(x2, y2, x0, y0, pox, poy) > 0 &&
             orient_i(x0, y0, x1, y1, pox, poy) > 0;
      // the exit is the CCW edge (a -> b) with s(a) = R, s(b) = L.  The origin
      // lies strictly inside, so the three vertices are not all on one side:
      // vertex 0 left leaves edge 0 (s2 = L) or edge 1 (s2 = R); vertex 0
      // right leaves edge 2 (s1 = L) or edge 0 (s1 = R).  Two side tests.
      const bool s0 = side_L_cw<kExact>(pkx, pky, oxw, oyw, coord_word(x0), coord_word(y0), n_fb);
      const bool sv = side_L_cw<kExact>(pkx, pky, oxw, oyw, coord_word(s0 ? x2 : x1), coord_word(s0 ? y2 : y1),
                                        n_fb);
      e = s0 ? (sv ? 0 : 1) : (sv ? 2 : 0);
      w = nb_of(r, e);
      if (ok && w >= 0 && idx_bad(w, n_he)) {
        ok = false;
        bad = true;
      }
    }
    const bool to_ready = ok && w >= 0;
    const bool to_done = v && !to_ready;
    const unsigned mr = __ballot_sync(FULL, to_ready), md = __ballot_sync(FULL, to_done);
    const unsigned mv = __ballot_sync(FULL, v), minv = __ballot_sync(FULL, v && !ok && !bad);
    if (kLocate) {
      const unsigned ls = __reduce_add_sync(FULL, (unsigned)lsteps);
      if (lane == 0) {
        W.cnt[kCntLocated] += __popc(m_loc);
        W.cnt[kCntLocSteps] += ls;
      }
    }
    if (lane == 0) {
      W.cnt[kCntRays] += __popc(mv);
      W.cnt[kCntInvalid] += __popc(minv);
    }
    if (to_ready) {
      const int k = n_ready + __popc(mr & lt);
      W.r_a[k] = make_int4(oxw, oyw, pkx, pky);
      W.r_b[k] = make_int2(w, pid);
    } else if (to_done) {
      const int k = n_done + __popc(md & lt);
      W.d_a[k] = make_int4(oxw, oyw, pkx, pky);
      W.d_b[k] = make_int2(pid, (T0 << 2) | e);
      W.d_st[k] = ok ? 1 : (bad ? CCT_RAY_BAD_INDEX : CCT_RAY_INVALID);
    }
    n_ready += __popc(mr);
    n_done += __popc(md);
    __syncwarp();
  };

  // One apex step of a walking slot on its half-edge record q (Sec. 5.1):
  // s(c) = L -> leave through edge nxt(j) (word q.z), else through prv(j) (q.w).
  auto step = [&](Slot& s, const int4& q) {
    const bool sc = side_L_cw<kExact>(s.kx, s.ky, s.ox, s.oy, q.x, q.y, n_fb);
    ++s.ns;
    const int32_t w = sc ? q.z : q.w;
    if (w >= 0 && s.ns < max_steps && !idx_bad(w, n_he)) {
      s.h = w;
      return;
    }
    if (w >= 0 && idx_bad(w, n_he)) {
      s.ns = CCT_RAY_BAD_INDEX;
    } else if (w >= 0) {
      s.ns = CCT_RAY_WALK_LIMIT;
      ++n_lim;
    } else {
      // hit or miss: park the final triangle and its exit edge
      const int T = he_tri(s.h), j = s.h - 3 * T;
      const int e = sc ? (j == 2 ? 0 : j + 1) : (j == 0 ? 2 : j - 1);
      s.h = (T << 2) | e;
    }
    s.act = false;
    s.dn = true;
  };

  prefetch();
  while (true) {
    // ---------------------------------------------------------------- serve idle slots
    const unsigned idle0 = __ballot_sync(FULL, !sl[0].act), idle1 = __ballot_sync(FULL, !sl[1].act);
    const int n_idle = __popc(idle0) + __popc(idle1);
    if (n_idle != 0 && (n_idle >= P.refill_min || (idle0 & idle1) == FULL)) {
      // park finished rays; complete them 32 at a time
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const unsigned dm = __ballot_sync(FULL, sl[q].dn);
        if (dm != 0u) {
          if (sl[q].dn) {
            const int k = n_done + __popc(dm & lt);
            W.d_a[k] = make_int4(sl[q].ox, sl[q].oy, sl[q].kx, sl[q].ky);
            W.d_b[k] = make_int2(sl[q].id, sl[q].h);
            W.d_st[k] = sl[q].ns;
            sl[q].dn = false;
          }
          n_done += __popc(dm);
          if (n_done >= 32) {
            flush(32, n_done);
            n_done -= 32;
          }
        }
      }
      const int want = min(n_idle, 32);
      if (n_ready < want && !exhausted) {
        prepare();
        if (n_done >= 32) {
          flush(32, n_done);
          n_done -= 32;
        }
      }
      // slot 0's idle lanes first, then slot 1's
      const int take = min(want, n_ready);
      const int rank0 = __popc(idle0 & lt), rank1 = __popc(idle0) + __popc(idle1 & lt);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int rank = q == 0 ? rank0 : rank1;
        if (!sl[q].act && rank < take) {
          const int k = n_ready - 1 - rank;
          const int4 a = W.r_a[k];
          const int2 b = W.r_b[k];
          sl[q].ox = a.x;
          sl[q].oy = a.y;
          sl[q].kx = a.z;
          sl[q].ky = a.w;
          sl[q].h = b.x;
          sl[q].id = b.y;
          sl[q].ns = 1;
          sl[q].act = true;
        }
      }
      n_ready -= take;
      __syncwarp();
    }
    if (!__any_sync(FULL, sl[0].act || sl[1].act)) {
      if (exhausted && n_ready == 0) break;
      continue;
    }

    // ---------------------------------------------------------------- one step per walking slot
    // both slots' loads first: two independent rays, two loads in flight
    // kStepsPerServe steps per slot before the next serve check: a slot that
    // finishes in one of them idles until then, but the warp runs a third of
    // the checks (ballots, counts, branch) it would otherwise
#pragma unroll
    for (int rep = 0; rep < kStepsPerServe; ++rep) {
      int4 q0 = make_int4(0, 0, 0, 0), q1 = make_int4(0, 0, 0, 0);
      if (kStage) {
        if (sl[0].act) q0 = sm_he[sl[0].h];
        if (sl[1].act) q1 = sm_he[sl[1].h];
      } else {
        if (sl[0].act) q0 = load_he(he_tab + sl[0].h);
        if (sl[1].act) q1 = load_he(he_tab + sl[1].h);
      }
      if (sl[0].act) step(sl[0], q0);
      if (sl[1].act) step(sl[1], q1);
    }
  }
  // the last parked rays (the final serve round parked every finished slot)
  while (n_done > 0) {
    const int m = min(32, n_done);
    flush(m, n_done);
    n_done -= m;
  }
  // ---------------------------------------------------------------- counters: one atomic per warp and counter
  __syncwarp();
  const unsigned w_fb = __reduce_add_sync(FULL, n_fb), w_limit = __reduce_add_sync(FULL, n_lim);
  // two side tests in the first triangle of every ray that reached it (the valid ones)
  const unsigned long long w_rays = W.cnt[kCntRays], w_inv = W.cnt[kCntInvalid];
  const unsigned long long w_steps = W.steps, w_side = W.sides + 2ull * (w_rays - w_inv);
  const unsigned long long w_loc = W.cnt[kCntLocated], w_lst = W.cnt[kCntLocSteps];
  if (lane == 0) {
    if (w_rays) atomicAdd(&S.stats->rays, w_rays);
    if (w_steps) atomicAdd(&S.stats->steps, w_steps);
    if (w_side) atomicAdd(&S.stats->side_tests, w_side);
    if (w_fb) atomicAdd(&S.stats->exact_fallbacks, (unsigned long long)w_fb);
    if (w_inv) atomicAdd(&S.stats->invalid_rays, w_inv);
    if (w_limit) atomicAdd(&S.stats->walk_limit_rays, (unsigned long long)w_limit);
    if (w_loc) atomicAdd(&S.stats->located, w_loc);
    if (w_lst) atomicAdd(&S.stats->locate_steps, w_lst);
  }
}

template <int kSrc>
static size_t stacks_bytes(int threads) {
  return sizeof(WarpStacks<pf_rows<kSrc>()>) * (size_t)(threads / 32);
}

// Shared memory a block may use (the GB300 per-block maximum).
constexpr size_t kMaxBlockSmem = 227 * 1024;

template <bool kExact, int kSrc, bool kStage>
static cudaError_t launch_walk_t(const SceneDev& S, const RaySrc& R, const cct_tuning& tu, int32_t* hit, float* t,
                                 int32_t* steps, unsigned long long* counter, int dev, cudaStream_t stream) {
  auto k = walk_kernel<kExact, kSrc, kStage>;
  const int threads = tu.block_threads;
  const size_t smem = stacks_bytes<kSrc>(threads) + (kStage ? sizeof(int4) * 3 * (size_t)S.n_tri : 0);
  {
    // once per instantiation and device (function attributes belong to each
    // device's context; `dev` is current): the stacks of 16 warps (and a
    // staged table) exceed the default 48 KB of dynamic shared memory.  The
    // shared/L1 split is left to the CUDA runtime's choice: a maximal shared
    // carveout measured 1.5x slower (the L1 also holds the loads in flight).
    static std::mutex mu;
    static uint64_t configured = 0;  // bit d: done on device d (d < 64; others every call)
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || !((configured >> dev) & 1u)) {
      const size_t cap = kStage ? kMaxBlockSmem : stacks_bytes<kSrc>(kWalkMaxThreads);
      const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) configured |= 1ull << dev;
    }
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  // every warp takes 32 rays at a time
  const long long want = (R.n + threads - 1) / threads;
  long long grid = std::min<long long>((long long)sm_count(dev) * per_sm, want);
  if (grid < 1) grid = 1;
  WalkParams P{std::max(1, std::min(32, tu.refill_min)), std::max(32, tu.chunk)};
  k<<<(unsigned)grid, threads, smem, stream>>>(S, R, P, hit, t, steps, counter);
  return cudaGetLastError();
}

bool walk_stage_fits(int32_t n_tri, int block_threads) {
  return stacks_bytes<kSrcPlainUser>(block_threads) + sizeof(int4) * 3 * (size_t)n_tri <= kMaxBlockSmem;
}

cudaError_t launch_walk_src(bool exact, int src, const SceneDev& S, const RaySrc& R, const cct_tuning& tu,
                            int32_t* hit, float* t, int32_t* steps, unsigned long long* counter, int dev,
                            cudaStream_t stream) {
  // the staged table only for unsorted rays, and only when it fits beside the stacks
  const bool stage = (tu.trace_flags & CCT_TRACE_STAGE) != 0 && src != kSrcSorted &&
                     walk_stage_fits(S.n_tri, tu.block_threads);
#define CCT_WALK_CASE(SRC)                                                                                  \
  case SRC:                                                                                                 \
    if (stage)                                                                                              \
      return exact ? launch_walk_t<true, SRC, true>(S, R, tu, hit, t, steps, counter, dev, stream)          \
                   : launch_walk_t<false, SRC, true>(S, R, tu, hit, t, steps, counter, dev, stream);        \
    return exact ? launch_walk_t<true, SRC, false>(S, R, tu, hit, t, steps, counter, dev, stream)           \
                 : launch_walk_t<false, SRC, false>(S, R, tu, hit, t, steps, counter, dev, stream);
  switch (src) {
    CCT_WALK_CASE(kSrcPlainUser)
    CCT_WALK_CASE(kSrcPlainDev)
    CCT_WALK_CASE(kSrcLocate)
    case kSrcSorted:
      return exact ? launch_walk_t<true, kSrcSorted, false>(S, R, tu, hit, t, steps, counter, dev, stream)
                   : launch_walk_t<false, kSrcSorted, false>(S, R, tu, hit, t, steps, counter, dev, stream);
    default:
      return cudaErrorInvalidValue;
  }
#undef CCT_WALK_CASE
}

cct_tuning default_tuning() {
  cct_tuning tu{};
  tu.block_threads = 256;
  tu.refill_min = 8;
  tu.chunk = 128;
  tu.bin_shift = -1;
  tu.trace_flags = 0;
  return tu;
}

cudaError_t launch_walk(bool exact, bool sorted, bool start_user, const SceneDev& S, const RaySrc& R, int32_t* hit,
                        float* t, int32_t* steps, unsigned long long* counter, int dev, cudaStream_t stream) {
  const int src = sorted ? kSrcSorted : (start_user ? kSrcPlainUser : kSrcPlainDev);
  return launch_walk_src(exact, src, S, R, default_tuning(), hit, t, steps, counter, dev, stream);
}

// Bin granularity: record indices >> shift, so that bins hold ~64 rays on average.
static int default_bin_shift(int64_t n, int32_t n_tri) {
  int shift = 0;
  const int64_t target = std::max<int64_t>(1024, n / 64);
  while (((int64_t)n_tri >> shift) > target && shift < 30) ++shift;
  return shift;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static int trace_impl(cct_scene scene, const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                      const int32_t* start, int64_t n, int32_t* hit, float* t, int32_t* steps, uint32_t flags,
                      cudaStream_t stream) {
  const SceneDev& S = scene->dev;
  cct_tuning tu = scene->tuning;
  flags |= tu.trace_flags;
  tu.trace_flags = flags;  // the launch sees the call's flags too
  const bool exact = (flags & CCT_TRACE_EXACT_ONLY) != 0;
  const bool bin = (flags & CCT_TRACE_BIN) != 0;
  const bool split = !start && !bin && (flags & CCT_TRACE_SPLIT_LOCATE) != 0;
  // launches of at most 2^30 rays keep every in-kernel index in 32 bits
  constexpr int64_t kMaxLaunch = 1ll << 30;
  const int64_t n_max = std::min<int64_t>(n, kMaxLaunch);
  const int shift = bin ? (tu.bin_shift >= 0 ? tu.bin_shift : default_bin_shift(n_max, S.n_tri)) : 0;
  const size_t o_start = 256;
  const size_t o_bin = o_start + (((bin || split) && !start) ? al256(sizeof(int32_t) * (size_t)n_max) : 0);
  const size_t total = o_bin + (bin ? bin_scratch_bytes(n_max, S.n_tri, shift) : 0);
  Scratch sc;
  sc.stream = stream;
  if (cudaMallocAsync((void**)&sc.base, total, stream) != cudaSuccess) {
    cudaGetLastError();
    sc.base = nullptr;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  unsigned long long* counter = (unsigned long long*)sc.base;
  for (int64_t off = 0; off < n; off += kMaxLaunch) {
    const int64_t m = std::min<int64_t>(kMaxLaunch, n - off);
    if (cudaMemsetAsync(counter, 0, 8, stream) != cudaSuccess) return CCT_ERR_CUDA;
    const int32_t* sx = ox + off;
    const int32_t* sy = oy + off;
    const float* sdx = dx + off;
    const float* sdy = dy + off;
    const int32_t* sst = start ? start + off : nullptr;
    int32_t* h = hit + off;
    int32_t* s = steps + off;
    float* tt = t + off;
    if (split) {
      // start cells from the locate kernel (record numbering), then the walk
      int32_t* sbuf = (int32_t*)(sc.base + o_start);
      if (launch_locate(S, sx, sy, m, sbuf, false, stream) != cudaSuccess) return CCT_ERR_CUDA;
      RaySrc R{sx, sy, sdx, sdy, sbuf, nullptr, nullptr, m};
      if (launch_walk_src(exact, kSrcPlainDev, S, R, tu, h, tt, s, counter, scene->device, stream) != cudaSuccess)
        return CCT_ERR_CUDA;
      continue;
    }
    if (!bin) {
      RaySrc R{sx, sy, sdx, sdy, sst, nullptr, nullptr, m};
      const int src = sst ? kSrcPlainUser : kSrcLocate;
      if (launch_walk_src(exact, src, S, R, tu, h, tt, s, counter, scene->device, stream) != cudaSuccess)
        return CCT_ERR_CUDA;
      continue;
    }
    // binned: start cells first (given or located), sort, then walk the sorted rays
    const int32_t* st = sst;
    bool st_user = true;
    if (!st) {
      int32_t* sbuf = (int32_t*)(sc.base + o_start);
      if (launch_locate(S, sx, sy, m, sbuf, false, stream) != cudaSuccess) return CCT_ERR_CUDA;
      st = sbuf;
      st_user = false;
    }
    BinOut bo{};
    if (launch_bin(S, sx, sy, sdx, sdy, st, st_user, m, shift, sc.base + o_bin, bo, stream) != cudaSuccess)
      return CCT_ERR_CUDA;
    // the sorted walk writes results at original indices relative to this launch
    RaySrc R{nullptr, nullptr, nullptr, nullptr, bo.start, bo.rays, bo.orig, m};
    if (launch_walk_src(exact, kSrcSorted, S, R, tu, h, tt, s, counter, scene->device, stream) != cudaSuccess)
      return CCT_ERR_CUDA;
  }
  return CCT_OK;
}

}  // namespace cct

using namespace cct;

extern "C" int cct_trace(cct_scene scene, const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                         const int32_t* start, int64_t n, int32_t* hit, float* t, int32_t* steps, uint32_t flags,
                         void* stream_v) {
  if (!scene || n < 0) return CCT_ERR_INVALID_ARGUMENT;
  if (n == 0) return CCT_OK;
  if (!ox || !oy || !dx || !dy || !hit || !t || !steps) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(scene->device);
  return trace_impl(scene, ox, oy, dx, dy, start, n, hit, t, steps, flags, (cudaStream_t)stream_v);
}

extern "C" int cct_scene_set_tuning(cct_scene scene, const cct_tuning* tu) {
  if (!scene) return CCT_ERR_INVALID_ARGUMENT;
  if (!tu) {
    scene->tuning = default_tuning();
    return CCT_OK;
  }
  if (tu->block_threads < 32 || tu->block_threads > kWalkMaxThreads || tu->block_threads % 32 != 0 ||
      tu->refill_min < 1 || tu->refill_min > 32 || tu->chunk < 32 || tu->chunk > (1 << 20) || tu->bin_shift > 30 ||
      (tu->trace_flags & ~(CCT_TRACE_EXACT_ONLY | CCT_TRACE_BIN | CCT_TRACE_SPLIT_LOCATE | CCT_TRACE_STAGE)) != 0)
    return CCT_ERR_INVALID_ARGUMENT;
  scene->tuning = *tu;
  return CCT_OK;
}

extern "C" int cct_scene_get_tuning(cct_scene scene, cct_tuning* out) {
  if (!scene || !out) return CCT_ERR_INVALID_ARGUMENT;
  *out = scene->tuning;
  return CCT_OK;
}
