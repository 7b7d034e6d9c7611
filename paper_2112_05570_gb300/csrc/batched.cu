// Multi-scene persistent walk: one launch serves many (scene, ray batch) items.
//
// The work list is a device table of items (scene index, ray arrays, output
// arrays, ray count); items are cut into chunks of `chunk` rays and the grid's
// warps draw chunk indices from one global counter, so scenes of very
// different sizes and batches of very different lengths share the GPU without
// per-item launches.  A warp serves its idle lanes from its current chunk;
// each lane carries its own scene (record base, step limit), so lanes of one
// warp may walk different scenes.  The per-ray work is the walk of Sec. 5.1
// (and the seed locate of Sec. 5.2 when an item has no start cells), exactly
// as in walk.cu.
//
// The table is filled from a pinned, device-mapped host staging buffer by
// cct_batch_enqueue (a small kernel that copies it and resets the work
// counter, then the walk), so the enqueue can be captured once in a CUDA graph
// and replayed after each cct_batch_stage.  No copy engine is involved: a
// launch does not wait behind the caller's bulk transfers.
#include <algorithm>
#include <cstring>
#include <vector>

#include "cct_internal.cuh"

namespace cct {

struct BatchItemDev {
  const int32_t* ox;
  const int32_t* oy;
  const float* dx;
  const float* dy;
  const int32_t* start;  // caller ids, or NULL: locate
  int32_t* hit;
  float* t;
  int32_t* steps;
  int32_t n;
  int32_t scene;
  int32_t chunk_begin;  // first global chunk index of this item
  int32_t stride;       // ray element stride (1: arrays, 4: interleaved records)
};

struct BatchHeader {
  int32_t n_items;
  int32_t total_chunks;
  int32_t chunk;
  int32_t pad;
};

constexpr int kBatchMaxThreads = 512;

__device__ __forceinline__ int find_item(const BatchItemDev* items, int n_items, int c) {
  int lo = 0, hi = n_items - 1;  // last item with chunk_begin <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].chunk_begin <= c)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Per-warp stacks in shared memory, as in the single-scene walk: `ready`
// holds rays past their first triangle, `parked` finished rays awaiting
// their results; each entry carries its item and scene.
constexpr int kBStack = 64;
enum : int { kBRays = 0, kBInvalid, kBLocated, kBLocSteps, kBCounters };
struct BatchStacks {
  int4 r_a[kBStack];  // ready: ox word, oy word, kx word, ky word
  int4 r_b[kBStack];  // ready: half-edge index, ray index, item, scene
  int4 d_a[kBStack];  // parked: ox word, oy word, kx word, ky word
  int4 d_b[kBStack];  // parked: ray index, final record << 2 | exit edge, steps or status, item
  int pf[5][32];      // the next batch's ray inputs (ox, oy, dx, dy, start), copied in while the warp walks
  int l_idx[2][32], l_item[2][32];  // the walk slots' ray indices and items (read when they park)
  unsigned cnt[kBCounters];
  unsigned long long steps, sides;
};

// One walk slot (see walk.cu), plus its scene's half-edge table; its ray
// index and item wait in shared memory until it parks.
struct BSlot {
  const int4* he;
  int ox, oy, kx, ky, h, ns;
  int n_he;  // the checked build's bound on h (unused otherwise)
  bool act, dn;
};

// max_steps: the largest step limit of the batch's scenes.  A slot walks
// until that limit; a ray that needed more than its own scene's limit
// becomes a walk-limit ray when its result is written, exactly as if it had
// stopped at its own limit.
// 72 registers per thread (no spills): at the compiler's own choice (83) the
// kernel holds 24 warps per SM and ran 13 % slower on 512 scenes; at 64 it
// spills and ran 13 % slower.  72 x 512 threads still fits one block per SM.
template <bool kExact>
__global__ void __maxnreg__(72) batch_kernel(const SceneDev* __restrict__ scenes,
                                                                 const BatchHeader* __restrict__ hdr,
                                                                 const BatchItemDev* __restrict__ items,
                                                                 int refill_min, int max_steps,
                                                                 unsigned long long* counter, DevStats* bstats) {
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchStacks& W = reinterpret_cast<BatchStacks*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int n_items = hdr->n_items, total = hdr->total_chunks, chunk = hdr->chunk;
  // warp-uniform pool: a range of rays of one item; the batch in `pf`:
  // [pf_base, pf_end) of item pf_item (pf_base < 0: none left)
  int p_item = 0, p_next = 0, p_end = 0;
  int pf_item = 0, pf_base = 0, pf_end = 0;
  int n_ready = 0, n_done = 0;
  bool exhausted = n_items <= 0;
  unsigned n_fb = 0;  // this lane's int64 fallbacks
  BSlot sl[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) sl[q] = BSlot{nullptr, 0, 0, 0, 0, 0, 0, 0, false, false};
  if (lane < kBCounters) W.cnt[lane] = 0;
  if (lane == 0) W.steps = W.sides = 0;
  __syncwarp();

  unsigned n_lim = 0;  // walk-limit rays completed by this lane
  auto flush = [&](int m, int top) {
    __syncwarp();
    unsigned f_steps = 0, f_sides = 0;
    if (lane < m) {
      const int k = top - m + lane;
      const int4 pb = W.d_b[k];
      const int id = pb.x, te = pb.y;
      int st = pb.z;
      const BatchItemDev& it = items[pb.w];
      const SceneDev& S = scenes[it.scene];
      if (st > S.max_steps) st = CCT_RAY_WALK_LIMIT;  // walked past its own scene's limit
      int32_t h = -1;
      float tv = __int_as_float(0x7fc00000);
      if (st > 0) {
        f_steps = (unsigned)st;
        f_sides = (unsigned)st - 1u;
        const TriRec r = load_rec(S.rec + (te >> 2));
        const int e = te & 3;
        const int32_t w = nb_of(r, e);
        if (w >= 0 && idx_bad(w, 3 * S.n_tri)) {
          st = CCT_RAY_BAD_INDEX;  // the exit word of the final triangle is out of range
        } else if (w <= -2) {
          h = -2 - w;
          const int a = (e == 2) ? 0 : e + 1, b = (e == 0) ? 2 : e - 1;
          const int4 o = W.d_a[k];
          tv = hit_param_fast(vx_of(r, a), vy_of(r, a), vx_of(r, b), vy_of(r, b), o_of_word<kExact>(o.x),
                              o_of_word<kExact>(o.y), k_of_word<kExact>(o.z), k_of_word<kExact>(o.w));
        } else {
          tv = __int_as_float(0x7f800000);
        }
      } else if (st == CCT_RAY_WALK_LIMIT) {
        f_sides = (unsigned)S.max_steps - 1u;
        ++n_lim;
      }
      const unsigned long long pol = l2_evict_first();
      st_stream(it.hit + id, h, pol);
      st_stream(it.t + id, __float_as_int(tv), pol);
      st_stream(it.steps + id, st, pol);
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
    if (p_next >= p_end) {
      int c = 0;
      if (lane == 0) c = (int)atomicAdd(counter, 1ull);
      c = __shfl_sync(FULL, c, 0);
      if (c >= total) {
        pf_base = -1;
        return;
      }
      p_item = find_item(items, n_items, c);
      const BatchItemDev& it = items[p_item];
      p_next = (c - it.chunk_begin) * chunk;
      p_end = min(p_next + chunk, it.n);
    }
    pf_item = p_item;
    pf_base = p_next;
    pf_end = min(p_next + 32, p_end);
    p_next = pf_end;
    const int i = pf_base + lane;
    if (i < pf_end) {
      const BatchItemDev& it = items[pf_item];
      const long long ri = (long long)i * it.stride;
      const unsigned long long pol = l2_evict_first();
      cp_async4_stream(&W.pf[0][lane], it.ox + ri, pol);
      cp_async4_stream(&W.pf[1][lane], it.oy + ri, pol);
      cp_async4_stream(&W.pf[2][lane], it.dx + ri, pol);
      cp_async4_stream(&W.pf[3][lane], it.dy + ri, pol);
      if (it.start) cp_async4_stream(&W.pf[4][lane], it.start + i, pol);
    }
    cp_async_commit();
  };

  // 32 rays of one item at once (the prefetched batch): start triangle
  // (given, or the Sec. 5.2 locate walk), first step; onto `ready` or `parked`
  auto prepare = [&]() {
    if (pf_base < 0) {
      exhausted = true;
      return;
    }
    cp_async_wait_all();
    const int it_idx = pf_item;
    const BatchItemDev& it = items[it_idx];
    const int sc = it.scene;
    const SceneDev& S = scenes[sc];
    const int i = pf_base + lane;
    const bool v = i < pf_end;
    const bool locate = it.start == nullptr;
    int pox = 0, poy = 0, pkx = 0, pky = 0, T0 = -1;  // pkx, pky: direction words
    float pdx = 0.f, pdy = 0.f;
    if (v) {
      pox = W.pf[0][lane];
      poy = W.pf[1][lane];
      pdx = __int_as_float(W.pf[2][lane]);
      pdy = __int_as_float(W.pf[3][lane]);
      if (!locate) T0 = W.pf[4][lane];
    }
    __syncwarp();
    prefetch();  // the next batch arrives while this one is prepared and walked
    bool ok = false, bad = false;  // bad: the checked build met an out-of-range table index
    if (v) {
      ok = dir_to_k(pdx, pkx) && dir_to_k(pdy, pky) && (pkx | pky) != 0 && pox >= 0 && poy >= 0 && pox <= S.D &&
           poy <= S.D;
      pkx = k_word<kExact>(pkx);
      pky = k_word<kExact>(pky);
      if (locate) {
        if (ok) {
          T0 = S.seeds[seed_cell(S, pox, poy)];
          if (idx_bad(T0, S.n_tri)) {
            ok = false;
            bad = true;
          }
        }
      } else {
        if (T0 >= 0 && T0 < S.n_tri) {
          T0 = S.user2dev[T0];
          bad = idx_bad(T0, S.n_tri);
        } else {
          T0 = -1;
        }
        ok = ok && !bad && T0 >= 0;
      }
    }
    const unsigned m_loc = locate ? __ballot_sync(FULL, ok) : 0u;
    TriRec r;
    if (ok) r = load_rec(S.rec + T0);
    int lsteps = 0;
    if (locate) {
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
          ok = false;
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
    const int oxw = o_word<kExact>(pox), oyw = o_word<kExact>(poy);
    int e = 0;
    int32_t w = -1;
    if (ok) {
      const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
      const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
      if (!locate)
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
      if (ok && w >= 0 && idx_bad(w, 3 * S.n_tri)) {
        ok = false;
        bad = true;
      }
    }
    const bool to_ready = ok && w >= 0;
    const bool to_done = v && !to_ready;
    const unsigned mr = __ballot_sync(FULL, to_ready), md = __ballot_sync(FULL, to_done);
    const unsigned mv = __ballot_sync(FULL, v), minv = __ballot_sync(FULL, v && !ok && !bad);
    if (locate) {
      const unsigned ls = __reduce_add_sync(FULL, (unsigned)lsteps);
      if (lane == 0) {
        W.cnt[kBLocated] += __popc(m_loc);
        W.cnt[kBLocSteps] += ls;
      }
    }
    if (lane == 0) {
      W.cnt[kBRays] += __popc(mv);
      W.cnt[kBInvalid] += __popc(minv);
    }
    if (to_ready) {
      const int k = n_ready + __popc(mr & lt);
      W.r_a[k] = make_int4(oxw, oyw, pkx, pky);
      W.r_b[k] = make_int4(w, i, it_idx, sc);
    } else if (to_done) {
      const int k = n_done + __popc(md & lt);
      W.d_a[k] = make_int4(oxw, oyw, pkx, pky);
      W.d_b[k] = make_int4(i, (T0 << 2) | e, ok ? 1 : (bad ? CCT_RAY_BAD_INDEX : CCT_RAY_INVALID), it_idx);
    }
    n_ready += __popc(mr);
    n_done += __popc(md);
    __syncwarp();
  };

  // One apex step of a walking slot on its half-edge record q (Sec. 5.1).
  auto step = [&](BSlot& s, const int4& q) {
    const bool sc = side_L_cw<kExact>(s.kx, s.ky, s.ox, s.oy, q.x, q.y, n_fb);
    ++s.ns;
    const int32_t w = sc ? q.z : q.w;
    if (w >= 0 && s.ns < max_steps && !idx_bad(w, s.n_he)) {
      s.h = w;
      return;
    }
    if (w >= 0 && idx_bad(w, s.n_he)) {
      s.ns = CCT_RAY_BAD_INDEX;
    } else if (w >= 0) {
      s.ns = CCT_RAY_WALK_LIMIT;
    } else {
      const int T = he_tri(s.h), j = s.h - 3 * T;
      const int e = sc ? (j == 2 ? 0 : j + 1) : (j == 0 ? 2 : j - 1);
      s.h = (T << 2) | e;
    }
    s.act = false;
    s.dn = true;
  };

  if (!exhausted) prefetch();
  while (true) {
    const unsigned idle0 = __ballot_sync(FULL, !sl[0].act), idle1 = __ballot_sync(FULL, !sl[1].act);
    const int n_idle = __popc(idle0) + __popc(idle1);
    if (n_idle != 0 && (n_idle >= refill_min || (idle0 & idle1) == FULL)) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const unsigned dm = __ballot_sync(FULL, sl[q].dn);
        if (dm != 0u) {
          if (sl[q].dn) {
            const int k = n_done + __popc(dm & lt);
            W.d_a[k] = make_int4(sl[q].ox, sl[q].oy, sl[q].kx, sl[q].ky);
            W.d_b[k] = make_int4(W.l_idx[q][lane], sl[q].h, sl[q].ns, W.l_item[q][lane]);
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
      const int take = min(want, n_ready);
      const int rank0 = __popc(idle0 & lt), rank1 = __popc(idle0) + __popc(idle1 & lt);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int rank = q == 0 ? rank0 : rank1;
        if (!sl[q].act && rank < take) {
          const int k = n_ready - 1 - rank;
          const int4 a = W.r_a[k];
          const int4 b = W.r_b[k];
          sl[q].ox = a.x;
          sl[q].oy = a.y;
          sl[q].kx = a.z;
          sl[q].ky = a.w;
          sl[q].h = b.x;
          W.l_idx[q][lane] = b.y;
          W.l_item[q][lane] = b.z;
          sl[q].he = scenes[b.w].he;
          if (kChecked) sl[q].n_he = 3 * scenes[b.w].n_tri;
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
    // kStepsPerServe steps per slot before the next serve check (see cct_internal.cuh)
#pragma unroll
    for (int rep = 0; rep < kStepsPerServe; ++rep) {
      int4 q0 = make_int4(0, 0, 0, 0), q1 = make_int4(0, 0, 0, 0);
      if (sl[0].act) q0 = load_he(sl[0].he + sl[0].h);
      if (sl[1].act) q1 = load_he(sl[1].he + sl[1].h);
      if (sl[0].act) step(sl[0], q0);
      if (sl[1].act) step(sl[1], q1);
    }
  }
  while (n_done > 0) {
    const int m = min(32, n_done);
    flush(m, n_done);
    n_done -= m;
  }
  __syncwarp();
  const unsigned w_fb = __reduce_add_sync(FULL, n_fb), w_limit = __reduce_add_sync(FULL, n_lim);
  // two side tests in the first triangle of every ray that reached it (the valid ones)
  const unsigned long long w_rays = W.cnt[kBRays], w_inv = W.cnt[kBInvalid];
  const unsigned long long w_steps = W.steps, w_side = W.sides + 2ull * (w_rays - w_inv);
  const unsigned long long w_loc = W.cnt[kBLocated], w_lst = W.cnt[kBLocSteps];
  if (lane == 0) {
    if (w_rays) atomicAdd(&bstats->rays, w_rays);
    if (w_steps) atomicAdd(&bstats->steps, w_steps);
    if (w_side) atomicAdd(&bstats->side_tests, w_side);
    if (w_fb) atomicAdd(&bstats->exact_fallbacks, (unsigned long long)w_fb);
    if (w_inv) atomicAdd(&bstats->invalid_rays, w_inv);
    if (w_limit) atomicAdd(&bstats->walk_limit_rays, (unsigned long long)w_limit);
    if (w_loc) atomicAdd(&bstats->located, w_loc);
    if (w_lst) atomicAdd(&bstats->locate_steps, w_lst);
  }
}

static size_t al256d(size_t x) { return (x + 255) & ~(size_t)255; }

// The staged work list into device memory, read by the GPU straight from the
// pinned (device-mapped) host staging buffer, and the work counter reset.  A
// kernel rather than a copy: a copy would queue on a copy engine behind the
// caller's bulk ray transfers (measured: a serving tick's launch waited
// 22 ms behind 16 queued uploads).
__global__ void stage_table_kernel(int4* __restrict__ dst, const int4* __restrict__ src, int n16,
                                   unsigned long long* __restrict__ counter) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n16; k += gridDim.x * blockDim.x) dst[k] = src[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0ull;
}

}  // namespace cct

using namespace cct;

struct cct_batch_s {
  int device;
  int n_scenes;
  int max_items;
  uint32_t flags;
  cct_tuning tuning;
  char* d_base;          // scenes | header + items | counter | stats
  SceneDev* d_scenes;
  BatchHeader* d_hdr;    // followed by max_items BatchItemDev
  unsigned long long* d_counter;
  DevStats* d_stats;
  char* h_staging;       // pinned copy of header + items, mapped into the device's address space
  const int4* h_staging_dev;  // its device address
  size_t table_bytes;
  int grid;
  int staged;
  int max_steps;  // the largest step limit of the batch's scenes
};

static size_t batch_smem(int threads) { return sizeof(BatchStacks) * (size_t)(threads / 32); }

static int batch_grid(cct_batch b) {
  int per_sm = 0;
  const int threads = b->tuning.block_threads;
  auto k = (b->flags & CCT_TRACE_EXACT_ONLY) ? batch_kernel<true> : batch_kernel<false>;
  // the stacks of 16 warps exceed the default 48 KB of dynamic shared memory
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(kBatchMaxThreads)) !=
      cudaSuccess)
    cudaGetLastError();
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, batch_smem(threads)) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return sm_count(b->device) * per_sm;
}

extern "C" int cct_batch_create(const cct_scene* scenes, int32_t n_scenes, int32_t max_items, uint32_t flags,
                                cct_batch* out) {
  if (!scenes || !out || n_scenes < 1 || max_items < 1 || max_items > (1 << 20) ||
      (flags & ~(uint32_t)CCT_TRACE_EXACT_ONLY) != 0)
    return CCT_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  const int dev = scenes[0] ? scenes[0]->device : -1;
  for (int k = 0; k < n_scenes; ++k)
    if (!scenes[k] || scenes[k]->device != dev) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(dev);
  auto* b = new cct_batch_s{};
  b->device = dev;
  b->n_scenes = n_scenes;
  b->max_items = max_items;
  b->flags = flags;
  b->tuning = default_tuning();
  b->table_bytes = sizeof(BatchHeader) + sizeof(BatchItemDev) * (size_t)max_items;
  static_assert(sizeof(BatchHeader) % 16 == 0 && sizeof(BatchItemDev) % 16 == 0, "the table is copied as int4");
  const size_t o_scenes = 0, o_table = al256d(sizeof(SceneDev) * n_scenes);
  const size_t o_counter = o_table + al256d(b->table_bytes), o_stats = o_counter + 256;
  const size_t total = o_stats + al256d(sizeof(DevStats));
  if (cudaMalloc(&b->d_base, total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  void* staging_dev = nullptr;
  b->h_staging = nullptr;
  if (cudaHostAlloc(&b->h_staging, b->table_bytes, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&staging_dev, b->h_staging, 0) != cudaSuccess) {
    cudaGetLastError();
    if (b->h_staging) cudaFreeHost(b->h_staging);
    cudaFree(b->d_base);
    delete b;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  std::memset(b->h_staging, 0, b->table_bytes);
  b->h_staging_dev = (const int4*)staging_dev;
  b->d_scenes = (SceneDev*)(b->d_base + o_scenes);
  b->d_hdr = (BatchHeader*)(b->d_base + o_table);
  b->d_counter = (unsigned long long*)(b->d_base + o_counter);
  b->d_stats = (DevStats*)(b->d_base + o_stats);
  std::vector<SceneDev> sd(n_scenes);
  b->max_steps = 1;
  for (int k = 0; k < n_scenes; ++k) {
    sd[k] = scenes[k]->dev;
    b->max_steps = std::max(b->max_steps, sd[k].max_steps);
  }
  cudaError_t e = cudaMemcpy(b->d_scenes, sd.data(), sizeof(SceneDev) * n_scenes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_hdr, 0, b->table_bytes);
  if (e == cudaSuccess) e = cudaMemset(b->d_stats, 0, sizeof(DevStats));
  if (e != cudaSuccess) {
    cudaFreeHost(b->h_staging);
    cudaFree(b->d_base);
    delete b;
    return CCT_ERR_CUDA;
  }
  b->grid = batch_grid(b);
  *out = b;
  return CCT_OK;
}

extern "C" int cct_batch_free(cct_batch b) {
  if (!b) return CCT_OK;
  int rc = CCT_OK;
  {
    DeviceGuard g(b->device);
    if (cudaFreeHost(b->h_staging) != cudaSuccess) rc = CCT_ERR_CUDA;
    if (cudaFree(b->d_base) != cudaSuccess) rc = CCT_ERR_CUDA;
  }
  delete b;
  return rc;
}

extern "C" int cct_batch_set_tuning(cct_batch b, const cct_tuning* tu) {
  if (!b) return CCT_ERR_INVALID_ARGUMENT;
  cct_tuning t = tu ? *tu : default_tuning();
  if (t.block_threads < 32 || t.block_threads > kBatchMaxThreads || t.block_threads % 32 != 0 || t.refill_min < 1 ||
      t.refill_min > 32 || t.chunk < 32 || t.chunk > (1 << 20))
    return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(b->device);
  b->tuning = t;
  b->grid = batch_grid(b);
  return CCT_OK;
}

extern "C" int cct_batch_stage(cct_batch b, const cct_batch_item* items, int32_t n_items) {
  if (!b || n_items < 0 || n_items > b->max_items || (n_items > 0 && !items)) return CCT_ERR_INVALID_ARGUMENT;
  const int chunk = b->tuning.chunk;
  auto* hdr = (BatchHeader*)b->h_staging;
  auto* it = (BatchItemDev*)(b->h_staging + sizeof(BatchHeader));
  long long chunks = 0;
  for (int k = 0; k < n_items; ++k) {
    const cct_batch_item& s = items[k];
    if (s.scene < 0 || s.scene >= b->n_scenes || s.n < 0 || s.n > 0x7fffffffll ||
        !(s.ray_stride == 0 || s.ray_stride == 1 || s.ray_stride == 4) || (s.ray_stride == 4 && s.n > 0x1fffffffll))
      return CCT_ERR_INVALID_ARGUMENT;
    if (s.n > 0 && (!s.d_ox || !s.d_oy || !s.d_dx || !s.d_dy || !s.d_hit_seg || !s.d_t || !s.d_steps))
      return CCT_ERR_INVALID_ARGUMENT;
    chunks += (s.n + chunk - 1) / chunk;
    if (chunks > 0x7fffffffll) return CCT_ERR_INVALID_ARGUMENT;
  }
  chunks = 0;
  for (int k = 0; k < n_items; ++k) {
    const cct_batch_item& s = items[k];
    it[k] = BatchItemDev{s.d_ox, s.d_oy, s.d_dx, s.d_dy, s.d_start_tri, s.d_hit_seg, s.d_t, s.d_steps, (int32_t)s.n,
                         s.scene, (int32_t)chunks, s.ray_stride == 4 ? 4 : 1};
    chunks += (s.n + chunk - 1) / chunk;
  }
  hdr->n_items = n_items;
  hdr->total_chunks = (int32_t)chunks;
  hdr->chunk = chunk;
  b->staged = 1;
  return CCT_OK;
}

extern "C" int cct_batch_enqueue(cct_batch b, void* stream_v) {
  if (!b || !b->staged) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(b->device);
  cudaStream_t stream = (cudaStream_t)stream_v;
  const int n16 = (int)(b->table_bytes / 16);
  stage_table_kernel<<<std::min(152, (n16 + 255) / 256), 256, 0, stream>>>((int4*)b->d_hdr, b->h_staging_dev, n16,
                                                                          b->d_counter);
  if (cudaGetLastError() != cudaSuccess) return CCT_ERR_CUDA;
  const auto* items = (const BatchItemDev*)((const char*)b->d_hdr + sizeof(BatchHeader));
  const size_t smem = batch_smem(b->tuning.block_threads);
  auto k = (b->flags & CCT_TRACE_EXACT_ONLY) ? batch_kernel<true> : batch_kernel<false>;
  k<<<b->grid, b->tuning.block_threads, smem, stream>>>(b->d_scenes, b->d_hdr, items, b->tuning.refill_min,
                                                        b->max_steps, b->d_counter, b->d_stats);
  return cudaGetLastError() == cudaSuccess ? CCT_OK : CCT_ERR_CUDA;
}

extern "C" int cct_batch_get_stats(cct_batch b, cct_stats* out, int reset, void* stream_v) {
  if (!b || !out) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(b->device);
  cudaStream_t stream = (cudaStream_t)stream_v;
  DevStats h{};
  if (cudaMemcpyAsync(&h, b->d_stats, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return CCT_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return CCT_ERR_CUDA;
  if (reset && (cudaMemsetAsync(b->d_stats, 0, sizeof(DevStats), stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess))
    return CCT_ERR_CUDA;
  *out = cct_stats{h.rays, h.steps, h.side_tests, h.exact_fallbacks, h.invalid_rays, h.walk_limit_rays, h.located,
                   h.locate_steps};
  return CCT_OK;
}

extern "C" int cct_trace_batched(const cct_scene* scenes, int32_t n_scenes, const cct_batch_item* items,
                                 int32_t n_items, uint32_t flags, void* stream_v) {
  if (n_items == 0) return CCT_OK;
  cct_batch b = nullptr;
  int rc = cct_batch_create(scenes, n_scenes, std::max(1, n_items), flags, &b);
  if (rc != CCT_OK) return rc;
  rc = cct_batch_stage(b, items, n_items);
  if (rc == CCT_OK) rc = cct_batch_enqueue(b, stream_v);
  if (rc == CCT_OK) {
    DeviceGuard g(b->device);
    if (cudaStreamSynchronize((cudaStream_t)stream_v) != cudaSuccess) rc = CCT_ERR_CUDA;
  }
  const int rc2 = cct_batch_free(b);
  return rc != CCT_OK ? rc : rc2;
}
