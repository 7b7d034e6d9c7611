// The stackless walk (Sec. 5.1) and cct_trace.
//
// Per ray: in the start triangle decide the side (L/R) of all three vertices
// and leave through the CCW edge (a -> b) with s(a) = R, s(b) = L.  Across an
// interior edge the neighbour shares the two decided vertices, so each later
// step decides only the new apex c: s(c) = L -> leave through (R-vertex, c),
// else through (c, L-vertex) -- the two remaining candidates of Sec. 7.2.  A
// constrained edge ends the walk with a hit (t from the edge's line), a hull
// edge with a miss.  Step count = triangles visited (Sec. 5.4).
//
// GPU mapping.  One ray per lane.  A warp draws ray indices from a global
// counter in chunks and serves idle lanes (ballot + prefix popcount) once at
// least `refill_min` of them are idle, so divergent ray lengths do not idle
// the warp.  A served lane starts in first-triangle mode, in the given start
// triangle or -- no start cells given: the Sec. 5.2 seed walk runs inside this
// kernel -- in the seed triangle of its origin's grid cell.  The seed
// triangle's inside test is the first-triangle step's own (the given start
// triangle is checked the same way), so only origins outside it take further
// locate iterations.  Every loop iteration issues exactly one dependent
// 32-byte record load per active lane, whatever its mode.
#include <algorithm>
#include <cmath>

#include "cct_internal.cuh"

namespace cct {

enum : int { kModeLocate = 0, kModeFirst = 1, kModeWalk = 2, kModeSeed = 3 };
enum : int { kSrcPlainUser = 0, kSrcPlainDev = 1, kSrcSorted = 2, kSrcLocate = 3 };
// rare per-warp counters (shared memory)
enum : int { kCntRays = 0, kCntFallback, kCntInvalid, kCntLimit, kCntLocated, kCntLocSteps, kRareCounters };

constexpr int kWalkMaxThreads = 512;

struct WalkParams {
  int refill_min;  // serve idle lanes once this many are idle (or the whole warp is)
  int chunk;       // ray indices a warp takes from the global counter at once
};

// Writes the parked result of a finished lane: hit id and t come from its
// final record (reloaded: it was read one iteration ago, so from L1/L2),
// `st` is the step count or a negative per-ray status.
__device__ __forceinline__ void complete_ray(const TriRec* __restrict__ rec, int T, int e, int st, int ox, int oy,
                                             int kx, int ky, int idx, int32_t* __restrict__ hit_out,
                                             float* __restrict__ t_out, int32_t* __restrict__ steps_out) {
  int32_t h = -1;
  float t = __int_as_float(0x7fc00000);  // NaN: invalid ray
  if (st > 0) {
    const TriRec r = load_rec(rec + T);
    const int32_t w = nb_of(r, e);
    if (w <= -2) {
      h = -2 - w;
      const int a = (e == 2) ? 0 : e + 1, b = (e == 0) ? 2 : e - 1;
      t = hit_param_fast(vx_of(r, a), vy_of(r, a), vx_of(r, b), vy_of(r, b), ox, oy, kx, ky);
    } else {
      t = __int_as_float(0x7f800000);  // +inf: left through the hull
    }
  }
  hit_out[idx] = h;
  t_out[idx] = t;
  steps_out[idx] = st;
}

template <bool kExact, int kSrc>
__global__ void __launch_bounds__(kWalkMaxThreads) walk_kernel(SceneDev S, RaySrc R, WalkParams P,
                                                               int32_t* __restrict__ hit_out,
                                                               float* __restrict__ t_out,
                                                               int32_t* __restrict__ steps_out,
                                                               unsigned long long* __restrict__ counter) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr bool kLocate = (kSrc == kSrcLocate);
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int n = (int)R.n;
  int pool_next = 0, pool_end = 0;
  bool exhausted = false;

  // lane state: walking (active), finished with a parked result (done), or idle;
  // in locate mode nsteps counts locate steps
  bool active = false, done = false;
  int mode = kModeFirst;
  int idx = 0, ox = 0, oy = 0, kx = 0, ky = 0, T = 0, j = 0, nsteps = 0;
  float fdx = 0.f, fdy = 0.f;

  // hot counters in registers, rare ones per warp in shared memory
  unsigned c_steps = 0, c_side = 0;
  __shared__ unsigned s_cnt[kWalkMaxThreads / 32][kRareCounters];
  unsigned* cnt = s_cnt[threadIdx.x >> 5];
  if (lane < kRareCounters) cnt[lane] = 0;
  __syncwarp();

  while (true) {
    // ---------------------------------------------------------------- serve idle lanes
    // (also where finished lanes write their parked results: a batch of
    // completions costs the warp one pass, not one per iteration)
    while (!exhausted) {
      const unsigned need = __ballot_sync(FULL, !active);
      if (need == 0u) break;
      if (__popc(need) < P.refill_min && need != FULL) break;
      if (done) {
        complete_ray(S.rec, T, j, nsteps, ox, oy, kx, ky, idx, hit_out, t_out, steps_out);
        done = false;
      }
      if (pool_next >= pool_end) {
        int base = 0;
        if (lane == 0) base = (int)atomicAdd(counter, (unsigned long long)P.chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n) {
          exhausted = true;
          break;
        }
        pool_next = base;
        pool_end = min(base + P.chunk, n);
      }
      const int avail = pool_end - pool_next;
      const int rank = __popc(need & lt);
      if (!active && rank < avail) {
        idx = pool_next + rank;
        int s = -1;
        if (kSrc == kSrcSorted) {
          const int4 rr = R.rays[idx];
          ox = rr.x;
          oy = rr.y;
          fdx = __int_as_float(rr.z);
          fdy = __int_as_float(rr.w);
          s = R.start[idx];
        } else {
          ox = R.ox[idx];
          oy = R.oy[idx];
          fdx = R.dx[idx];
          fdy = R.dy[idx];
          if (!kLocate) {
            s = R.start[idx];
            if (kSrc == kSrcPlainUser) s = (s >= 0 && s < S.n_tri) ? S.user2dev[s] : -1;
          }
        }
        // origins outside the domain lie in no triangle; rejecting them here
        // keeps every coordinate difference of the walk within int32
        bool ok = dir_to_k(fdx, kx) && dir_to_k(fdy, ky) && (kx | ky) != 0 && ox >= 0 && oy >= 0 && ox <= S.D &&
                  oy <= S.D;
        if (kLocate) {
          if (ok) {
            s = S.seeds[seed_cell(S, ox, oy)];
            mode = kModeSeed;
            atomicAdd(&cnt[kCntLocated], 1u);
          }
        } else {
          mode = kModeFirst;
          ok = ok && s >= 0 && s < S.n_tri;
        }
        if (kSrc == kSrcSorted) idx = R.orig[idx];
        atomicAdd(&cnt[kCntRays], 1u);
        if (ok) {
          T = s;
          nsteps = 0;
          active = true;
        } else {
          hit_out[idx] = -1;
          t_out[idx] = __int_as_float(0x7fc00000);
          steps_out[idx] = CCT_RAY_INVALID;
          atomicAdd(&cnt[kCntInvalid], 1u);
        }
      }
      pool_next += min(__popc(need), avail);
    }
    if (!__any_sync(FULL, active)) {
      if (exhausted) break;
      continue;
    }

    // ---------------------------------------------------------------- one record per active lane
    if (active) {
      const TriRec r = load_rec(S.rec + T);
      int status = 0;  // 0 walking on, > 0 finished (steps), < 0 per-ray status
      bool step = true;  // take a walk step in T this iteration
      if (kLocate && mode == kModeLocate) {
        // Sec. 5.2 past the seed triangle: T was entered through edge j on the
        // way from the seed point to the origin; nsteps counts locate steps
        ++nsteps;
        int cx, cy;
        seed_point(S, ox, oy, cx, cy);
        const int res = locate_step_entered(S, r, T, j, ox, oy, cx, cy);
        step = false;
        if (res != 0 || nsteps > S.max_steps) {
          atomicAdd(&cnt[kCntLocSteps], (unsigned)nsteps);
          nsteps = 0;
          if (res > 0) {
            mode = kModeFirst;  // T holds the origin: its first walk step follows
            step = true;
          } else {
            status = CCT_RAY_INVALID;  // origin on an edge or a vertex: not a valid ray origin
            atomicAdd(&cnt[kCntInvalid], 1u);
          }
        }
      }
      if (step) {
        int e = 0;
        if (mode != kModeWalk) {
          // first triangle: the given start triangle, the seed triangle
          // (kModeSeed) or the triangle where the locate walk found the origin
          const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
          const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
          bool inside = true;
          if (!kLocate || mode == kModeSeed) {
            const long long o0 = orient_i(x1, y1, x2, y2, ox, oy), o1 = orient_i(x2, y2, x0, y0, ox, oy);
            const long long o2 = orient_i(x0, y0, x1, y1, ox, oy);
            inside = o0 > 0 && o1 > 0 && o2 > 0;
            if (kLocate) {
              if (!inside && (o0 < 0 || o1 < 0 || o2 < 0)) {
                // the origin lies outside the seed triangle: the locate walk
                // leaves it towards the origin
                int cx, cy;
                seed_point(S, ox, oy, cx, cy);
                nsteps = 1;
                step = false;
                if (locate_hop(S, r, T, j, seed_exit(r, cx, cy, ox, oy))) {
                  mode = kModeLocate;
                } else {
                  status = CCT_RAY_INVALID;
                  atomicAdd(&cnt[kCntInvalid], 1u);
                  atomicAdd(&cnt[kCntLocSteps], 1u);
                }
              } else {
                atomicAdd(&cnt[kCntLocSteps], 1u);  // located in one step (or on the seed triangle's boundary)
              }
            }
          }
          if (step) {
            unsigned fb = 0;
            const bool s0 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x0, y0, fb);
            const bool s1 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x1, y1, fb);
            const bool s2 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x2, y2, fb);
            if (fb) atomicAdd(&cnt[kCntFallback], fb);
            c_side += 3;
            e = (!s1 && s2) ? 0 : ((!s2 && s0) ? 1 : 2);
            mode = kModeWalk;
            if (!inside) {
              status = CCT_RAY_INVALID;
              atomicAdd(&cnt[kCntInvalid], 1u);
            }
          }
        } else {
          unsigned fb = 0;
          const bool sc = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, vx_of(r, j), vy_of(r, j), fb);
          if (fb) atomicAdd(&cnt[kCntFallback], fb);
          ++c_side;
          e = sc ? (j == 2 ? 0 : j + 1) : (j == 0 ? 2 : j - 1);
        }
        if (step && status == 0) {
          ++nsteps;
          const int32_t w = nb_of(r, e);
          if (w >= 0) {
            if (nsteps >= S.max_steps) {
              status = CCT_RAY_WALK_LIMIT;
              atomicAdd(&cnt[kCntLimit], 1u);
            } else {
              T = w >> 2;
              j = w & 3;
            }
          } else {
            status = nsteps;  // hit or miss: park T (the final triangle) and e
            j = e;
            c_steps += (unsigned)nsteps;
          }
        }
      }
      if (status != 0) {
        nsteps = status;
        active = false;
        done = true;
      }
    }
  }
  if (done) complete_ray(S.rec, T, j, nsteps, ox, oy, kx, ky, idx, hit_out, t_out, steps_out);
  // ---------------------------------------------------------------- counters: one atomic per warp and counter
  const unsigned long long w_steps = warp_sum((unsigned long long)c_steps);
  const unsigned long long w_side = warp_sum((unsigned long long)c_side);
  __syncwarp();
  const unsigned long long w_rays = cnt[kCntRays], w_fb = cnt[kCntFallback], w_inv = cnt[kCntInvalid];
  const unsigned long long w_lim = cnt[kCntLimit], w_loc = cnt[kCntLocated], w_lst = cnt[kCntLocSteps];
  if (lane == 0) {
    if (w_rays) atomicAdd(&S.stats->rays, w_rays);
    if (w_steps) atomicAdd(&S.stats->steps, w_steps);
    if (w_side) atomicAdd(&S.stats->side_tests, w_side);
    if (w_fb) atomicAdd(&S.stats->exact_fallbacks, w_fb);
    if (w_inv) atomicAdd(&S.stats->invalid_rays, w_inv);
    if (w_lim) atomicAdd(&S.stats->walk_limit_rays, w_lim);
    if (w_loc) atomicAdd(&S.stats->located, w_loc);
    if (w_lst) atomicAdd(&S.stats->locate_steps, w_lst);
  }
}

template <bool kExact, int kSrc>
static cudaError_t launch_walk_t(const SceneDev& S, const RaySrc& R, const cct_tuning& tu, int32_t* hit, float* t,
                                 int32_t* steps, unsigned long long* counter, int dev, cudaStream_t stream) {
  auto k = walk_kernel<kExact, kSrc>;
  const int threads = tu.block_threads;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  const long long want = (R.n + threads - 1) / threads;
  long long grid = std::min<long long>((long long)sm_count(dev) * per_sm, want);
  if (grid < 1) grid = 1;
  WalkParams P{std::max(1, std::min(32, tu.refill_min)), std::max(32, tu.chunk)};
  k<<<(unsigned)grid, threads, 0, stream>>>(S, R, P, hit, t, steps, counter);
  return cudaGetLastError();
}

static cudaError_t launch_walk_src(bool exact, int src, const SceneDev& S, const RaySrc& R, const cct_tuning& tu,
                                   int32_t* hit, float* t, int32_t* steps, unsigned long long* counter, int dev,
                                   cudaStream_t stream) {
#define CCT_WALK_CASE(SRC)                                                                 \
  case SRC:                                                                                \
    return exact ? launch_walk_t<true, SRC>(S, R, tu, hit, t, steps, counter, dev, stream) \
                 : launch_walk_t<false, SRC>(S, R, tu, hit, t, steps, counter, dev, stream);
  switch (src) {
    CCT_WALK_CASE(kSrcPlainUser)
    CCT_WALK_CASE(kSrcPlainDev)
    CCT_WALK_CASE(kSrcSorted)
    CCT_WALK_CASE(kSrcLocate)
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
  const cct_tuning& tu = scene->tuning;
  flags |= tu.trace_flags;
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
      (tu->trace_flags & ~(CCT_TRACE_EXACT_ONLY | CCT_TRACE_BIN | CCT_TRACE_SPLIT_LOCATE)) != 0)
    return CCT_ERR_INVALID_ARGUMENT;
  scene->tuning = *tu;
  return CCT_OK;
}

extern "C" int cct_scene_get_tuning(cct_scene scene, cct_tuning* out) {
  if (!scene || !out) return CCT_ERR_INVALID_ARGUMENT;
  *out = scene->tuning;
  return CCT_OK;
}
