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
// the warp; a served lane starts in locate mode (no start cells given: the
// Sec. 5.2 seed walk runs inside this kernel) or in first-triangle mode.
// Every loop iteration issues exactly one dependent 32-byte record load per
// active lane, whatever its mode.
#include <algorithm>
#include <cmath>

#include "cct_internal.cuh"

namespace cct {

enum : int { kModeLocate = 0, kModeFirst = 1, kModeWalk = 2 };
enum : int { kSrcPlainUser = 0, kSrcPlainDev = 1, kSrcSorted = 2, kSrcLocate = 3 };

constexpr int kWalkMaxThreads = 512;

struct WalkParams {
  int refill_min;  // serve idle lanes once this many are idle (or the whole warp is)
  int chunk;       // ray indices a warp takes from the global counter at once
};

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

  bool active = false;
  int mode = kModeFirst;
  int idx = 0, ox = 0, oy = 0, kx = 0, ky = 0, T = 0, j = 0, nsteps = 0, lsteps = 0;
  int px3 = 0, py3 = 0;  // locate seed point x 3 (kLocate)
  float fdx = 0.f, fdy = 0.f;

  unsigned c_steps = 0, c_side = 0, c_fb = 0, c_rays = 0, c_inv = 0, c_lim = 0, c_loc = 0, c_lsteps = 0;

  while (true) {
    // ---------------------------------------------------------------- serve idle lanes
    while (!exhausted) {
      const unsigned need = __ballot_sync(FULL, !active);
      if (need == 0u) break;
      if (__popc(need) < P.refill_min && need != FULL) break;
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
        bool ok = dir_to_k(fdx, kx) && dir_to_k(fdy, ky) && (kx | ky) != 0;
        if (kLocate) {
          if (ok && ox >= 0 && oy >= 0 && ox <= S.D && oy <= S.D) {
            const int G = S.G;
            const int ix = min(G - 1, (int)((long long)ox * G / S.D));
            const int iy = min(G - 1, (int)((long long)oy * G / S.D));
            const SeedCell sd = S.seeds[iy * G + ix];
            px3 = sd.px3;
            py3 = sd.py3;
            s = sd.tri;
            j = 3;
            mode = kModeLocate;
            lsteps = 0;
            ++c_loc;
          } else {
            ok = false;
          }
        } else {
          mode = kModeFirst;
          ok = ok && s >= 0 && s < S.n_tri;
        }
        if (kSrc == kSrcSorted) idx = R.orig[idx];
        if (ok) {
          T = s;
          nsteps = 0;
          active = true;
        } else {
          hit_out[idx] = -1;
          t_out[idx] = __int_as_float(0x7fc00000);
          steps_out[idx] = CCT_RAY_INVALID;
          ++c_inv;
          ++c_rays;
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
      bool done = false;
      int32_t res_hit = -1, res_steps = CCT_RAY_INVALID;
      float res_t = __int_as_float(0x7fc00000);
      bool advance = true;
      if (kLocate && mode == kModeLocate) {
        // Sec. 5.2: walk from the seed point towards the origin until the
        // current triangle holds it (this triangle is then the start triangle)
        ++lsteps;
        const int res = locate_step(S, r, T, j, ox, oy, px3, py3);
        if (res > 0) {
          mode = kModeFirst;
          c_lsteps += (unsigned)lsteps;
        } else if (res < 0 || lsteps > S.max_steps) {
          done = true;  // origin on an edge or a vertex: not a valid ray origin
          ++c_inv;
          c_lsteps += (unsigned)lsteps;
        } else {
          advance = false;
        }
      }
      if (!done && advance) {
        int e;
        if (mode == kModeFirst) {
          const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
          const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
          bool inside = true;
          if (!kLocate)
            inside = orient_ll(x1, y1, x2, y2, ox, oy) > 0 && orient_ll(x2, y2, x0, y0, ox, oy) > 0 &&
                     orient_ll(x0, y0, x1, y1, ox, oy) > 0;
          const bool s0 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x0, y0, c_fb);
          const bool s1 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x1, y1, c_fb);
          const bool s2 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x2, y2, c_fb);
          c_side += 3;
          e = (!s1 && s2) ? 0 : ((!s2 && s0) ? 1 : 2);
          mode = kModeWalk;
          if (!inside) {
            done = true;
            ++c_inv;
          }
        } else {
          const bool sc = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, vx_of(r, j), vy_of(r, j), c_fb);
          ++c_side;
          e = sc ? (j == 2 ? 0 : j + 1) : (j == 0 ? 2 : j - 1);
        }
        if (!done) {
          ++nsteps;
          const int32_t w = nb_of(r, e);
          if (w >= 0) {
            if (nsteps >= S.max_steps) {
              done = true;
              res_steps = CCT_RAY_WALK_LIMIT;
              ++c_lim;
            } else {
              T = w >> 2;
              j = w & 3;
            }
          } else {
            done = true;
            res_steps = nsteps;
            c_steps += (unsigned)nsteps;
            if (w <= -2) {
              res_hit = -2 - w;
              const int a = (e == 2) ? 0 : e + 1, b = (e == 0) ? 2 : e - 1;
              res_t = hit_param(vx_of(r, a), vy_of(r, a), vx_of(r, b), vy_of(r, b), ox, oy, kx, ky);
            } else {
              res_t = __int_as_float(0x7f800000);  // +inf: left through the hull
            }
          }
        }
      }
      if (done) {
        hit_out[idx] = res_hit;
        t_out[idx] = res_t;
        steps_out[idx] = res_steps;
        ++c_rays;
        active = false;
      }
    }
  }
  // ---------------------------------------------------------------- counters: one atomic per warp and counter
  const unsigned long long w_steps = warp_sum((unsigned long long)c_steps);
  const unsigned long long w_side = warp_sum((unsigned long long)c_side);
  const unsigned long long w_rays = warp_sum((unsigned long long)c_rays);
  const unsigned long long w_fb = warp_sum((unsigned long long)c_fb);
  const unsigned long long w_inv = warp_sum((unsigned long long)c_inv);
  const unsigned long long w_lim = warp_sum((unsigned long long)c_lim);
  const unsigned long long w_loc = warp_sum((unsigned long long)c_loc);
  const unsigned long long w_lst = warp_sum((unsigned long long)c_lsteps);
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
  // launches of at most 2^30 rays keep every in-kernel index in 32 bits
  constexpr int64_t kMaxLaunch = 1ll << 30;
  const int64_t n_max = std::min<int64_t>(n, kMaxLaunch);
  const int shift = bin ? (tu.bin_shift >= 0 ? tu.bin_shift : default_bin_shift(n_max, S.n_tri)) : 0;
  const size_t o_start = 256;
  const size_t o_bin = o_start + ((bin && !start) ? al256(sizeof(int32_t) * (size_t)n_max) : 0);
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
      (tu->trace_flags & ~(CCT_TRACE_EXACT_ONLY | CCT_TRACE_BIN)) != 0)
    return CCT_ERR_INVALID_ARGUMENT;
  scene->tuning = *tu;
  return CCT_OK;
}

extern "C" int cct_scene_get_tuning(cct_scene scene, cct_tuning* out) {
  if (!scene || !out) return CCT_ERR_INVALID_ARGUMENT;
  *out = scene->tuning;
  return CCT_OK;
}
