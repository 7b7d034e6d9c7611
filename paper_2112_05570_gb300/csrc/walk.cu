// The stackless walk (Sec. 5.1) and cct_trace.
//
// Per ray: in the start triangle decide the side (L/R) of all three vertices
// and leave through the CCW edge (a -> b) with s(a) = R, s(b) = L.  Across an
// interior edge the neighbour shares the two decided vertices, so each later
// step decides only the new apex c: s(c) = L -> leave through (R-vertex, c),
// else through (c, L-vertex) -- the "two remaining candidates" of Sec. 7.2.
// A constrained edge ends the walk with a hit (t from the edge's line), a
// hull edge with a miss.  Step count = triangles visited (Sec. 5.4).
//
// GPU mapping: one ray per lane; a warp keeps a pool of ray indices taken in
// chunks from a global counter, and lanes whose ray finished are refilled at
// the top of every iteration (ballot + prefix rank), so short rays do not idle
// lanes while long rays run.  Each iteration issues exactly one dependent
// 32-byte record load per active lane.
#include <algorithm>
#include <cmath>

#include "cct_internal.cuh"

namespace cct {

constexpr int kWalkThreads = 256;
constexpr int kChunk = 128;

template <bool kExact, bool kSorted, bool kStartUser>
__global__ void __launch_bounds__(kWalkThreads) walk_kernel(SceneDev S, RaySrc R, int32_t* __restrict__ hit_out,
                                                            float* __restrict__ t_out,
                                                            int32_t* __restrict__ steps_out,
                                                            unsigned long long* __restrict__ counter) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  long long pool_next = 0, pool_end = 0;
  bool exhausted = false;

  bool active = false, first = false, bad = false;
  long long out_idx = 0;
  int ox = 0, oy = 0, kx = 0, ky = 0, T = 0, j = 0, nsteps = 0;
  float fdx = 0.f, fdy = 0.f;

  unsigned long long c_steps = 0, c_side = 0;
  unsigned c_rays = 0, c_fb = 0, c_inv = 0, c_lim = 0;

  while (true) {
    // ---- refill lanes whose ray has finished
    const unsigned need = __ballot_sync(FULL, !active);
    if (need && !exhausted) {
      int rank = active ? -1 : __popc(need & lt);
      int cnt = __popc(need);
      while (cnt > 0) {
        long long avail = pool_end - pool_next;
        if (avail <= 0) {
          long long base = 0;
          if (lane == 0) base = (long long)atomicAdd(counter, (unsigned long long)kChunk);
          base = __shfl_sync(FULL, base, 0);
          if (base >= R.n) {
            exhausted = true;
            break;
          }
          pool_next = base;
          pool_end = (base + (long long)kChunk < (long long)R.n) ? base + (long long)kChunk : (long long)R.n;
          continue;
        }
        const int take = (avail < (long long)cnt) ? (int)avail : cnt;
        if (rank >= 0 && rank < take) {
          const long long i = pool_next + rank;
          int s;
          if (kSorted) {
            const int4 rr = R.rays[i];
            ox = rr.x;
            oy = rr.y;
            fdx = __int_as_float(rr.z);
            fdy = __int_as_float(rr.w);
            s = R.start[i];
            out_idx = R.orig[i];
          } else {
            ox = R.ox[i];
            oy = R.oy[i];
            fdx = R.dx[i];
            fdy = R.dy[i];
            s = R.start[i];
            out_idx = i;
            if (kStartUser) s = (s >= 0 && s < S.n_tri) ? S.user2dev[s] : -1;
          }
          T = s;
          bad = !(dir_to_k(fdx, kx) && dir_to_k(fdy, ky)) || (kx == 0 && ky == 0) || s < 0 || s >= S.n_tri;
          first = true;
          nsteps = 0;
          active = true;
        }
        pool_next += take;
        cnt -= take;
        rank -= take;
      }
    }
    if (!__any_sync(FULL, active)) break;

    // ---- one step per active lane
    if (active) {
      bool done = false;
      int32_t res_hit = -1, res_steps = CCT_RAY_INVALID;
      float res_t = __int_as_float(0x7fc00000);  // NaN
      if (bad) {
        done = true;
        ++c_inv;
      } else {
        const TriRec r = load_rec(S.rec + T);
        int e = 0;
        if (first) {
          const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
          const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
          const bool inside = orient_ll(x1, y1, x2, y2, ox, oy) > 0 && orient_ll(x2, y2, x0, y0, ox, oy) > 0 &&
                              orient_ll(x0, y0, x1, y1, ox, oy) > 0;
          if (!inside) {
            done = true;
            ++c_inv;
          } else {
            const bool s0 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x0, y0, c_fb);
            const bool s1 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x1, y1, c_fb);
            const bool s2 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x2, y2, c_fb);
            c_side += 3;
            e = (!s1 && s2) ? 0 : ((!s2 && s0) ? 1 : 2);
          }
          first = false;
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
              res_t = __int_as_float(0x7f800000);  // +inf
            }
          }
        }
      }
      if (done) {
        hit_out[out_idx] = res_hit;
        t_out[out_idx] = res_t;
        steps_out[out_idx] = res_steps;
        ++c_rays;
        active = false;
      }
    }
  }
  // ---- counters: one atomic per warp and counter
  c_steps = warp_sum(c_steps);
  c_side = warp_sum(c_side);
  const unsigned long long r_rays = warp_sum((unsigned long long)c_rays);
  const unsigned long long r_fb = warp_sum((unsigned long long)c_fb);
  const unsigned long long r_inv = warp_sum((unsigned long long)c_inv);
  const unsigned long long r_lim = warp_sum((unsigned long long)c_lim);
  if (lane == 0) {
    if (r_rays) atomicAdd(&S.stats->rays, r_rays);
    if (c_steps) atomicAdd(&S.stats->steps, c_steps);
    if (c_side) atomicAdd(&S.stats->side_tests, c_side);
    if (r_fb) atomicAdd(&S.stats->exact_fallbacks, r_fb);
    if (r_inv) atomicAdd(&S.stats->invalid_rays, r_inv);
    if (r_lim) atomicAdd(&S.stats->walk_limit_rays, r_lim);
  }
}

template <bool kExact, bool kSorted, bool kStartUser>
static cudaError_t launch_walk_t(const SceneDev& S, const RaySrc& R, int32_t* hit, float* t, int32_t* steps,
                                 unsigned long long* counter, int dev, cudaStream_t stream) {
  auto k = walk_kernel<kExact, kSorted, kStartUser>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWalkThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  long long want = (R.n + kWalkThreads - 1) / kWalkThreads;
  long long grid = std::min<long long>((long long)sm_count(dev) * per_sm, want);
  if (grid < 1) grid = 1;
  k<<<(unsigned)grid, kWalkThreads, 0, stream>>>(S, R, hit, t, steps, counter);
  return cudaGetLastError();
}

cudaError_t launch_walk(bool exact, bool sorted, bool start_user, const SceneDev& S, const RaySrc& R,
                               int32_t* hit, float* t, int32_t* steps, unsigned long long* counter, int dev,
                               cudaStream_t stream) {
  if (sorted)
    return exact ? launch_walk_t<true, true, false>(S, R, hit, t, steps, counter, dev, stream)
                 : launch_walk_t<false, true, false>(S, R, hit, t, steps, counter, dev, stream);
  if (start_user)
    return exact ? launch_walk_t<true, false, true>(S, R, hit, t, steps, counter, dev, stream)
                 : launch_walk_t<false, false, true>(S, R, hit, t, steps, counter, dev, stream);
  return exact ? launch_walk_t<true, false, false>(S, R, hit, t, steps, counter, dev, stream)
               : launch_walk_t<false, false, false>(S, R, hit, t, steps, counter, dev, stream);
}

// Bin granularity: record indices >> shift, so that bins hold ~64 rays on average.
static int default_bin_shift(int64_t n, int32_t n_tri) {
  int shift = 0;
  const int64_t target = std::max<int64_t>(1024, n / 64);
  while (((int64_t)n_tri >> shift) > target && shift < 30) ++shift;
  return shift;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace cct

using namespace cct;

extern "C" int cct_trace(cct_scene scene, const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                         const int32_t* start, int64_t n, int32_t* hit, float* t, int32_t* steps, uint32_t flags,
                         void* stream_v) {
  if (!scene || n < 0) return CCT_ERR_INVALID_ARGUMENT;
  if (n == 0) return CCT_OK;
  if (!ox || !oy || !dx || !dy || !hit || !t || !steps) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(scene->device);
  cudaStream_t stream = (cudaStream_t)stream_v;
  const SceneDev& S = scene->dev;
  const bool exact = (flags & CCT_TRACE_EXACT_ONLY) != 0;
  const bool bin = (flags & CCT_TRACE_BIN) != 0;
  const int shift = bin ? default_bin_shift(n, S.n_tri) : 0;
  const size_t o_cnt = 0;
  const size_t o_start = o_cnt + 256;
  const size_t o_bin = o_start + (start ? 0 : al256(sizeof(int32_t) * (size_t)n));
  const size_t total = o_bin + (bin ? bin_scratch_bytes(n, S.n_tri, shift) : 0);
  Scratch sc;
  sc.stream = stream;
  if (cudaMallocAsync((void**)&sc.base, total, stream) != cudaSuccess) {
    cudaGetLastError();
    sc.base = nullptr;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  if (cudaMemsetAsync(sc.base + o_cnt, 0, 8, stream) != cudaSuccess) return CCT_ERR_CUDA;
  unsigned long long* counter = (unsigned long long*)(sc.base + o_cnt);
  const int32_t* st = start;
  bool st_user = true;
  if (!start) {
    int32_t* sbuf = (int32_t*)(sc.base + o_start);
    if (launch_locate(S, ox, oy, n, sbuf, false, stream) != cudaSuccess) return CCT_ERR_CUDA;
    st = sbuf;
    st_user = false;
  }
  RaySrc R{ox, oy, dx, dy, st, nullptr, nullptr, n};
  if (bin) {
    BinOut bo{};
    if (launch_bin(S, ox, oy, dx, dy, st, st_user, n, shift, sc.base + o_bin, bo, stream) != cudaSuccess)
      return CCT_ERR_CUDA;
    R.rays = bo.rays;
    R.start = bo.start;
    R.orig = bo.orig;
  }
  if (launch_walk(exact, bin, !bin && st_user, S, R, hit, t, steps, counter, scene->device, stream) != cudaSuccess)
    return CCT_ERR_CUDA;
  return CCT_OK;
}
