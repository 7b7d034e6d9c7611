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
// The table is filled from a pinned host staging buffer by
// cct_batch_enqueue (a fixed-size copy, a counter reset, one kernel), so the
// enqueue can be captured once in a CUDA graph and replayed after each
// cct_batch_stage.
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

__device__ __forceinline__ void batch_complete(const BatchItemDev& it, const TriRec* __restrict__ rec, int T, int e,
                                               int st, int ox, int oy, int kx, int ky, int idx) {
  int32_t h = -1;
  float t = __int_as_float(0x7fc00000);
  if (st > 0) {
    const TriRec r = load_rec(rec + T);
    const int32_t w = nb_of(r, e);
    if (w <= -2) {
      h = -2 - w;
      const int a = (e == 2) ? 0 : e + 1, b = (e == 0) ? 2 : e - 1;
      t = hit_param_fast(vx_of(r, a), vy_of(r, a), vx_of(r, b), vy_of(r, b), ox, oy, kx, ky);
    } else {
      t = __int_as_float(0x7f800000);
    }
  }
  it.hit[idx] = h;
  it.t[idx] = t;
  it.steps[idx] = st;
}

template <bool kExact>
__global__ void __launch_bounds__(kBatchMaxThreads) batch_kernel(const SceneDev* __restrict__ scenes,
                                                                 const BatchHeader* __restrict__ hdr,
                                                                 const BatchItemDev* __restrict__ items,
                                                                 int refill_min, unsigned long long* counter,
                                                                 DevStats* bstats) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int n_items = hdr->n_items, total = hdr->total_chunks, chunk = hdr->chunk;
  // warp-uniform pool: a range of rays of one item
  int p_item = -1, p_next = 0, p_end = 0;
  bool exhausted = n_items <= 0;
  // lane state: walking (active), finished with a parked result (done), or idle
  bool active = false, done = false;
  // modes: 0 locate past the seed triangle, 1 first triangle, 2 walk, 3 seed triangle
  int mode = 1, item = 0, idx = 0, ox = 0, oy = 0, kx = 0, ky = 0, T = 0, j = 0, nsteps = 0, lsteps = 0;
  int max_steps = 0, scene = 0;
  float fdx = 0.f, fdy = 0.f;
  const TriRec* rec = nullptr;
  unsigned c_steps = 0, c_side = 0, c_fb = 0, c_rays = 0, c_inv = 0, c_lim = 0, c_loc = 0, c_lsteps = 0;

  while (true) {
    while (!exhausted) {
      const unsigned need = __ballot_sync(FULL, !active);
      if (need == 0u) break;
      if (__popc(need) < refill_min && need != FULL) break;
      if (done) {
        batch_complete(items[item], rec, T, j, nsteps, ox, oy, kx, ky, idx);
        done = false;
      }
      if (p_next >= p_end) {
        int c = 0;
        if (lane == 0) c = (int)atomicAdd(counter, 1ull);
        c = __shfl_sync(FULL, c, 0);
        if (c >= total) {
          exhausted = true;
          break;
        }
        p_item = find_item(items, n_items, c);
        const BatchItemDev& it = items[p_item];
        p_next = (c - it.chunk_begin) * chunk;
        p_end = min(p_next + chunk, it.n);
      }
      const int avail = p_end - p_next;
      const int rank = __popc(need & lt);
      if (!active && rank < avail) {
        const BatchItemDev& it = items[p_item];
        const SceneDev& S = scenes[it.scene];
        item = p_item;
        scene = it.scene;
        idx = p_next + rank;
        const long long ri = (long long)idx * it.stride;
        ox = it.ox[ri];
        oy = it.oy[ri];
        fdx = it.dx[ri];
        fdy = it.dy[ri];
        rec = S.rec;
        max_steps = S.max_steps;
        bool ok = dir_to_k(fdx, kx) && dir_to_k(fdy, ky) && (kx | ky) != 0;
        int s = -1;
        if (it.start == nullptr) {
          if (ok && ox >= 0 && oy >= 0 && ox <= S.D && oy <= S.D) {
            s = S.seeds[seed_cell(S, ox, oy)];
            mode = 3;
            lsteps = 0;
            ++c_loc;
          } else {
            ok = false;
          }
        } else {
          s = it.start[idx];
          s = (s >= 0 && s < S.n_tri) ? S.user2dev[s] : -1;
          ok = ok && s >= 0;
          mode = 1;
        }
        ++c_rays;
        if (ok) {
          T = s;
          nsteps = 0;
          active = true;
        } else {
          it.hit[idx] = -1;
          it.t[idx] = __int_as_float(0x7fc00000);
          it.steps[idx] = CCT_RAY_INVALID;
          ++c_inv;
        }
      }
      p_next += min(__popc(need), avail);
    }
    if (!__any_sync(FULL, active)) {
      if (exhausted) break;
      continue;
    }
    if (active) {
      const TriRec r = load_rec(rec + T);
      int status = 0;
      bool step = true;
      if (mode == 0) {
        ++lsteps;
        int cx, cy;
        seed_point(scenes[scene], ox, oy, cx, cy);
        const int res = locate_step_entered(scenes[scene], r, T, j, ox, oy, cx, cy);
        step = false;
        if (res > 0) {
          mode = 1;
          step = true;
          c_lsteps += (unsigned)lsteps;
        } else if (res < 0 || lsteps > max_steps) {
          status = CCT_RAY_INVALID;
          ++c_inv;
          c_lsteps += (unsigned)lsteps;
        }
      }
      if (step) {
        int e = 0;
        if (mode != 2) {
          const int x0 = vx_of(r, 0), y0 = vy_of(r, 0), x1 = vx_of(r, 1), y1 = vy_of(r, 1);
          const int x2 = vx_of(r, 2), y2 = vy_of(r, 2);
          bool inside = true;
          if (mode == 3 || mode == 1) {
            const long long o0 = orient_i(x1, y1, x2, y2, ox, oy), o1 = orient_i(x2, y2, x0, y0, ox, oy);
            const long long o2 = orient_i(x0, y0, x1, y1, ox, oy);
            inside = o0 > 0 && o1 > 0 && o2 > 0;
            if (mode == 3) {
              lsteps = 1;
              if (!inside && (o0 < 0 || o1 < 0 || o2 < 0)) {
                // outside the seed triangle: the Sec. 5.2 locate walk leaves it
                int cx, cy;
                seed_point(scenes[scene], ox, oy, cx, cy);
                step = false;
                if (locate_hop(scenes[scene], r, T, j, seed_exit(r, cx, cy, ox, oy))) {
                  mode = 0;
                } else {
                  status = CCT_RAY_INVALID;
                  ++c_inv;
                  c_lsteps += 1u;
                }
              } else {
                c_lsteps += 1u;
              }
            }
          }
          if (step) {
            const bool s0 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x0, y0, c_fb);
            const bool s1 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x1, y1, c_fb);
            const bool s2 = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, x2, y2, c_fb);
            c_side += 3;
            e = (!s1 && s2) ? 0 : ((!s2 && s0) ? 1 : 2);
            mode = 2;
            if (!inside) {
              status = CCT_RAY_INVALID;
              ++c_inv;
            }
          }
        } else {
          const bool sc = side_L<kExact>(fdx, fdy, kx, ky, ox, oy, vx_of(r, j), vy_of(r, j), c_fb);
          ++c_side;
          e = sc ? (j == 2 ? 0 : j + 1) : (j == 0 ? 2 : j - 1);
        }
        if (step && status == 0) {
          ++nsteps;
          const int32_t w = nb_of(r, e);
          if (w >= 0) {
            if (nsteps >= max_steps) {
              status = CCT_RAY_WALK_LIMIT;
              ++c_lim;
            } else {
              T = w >> 2;
              j = w & 3;
            }
          } else {
            status = nsteps;
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
  if (done) batch_complete(items[item], rec, T, j, nsteps, ox, oy, kx, ky, idx);
  const unsigned long long w_steps = warp_sum((unsigned long long)c_steps);
  const unsigned long long w_side = warp_sum((unsigned long long)c_side);
  const unsigned long long w_rays = warp_sum((unsigned long long)c_rays);
  const unsigned long long w_fb = warp_sum((unsigned long long)c_fb);
  const unsigned long long w_inv = warp_sum((unsigned long long)c_inv);
  const unsigned long long w_lim = warp_sum((unsigned long long)c_lim);
  const unsigned long long w_loc = warp_sum((unsigned long long)c_loc);
  const unsigned long long w_lst = warp_sum((unsigned long long)c_lsteps);
  if (lane == 0) {
    if (w_rays) atomicAdd(&bstats->rays, w_rays);
    if (w_steps) atomicAdd(&bstats->steps, w_steps);
    if (w_side) atomicAdd(&bstats->side_tests, w_side);
    if (w_fb) atomicAdd(&bstats->exact_fallbacks, w_fb);
    if (w_inv) atomicAdd(&bstats->invalid_rays, w_inv);
    if (w_lim) atomicAdd(&bstats->walk_limit_rays, w_lim);
    if (w_loc) atomicAdd(&bstats->located, w_loc);
    if (w_lst) atomicAdd(&bstats->locate_steps, w_lst);
  }
}

static size_t al256d(size_t x) { return (x + 255) & ~(size_t)255; }

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
  char* h_staging;       // pinned copy of header + items
  size_t table_bytes;
  int grid;
  int staged;
};

static int batch_grid(cct_batch b) {
  int per_sm = 0;
  const int threads = b->tuning.block_threads;
  auto k = (b->flags & CCT_TRACE_EXACT_ONLY) ? batch_kernel<true> : batch_kernel<false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
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
  const size_t o_scenes = 0, o_table = al256d(sizeof(SceneDev) * n_scenes);
  const size_t o_counter = o_table + al256d(b->table_bytes), o_stats = o_counter + 256;
  const size_t total = o_stats + al256d(sizeof(DevStats));
  if (cudaMalloc(&b->d_base, total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  if (cudaMallocHost(&b->h_staging, b->table_bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_base);
    delete b;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  std::memset(b->h_staging, 0, b->table_bytes);
  b->d_scenes = (SceneDev*)(b->d_base + o_scenes);
  b->d_hdr = (BatchHeader*)(b->d_base + o_table);
  b->d_counter = (unsigned long long*)(b->d_base + o_counter);
  b->d_stats = (DevStats*)(b->d_base + o_stats);
  std::vector<SceneDev> sd(n_scenes);
  for (int k = 0; k < n_scenes; ++k) sd[k] = scenes[k]->dev;
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
  if (cudaMemcpyAsync(b->d_hdr, b->h_staging, b->table_bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return CCT_ERR_CUDA;
  if (cudaMemsetAsync(b->d_counter, 0, 8, stream) != cudaSuccess) return CCT_ERR_CUDA;
  const auto* items = (const BatchItemDev*)((const char*)b->d_hdr + sizeof(BatchHeader));
  if (b->flags & CCT_TRACE_EXACT_ONLY)
    batch_kernel<true><<<b->grid, b->tuning.block_threads, 0, stream>>>(b->d_scenes, b->d_hdr, items,
                                                                        b->tuning.refill_min, b->d_counter,
                                                                        b->d_stats);
  else
    batch_kernel<false><<<b->grid, b->tuning.block_threads, 0, stream>>>(b->d_scenes, b->d_hdr, items,
                                                                         b->tuning.refill_min, b->d_counter,
                                                                         b->d_stats);
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
