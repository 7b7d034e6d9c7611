// Start-triangle location (Sec. 5.2) and cct_locate.
//
// The paper's option without an extra data structure: from a point p whose
// triangle is known, follow the traversal towards the origin o until the
// current triangle holds o.  Seeds sit on a regular grid of power-of-two
// cells: the seed point of a cell is its centre under a symbolic perturbation
// (computed from o with shifts, never stored), located exactly at load time,
// so a cell costs one 4-byte triangle index.  The locate walk crosses
// constrained edges (it is a point location, not a ray query), reading their
// neighbours from `cnb`.
#include <algorithm>

#include "cct_internal.cuh"

namespace cct {

constexpr int kLocateThreads = 256;

__global__ void __launch_bounds__(kLocateThreads) locate_kernel(SceneDev S, const int32_t* __restrict__ ox,
                                                                const int32_t* __restrict__ oy, int64_t n,
                                                                int32_t* __restrict__ out, bool to_user) {
  unsigned long long c_loc = 0, c_steps = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int qx = ox[i], qy = oy[i];
    int32_t res = -1;
    if (qx >= 0 && qy >= 0 && qx <= S.D && qy <= S.D) {
      int T = S.seeds[seed_cell(S, qx, qy)], j = 3, cx, cy;
      seed_point(S, qx, qy, cx, cy);
      int steps = 0;
      if (idx_bad(T, S.n_tri)) res = CCT_RAY_BAD_INDEX;
      while (res != CCT_RAY_BAD_INDEX) {
        if (++steps > S.max_steps) {
          res = -1;
          break;
        }
        const TriRec r = load_rec(S.rec + T);
        const int st = locate_step(S, r, T, j, qx, qy, cx, cy);
        if (st != 0) {
          res = st > 0 ? T : (kChecked && T < 0 ? CCT_RAY_BAD_INDEX : -1);
          break;
        }
      }
      ++c_loc;
      c_steps += (unsigned)steps;
    }
    out[i] = (res >= 0 && to_user) ? S.dev2user[res] : res;
  }
  c_loc = warp_sum(c_loc);
  c_steps = warp_sum(c_steps);
  if ((threadIdx.x & 31) == 0 && c_loc) {
    atomicAdd(&S.stats->located, c_loc);
    atomicAdd(&S.stats->locate_steps, c_steps);
  }
}

cudaError_t launch_locate(const SceneDev& S, const int32_t* ox, const int32_t* oy, int64_t n, int32_t* out,
                          bool to_user, cudaStream_t stream) {
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, locate_kernel, kLocateThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long long want = (n + kLocateThreads - 1) / kLocateThreads;
  long long grid = std::min<long long>((long long)sm_count(dev) * per_sm * 4, want);
  if (grid < 1) grid = 1;
  locate_kernel<<<(unsigned)grid, kLocateThreads, 0, stream>>>(S, ox, oy, n, out, to_user);
  return cudaGetLastError();
}

}  // namespace cct

using namespace cct;

extern "C" int cct_locate(cct_scene scene, const int32_t* ox, const int32_t* oy, int64_t n, int32_t* start,
                          void* stream_v) {
  if (!scene || n < 0) return CCT_ERR_INVALID_ARGUMENT;
  if (n == 0) return CCT_OK;
  if (!ox || !oy || !start) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(scene->device);
  if (launch_locate(scene->dev, ox, oy, n, start, true, (cudaStream_t)stream_v) != cudaSuccess) return CCT_ERR_CUDA;
  return CCT_OK;
}
