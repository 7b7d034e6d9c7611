// Ray binning: a counting sort of rays by start cell (record index >> shift).
// Records are in Hilbert order, so a bin is a compact patch of the plane and
// rays walked together by a warp start in the same few triangles.
//   1. histogram of bin keys (warp-aggregated atomics);
//   2. exclusive scan of the histogram (three-phase block scan);
//   3. scatter: each ray takes the next slot of its bin and is written in
//      packed form {ox, oy, dx bits, dy bits} with its start record and its
//      original index (results are written back at the original index).
// Rays with an invalid start go to the last bin.
#include <algorithm>

#include "cct_internal.cuh"

namespace cct {

constexpr int kBinThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

static size_t al256b(size_t x) { return (x + 255) & ~(size_t)255; }

static int64_t n_bins_of(int32_t n_tri, int shift) { return ((int64_t)n_tri >> shift) + 2; }

size_t bin_scratch_bytes(int64_t n, int32_t n_tri, int shift) {
  const int64_t nb = n_bins_of(n_tri, shift);
  const int64_t nblk = (nb + kScanTile - 1) / kScanTile;
  return al256b(sizeof(int32_t) * nb) * 2 + al256b(sizeof(int32_t) * (nblk + 1)) + al256b(sizeof(int4) * n) +
         al256b(sizeof(int32_t) * n) * 2;
}

__device__ __forceinline__ int32_t start_rec(const SceneDev& S, const int32_t* start, bool start_is_user,
                                             long long i) {
  int32_t s = start[i];
  if (kChecked && !start_is_user && s == CCT_RAY_BAD_INDEX) return s;  // marked by the locate kernel
  if (s < 0 || s >= S.n_tri) return -1;
  if (!start_is_user) return s;
  const int32_t r = S.user2dev[s];
  return idx_bad(r, S.n_tri) ? CCT_RAY_BAD_INDEX : r;
}

__device__ __forceinline__ int32_t bin_key(int32_t rec, int shift, int32_t nb) {
  return rec < 0 ? nb - 1 : (rec >> shift);
}

__global__ void bin_hist_kernel(SceneDev S, const int32_t* __restrict__ start, bool start_is_user, int64_t n,
                                int shift, int32_t nb, int32_t* __restrict__ hist) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t key = bin_key(start_rec(S, start, start_is_user, i), shift, nb);
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, key);
    const int leader = __ffs(same) - 1;
    if ((threadIdx.x & 31) == leader) atomicAdd(&hist[key], __popc(same));
  }
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_tot[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  const int before = wid > 0 ? warp_tot[wid - 1] : 0;
  const int res = before + x - v;
  __syncthreads();
  return res;
}

// Phase 1: per-tile totals.
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int32_t* __restrict__ in, int64_t nb,
                                                                  int32_t* __restrict__ tile_sum) {
  __shared__ int warp_tot[32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < nb) s += in[base + k];
  int ex = block_exclusive_scan(s, warp_tot);
  if (threadIdx.x == blockDim.x - 1) tile_sum[blockIdx.x] = ex + s;
}

// Phase 2: exclusive scan of the tile totals (one block, up to kScanTile tiles).
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int32_t* __restrict__ tile_sum, int64_t ntiles) {
  __shared__ int warp_tot[32];
  const long long base = (long long)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < ntiles) ? tile_sum[base + k] : 0;
    s += v[k];
  }
  int ex = block_exclusive_scan(s, warp_tot);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < ntiles) tile_sum[base + k] = ex;
    ex += v[k];
  }
}

// Phase 3: exclusive prefix of every bin.
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int32_t* __restrict__ in, int64_t nb,
                                                                  const int32_t* __restrict__ tile_sum,
                                                                  int32_t* __restrict__ out) {
  __shared__ int warp_tot[32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < nb) ? in[base + k] : 0;
    s += v[k];
  }
  int ex = block_exclusive_scan(s, warp_tot) + tile_sum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < nb) out[base + k] = ex;
    ex += v[k];
  }
}

__global__ void bin_scatter_kernel(SceneDev S, const int32_t* __restrict__ ox, const int32_t* __restrict__ oy,
                                   const float* __restrict__ dx, const float* __restrict__ dy,
                                   const int32_t* __restrict__ start, bool start_is_user, int64_t n, int shift,
                                   int32_t nb, int32_t* __restrict__ cursor, int4* __restrict__ rays,
                                   int32_t* __restrict__ sstart, int32_t* __restrict__ orig) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t rec = start_rec(S, start, start_is_user, i);
    const int32_t key = bin_key(rec, shift, nb);
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&cursor[key], __popc(same));
    base = __shfl_sync(same, base, leader);
    const int pos = base + __popc(same & lanemask_lt());
    rays[pos] = make_int4(ox[i], oy[i], __float_as_int(dx[i]), __float_as_int(dy[i]));
    sstart[pos] = rec;
    orig[pos] = (int32_t)i;
  }
}

cudaError_t launch_bin(const SceneDev& S, const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                       const int32_t* start, bool start_is_user, int64_t n, int shift, char* scratch, BinOut& out,
                       cudaStream_t stream) {
  if (n > 0x7fffffffll) return cudaErrorInvalidValue;
  const int64_t nb = n_bins_of(S.n_tri, shift);
  const int64_t ntiles = (nb + kScanTile - 1) / kScanTile;
  if (ntiles > kScanTile) return cudaErrorInvalidValue;
  char* p = scratch;
  int32_t* hist = (int32_t*)p;
  p += al256b(sizeof(int32_t) * nb);
  int32_t* cursor = (int32_t*)p;
  p += al256b(sizeof(int32_t) * nb);
  int32_t* tiles = (int32_t*)p;
  p += al256b(sizeof(int32_t) * (ntiles + 1));
  out.rays = (int4*)p;
  p += al256b(sizeof(int4) * n);
  out.start = (int32_t*)p;
  p += al256b(sizeof(int32_t) * n);
  out.orig = (int32_t*)p;
  int dev = 0;
  cudaGetDevice(&dev);
  const long long grid = std::min<long long>((long long)sm_count(dev) * 8, (n + kBinThreads - 1) / kBinThreads);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * nb, stream);
  if (e != cudaSuccess) return e;
  bin_hist_kernel<<<(unsigned)std::max(1ll, grid), kBinThreads, 0, stream>>>(S, start, start_is_user, n, shift,
                                                                          (int32_t)nb, hist);
  scan_tiles_kernel<<<(unsigned)ntiles, kScanThreads, 0, stream>>>(hist, nb, tiles);
  scan_sums_kernel<<<1, kScanThreads, 0, stream>>>(tiles, ntiles);
  scan_apply_kernel<<<(unsigned)ntiles, kScanThreads, 0, stream>>>(hist, nb, tiles, cursor);
  bin_scatter_kernel<<<(unsigned)std::max(1ll, grid), kBinThreads, 0, stream>>>(
      S, ox, oy, dx, dy, start, start_is_user, n, shift, (int32_t)nb, cursor, out.rays, out.start, out.orig);
  return cudaGetLastError();
}

}  // namespace cct
