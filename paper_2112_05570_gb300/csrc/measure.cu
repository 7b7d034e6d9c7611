// Random 32-byte sector gather peak (include/cct_measure.h): the roofline
// denominator of the walk, whose every step is one data-dependent 32-byte
// record load.  Loads here are independent (addresses are hashed, never read
// from memory), so the memory system sees its maximum sector parallelism.
#include <algorithm>

#include "cct_internal.cuh"
#include "cct_measure.h"

namespace cct {

constexpr int kGatherThreads = 256;
constexpr int kGatherUnroll = 8;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  // integer hash (Wang / Jenkins style avalanche)
  x = (x ^ 61u) ^ (x >> 16);
  x *= 9u;
  x ^= x >> 4;
  x *= 0x27d4eb2du;
  x ^= x >> 15;
  return x;
}

__global__ void __launch_bounds__(kGatherThreads) gather_kernel(const TriRec* __restrict__ table, uint32_t n_rec,
                                                                long long per_thread,
                                                                unsigned long long* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t h = mix32(tid * 0x9E3779B9u + 1u);
  unsigned long long acc = 0;
  for (long long k = 0; k < per_thread; k += kGatherUnroll) {
    TriRec r[kGatherUnroll];
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
      h = mix32(h + (uint32_t)u + 0x632BE5ABu);
      r[u] = load_rec(table + (h % n_rec));
    }
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) acc ^= r[u].X ^ r[u].Y ^ (unsigned long long)(uint32_t)r[u].nb[0];
  }
  if (acc == 0x5A5A5A5A5A5A5A5Aull) *sink = acc;  // keeps the loads alive
}

__global__ void fill_kernel(TriRec* t, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    TriRec r;
    r.X = mix32(i) | ((unsigned long long)mix32(i + 7) << 32);
    r.Y = mix32(i + 3);
    r.nb[0] = (int32_t)i;
    r.nb[1] = r.nb[2] = r.pad = 0;
    t[i] = r;
  }
}

}  // namespace cct

using namespace cct;

extern "C" int cct_measure_gather(size_t table_bytes, int64_t loads, int32_t reps, void* stream_v,
                                  float* ms_per_launch, double* bytes_per_s) {
  if (!ms_per_launch || !bytes_per_s || loads <= 0 || reps <= 0) return CCT_ERR_INVALID_ARGUMENT;
  size_t n_rec64 = std::max<size_t>(1, table_bytes / sizeof(TriRec));
  if (n_rec64 > 0xffffffffull) return CCT_ERR_INVALID_ARGUMENT;
  const uint32_t n_rec = (uint32_t)n_rec64;
  cudaStream_t stream = (cudaStream_t)stream_v;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CCT_ERR_CUDA;
  TriRec* table = nullptr;
  unsigned long long* sink = nullptr;
  if (cudaMalloc(&table, sizeof(TriRec) * (size_t)n_rec) != cudaSuccess) {
    cudaGetLastError();
    return CCT_ERR_OUT_OF_MEMORY;
  }
  if (cudaMalloc(&sink, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(table);
    return CCT_ERR_OUT_OF_MEMORY;
  }
  int rc = CCT_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  do {
    fill_kernel<<<sm_count(dev) * 4, 256, 0, stream>>>(table, n_rec);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_kernel, kGatherThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const long long threads = (long long)sm_count(dev) * per_sm * kGatherThreads;
    long long per_thread = (loads + threads - 1) / threads;
    per_thread = ((per_thread + kGatherUnroll - 1) / kGatherUnroll) * kGatherUnroll;
    const unsigned grid = (unsigned)(threads / kGatherThreads);
    gather_kernel<<<grid, kGatherThreads, 0, stream>>>(table, n_rec, per_thread, sink);  // warm-up
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = CCT_ERR_CUDA;
      break;
    }
    cudaEventRecord(e0, stream);
    for (int r = 0; r < reps; ++r) gather_kernel<<<grid, kGatherThreads, 0, stream>>>(table, n_rec, per_thread, sink);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = CCT_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    *ms_per_launch = ms;
    *bytes_per_s = (double)threads * (double)per_thread * 32.0 / ((double)ms * 1e-3);
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(table);
  cudaFree(sink);
  return rc;
}
