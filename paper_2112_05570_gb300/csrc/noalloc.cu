// cct_trace_noalloc: cct_trace for callers that cannot allocate device memory.
//
// cct_trace takes its scratch (the walk's ray-chunk counter and, when the
// caller passes no start cells, the located start triangles) from the
// stream-ordered allocator.  Some callers must not enter an allocator during a
// query: a process that reserved all device memory for its own pool at
// start-up, or a latency-critical loop that may not take the allocator's
// locks or trigger a pool growth.  This variant takes the same scratch from
// one file-scope device array instead, so a call allocates nothing.
//
// The array is CCT_NOALLOC_SCRATCH_BYTES long and lives on every GPU that
// loads this library until the process exits.  Every call on a device uses
// the same array: two calls whose GPU work overlaps (different streams, or
// different host threads) race on it and return wrong results.  The counter
// that must start at zero is cleared by every call (cudaMemsetAsync on the
// caller's stream); the start-cell area is fully rewritten before it is read.
#include <mutex>

#include "cct_internal.cuh"

namespace cct {

constexpr size_t kNoallocCounterBytes = 256;
constexpr size_t kNoallocBytes = kNoallocCounterBytes + sizeof(int32_t) * (size_t)CCT_NOALLOC_MAX_RAYS;
static_assert(kNoallocBytes == CCT_NOALLOC_SCRATCH_BYTES, "header and implementation disagree on the size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on `dev` (which must be current).  The
// host-side symbol is only a stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress and cached.
static int noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return CCT_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return CCT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_ptr[dev];
  return CCT_OK;
}

}  // namespace cct

using namespace cct;

extern "C" int cct_trace_noalloc(cct_scene scene, const int32_t* ox, const int32_t* oy, const float* dx,
                                 const float* dy, const int32_t* start, int64_t n, int32_t* hit, float* t,
                                 int32_t* steps, uint32_t flags, void* stream_v) {
  if (!scene || n < 0 || n > (int64_t)CCT_NOALLOC_MAX_RAYS) return CCT_ERR_INVALID_ARGUMENT;
  if (flags & CCT_TRACE_BIN) return CCT_ERR_INVALID_ARGUMENT;  // binning needs scratch per ray: use cct_trace
  if (n == 0) return CCT_OK;
  if (!ox || !oy || !dx || !dy || !hit || !t || !steps) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(scene->device);
  unsigned char* base = nullptr;
  const int rc = noalloc_scratch(scene->device, &base);
  if (rc != CCT_OK) return rc;
  cudaStream_t stream = (cudaStream_t)stream_v;
  unsigned long long* counter = (unsigned long long*)base;
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream) != cudaSuccess) return CCT_ERR_CUDA;
  // the scene's launch configuration and predicate choice, as cct_trace uses
  // them; binning (which needs scratch per ray) is left out
  cct_tuning tu = scene->tuning;
  flags |= tu.trace_flags & ~(uint32_t)CCT_TRACE_BIN;
  tu.trace_flags = flags;
  const bool exact = (flags & CCT_TRACE_EXACT_ONLY) != 0;
  const SceneDev& S = scene->dev;
  if (start) {
    RaySrc R{ox, oy, dx, dy, start, nullptr, nullptr, n};
    return launch_walk_src(exact, kSrcPlainUser, S, R, tu, hit, t, steps, counter, scene->device, stream) ==
                   cudaSuccess
               ? CCT_OK
               : CCT_ERR_CUDA;
  }
  if (flags & CCT_TRACE_SPLIT_LOCATE) {
    // start cells from the locate kernel into the array, then the walk
    int32_t* sbuf = (int32_t*)(base + kNoallocCounterBytes);
    if (launch_locate(S, ox, oy, n, sbuf, false, stream) != cudaSuccess) return CCT_ERR_CUDA;
    RaySrc R{ox, oy, dx, dy, sbuf, nullptr, nullptr, n};
    return launch_walk_src(exact, kSrcPlainDev, S, R, tu, hit, t, steps, counter, scene->device, stream) ==
                   cudaSuccess
               ? CCT_OK
               : CCT_ERR_CUDA;
  }
  // the walk kernel locates each origin itself (no start-cell scratch)
  RaySrc R{ox, oy, dx, dy, nullptr, nullptr, nullptr, n};
  return launch_walk_src(exact, kSrcLocate, S, R, tu, hit, t, steps, counter, scene->device, stream) == cudaSuccess
             ? CCT_OK
             : CCT_ERR_CUDA;
}
