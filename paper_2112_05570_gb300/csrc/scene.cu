// Scene load / free / info / stats of libcct (include/cct.h).
//
// cct_scene_load turns the caller's triangulation (Sec. 5.1: triangles with
// neighbours, some edges belonging to the original geometry) into the device
// layout described in cct_internal.cuh:
//   1. validation (exact integer checks, host);
//   2. Hilbert order of the triangle centroids, so that triangles adjacent in
//      space are adjacent in memory (walk and locate locality);
//   3. one 32-byte record per triangle (coordinates + neighbour words) and
//      one 16-byte half-edge record per (triangle, entry edge) for the walk
//      steps after the first;
//   4. the locate seed grid of Sec. 5.2: G x G square cells of side 2^s, each
//      holding the triangle of its seed point (the cell centre, symbolically
//      perturbed: see seed_point in cct_internal.cuh), found by exact walks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cct_internal.cuh"

namespace cct {

int sm_count(int dev) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  return n;
}

static uint64_t hilbert_d(int order, uint32_t x, uint32_t y) {
  uint64_t d = 0;
  for (uint32_t s = 1u << (order - 1); s > 0; s >>= 1) {
    uint32_t rx = (x & s) > 0, ry = (y & s) > 0;
    d += (uint64_t)s * s * ((3 * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = s - 1 - x;
        y = s - 1 - y;
      }
      uint32_t t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

static inline long long orient_h(long long ax, long long ay, long long bx, long long by, long long cx, long long cy) {
  return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

// Index ranges and coordinates: always checked (even with CCT_LOAD_NO_VALIDATE),
// so every record and neighbour word the kernels can reach is in bounds.
static int check_ranges(const cct_tri_desc& d) {
  const long long D = d.domain;
  for (int v = 0; v < d.n_vert; ++v)
    if (d.vx[v] < 0 || d.vy[v] < 0 || d.vx[v] > D || d.vy[v] > D) return CCT_ERR_BAD_TRIANGULATION;
  for (long long k = 0; k < 3ll * d.n_tri; ++k) {
    int32_t v = d.tri_v[k], nb = d.tri_nb[k], s = d.tri_seg[k];
    if (v < 0 || v >= d.n_vert || nb < -1 || nb >= d.n_tri || s < -1 || s >= d.n_seg)
      return CCT_ERR_BAD_TRIANGULATION;
  }
  return CCT_OK;
}

static int validate(const cct_tri_desc& d) {
  const long long D = d.domain;
  const int nt = d.n_tri;
  long long area2 = 0;
  for (int t = 0; t < nt; ++t) {
    const int32_t* tv = d.tri_v + 3 * t;
    long long o = orient_h(d.vx[tv[0]], d.vy[tv[0]], d.vx[tv[1]], d.vy[tv[1]], d.vx[tv[2]], d.vy[tv[2]]);
    if (o <= 0) return CCT_ERR_BAD_TRIANGULATION;
    area2 += o;
  }
  if (area2 != 2 * D * D) return CCT_ERR_BAD_TRIANGULATION;
  for (int t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      int32_t a = d.tri_v[3 * t + (i + 1) % 3], b = d.tri_v[3 * t + (i + 2) % 3];
      int32_t u = d.tri_nb[3 * t + i];
      if (u < 0) {
        long long ax = d.vx[a], ay = d.vy[a], bx = d.vx[b], by = d.vy[b];
        bool on_side = (ax == 0 && bx == 0) || (ay == 0 && by == 0) || (ax == D && bx == D) || (ay == D && by == D);
        if (!on_side) return CCT_ERR_BAD_TRIANGULATION;
        continue;
      }
      int j = -1;
      for (int k = 0; k < 3; ++k)
        if (d.tri_v[3 * u + (k + 1) % 3] == b && d.tri_v[3 * u + (k + 2) % 3] == a) j = k;
      if (j < 0 || d.tri_nb[3 * u + j] != t || d.tri_seg[3 * u + j] != d.tri_seg[3 * t + i])
        return CCT_ERR_BAD_TRIANGULATION;
    }
  return CCT_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Exact host point location of perturbed seed points c + eps (1, delta)
// (0 < eps << delta << 1) over the packed records (used once, at load).
struct HostLocator {
  const std::vector<TriRec>& rec;
  const std::vector<int32_t>& cnb;
  HostLocator(const std::vector<TriRec>& r, const std::vector<int32_t>& c) : rec(r), cnb(c) {}
  static long long vx(const TriRec& r, int i) { return (long long)((r.X >> (kCoordBits * i)) & kCoordMask); }
  static long long vy(const TriRec& r, int i) { return (long long)((r.Y >> (kCoordBits * i)) & kCoordMask); }
  // orientation of (a, b, c + eps (1, delta)): orient(a, b, c) + eps ((bx - ax) delta - (by - ay)); never 0
  static bool left_sos(long long ax, long long ay, long long bx, long long by, long long cx, long long cy) {
    const long long o = orient_h(ax, ay, bx, by, cx, cy);
    if (o != 0) return o > 0;
    return ay != by ? ay > by : bx > ax;
  }
  bool contains(int T, long long x, long long y) const {
    const TriRec& r = rec[T];
    for (int i = 0; i < 3; ++i) {
      const int a = (i + 1) % 3, b = (i + 2) % 3;
      if (!left_sos(vx(r, a), vy(r, a), vx(r, b), vy(r, b), x, y)) return false;
    }
    return true;
  }
  int scan(long long x, long long y) const {
    for (int T = 0; T < (int)rec.size(); ++T)
      if (contains(T, x, y)) return T;
    return -1;
  }
  // From the perturbed p (inside T) along the segment to the perturbed q (both
  // moved by the same eps (1, delta)); the triangle holding q, or -1 if the
  // walk leaves the domain (a triangulation loaded without validation).
  int walk(int T, long long px, long long py, long long qx, long long qy) const {
    const long long kx = qx - px, ky = qy - py;
    // side of v: k x (v - p) - eps (kx delta - ky); tie: sign of ky, else of -kx
    const bool tie_left = ky != 0 ? ky > 0 : kx < 0;
    for (size_t guard = 0; guard <= rec.size() + 8; ++guard) {
      if (contains(T, qx, qy)) return T;
      const TriRec& r = rec[T];
      bool s[3];
      for (int i = 0; i < 3; ++i) {
        const long long e = kx * (vy(r, i) - py) - ky * (vx(r, i) - px);
        s[i] = e != 0 ? e > 0 : tie_left;
      }
      const int e = (!s[1] && s[2]) ? 0 : ((!s[2] && s[0]) ? 1 : 2);
      int32_t w = r.nb[e];
      if (w <= -2) w = cnb[3 * (size_t)T + e];
      if (w < 0) return -1;
      T = w / 3;
    }
    return -1;
  }
};

}  // namespace cct

using namespace cct;

extern "C" int cct_scene_load(const cct_tri_desc* desc, uint32_t flags, void* stream_v, cct_scene* out) {
  if (!desc || !out) return CCT_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  const cct_tri_desc& d = *desc;
  if (d.n_tri < 1 || d.n_vert < 3 || d.n_seg < 0 || d.domain < 1 || d.domain > (1 << 20) || !d.vx || !d.vy ||
      !d.tri_v || !d.tri_nb || !d.tri_seg)
    return CCT_ERR_INVALID_ARGUMENT;
  if ((int64_t)d.n_tri >= (1ll << 29)) return CCT_ERR_INVALID_ARGUMENT;
  {
    int v = check_ranges(d);
    if (v == CCT_OK && !(flags & CCT_LOAD_NO_VALIDATE)) v = validate(d);
    if (v != CCT_OK) return v;
  }
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return CCT_ERR_NO_DEVICE;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return CCT_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_v;
  const int nt = d.n_tri;
  try {
    // ---- order
    std::vector<int32_t> dev2user(nt), user2dev(nt);
    if (flags & CCT_LOAD_NO_REORDER) {
      for (int t = 0; t < nt; ++t) dev2user[t] = t;
    } else {
      std::vector<std::pair<uint64_t, int32_t>> key(nt);
      for (int t = 0; t < nt; ++t) {
        const int32_t* tv = d.tri_v + 3 * t;
        uint32_t cx = (uint32_t)(d.vx[tv[0]] + d.vx[tv[1]] + d.vx[tv[2]]);
        uint32_t cy = (uint32_t)(d.vy[tv[0]] + d.vy[tv[1]] + d.vy[tv[2]]);
        key[t] = {hilbert_d(22, cx, cy), t};
      }
      std::sort(key.begin(), key.end());
      for (int t = 0; t < nt; ++t) dev2user[t] = key[t].second;
    }
    for (int t = 0; t < nt; ++t) user2dev[dev2user[t]] = t;
    // ---- records
    std::vector<TriRec> rec(nt);
    std::vector<int32_t> cnb(3 * (size_t)nt, -1);
    for (int T = 0; T < nt; ++T) {
      const int u = dev2user[T];
      const int32_t* tv = d.tri_v + 3 * u;
      TriRec r{};
      for (int i = 0; i < 3; ++i) {
        r.X |= (uint64_t)(uint32_t)d.vx[tv[i]] << (kCoordBits * i);
        r.Y |= (uint64_t)(uint32_t)d.vy[tv[i]] << (kCoordBits * i);
      }
      for (int i = 0; i < 3; ++i) {
        int32_t nbu = d.tri_nb[3 * u + i], seg = d.tri_seg[3 * u + i];
        int32_t word = -1;
        if (nbu >= 0) {
          int32_t a = tv[(i + 1) % 3], b = tv[(i + 2) % 3];
          int j = 0;
          for (int k = 0; k < 3; ++k)
            if (d.tri_v[3 * nbu + (k + 1) % 3] == b && d.tri_v[3 * nbu + (k + 2) % 3] == a) j = k;
          word = 3 * user2dev[nbu] + j;
        }
        if (seg >= 0) {
          cnb[3 * (size_t)T + i] = word;
          r.nb[i] = -2 - seg;
        } else {
          r.nb[i] = word;
        }
      }
      rec[T] = r;
    }
    // half-edge records 3 T + j: apex j and the exit words of edges nxt(j), prv(j)
    std::vector<int4> he(3 * (size_t)nt);
    for (int T = 0; T < nt; ++T) {
      const TriRec& r = rec[T];
      for (int j = 0; j < 3; ++j) {
        const int ax = (int)((r.X >> (kCoordBits * j)) & kCoordMask), ay = (int)((r.Y >> (kCoordBits * j)) & kCoordMask);
        he[3 * (size_t)T + j] = make_int4(coord_word(ax), coord_word(ay), r.nb[(j + 1) % 3], r.nb[(j + 2) % 3]);
      }
    }
    // ---- seed grid (Sec. 5.2): per cell, the triangle whose interior holds
    // the perturbed cell centre; about 2^k cells per triangle, k from the flags
    const long long D = d.domain;
    int shift = 0, G = 1;
    {
      const unsigned kd = (flags >> 8) & 15u;
      const int k = kd == 0 ? 5 : std::min(8, (int)kd - 1);
      const double h = (double)D / std::sqrt(std::ldexp(1.0, k) * (double)nt);
      shift = std::max(0, (int)std::lround(std::log2(std::max(1.0, h))));
      while (((D + (1ll << shift) - 1) >> shift) > 8192) ++shift;
      G = (int)((D + (1ll << shift) - 1) >> shift);
    }
    std::vector<int32_t> seeds((size_t)G * G, 0);
    {
      HostLocator loc(rec, cnb);
      const long long half = (1ll << shift) >> 1;
      int prev_tri = -1;
      long long prev_x = 0, prev_y = 0;
      for (int iy = 0; iy < G; ++iy)
        for (int jx = 0; jx < G; ++jx) {
          const int ix = (iy & 1) ? G - 1 - jx : jx;  // boustrophedon: short walks
          const long long cx = std::min(((long long)ix << shift) + half, D - 1);
          const long long cy = std::min(((long long)iy << shift) + half, D - 1);
          const int tri = prev_tri < 0 ? loc.scan(cx, cy) : loc.walk(prev_tri, prev_x, prev_y, cx, cy);
          if (tri < 0) {
            // only on a triangulation loaded without validation: keep the
            // previous cell's triangle (or record 0); locate walks from there
            // end at their step limit or report the origin invalid, and every
            // index they follow was range-checked
            seeds[(size_t)iy * G + ix] = std::max(prev_tri, 0);
            continue;
          }
          seeds[(size_t)iy * G + ix] = tri;
          prev_tri = tri;
          prev_x = cx;
          prev_y = cy;
        }
    }
    // ---- device allocation and upload
    size_t o_rec = 0;
    size_t o_he = o_rec + align256(sizeof(TriRec) * (size_t)nt);
    size_t o_cnb = o_he + align256(sizeof(int4) * 3 * (size_t)nt);
    size_t o_u2d = o_cnb + align256(sizeof(int32_t) * 3 * (size_t)nt);
    size_t o_d2u = o_u2d + align256(sizeof(int32_t) * (size_t)nt);
    size_t o_seed = o_d2u + align256(sizeof(int32_t) * (size_t)nt);
    const bool two = (flags & CCT_LOAD_TWO_STEP) != 0;
    size_t o_he2 = o_seed + align256(sizeof(int32_t) * (size_t)G * G);
    size_t o_stats = o_he2 + (two ? align256(sizeof(int4) * 12 * (size_t)nt) : 0);
    size_t total = o_stats + align256(sizeof(DevStats));
    char* base = nullptr;
    if (cudaMalloc(&base, total) != cudaSuccess) {
      cudaGetLastError();
      return CCT_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](size_t off, const void* src, size_t n) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, stream);
    };
    up(o_rec, rec.data(), sizeof(TriRec) * (size_t)nt);
    up(o_he, he.data(), sizeof(int4) * 3 * (size_t)nt);
    up(o_cnb, cnb.data(), sizeof(int32_t) * 3 * (size_t)nt);
    up(o_u2d, user2dev.data(), sizeof(int32_t) * (size_t)nt);
    up(o_d2u, dev2user.data(), sizeof(int32_t) * (size_t)nt);
    up(o_seed, seeds.data(), sizeof(int32_t) * (size_t)G * G);
    std::vector<int4> he2;
    if (two) {
      // two-step records: he[h], then the records behind its L and R exits
      he2.assign(12 * (size_t)nt, make_int4(0, 0, 0, 0));
      for (size_t h = 0; h < 3 * (size_t)nt; ++h) {
        const int4 q = he[h];
        he2[4 * h] = q;
        if (q.z >= 0) he2[4 * h + 1] = he[q.z];
        if (q.w >= 0) he2[4 * h + 2] = he[q.w];
      }
      up(o_he2, he2.data(), sizeof(int4) * 12 * (size_t)nt);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_stats, 0, sizeof(DevStats), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      cudaFree(base);
      return CCT_ERR_CUDA;
    }
    auto* s = new cct_scene_s;
    s->d_base = base;
    s->bytes = total;
    s->device = dev;
    s->dev.rec = (const TriRec*)(base + o_rec);
    s->dev.he = (const int4*)(base + o_he);
    s->dev.he2 = two ? (const int4*)(base + o_he2) : nullptr;
    s->dev.cnb = (const int32_t*)(base + o_cnb);
    s->dev.user2dev = (const int32_t*)(base + o_u2d);
    s->dev.dev2user = (const int32_t*)(base + o_d2u);
    s->dev.seeds = (const int32_t*)(base + o_seed);
    s->dev.stats = (DevStats*)(base + o_stats);
    s->dev.n_tri = nt;
    s->dev.G = G;
    s->dev.seed_shift = shift;
    s->dev.D = d.domain;
    s->dev.max_steps = nt + 8;
    s->tuning = default_tuning();
    *out = s;
    return CCT_OK;
  } catch (const std::bad_alloc&) {
    return CCT_ERR_OUT_OF_MEMORY;
  }
}

extern "C" int cct_scene_load_file(const char* path, uint32_t flags, void* stream_v, cct_scene* out) {
  if (!path || !out) return CCT_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return CCT_ERR_IO;
  struct Closer {
    FILE* f;
    ~Closer() { std::fclose(f); }
  } closer{f};
  char magic[8];
  int32_t hdr[4];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, CCT_FILE_MAGIC, 8) != 0) return CCT_ERR_IO;
  if (std::fread(hdr, sizeof(int32_t), 4, f) != 4) return CCT_ERR_IO;
  const int64_t nv = hdr[0], nt = hdr[1], ns = hdr[2], D = hdr[3];
  if (nv < 3 || nt < 1 || nt >= (1ll << 29) || ns < 0 || D < 1 || D > (1 << 20)) return CCT_ERR_IO;
  // the size must match the counts exactly before anything is allocated
  const int64_t body = 4ll * (2 * nv + 9 * nt);
  if (std::fseek(f, 0, SEEK_END) != 0) return CCT_ERR_IO;
  const long long size = std::ftell(f);
  if (size != 8 + 16 + body || std::fseek(f, 24, SEEK_SET) != 0) return CCT_ERR_IO;
  try {
    std::vector<int32_t> vx(nv), vy(nv), tv(3 * nt), tn(3 * nt), ts(3 * nt);
    for (auto* v : {&vx, &vy, &tv, &tn, &ts})
      if (std::fread(v->data(), sizeof(int32_t), v->size(), f) != v->size()) return CCT_ERR_IO;
    cct_tri_desc d{};
    d.n_vert = (int32_t)nv;
    d.n_tri = (int32_t)nt;
    d.n_seg = (int32_t)ns;
    d.domain = (int32_t)D;
    d.vx = vx.data();
    d.vy = vy.data();
    d.tri_v = tv.data();
    d.tri_nb = tn.data();
    d.tri_seg = ts.data();
    return cct_scene_load(&d, flags, stream_v, out);
  } catch (const std::bad_alloc&) {
    return CCT_ERR_OUT_OF_MEMORY;
  }
}

extern "C" int cct_scene_free(cct_scene s) {
  if (!s) return CCT_OK;
  int rc = CCT_OK;
  {
    DeviceGuard g(s->device);
    if (cudaFree(s->d_base) != cudaSuccess) rc = CCT_ERR_CUDA;
  }
  delete s;
  return rc;
}

extern "C" int cct_scene_info(cct_scene s, size_t* device_bytes, int32_t* n_tri) {
  if (!s) return CCT_ERR_INVALID_ARGUMENT;
  if (device_bytes) *device_bytes = s->bytes;
  if (n_tri) *n_tri = s->dev.n_tri;
  return CCT_OK;
}

extern "C" int cct_get_stats(cct_scene s, cct_stats* out, int reset, void* stream_v) {
  if (!s || !out) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(s->device);
  cudaStream_t stream = (cudaStream_t)stream_v;
  DevStats h{};
  if (cudaMemcpyAsync(&h, s->dev.stats, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return CCT_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return CCT_ERR_CUDA;
  if (reset) {
    if (cudaMemsetAsync(s->dev.stats, 0, sizeof(DevStats), stream) != cudaSuccess) return CCT_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return CCT_ERR_CUDA;
  }
  out->rays = h.rays;
  out->steps = h.steps;
  out->side_tests = h.side_tests;
  out->exact_fallbacks = h.exact_fallbacks;
  out->invalid_rays = h.invalid_rays;
  out->walk_limit_rays = h.walk_limit_rays;
  out->located = h.located;
  out->locate_steps = h.locate_steps;
  return CCT_OK;
}

extern "C" const char* cct_error_string(int code) {
  switch (code) {
    case CCT_OK: return "ok";
    case CCT_ERR_INVALID_ARGUMENT: return "invalid argument";
    case CCT_ERR_BAD_TRIANGULATION: return "triangulation failed validation";
    case CCT_ERR_OUT_OF_MEMORY: return "out of memory";
    case CCT_ERR_CUDA: return "CUDA runtime error";
    case CCT_ERR_WALK_LIMIT: return "walk step limit exceeded";
    case CCT_ERR_NO_DEVICE: return "no CUDA device";
    case CCT_ERR_IO: return "scene file missing, unreadable or malformed";
    case CCT_ERR_UNSUPPORTED: return "needs the checked build (libcct_checked.so)";
    default: return "unknown status";
  }
}

extern "C" int cct_version(void) { return (0 << 16) | 1; }

extern "C" int cct_is_checked(void) { return kChecked ? 1 : 0; }

namespace cct {

int poke_word(int device, const void* base, int64_t n, int64_t index, int64_t word, int32_t value, int32_t* old,
              int64_t* len) {
  if (index < 0) {
    if (len) *len = n;
    return CCT_OK;
  }
  if (index >= n) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(device);
  int32_t* p = (int32_t*)base + word;
  if (cudaDeviceSynchronize() != cudaSuccess) return CCT_ERR_CUDA;
  if (old && cudaMemcpy(old, p, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return CCT_ERR_CUDA;
  if (cudaMemcpy(p, &value, sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) return CCT_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? CCT_OK : CCT_ERR_CUDA;
}

}  // namespace cct

extern "C" int cct_scene_poke(cct_scene scene, int32_t table, int64_t index, int32_t value, int32_t* old,
                              int64_t* len) {
  if (!scene) return CCT_ERR_INVALID_ARGUMENT;
  if (!kChecked) return CCT_ERR_UNSUPPORTED;
  const SceneDev& S = scene->dev;
  const int64_t nt = S.n_tri;
  switch (table) {
    case CCT_TABLE_NEIGHBOUR:  // nb[e] is word 4 + e of the 8-word record
      return poke_word(scene->device, S.rec, 3 * nt, index, 8 * (index / 3) + 4 + index % 3, value, old, len);
    case CCT_TABLE_HALF_EDGE_EXIT:  // the exits are words 2 and 3 of the 4-word half-edge record
      return poke_word(scene->device, S.he, 6 * nt, index, 4 * (index / 2) + 2 + index % 2, value, old, len);
    case CCT_TABLE_CONSTRAINED:
      return poke_word(scene->device, S.cnb, 3 * nt, index, index, value, old, len);
    case CCT_TABLE_SEED:
      return poke_word(scene->device, S.seeds, (int64_t)S.G * S.G, index, index, value, old, len);
    case CCT_TABLE_USER_TO_RECORD:
      return poke_word(scene->device, S.user2dev, nt, index, index, value, old, len);
    case CCT_TABLE_TWO_STEP_EXIT:  // exit c of sub-record k of half-edge h: word 16 h + 4 k + 2 + c
      if (!S.he2) return CCT_ERR_INVALID_ARGUMENT;
      return poke_word(scene->device, S.he2, 18 * nt, index, 16 * (index / 6) + 4 * (index % 6 / 2) + 2 + index % 2,
                       value, old, len);
    default:
      return CCT_ERR_INVALID_ARGUMENT;
  }
}

extern "C" int cct_copies_async(int32_t n, void* const* dst, const void* const* src, const size_t* bytes,
                                void* stream_v) {
  if (n < 0 || (n > 0 && (!dst || !src || !bytes))) return CCT_ERR_INVALID_ARGUMENT;
  cudaStream_t stream = (cudaStream_t)stream_v;
  for (int32_t k = 0; k < n; ++k) {
    if (bytes[k] == 0) continue;
    if (cudaMemcpyAsync(dst[k], src[k], bytes[k], cudaMemcpyDefault, stream) != cudaSuccess) {
      cudaGetLastError();
      return CCT_ERR_CUDA;
    }
  }
  return CCT_OK;
}
