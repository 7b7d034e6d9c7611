// Comparison structures of Sec. 5.3, traversed on the GPU with the same exact
// hit rule as the walk (the side rule of include/cct.h), so all three
// structures return the same closest hit; each counts its traversal
// operations the way Sec. 5.3/5.4 does.
//
//   BVH (Sec. 5.3.1): stack traversal from the root, nearer child first;
//     operations = AABB tests + segment tests.
//   Roped kd-tree (Sec. 5.3.2): stackless traversal from the leaf holding the
//     origin (known a priori, Sec. 5.4); in each leaf test its segments,
//     accepting hits up to the leaf's exit; else follow the rope of the exit
//     face and descend to the leaf holding the exit point.  Reported per ray:
//     leaves visited, inner nodes passed in rope descents, segment tests,
//     unique segment tests (the ideal mailbox: a per-thread hash set), the sum
//     of ceil(log2 #ropes) over the faces crossed (the ideal rope tree), and a
//     mailbox-overflow flag.
//
// Parameters t are kept as exact rationals: a slab parameter (X - o_x) / k_x
// (int32 / int32) and a segment parameter num / den (int64 / int64) are both
// t / 2^22; comparisons between them need 128-bit products.
#include <algorithm>
#include <vector>

#include "cct_internal.cuh"

namespace cct {

typedef __int128 i128;

struct BvhDev {
  const int4* box;
  const int32_t* c0;
  const int32_t* c1;
  const int32_t* prims;
  const int4* seg;
  int32_t n_nodes;
  int32_t n_prims;  // the checked build's bounds
  int32_t n_seg;
};

struct KdDev {
  const int32_t* axis;
  const int32_t* split;
  const int32_t* child;
  const int32_t* count;
  const int4* box;
  const int4* rope;
  const int32_t* rope_log2;  // 4 x 8 bits per node
  const int32_t* refs;
  const int4* seg;
  int32_t n_nodes;
  int32_t n_refs;  // the checked build's bounds
  int32_t n_seg;
};

struct Frac {  // num / den, den > 0; den == 0 means +infinity
  int num, den;
};

__device__ __forceinline__ bool frac_lt(Frac a, Frac b) {
  if (b.den == 0) return a.den != 0;
  if (a.den == 0) return false;
  return (long long)a.num * b.den < (long long)b.num * a.den;
}

struct Best {
  long long num, den;  // segment parameter, den > 0
  int seg;             // -1: none
  int wx, wy;          // right-hand endpoint of the best segment (tie order)
  int vx, vy;          // its endpoint on the ray's line side (common point at a tie)
};

// sign of (slab a / b) - (segment num / den)
__device__ __forceinline__ int cmp_frac_seg(Frac a, long long num, long long den) {
  if (a.den == 0) return 1;
  const i128 l = (i128)a.num * den, r = (i128)num * a.den;
  return (l > r) - (l < r);
}

__device__ __forceinline__ int tie_order(int kx, int ky, long long u1x, long long u1y, long long u2x,
                                         long long u2y) {
  const i128 d1 = (i128)kx * u1x + (i128)ky * u1y, d2 = (i128)kx * u2x + (i128)ky * u2y;
  i128 c1 = (i128)kx * u1y - (i128)ky * u1x, c2 = (i128)kx * u2y - (i128)ky * u2x;
  if (c1 < 0) c1 = -c1;
  if (c2 < 0) c2 = -c2;
  const i128 l = d1 * c2, r = d2 * c1;
  return (l > r) - (l < r);
}

// Exact segment test (the side rule), updating the closest hit.  `limit`
// (optional) bounds the accepted parameter from above (inclusive).
__device__ __forceinline__ void seg_test(const int4 q, int sid, int ox, int oy, int kx, int ky, Best& b,
                                         const Frac* limit) {
  const long long va = (long long)kx * (q.y - oy) - (long long)ky * (q.x - ox);
  const long long vb = (long long)kx * (q.w - oy) - (long long)ky * (q.z - ox);
  const bool la = va >= 0, lb = vb >= 0;
  if (la == lb) return;
  const long long ex = q.z - q.x, ey = q.w - q.y;
  long long num = ex * (long long)(q.y - oy) - ey * (long long)(q.x - ox);
  long long den = ex * (long long)ky - ey * (long long)kx;
  if (den < 0) {
    num = -num;
    den = -den;
  }
  if (num <= 0) return;
  if (limit && cmp_frac_seg(*limit, num, den) < 0) return;  // beyond the limit
  const int wx = la ? q.z : q.x, wy = la ? q.w : q.y;       // right-hand endpoint
  const int vx = la ? q.x : q.z, vy = la ? q.y : q.w;
  bool take = b.seg < 0;
  if (!take) {
    const i128 l = (i128)num * b.den, r = (i128)b.num * den;
    if (l < r)
      take = true;
    else if (l == r)
      take = tie_order(kx, ky, wx - vx, wy - vy, b.wx - vx, b.wy - vy) < 0;
  }
  if (take) {
    b.num = num;
    b.den = den;
    b.seg = sid;
    b.wx = wx;
    b.wy = wy;
    b.vx = vx;
    b.vy = vy;
  }
}

__device__ __forceinline__ float best_t(const Best& b) {
  if (b.seg < 0) return __int_as_float(0x7f800000);
  return __fmul_rn(__fdiv_rn(__ll2float_rn(b.num), __ll2float_rn(b.den)), kDirScale);
}

// Closed-box slab test; on a hit, tn = entry parameter (>= 0).
__device__ __forceinline__ bool box_hit(const int4 B, int ox, int oy, int kx, int ky, Frac& tn) {
  Frac nr{0, 1}, fr{0, 0};
  if (kx == 0) {
    if (ox < B.x || ox > B.z) return false;
  } else {
    const Frac a = kx > 0 ? Frac{B.x - ox, kx} : Frac{ox - B.z, -kx};
    const Frac c = kx > 0 ? Frac{B.z - ox, kx} : Frac{ox - B.x, -kx};
    if (frac_lt(nr, a)) nr = a;
    if (frac_lt(c, fr)) fr = c;
  }
  if (ky == 0) {
    if (oy < B.y || oy > B.w) return false;
  } else {
    const Frac a = ky > 0 ? Frac{B.y - oy, ky} : Frac{oy - B.w, -ky};
    const Frac c = ky > 0 ? Frac{B.w - oy, ky} : Frac{oy - B.y, -ky};
    if (frac_lt(nr, a)) nr = a;
    if (frac_lt(c, fr)) fr = c;
  }
  if (frac_lt(fr, nr)) return false;
  tn = nr;
  return true;
}

constexpr int kBvhStack = 64;
constexpr int kBaseThreads = 128;

__global__ void __launch_bounds__(kBaseThreads) bvh_kernel(BvhDev B, const int32_t* __restrict__ rox,
                                                           const int32_t* __restrict__ roy,
                                                           const float* __restrict__ rdx,
                                                           const float* __restrict__ rdy, int64_t n,
                                                           int32_t* __restrict__ hit, float* __restrict__ tout,
                                                           int32_t* __restrict__ ops) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int ox = rox[i], oy = roy[i];
    int kx, ky;
    if (!dir_to_k(rdx[i], kx) || !dir_to_k(rdy[i], ky) || (kx | ky) == 0) {
      hit[i] = -1;
      tout[i] = __int_as_float(0x7fc00000);
      ops[2 * i] = -1;
      ops[2 * i + 1] = -1;
      continue;
    }
    Best b;
    b.seg = -1;
    b.num = 0;
    b.den = 1;
    b.wx = b.wy = b.vx = b.vy = 0;
    int n_aabb = 1, n_prim = 0;
    int st_node[kBvhStack];
    Frac st_t[kBvhStack];
    int sp = 0;
    bool bad = false;  // the checked build met an out-of-range table index
    Frac tn;
    if (box_hit(B.box[0], ox, oy, kx, ky, tn)) {
      st_node[0] = 0;
      st_t[0] = tn;
      sp = 1;
    }
    while (sp > 0) {
      --sp;
      const int N = st_node[sp];
      if (b.seg >= 0 && cmp_frac_seg(st_t[sp], b.num, b.den) > 0) continue;
      const int c0 = B.c0[N];
      if (c0 < 0) {
        const int first = -1 - c0, cnt = B.c1[N];
        if (kChecked && (cnt < 0 || first > B.n_prims - cnt)) {
          bad = true;
          break;
        }
        for (int k = 0; k < cnt; ++k) {
          const int sid = B.prims[first + k];
          if (idx_bad(sid, B.n_seg)) {
            bad = true;
            break;
          }
          ++n_prim;
          seg_test(B.seg[sid], sid, ox, oy, kx, ky, b, nullptr);
        }
        if (bad) break;
        continue;
      }
      const int c1 = B.c1[N];
      // children after their parent (so the traversal ends) and room on the stack
      if (kChecked && (c0 <= N || c1 <= N || c0 >= B.n_nodes || c1 >= B.n_nodes || sp + 2 > kBvhStack)) {
        bad = true;
        break;
      }
      Frac t0, t1;
      n_aabb += 2;
      bool h0 = box_hit(B.box[c0], ox, oy, kx, ky, t0);
      bool h1 = box_hit(B.box[c1], ox, oy, kx, ky, t1);
      if (h0 && b.seg >= 0 && cmp_frac_seg(t0, b.num, b.den) > 0) h0 = false;
      if (h1 && b.seg >= 0 && cmp_frac_seg(t1, b.num, b.den) > 0) h1 = false;
      if (h0 && h1) {
        const bool first0 = !frac_lt(t1, t0);  // nearer first; left on equal entry
        st_node[sp] = first0 ? c1 : c0;
        st_t[sp] = first0 ? t1 : t0;
        ++sp;
        st_node[sp] = first0 ? c0 : c1;
        st_t[sp] = first0 ? t0 : t1;
        ++sp;
      } else if (h0) {
        st_node[sp] = c0;
        st_t[sp] = t0;
        ++sp;
      } else if (h1) {
        st_node[sp] = c1;
        st_t[sp] = t1;
        ++sp;
      }
    }
    if (bad) {
      hit[i] = -1;
      tout[i] = __int_as_float(0x7fc00000);
      ops[2 * i] = CCT_RAY_BAD_INDEX;
      ops[2 * i + 1] = CCT_RAY_BAD_INDEX;
      continue;
    }
    hit[i] = b.seg;
    tout[i] = best_t(b);
    ops[2 * i] = n_aabb;
    ops[2 * i + 1] = n_prim;
  }
}

constexpr int kMailboxSlots = 256;  // per thread; a ray with more unique tests overflows (flagged)

// Side of the split plane value s on axis a for a point moving with k (a tie
// at the plane goes the way the ray moves; with k_a = 0 the way the ray is
// shifted, to its right).  Returns true for the child with coordinates >= s.
__device__ __forceinline__ bool tie_side(int a, int kx, int ky) {
  const int ka = a == 0 ? kx : ky;
  if (ka != 0) return ka > 0;
  const int right_normal = a == 0 ? ky : -kx;  // right-hand normal (ky, -kx), component a
  return right_normal > 0;
}

__global__ void __launch_bounds__(kBaseThreads) kd_kernel(KdDev K, const int32_t* __restrict__ rox,
                                                          const int32_t* __restrict__ roy,
                                                          const float* __restrict__ rdx,
                                                          const float* __restrict__ rdy, int64_t n,
                                                          int32_t* __restrict__ hit, float* __restrict__ tout,
                                                          int32_t* __restrict__ ops,
                                                          unsigned long long* __restrict__ mailbox) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long* mb = mailbox + tid * kMailboxSlots;
  unsigned stamp = 0;
  for (long long i = tid; i < n; i += stride) {
    int32_t* o = ops + 6 * i;
    const int ox = rox[i], oy = roy[i];
    int kx, ky;
    const int4 root = K.box[0];
    if (!dir_to_k(rdx[i], kx) || !dir_to_k(rdy[i], ky) || (kx | ky) == 0 || ox < root.x || ox > root.z ||
        oy < root.y || oy > root.w) {
      hit[i] = -1;
      tout[i] = __int_as_float(0x7fc00000);
      for (int q = 0; q < 6; ++q) o[q] = -1;
      continue;
    }
    ++stamp;
    // start leaf: descend with the origin (not counted: known a priori, Sec. 5.4)
    int L = 0;
    bool bad = false;  // the checked build met an out-of-range table index
    while (K.axis[L] != 2) {
      const int a = K.axis[L], s = K.split[L];
      const int c = (a == 0 ? ox : oy) - s;
      const bool right = c > 0 || (c == 0 && tie_side(a, kx, ky));
      const int ch = K.child[L];
      if (kChecked && (ch <= L || ch >= K.n_nodes - 1)) {  // children follow their parent
        bad = true;
        break;
      }
      L = ch + (right ? 1 : 0);
    }
    Best b;
    b.seg = -1;
    b.num = 0;
    b.den = 1;
    b.wx = b.wy = b.vx = b.vy = 0;
    int leaves = 0, desc = 0, tests = 0, uniq = 0, ropes = 0, overflow = 0;
    const int guard = K.n_nodes + 8;
    while (!bad) {
      if (++leaves > guard) {
        b.seg = -1;
        overflow = 2;  // corrupt ropes: reported as a mailbox/traversal fault
        break;
      }
      const int4 B = K.box[L];
      const Frac tx = kx > 0 ? Frac{B.z - ox, kx} : (kx < 0 ? Frac{ox - B.x, -kx} : Frac{0, 0});
      const Frac ty = ky > 0 ? Frac{B.w - oy, ky} : (ky < 0 ? Frac{oy - B.y, -ky} : Frac{0, 0});
      const bool xface = !frac_lt(ty, tx);  // x face unless the y face is strictly nearer
      const Frac te = xface ? tx : ty;
      const int face = xface ? (kx > 0 ? 1 : 0) : (ky > 0 ? 3 : 2);
      const int first = K.child[L], cnt = K.count[L];
      if (kChecked && (first < 0 || cnt < 0 || first > K.n_refs - cnt)) {
        bad = true;
        break;
      }
      for (int q = 0; q < cnt; ++q) {
        const int sid = K.refs[first + q];
        if (idx_bad(sid, K.n_seg)) {
          bad = true;
          break;
        }
        ++tests;
        // ideal mailbox: count each segment once per ray
        unsigned h = ((unsigned)sid * 2654435761u) >> 24;
        bool seen = false, placed = false;
        for (int p = 0; p < kMailboxSlots; ++p) {
          const unsigned slot = (h + p) & (kMailboxSlots - 1);
          const unsigned long long v = mb[slot];
          if ((unsigned)(v >> 32) != stamp) {
            mb[slot] = ((unsigned long long)stamp << 32) | (unsigned)sid;
            placed = true;
            break;
          }
          if ((int)(unsigned)v == sid) {
            seen = true;
            break;
          }
        }
        if (!seen) ++uniq;
        if (!seen && !placed) overflow = 1;
        seg_test(K.seg[sid], sid, ox, oy, kx, ky, b, &te);
      }
      if (bad || b.seg >= 0) break;
      const int4 R = K.rope[L];
      const int nxt = face == 0 ? R.x : (face == 1 ? R.y : (face == 2 ? R.z : R.w));
      if (nxt < 0) break;  // left the domain: a miss
      if (idx_bad(nxt, K.n_nodes)) {
        bad = true;
        break;
      }
      ropes += (K.rope_log2[L] >> (8 * face)) & 0xff;
      // descend to the leaf holding the exit point P = o + te * k
      int N = nxt;
      const int fa = face >> 1;
      const int plane = face == 0 ? B.x : (face == 1 ? B.z : (face == 2 ? B.y : B.w));
      while (K.axis[N] != 2) {
        const int a = K.axis[N], s = K.split[N];
        bool right;
        if (a == fa) {
          right = plane > s || (plane == s && tie_side(a, kx, ky));
        } else {
          const int oa = a == 0 ? ox : oy, ka = a == 0 ? kx : ky;
          const long long v = (long long)(oa - s) * te.den + (long long)te.num * ka;  // (P_a - s) * den
          right = v > 0 || (v == 0 && tie_side(a, kx, ky));
        }
        const int ch = K.child[N];
        if (kChecked && (ch <= N || ch >= K.n_nodes - 1)) {
          bad = true;
          break;
        }
        N = ch + (right ? 1 : 0);
        ++desc;
      }
      L = N;
    }
    if (bad) {
      hit[i] = -1;
      tout[i] = __int_as_float(0x7fc00000);
      for (int q = 0; q < 6; ++q) o[q] = CCT_RAY_BAD_INDEX;
      continue;
    }
    hit[i] = b.seg;
    tout[i] = best_t(b);
    o[0] = leaves;
    o[1] = desc;
    o[2] = tests;
    o[3] = uniq;
    o[4] = ropes;
    o[5] = overflow;
  }
}

static size_t al256c(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace cct

using namespace cct;

struct cct_bvh_s {
  BvhDev dev;
  void* base;
  int device;
};

struct cct_kdtree_s {
  KdDev dev;
  void* base;
  int device;
};

template <typename T>
static int upload(cudaStream_t st, char* base, size_t off, const T* src, size_t count) {
  if (count == 0) return CCT_OK;
  return cudaMemcpyAsync(base + off, src, sizeof(T) * count, cudaMemcpyHostToDevice, st) == cudaSuccess
             ? CCT_OK
             : CCT_ERR_CUDA;
}

extern "C" int cct_bvh_load(const cct_bvh_desc* d, void* stream_v, cct_bvh* out) {
  if (!d || !out || d->n_nodes < 1 || d->n_prims < 0 || d->n_seg < 0 || !d->box || !d->child0 || !d->child1 ||
      (d->n_prims > 0 && !d->prims) || (d->n_seg > 0 && !d->seg))
    return CCT_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  // indices in range, children after their parent (descents terminate), depth
  // within the traversal stack, leaf ranges inside the primitive list
  std::vector<int> depth(d->n_nodes, 0);
  for (int v = 0; v < d->n_nodes; ++v) {
    const int c0 = d->child0[v], c1 = d->child1[v];
    if (c0 < 0) {
      const long long first = -1ll - c0;
      if (c1 < 0 || first + c1 > d->n_prims) return CCT_ERR_INVALID_ARGUMENT;
    } else {
      if (c0 <= v || c1 <= v || c0 >= d->n_nodes || c1 >= d->n_nodes) return CCT_ERR_INVALID_ARGUMENT;
      depth[c0] = std::max(depth[c0], depth[v] + 1);
      depth[c1] = std::max(depth[c1], depth[v] + 1);
      if (depth[c0] >= kBvhStack - 2) return CCT_ERR_INVALID_ARGUMENT;
    }
  }
  for (int k = 0; k < d->n_prims; ++k)
    if (d->prims[k] < 0 || d->prims[k] >= d->n_seg) return CCT_ERR_INVALID_ARGUMENT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CCT_ERR_NO_DEVICE;
  cudaStream_t st = (cudaStream_t)stream_v;
  const size_t o_box = 0, o_c0 = o_box + al256c(16ull * d->n_nodes), o_c1 = o_c0 + al256c(4ull * d->n_nodes);
  const size_t o_pr = o_c1 + al256c(4ull * d->n_nodes), o_seg = o_pr + al256c(4ull * d->n_prims + 4);
  const size_t total = o_seg + al256c(16ull * d->n_seg + 16);
  char* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) {
    cudaGetLastError();
    return CCT_ERR_OUT_OF_MEMORY;
  }
  int rc = upload(st, base, o_box, d->box, 4ull * d->n_nodes);
  if (rc == CCT_OK) rc = upload(st, base, o_c0, d->child0, d->n_nodes);
  if (rc == CCT_OK) rc = upload(st, base, o_c1, d->child1, d->n_nodes);
  if (rc == CCT_OK) rc = upload(st, base, o_pr, d->prims, d->n_prims);
  if (rc == CCT_OK) rc = upload(st, base, o_seg, d->seg, 4ull * d->n_seg);
  if (rc == CCT_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = CCT_ERR_CUDA;
  if (rc != CCT_OK) {
    cudaFree(base);
    return rc;
  }
  auto* b = new cct_bvh_s;
  b->base = base;
  b->device = dev;
  b->dev = BvhDev{(const int4*)(base + o_box), (const int32_t*)(base + o_c0), (const int32_t*)(base + o_c1),
                  (const int32_t*)(base + o_pr), (const int4*)(base + o_seg), d->n_nodes, d->n_prims, d->n_seg};
  *out = b;
  return CCT_OK;
}

extern "C" int cct_bvh_poke(cct_bvh b, int32_t table, int64_t index, int32_t value, int32_t* old, int64_t* len) {
  if (!b) return CCT_ERR_INVALID_ARGUMENT;
  if (!kChecked) return CCT_ERR_UNSUPPORTED;
  const BvhDev& B = b->dev;
  switch (table) {
    case CCT_TABLE_BVH_CHILD0:
      return poke_word(b->device, B.c0, B.n_nodes, index, index, value, old, len);
    case CCT_TABLE_BVH_CHILD1:
      return poke_word(b->device, B.c1, B.n_nodes, index, index, value, old, len);
    case CCT_TABLE_BVH_PRIM:
      return poke_word(b->device, B.prims, B.n_prims, index, index, value, old, len);
    default:
      return CCT_ERR_INVALID_ARGUMENT;
  }
}

extern "C" int cct_bvh_free(cct_bvh b) {
  if (!b) return CCT_OK;
  int rc = CCT_OK;
  {
    DeviceGuard g(b->device);
    if (cudaFree(b->base) != cudaSuccess) rc = CCT_ERR_CUDA;
  }
  delete b;
  return rc;
}

extern "C" int cct_trace_bvh(cct_bvh b, const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                             int64_t n, int32_t* hit, float* t, int32_t* ops, void* stream_v) {
  if (!b || n < 0) return CCT_ERR_INVALID_ARGUMENT;
  if (n == 0) return CCT_OK;
  if (!ox || !oy || !dx || !dy || !hit || !t || !ops) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(b->device);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bvh_kernel, kBaseThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const long long grid =
      std::max(1ll, std::min<long long>((long long)sm_count(b->device) * per_sm, (n + kBaseThreads - 1) / kBaseThreads));
  bvh_kernel<<<(unsigned)grid, kBaseThreads, 0, (cudaStream_t)stream_v>>>(b->dev, ox, oy, dx, dy, n, hit, t, ops);
  return cudaGetLastError() == cudaSuccess ? CCT_OK : CCT_ERR_CUDA;
}

extern "C" int cct_kdtree_load(const cct_kdtree_desc* d, void* stream_v, cct_kdtree* out) {
  if (!d || !out || d->n_nodes < 1 || d->n_refs < 0 || d->n_seg < 0 || !d->axis || !d->split || !d->child ||
      !d->count || !d->box || !d->rope || !d->rope_log2 || (d->n_refs > 0 && !d->refs) || (d->n_seg > 0 && !d->seg))
    return CCT_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  const int nn = d->n_nodes;
  std::vector<int32_t> packed_log2(nn, 0);
  for (int v = 0; v < nn; ++v) {
    const int a = d->axis[v];
    if (a < 0 || a > 2) return CCT_ERR_INVALID_ARGUMENT;
    if (a == 2) {
      const long long first = d->child[v], cnt = d->count[v];
      if (first < 0 || cnt < 0 || first + cnt > d->n_refs) return CCT_ERR_INVALID_ARGUMENT;
    } else if (d->child[v] <= v || d->child[v] + 1 >= nn) {
      return CCT_ERR_INVALID_ARGUMENT;
    }
    for (int f = 0; f < 4; ++f) {
      const int r = d->rope[4 * v + f], lg = d->rope_log2[4 * v + f];
      if (r < -1 || r >= nn || lg < 0 || lg > 255) return CCT_ERR_INVALID_ARGUMENT;
      packed_log2[v] |= lg << (8 * f);
    }
  }
  for (int k = 0; k < d->n_refs; ++k)
    if (d->refs[k] < 0 || d->refs[k] >= d->n_seg) return CCT_ERR_INVALID_ARGUMENT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CCT_ERR_NO_DEVICE;
  cudaStream_t st = (cudaStream_t)stream_v;
  size_t off = 0;
  const size_t o_axis = off;
  off += al256c(4ull * nn);
  const size_t o_split = off;
  off += al256c(4ull * nn);
  const size_t o_child = off;
  off += al256c(4ull * nn);
  const size_t o_count = off;
  off += al256c(4ull * nn);
  const size_t o_box = off;
  off += al256c(16ull * nn);
  const size_t o_rope = off;
  off += al256c(16ull * nn);
  const size_t o_lg = off;
  off += al256c(4ull * nn);
  const size_t o_refs = off;
  off += al256c(4ull * d->n_refs + 4);
  const size_t o_seg = off;
  off += al256c(16ull * d->n_seg + 16);
  char* base = nullptr;
  if (cudaMalloc(&base, off) != cudaSuccess) {
    cudaGetLastError();
    return CCT_ERR_OUT_OF_MEMORY;
  }
  int rc = upload(st, base, o_axis, d->axis, nn);
  if (rc == CCT_OK) rc = upload(st, base, o_split, d->split, nn);
  if (rc == CCT_OK) rc = upload(st, base, o_child, d->child, nn);
  if (rc == CCT_OK) rc = upload(st, base, o_count, d->count, nn);
  if (rc == CCT_OK) rc = upload(st, base, o_box, d->box, 4ull * nn);
  if (rc == CCT_OK) rc = upload(st, base, o_rope, d->rope, 4ull * nn);
  if (rc == CCT_OK) rc = upload(st, base, o_lg, packed_log2.data(), nn);
  if (rc == CCT_OK) rc = upload(st, base, o_refs, d->refs, d->n_refs);
  if (rc == CCT_OK) rc = upload(st, base, o_seg, d->seg, 4ull * d->n_seg);
  if (rc == CCT_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = CCT_ERR_CUDA;
  if (rc != CCT_OK) {
    cudaFree(base);
    return rc;
  }
  auto* k = new cct_kdtree_s;
  k->base = base;
  k->device = dev;
  k->dev = KdDev{(const int32_t*)(base + o_axis), (const int32_t*)(base + o_split), (const int32_t*)(base + o_child),
                 (const int32_t*)(base + o_count), (const int4*)(base + o_box),     (const int4*)(base + o_rope),
                 (const int32_t*)(base + o_lg),    (const int32_t*)(base + o_refs), (const int4*)(base + o_seg),
                 nn,                               d->n_refs,                       d->n_seg};
  *out = k;
  return CCT_OK;
}

extern "C" int cct_kdtree_poke(cct_kdtree k, int32_t table, int64_t index, int32_t value, int32_t* old,
                               int64_t* len) {
  if (!k) return CCT_ERR_INVALID_ARGUMENT;
  if (!kChecked) return CCT_ERR_UNSUPPORTED;
  const KdDev& K = k->dev;
  switch (table) {
    case CCT_TABLE_KD_CHILD:
      return poke_word(k->device, K.child, K.n_nodes, index, index, value, old, len);
    case CCT_TABLE_KD_ROPE:
      return poke_word(k->device, K.rope, 4ll * K.n_nodes, index, index, value, old, len);
    case CCT_TABLE_KD_REF:
      return poke_word(k->device, K.refs, K.n_refs, index, index, value, old, len);
    default:
      return CCT_ERR_INVALID_ARGUMENT;
  }
}

extern "C" int cct_kdtree_free(cct_kdtree k) {
  if (!k) return CCT_OK;
  int rc = CCT_OK;
  {
    DeviceGuard g(k->device);
    if (cudaFree(k->base) != cudaSuccess) rc = CCT_ERR_CUDA;
  }
  delete k;
  return rc;
}

extern "C" int cct_trace_kdtree(cct_kdtree k, const int32_t* ox, const int32_t* oy, const float* dx, const float* dy,
                                int64_t n, int32_t* hit, float* t, int32_t* ops, void* stream_v) {
  if (!k || n < 0) return CCT_ERR_INVALID_ARGUMENT;
  if (n == 0) return CCT_OK;
  if (!ox || !oy || !dx || !dy || !hit || !t || !ops) return CCT_ERR_INVALID_ARGUMENT;
  DeviceGuard g(k->device);
  cudaStream_t stream = (cudaStream_t)stream_v;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kd_kernel, kBaseThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long long grid =
      std::max(1ll, std::min<long long>((long long)sm_count(k->device) * per_sm, (n + kBaseThreads - 1) / kBaseThreads));
  const size_t mb_bytes = (size_t)grid * kBaseThreads * kMailboxSlots * sizeof(unsigned long long);
  Scratch sc;
  sc.stream = stream;
  if (cudaMallocAsync((void**)&sc.base, mb_bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    sc.base = nullptr;
    return CCT_ERR_OUT_OF_MEMORY;
  }
  if (cudaMemsetAsync(sc.base, 0, mb_bytes, stream) != cudaSuccess) return CCT_ERR_CUDA;
  kd_kernel<<<(unsigned)grid, kBaseThreads, 0, stream>>>(k->dev, ox, oy, dx, dy, n, hit, t, ops,
                                                         (unsigned long long*)sc.base);
  return cudaGetLastError() == cudaSuccess ? CCT_OK : CCT_ERR_CUDA;
}
