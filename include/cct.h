/* cct.h -- C ABI of libcct: closest-hit queries of 2D rays against a scene of
 * line segments, answered by a stackless walk through a constrained
 * triangulation whose edges contain every segment, on one GB300 (sm_103a).
 *
 * Method: Frederickx & Dutre, "Stackless Ray-Object Intersections Using
 * Approximate Minimum Weight Triangulations" (arXiv 2112.05570).
 *   Sec. 5.1  ray traversal: in the triangle that holds the ray, find the edge
 *             the ray leaves through; an edge of the original geometry is the
 *             closest hit, an edge with no neighbour (the hull) is a miss,
 *             otherwise continue in the neighbour across that edge.
 *   Sec. 5.2  the start triangle: known a priori, or found by walking from a
 *             point with a known triangle; seed points on a regular grid.
 *   Sec. 5.4  one traversal operation = one exit-edge determination in one
 *             visited triangle; start cells known a priori for the count.
 *
 * Geometry and exactness.  Vertices are integer points of [0, D]^2 with
 * D <= 2^20; the hull of the triangulation is that square.  Ray origins are
 * integer points; a direction d = (dx, dy) is fp32 with each component a
 * multiple of 2^-22 and |dx|, |dy| <= 1, so k = 2^22 d is an exact integer
 * vector.  The side of a point v is L iff k.x (v.y - o.y) - k.y (v.x - o.x) >= 0
 * (a point on the ray's line counts as left: the ray is shifted infinitesimally
 * to its right), which makes the walk consistent across neighbouring triangles
 * (Sec. 5.1 requires consistency).  Sides are decided in fp32 under a static
 * error bound and, only where that is inconclusive, in exact int64 arithmetic:
 * hit ids and step counts are exact; t is fp32 (within 4 ulp of the exact
 * rational parameter of the hit).
 *
 * Conventions for every function:
 *   - returns CCT_OK (0) or a negative CCT_ERR_* code; no function aborts,
 *     throws or traps the GPU;
 *   - pointers named d_* are device memory owned by the caller; cct_tri_desc
 *     arrays are host memory owned by the caller, only read during the call;
 *   - work is enqueued on `stream` (a cudaStream_t, NULL = legacy default) and
 *     the call returns without waiting, except cct_scene_load (waits for its
 *     upload), cct_get_stats (waits for `stream`) and cct_scene_free;
 *   - a scene is immutable after loading and may be used from several streams
 *     at once; free it only after all work using it has completed.
 */
#ifndef CCT_H
#define CCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define CCT_OK 0
#define CCT_ERR_INVALID_ARGUMENT -1    /* null pointer, negative count, size out of range */
#define CCT_ERR_BAD_TRIANGULATION -2   /* cct_scene_load validation failed */
#define CCT_ERR_OUT_OF_MEMORY -3       /* a device or host allocation failed */
#define CCT_ERR_CUDA -4                /* a CUDA runtime call failed */
#define CCT_ERR_WALK_LIMIT -5          /* reported by cct_get_stats' counters only */
#define CCT_ERR_NO_DEVICE -6           /* no usable CUDA device */
#define CCT_ERR_IO -7                  /* cct_scene_load_file: file missing, unreadable or malformed */
#define CCT_ERR_UNSUPPORTED -8         /* the call needs the checked build (libcct_checked.so) */

/* Per-ray status, written to d_steps instead of a step count. */
#define CCT_RAY_INVALID -1    /* direction off the 2^-22 grid, |component| > 1, zero, or the
                                 start triangle does not strictly contain the origin */
#define CCT_RAY_WALK_LIMIT -2 /* more than n_tri + 8 steps (only on a corrupt triangulation) */
#define CCT_RAY_NONE -3       /* cct_trace_bounces: no ray at this bounce (the path ended before it) */
#define CCT_RAY_BAD_INDEX -4  /* checked build only: the ray met an out-of-range index in a device
                                 table (a corrupted table), which was not read */

/* ------------------------------------------------------------------ flags */
/* cct_scene_load */
#define CCT_LOAD_NO_REORDER 1u  /* keep the caller's triangle order (default: Hilbert order) */
#define CCT_LOAD_NO_VALIDATE 2u /* skip the geometric checks of cct_scene_load (fault-injection tests);
                                   index ranges are always checked */
#define CCT_LOAD_TWO_STEP 4u    /* also build two-step half-edge records (64 bytes per half-edge, 192
                                   per triangle): the record of a half-edge together with the records
                                   behind its two exits, so that the paths of cct_trace_bounces decide
                                   two triangles per dependent load (see there) */

/* Density of the locate seed grid (Sec. 5.2): square cells of side 2^s with
 * about 2^k cells per triangle, k in [0, 8] (at most 8192 cells per side; 4
 * bytes per cell), encoded in bits 8..11 of the load flags.  Without it k = 5
 * (about 1.1 locate steps per uniformly placed origin). */
#define CCT_LOAD_SEED_DENSITY(k) ((uint32_t)((k) + 1) << 8)

/* cct_trace */
#define CCT_TRACE_EXACT_ONLY 1u /* decide every side in int64 (no fp32 filter) */
#define CCT_TRACE_BIN 2u        /* sort rays by start cell before walking (ray binning) */
#define CCT_TRACE_SPLIT_LOCATE 4u /* without start cells: locate all origins in a separate kernel
                                     first (default: inside the walk kernel) */
#define CCT_TRACE_STAGE 8u      /* each block first copies the scene's half-edge table (48 bytes per
                                   triangle) into shared memory and walks from there; used only when
                                   it fits beside the block's stacks (about 3,500 triangles at 64
                                   threads per block, fewer for larger blocks) and the rays are not
                                   binned, ignored otherwise.  Pays on small scenes only */
#define CCT_TRACE_ONE_STEP 16u  /* cct_trace_bounces on a scene loaded with CCT_LOAD_TWO_STEP: walk one
                                   triangle per load on the 16-byte records anyway */

/* ------------------------------------------------------------------ types */
typedef struct cct_scene_s* cct_scene; /* opaque; the library owns all device memory of a scene */

/* A triangulation of [0, D]^2 whose constrained edges cover the scene
 * segments (Sec. 1.3: the primitives lie on cell boundaries).  Host arrays:
 *   vx, vy   [n_vert]   integer coordinates in [0, D]
 *   tri_v    [3*n_tri]  vertex ids of triangle t, counter-clockwise
 *   tri_nb   [3*n_tri]  triangle across edge i of t (the edge opposite
 *                       vertex i), or -1 on the hull
 *   tri_seg  [3*n_tri]  scene segment id carried by edge i (a constrained edge)
 *                       or -1; equal on both sides of an edge
 * Triangle ids used by cct_trace / cct_locate are indices into this array. */
typedef struct {
  int32_t n_vert;
  int32_t n_tri;
  int32_t n_seg;  /* segment ids in tri_seg lie in [0, n_seg) */
  int32_t domain; /* D, 1 <= D <= 2^20 */
  const int32_t* vx;
  const int32_t* vy;
  const int32_t* tri_v;
  const int32_t* tri_nb;
  const int32_t* tri_seg;
} cct_tri_desc;

/* Device-side counters of a scene, accumulated by every call that uses it. */
typedef struct {
  uint64_t rays;           /* rays walked by cct_trace */
  uint64_t steps;          /* sum of step counts of valid rays (Sec. 5.4 operations) */
  uint64_t side_tests;     /* side-of-line decisions taken by the walk */
  uint64_t exact_fallbacks;/* of those, decided in int64 because the fp32 filter was inconclusive */
  uint64_t invalid_rays;   /* rays reported CCT_RAY_INVALID */
  uint64_t walk_limit_rays;/* rays reported CCT_RAY_WALK_LIMIT */
  uint64_t located;        /* origins located by cct_locate or cct_trace(start = NULL) */
  uint64_t locate_steps;   /* triangles visited by those locate walks (not part of `steps`) */
} cct_stats;

/* Launch configuration of the walk for one scene (no counterpart in the paper;
 * chosen by an autotuner, defaults are used otherwise).
 *   block_threads  threads per block, a multiple of 32 in [32, 512]      (256)
 *   refill_min     a warp serves its idle lanes new rays once this many of
 *                  them are idle, or all of them (the warp-level ray
 *                  retirement / refill), in [1, 32]                          (8)
 *   chunk          rays a warp takes from the global work counter at once,
 *                  in [32, 2^20]                                            (128)
 *   bin_shift      ray-binning granularity: rays are sorted by start record
 *                  index >> bin_shift; -1 = automatic (~64 rays per bin)     (-1)
 *   trace_flags    CCT_TRACE_* flags OR-ed into every cct_trace of the scene  (0) */
typedef struct {
  int32_t block_threads;
  int32_t refill_min;
  int32_t chunk;
  int32_t bin_shift;
  uint32_t trace_flags;
} cct_tuning;

/* ------------------------------------------------------------------ scene */
/* Validates and uploads a triangulation (Sec. 5.1's structure).  Checks: index
 * ranges, strictly CCW triangles, neighbour symmetry, equal labels on both
 * sides, hull edges on the square's sides, sum of areas = D^2.  Reorders the
 * triangles along a Hilbert curve (unless CCT_LOAD_NO_REORDER), packs one
 * 32-byte record per triangle (coordinates and neighbours) and three 16-byte
 * half-edge records (one per entry edge: the apex and the two candidate exits,
 * all a walk step reads) and builds the locate seed grid (Sec. 5.2).
 * Waits for its upload on `stream`.  *out receives the handle.
 * Errors: CCT_ERR_INVALID_ARGUMENT, CCT_ERR_BAD_TRIANGULATION,
 * CCT_ERR_OUT_OF_MEMORY, CCT_ERR_CUDA, CCT_ERR_NO_DEVICE. */
int cct_scene_load(const cct_tri_desc* desc, uint32_t flags, void* stream, cct_scene* out);

/* cct_scene_load from a file holding the triangulation (the offline build of
 * Sec. 4 writes it once; queries load it).  Layout, little-endian: the 8
 * bytes "CCTTRI1" + NUL; int32 n_vert, n_tri, n_seg, domain; then the int32
 * arrays of cct_tri_desc in order: vx[n_vert], vy[n_vert], tri_v[3 n_tri],
 * tri_nb[3 n_tri], tri_seg[3 n_tri].  The header and the file size are checked
 * before anything is allocated; the arrays are then validated by
 * cct_scene_load.  Errors: CCT_ERR_INVALID_ARGUMENT (null argument), CCT_ERR_IO
 * (cannot open or read, wrong magic, counts out of range, size not matching
 * the counts), then those of cct_scene_load. */
#define CCT_FILE_MAGIC "CCTTRI1"
int cct_scene_load_file(const char* path, uint32_t flags, void* stream, cct_scene* out);

/* Releases a scene's device memory.  The caller guarantees no work using it
 * is pending.  NULL is accepted. */
int cct_scene_free(cct_scene scene);

/* Sets (tuning != NULL) or resets to the defaults (NULL) the walk's launch
 * configuration of a scene; takes effect for calls enqueued afterwards.  Not
 * thread-safe against concurrent cct_trace calls on the same scene from other
 * host threads.  Errors: CCT_ERR_INVALID_ARGUMENT (a field out of range). */
int cct_scene_set_tuning(cct_scene scene, const cct_tuning* tuning);

/* Copies the scene's current launch configuration to *out. */
int cct_scene_get_tuning(cct_scene scene, cct_tuning* out);

/* Device bytes held by the scene and its number of triangles (either output
 * pointer may be NULL). */
int cct_scene_info(cct_scene scene, size_t* device_bytes, int32_t* n_tri);

/* Start triangles (Sec. 5.2): for each of n origins (d_ox, d_oy, device int32),
 * walks from the seed point of its grid cell to the origin and writes the id
 * (caller numbering) of the triangle whose interior holds it to
 * d_start_tri[i], or -1 if the origin lies on an edge or a vertex or outside
 * the domain.  n = 0 is a no-op.  Errors: CCT_ERR_INVALID_ARGUMENT,
 * CCT_ERR_CUDA. */
int cct_locate(cct_scene scene, const int32_t* d_ox, const int32_t* d_oy, int64_t n, int32_t* d_start_tri,
               void* stream);

/* Closest hit of n rays (Sec. 5.1).  Inputs (device): origins d_ox, d_oy
 * (int32), directions d_dx, d_dy (fp32 on the 2^-22 grid), and d_start_tri,
 * the triangle (caller numbering) that holds each origin -- or NULL, in which
 * case the origins are located first as by cct_locate.  Outputs (device, all
 * n entries written): d_hit_seg = segment id of the closest hit or -1 (miss
 * or invalid ray); d_t = hit parameter (o + t d), +inf on a miss, NaN on an
 * invalid ray; d_steps = triangles visited including the start triangle
 * (Sec. 5.4), or CCT_RAY_INVALID / CCT_RAY_WALK_LIMIT (CCT_RAY_BAD_INDEX in the checked
 * build).  flags: CCT_TRACE_*.
 * Scratch memory (ray binning, start cells) is taken from the stream-ordered
 * allocator on `stream` and released on it.  n = 0 is a no-op.
 * Errors: CCT_ERR_INVALID_ARGUMENT, CCT_ERR_OUT_OF_MEMORY, CCT_ERR_CUDA. */
int cct_trace(cct_scene scene, const int32_t* d_ox, const int32_t* d_oy, const float* d_dx, const float* d_dy,
              const int32_t* d_start_tri, int64_t n, int32_t* d_hit_seg, float* d_t, int32_t* d_steps,
              uint32_t flags, void* stream);

/* No counterpart in the paper: cct_trace for callers that cannot allocate
 * device memory during a query -- e.g. a process that reserved the GPU's memory
 * for its own pool at start-up, or a latency-critical loop that must not enter
 * an allocator.  Same arguments, outputs and per-ray statuses as cct_trace,
 * and the same launch configuration: the scene's tuning (block size, refill
 * threshold, chunk, and its trace_flags: exact-only predicates, split locate)
 * applies as in cct_trace, except that binning is never used.  The scratch it
 * needs (a work counter and, with CCT_TRACE_SPLIT_LOCATE and no d_start_tri,
 * the located start cells) lives in one file-scope device array of
 * CCT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  Nothing is allocated: no cudaMalloc, cudaFree or allocating
 * library routine is called.
 * Limits: n <= CCT_NOALLOC_MAX_RAYS and no CCT_TRACE_BIN (binning needs scratch
 * per ray); otherwise CCT_ERR_INVALID_ARGUMENT.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make that
 * first call before any stream capture.  All calls share the array and each
 * call clears the part that must start at zero, so calls whose GPU work
 * overlaps (other streams or host threads) race and give wrong results:
 * serialise them.  Errors: those of cct_trace. */
#define CCT_NOALLOC_MAX_RAYS (1 << 20)
#define CCT_NOALLOC_SCRATCH_BYTES (256 + 4 * CCT_NOALLOC_MAX_RAYS)
int cct_trace_noalloc(cct_scene scene, const int32_t* d_ox, const int32_t* d_oy, const float* d_dx,
                      const float* d_dy, const int32_t* d_start_tri, int64_t n, int32_t* d_hit_seg, float* d_t,
                      int32_t* d_steps, uint32_t flags, void* stream);

/* Mirror paths of n primary rays (Sec. 5.2: a secondary ray starts where its
 * parent hit the geometry, and the final triangle of the parent's walk is its
 * start triangle, so secondary rays need no locate).  Each primary ray (inputs
 * and start cells as cct_trace; d_start_tri NULL = located first) is followed
 * by up to n_bounce secondary rays, each the mirror image of its parent about
 * the hit segment (or, with d_frame, a direction the caller gives in the hit
 * edge's frame):
 *   origin     the parent's exact hit point moved onto the hit constrained
 *              edge (a -> b) of the final triangle (a right of the parent ray,
 *              b left or on its line): a + (i / 2^32)(b - a),
 *              i = round(2^32 mu) (halves up) clamped to [1, 2^32 - 1], mu the
 *              exact parameter of the hit point on the edge;
 *   direction  k' = 2 (k.u) u / |u|^2 - k for k = 2^22 d and u = b - a,
 *              rounded to integers (halves up), clamped to [-2^22, 2^22],
 *              then d' = k' / 2^22;  with d_frame (device, 2 * n_bounce * n
 *              floats, the pair (c, s) of ray b >= 1 of path r at
 *              2 ((b - 1) n + r)): k' = 2^22 (c u + s m) / |u| rounded to
 *              integers (halves up, decided exactly) and clamped, m = (-u_y, u_x)
 *              the normal on the parent's side; c and s must lie on the
 *              2^-22 grid with |c|, |s| <= 1 and s > 0, else that ray is
 *              CCT_RAY_INVALID and the path ends (a diffuse or glossy bounce
 *              samples (c, s) without knowing which segment is hit);
 *   walk       Sec. 5.1 from that triangle, entered through the hit edge; the
 *              side rule, hit rule and tie order of cct_trace apply with the
 *              origin in units of 2^-32 (all decisions exact).
 * A path ends at a miss, an invalid primary ray, a walk limit, after n_bounce
 * secondary rays, or when k' does not point strictly back to the parent's side
 * of the segment (a grazing reflection).
 * Outputs (device, (1 + n_bounce) * n entries, entry b * n + r for ray b of
 * path r; b = 0 is the primary ray): d_hit_seg, d_t, d_steps as cct_trace, and
 * CCT_RAY_NONE in d_steps (hit -1, t NaN) where the path ended earlier.
 * Optional outputs (NULL: not written): d_org_x, d_org_y = the ray's origin in
 * units of 2^-32 (int64; 0 where there is no ray or the ray is invalid),
 * d_dir_x, d_dir_y = its direction (0 likewise).
 * Launch: blocks of 256 threads, one path per lane; the scene tuning's chunk
 * applies.  flags: CCT_TRACE_EXACT_ONLY (every decision is exact here anyway) and
 * CCT_TRACE_ONE_STEP (on a scene loaded with CCT_LOAD_TWO_STEP the paths walk
 * the two-step records unless this flag is given: after deciding the exit of
 * a triangle a lane already holds the next triangle's apex and exits, in the
 * same 32-byte sector after a left exit, 16 more bytes of the same record
 * after a right one; 7-12 % faster, identical results).  Scratch
 * (a work counter, located start cells) comes from the stream-ordered
 * allocator on `stream`.  n = 0 is a no-op.
 * Errors: CCT_ERR_INVALID_ARGUMENT (n < 0, n_bounce outside
 * [0, CCT_MAX_BOUNCES], other flags, a null required pointer),
 * CCT_ERR_OUT_OF_MEMORY, CCT_ERR_CUDA. */
#define CCT_MAX_BOUNCES 1024
int cct_trace_bounces(cct_scene scene, const int32_t* d_ox, const int32_t* d_oy, const float* d_dx,
                      const float* d_dy, const int32_t* d_start_tri, int64_t n, int32_t n_bounce,
                      const float* d_frame, int32_t* d_hit_seg,
                      float* d_t, int32_t* d_steps, int64_t* d_org_x, int64_t* d_org_y, float* d_dir_x,
                      float* d_dir_y, uint32_t flags, void* stream);

/* Copies the scene's counters to *out after waiting for `stream`; reset != 0
 * zeroes them afterwards.  Errors: CCT_ERR_INVALID_ARGUMENT, CCT_ERR_CUDA. */
int cct_get_stats(cct_scene scene, cct_stats* out, int reset, void* stream);

/* ------------------------------------------------------------------ many scenes in one launch */
/* No counterpart in the paper (a GPU batching layer over Sec. 5.1/5.2): one
 * persistent launch walks the rays of many items, each item a ray batch
 * against one of a set of device-resident scenes.  Items are cut into chunks
 * of `chunk` rays (cct_tuning) that the launch's warps take from one work
 * counter, so scenes and batches of very different sizes share the GPU. */
typedef struct {
  int32_t scene;              /* index into the scene array of the batch */
  int32_t ray_stride;         /* 0 or 1: separate ray arrays; 4: ray i's ox, oy, dx, dy are 4
                                 consecutive 32-bit words (d_ox = record base, d_oy = d_ox + 1, ...) */
  int64_t n;                  /* rays, < 2^31 */
  const int32_t* d_ox;        /* device arrays as in cct_trace */
  const int32_t* d_oy;
  const float* d_dx;
  const float* d_dy;
  const int32_t* d_start_tri; /* caller numbering of that scene, or NULL: locate */
  int32_t* d_hit_seg;
  float* d_t;
  int32_t* d_steps;
} cct_batch_item;

typedef struct cct_batch_s* cct_batch;

/* A reusable batch over n_scenes loaded scenes (all on one device) for up to
 * max_items items; flags: 0 or CCT_TRACE_EXACT_ONLY.  Holds a device work table
 * and a pinned, device-mapped host staging copy of it.  The scenes must outlive
 * the batch. */
int cct_batch_create(const cct_scene* scenes, int32_t n_scenes, int32_t max_items, uint32_t flags, cct_batch* out);
int cct_batch_free(cct_batch batch);

/* Block size, refill threshold and chunk of later stages and enqueues (bin_shift
 * and trace_flags are ignored); NULL = defaults. */
int cct_batch_set_tuning(cct_batch batch, const cct_tuning* tuning);

/* Writes the work list into the host staging copy (host only, no GPU work).
 * Must not be called while an enqueued copy of the staging buffer may still be
 * pending on the GPU.  Errors: CCT_ERR_INVALID_ARGUMENT (scene index, counts,
 * null arrays, more than max_items). */
int cct_batch_stage(cct_batch batch, const cct_batch_item* items, int32_t n_items);

/* Enqueues on `stream` two kernels: one that copies the staged table (its full
 * fixed size, read by the GPU from the mapped staging buffer) to the device and
 * resets the work counter, then the persistent walk.  No copy engine is used,
 * so the launch does not queue behind the caller's bulk transfers on other
 * streams.  Both have fixed arguments, so one stream capture of this call can
 * be replayed after every cct_batch_stage. */
int cct_batch_enqueue(cct_batch batch, void* stream);

/* Counters accumulated by this batch's launches (per-scene counters of
 * cct_get_stats do not include batched work); waits for `stream`. */
int cct_batch_get_stats(cct_batch batch, cct_stats* out, int reset, void* stream);

/* One-shot convenience: create, stage, enqueue, wait for `stream`, free. */
int cct_trace_batched(const cct_scene* scenes, int32_t n_scenes, const cct_batch_item* items, int32_t n_items,
                      uint32_t flags, void* stream);

/* ------------------------------------------------------------------ comparison structures (Sec. 5.3) */
/* The two classical structures the paper compares against, traversed on the
 * GPU with the same exact hit rule as the walk, so all three return the same
 * closest hit (segment id and t).  They exist to measure operations per ray
 * the way Sec. 5.3/5.4 counts them, on the same rays. */

typedef struct cct_bvh_s* cct_bvh;

/* SAH BVH over the scene segments (Sec. 5.3.1), host arrays:
 *   box     [4*n_nodes]  closed integer box x0 y0 x1 y1 of every node
 *   child0  [n_nodes]    >= 0: inner node, left child; < 0: leaf whose first
 *                        primitive is prims[-child0 - 1]
 *   child1  [n_nodes]    inner: right child; leaf: primitive count
 *   prims   [n_prims]    segment ids
 *   seg     [4*n_seg]    segments x0 y0 x1 y1
 * Children must follow their parent in the arrays; depth <= 61. */
typedef struct {
  int32_t n_nodes;
  int32_t n_prims;
  int32_t n_seg;
  const int32_t* box;
  const int32_t* child0;
  const int32_t* child1;
  const int32_t* prims;
  const int32_t* seg;
} cct_bvh_desc;

/* Validates (index ranges, child order, depth) and uploads; waits for the
 * upload on `stream`.  Errors: CCT_ERR_INVALID_ARGUMENT, CCT_ERR_OUT_OF_MEMORY,
 * CCT_ERR_CUDA, CCT_ERR_NO_DEVICE. */
int cct_bvh_load(const cct_bvh_desc* desc, void* stream, cct_bvh* out);
int cct_bvh_free(cct_bvh bvh);

/* Closest hit of n rays (device arrays as cct_trace) by stack traversal from
 * the root, nearer child first.  d_ops[2i] = AABB tests, d_ops[2i+1] = segment
 * tests of ray i (Sec. 5.3.1's two operation kinds); -1 for an invalid ray
 * (direction off the 2^-22 grid or zero; hit -1, t NaN). */
int cct_trace_bvh(cct_bvh bvh, const int32_t* d_ox, const int32_t* d_oy, const float* d_dx, const float* d_dy,
                  int64_t n, int32_t* d_hit_seg, float* d_t, int32_t* d_ops, void* stream);

typedef struct cct_kdtree_s* cct_kdtree;

/* Roped kd-tree over the scene segments in [0, D]^2 (Sec. 5.3.2), host arrays:
 *   axis      [n_nodes]    0: split on x, 1: split on y, 2: leaf
 *   split     [n_nodes]    split coordinate of an inner node
 *   child     [n_nodes]    inner: left child (right child = left + 1, after
 *                          the parent); leaf: first index into refs
 *   count     [n_nodes]    leaf: number of refs
 *   box       [4*n_nodes]  node region x0 y0 x1 y1 (closed)
 *   rope      [4*n_nodes]  leaf ropes across faces x-min, x-max, y-min, y-max:
 *                          the deepest node holding the whole region across
 *                          the face, or -1 outside the domain
 *   rope_log2 [4*n_nodes]  ceil(log2 of the leaves adjacent across each face),
 *                          the cost of an ideal rope tree (0..255)
 *   refs      [n_refs]     segment ids (a segment is in every leaf it touches)
 *   seg       [4*n_seg]    segments */
typedef struct {
  int32_t n_nodes;
  int32_t n_refs;
  int32_t n_seg;
  int32_t domain;
  const int32_t* axis;
  const int32_t* split;
  const int32_t* child;
  const int32_t* count;
  const int32_t* box;
  const int32_t* rope;
  const int32_t* rope_log2;
  const int32_t* refs;
  const int32_t* seg;
} cct_kdtree_desc;

/* Validates (index ranges, child order) and uploads; waits on `stream`. */
int cct_kdtree_load(const cct_kdtree_desc* desc, void* stream, cct_kdtree* out);
int cct_kdtree_free(cct_kdtree kd);

/* Closest hit of n rays by stackless rope traversal from the leaf holding the
 * origin (known a priori, Sec. 5.4): segments of a leaf are accepted up to the
 * leaf's exit; otherwise the rope of the exit face is followed and the leaf
 * holding the exit point is found by descending (exit through a corner: the
 * x face; a point on a split plane: the side the ray moves to).  Six counts
 * per ray in d_ops[6i..6i+5]: leaves visited, inner nodes passed in rope
 * descents, segment tests, unique segment tests (ideal mailbox), sum of the
 * crossed faces' rope_log2 (ideal rope tree), mailbox overflow flag (1 when a
 * ray tested more than 256 distinct segments: its unique count is then an
 * upper bound).  The paper's ideal operation count is leaves + rope_log2 sum
 * + unique tests.  -1 in all six for an invalid ray.  Scratch (the mailboxes)
 * from the stream-ordered allocator on `stream`. */
int cct_trace_kdtree(cct_kdtree kd, const int32_t* d_ox, const int32_t* d_oy, const float* d_dx, const float* d_dy,
                     int64_t n, int32_t* d_hit_seg, float* d_t, int32_t* d_ops, void* stream);

/* ------------------------------------------------------------------ checked build */
/* No counterpart in the paper: a checked build and fault injection for it.
 *
 * libcct_checked.so is this library compiled with -DCCT_CHECKED: every index
 * its kernels read out of a device table (a seed cell's triangle, a neighbour
 * or half-edge exit word, a constrained-edge neighbour, the caller-id map, the
 * kd-tree's and BVH's child, rope, reference and primitive entries) is
 * range-checked before it addresses memory.  A ray that meets an index out of
 * range -- possible only in a corrupted table -- ends with CCT_RAY_BAD_INDEX
 * in d_steps (hit -1, t NaN; in every op count of cct_trace_kdtree and
 * cct_trace_bvh) instead of reading outside the table, and cct_locate reports
 * CCT_RAY_BAD_INDEX for its origin.  Every other result equals libcct.so's.
 * libcct.so leaves the checks out: its loaders validate every table, so its
 * indices are in range by construction.  The checked kernels are slower; the
 * build exists to test that claim and to run suspect data. */

/* 1 in libcct_checked.so, 0 in libcct.so. */
int cct_is_checked(void);

/* Device tables the poke calls may overwrite, one 32-bit word at a time:
 *   CCT_TABLE_NEIGHBOUR       scene: neighbour word of edge e of triangle
 *                             record r, index 3 r + e (records in the scene's
 *                             device order, which need not be the caller's)
 *   CCT_TABLE_HALF_EDGE_EXIT  scene: exit word c of half-edge record h (c = 0:
 *                             the exit when the apex is left, 1: right),
 *                             index 2 h + c, h in [0, 3 n_tri)
 *   CCT_TABLE_CONSTRAINED     scene: neighbour across constrained edge e of
 *                             record r (read by the locate walk), index 3 r + e
 *   CCT_TABLE_SEED            scene: the triangle record of locate seed cell c
 *   CCT_TABLE_USER_TO_RECORD  scene: the record of caller triangle id u
 *   CCT_TABLE_KD_CHILD        kd-tree: child of inner node v, first ref of
 *                             leaf v, index v
 *   CCT_TABLE_KD_ROPE         kd-tree: rope across face f of node v, index 4 v + f
 *   CCT_TABLE_KD_REF          kd-tree: ref k
 *   CCT_TABLE_BVH_CHILD0      BVH: child0 of node v
 *   CCT_TABLE_BVH_CHILD1      BVH: child1 of node v
 *   CCT_TABLE_BVH_PRIM        BVH: primitive k
 *   CCT_TABLE_TWO_STEP_EXIT   scene loaded with CCT_LOAD_TWO_STEP: exit word c
 *                             of sub-record k of the two-step record of
 *                             half-edge h (k = 0: h itself, 1: the record
 *                             behind its left exit, 2: behind its right exit),
 *                             index 6 h + 2 k + c */
#define CCT_TABLE_NEIGHBOUR 1
#define CCT_TABLE_HALF_EDGE_EXIT 2
#define CCT_TABLE_CONSTRAINED 3
#define CCT_TABLE_SEED 4
#define CCT_TABLE_USER_TO_RECORD 5
#define CCT_TABLE_KD_CHILD 6
#define CCT_TABLE_KD_ROPE 7
#define CCT_TABLE_KD_REF 8
#define CCT_TABLE_BVH_CHILD0 9
#define CCT_TABLE_BVH_CHILD1 10
#define CCT_TABLE_BVH_PRIM 11
#define CCT_TABLE_TWO_STEP_EXIT 12

/* Fault injection (checked build only): writes `value` at `index` of one of
 * the object's tables, after reading the word it replaces into *old (when old
 * is not NULL).  With index < 0 nothing is written and the table's length is
 * reported in *len (when len is not NULL).  Synchronous: waits for the whole
 * device before and after.  Any value may be written: the checked kernels
 * report each ray that reads an out-of-range one.
 * Errors: CCT_ERR_UNSUPPORTED in libcct.so (its kernels do not check, so it
 * refuses to corrupt a table); CCT_ERR_INVALID_ARGUMENT (NULL object, a table
 * of another kind of object, index beyond the table); CCT_ERR_CUDA. */
int cct_scene_poke(cct_scene scene, int32_t table, int64_t index, int32_t value, int32_t* old, int64_t* len);
int cct_kdtree_poke(cct_kdtree kd, int32_t table, int64_t index, int32_t value, int32_t* old, int64_t* len);
int cct_bvh_poke(cct_bvh bvh, int32_t table, int64_t index, int32_t value, int32_t* old, int64_t* len);

/* No counterpart in the paper: a host utility for a serving loop that moves
 * many requests' rays and results at once.  Enqueues n asynchronous copies on
 * `stream`, in order, one runtime copy call each: copy k moves bytes[k] bytes
 * from src[k] to dst[k] (host or device addresses, resolved by the CUDA
 * runtime's unified addressing; host memory should be pinned for the copies to
 * overlap other work).  The three arrays are host arrays, read before the call
 * returns; the memory they point to must stay valid until the copies have run
 * on the stream.  n = 0 is a no-op.  Errors: CCT_ERR_INVALID_ARGUMENT (n < 0,
 * or a NULL array with n > 0), CCT_ERR_CUDA (a copy could not be enqueued; the
 * copies before it stay enqueued). */
int cct_copies_async(int32_t n, void* const* dst, const void* const* src, const size_t* bytes, void* stream);

/* Static text for a status code. */
const char* cct_error_string(int code);

/* Library version, (major << 16) | minor. */
int cct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CCT_H */
