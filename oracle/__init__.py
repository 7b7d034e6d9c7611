"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
The product package never does and has no CPU fallback.

A plain, slow, exact CPU implementation (``oracle.c``) of what the GPU path
computes, written from the paper (Frederickx & Dutre, arXiv 2112.05570, Sec. 5.1
and 5.4) and sharing no code with the CUDA path.  See ``oracle.c`` for the
degeneracy rule and the per-function citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_libs: dict[int, ctypes.CDLL] = {}

# failure bits of check_triangulation
BAD_INDEX, NOT_CCW, AREA, NB_ASYM, HULL, EULER, CONSTRAINT_ASYM, COVERAGE, NOT_DELAUNAY = (
    1, 2, 4, 8, 16, 32, 64, 128, 256)
N_MUTANTS = 11
PRIMARY_MUTANTS = (1, 2, 3, 4)  # planted in the primary-ray predicates and walk
BOUNCE_MUTANTS = (5, 6, 7)  # planted in the secondary-ray construction
KD_MUTANTS = (8, 9)  # planted in the kd-tree's rope-search count
BVH_MUTANTS = (10, 11)  # planted in the BVH's traversal order and pruning
BOUNCE_NONE = -3  # steps of a path entry with no ray


def _libpath(mutant: int) -> str:
    return os.path.join(_LIBDIR, "liboracle.so" if mutant == 0 else f"liboracle_m{mutant}.so")


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile the oracle (plain C, gcc).  mutant > 0 builds a copy with a
    planted mistake, used only by the tests that show the pins catch it."""
    out = _libpath(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
                           f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def _load(mutant: int = 0) -> ctypes.CDLL:
    if mutant in _libs:
        return _libs[mutant]
    L = ctypes.CDLL(build(mutant=mutant))
    i64, i32, vp, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double
    L.oracle_closest_bruteforce.restype = ctypes.c_int
    L.oracle_closest_bruteforce.argtypes = [i64, vp, i64, vp, vp, vp, vp, vp, vp, i32]
    L.oracle_walk.restype = ctypes.c_int
    L.oracle_walk.argtypes = [i64, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, i32, i32]
    L.oracle_steps_bruteforce.restype = ctypes.c_int
    L.oracle_steps_bruteforce.argtypes = [i64, vp, vp, vp, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, i32]
    L.oracle_locate_bruteforce.restype = ctypes.c_int
    L.oracle_locate_bruteforce.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, i32]
    L.oracle_check_triangulation.restype = i32
    L.oracle_check_triangulation.argtypes = [i64, i64, vp, vp, i64, vp, vp, vp, i64, vp, i32]
    L.oracle_interior_length.restype = dbl
    L.oracle_interior_length.argtypes = [i64, vp, vp, vp, vp]
    L.oracle_count_line_crossings.restype = ctypes.c_int
    L.oracle_count_line_crossings.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, vp, vp]
    L.oracle_bvh_trace.restype = ctypes.c_int
    L.oracle_bvh_trace.argtypes = [i32, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, i32]
    L.oracle_kd_trace.restype = ctypes.c_int
    L.oracle_kd_trace.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, i32]
    L.oracle_bounce_walk.restype = ctypes.c_int
    L.oracle_bounce_walk.argtypes = [i64, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp,
                                     vp, i64, vp, i32]
    L.oracle_bounce_bruteforce.restype = ctypes.c_int
    L.oracle_bounce_bruteforce.argtypes = [i64, vp, vp, vp, vp, i64, vp, i64, vp, vp, vp, vp, i32, vp, vp, vp, vp,
                                           vp, vp, vp, i32]
    L.oracle_mutant.restype = i32
    _libs[mutant] = L
    return L


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _p(a):
    return a.ctypes.data


def _nthreads(n_threads):
    return int(n_threads if n_threads is not None else (os.cpu_count() or 1))


def closest_bruteforce(segs, ox, oy, dx, dy, n_threads=None, mutant=0):
    """Closest hit over all segments: (hit id or -1, t fp32 (+inf miss, NaN invalid))."""
    L = _load(mutant)
    segs = _c(segs, np.int32).reshape(-1, 4)
    ox, oy, dx, dy = _c(ox, np.int32), _c(oy, np.int32), _c(dx, np.float32), _c(dy, np.float32)
    n = ox.size
    hit = np.empty(n, np.int32)
    t = np.empty(n, np.float32)
    L.oracle_closest_bruteforce(segs.shape[0], _p(segs), n, _p(ox), _p(oy), _p(dx), _p(dy), _p(hit), _p(t),
                                _nthreads(n_threads))
    return hit, t


def walk(tri, ox, oy, dx, dy, start, max_steps=None, through=False, n_threads=None, mutant=0,
         want_last=False):
    """The walk of Sec. 5.1 from given start triangles: (hit, t, steps[, last])."""
    L = _load(mutant)
    vx, vy = _c(tri.vx, np.int32), _c(tri.vy, np.int32)
    tv, tn, ts = _c(tri.tri_v, np.int32), _c(tri.tri_nb, np.int32), _c(tri.tri_seg, np.int32)
    ox, oy, dx, dy = _c(ox, np.int32), _c(oy, np.int32), _c(dx, np.float32), _c(dy, np.float32)
    start = _c(start, np.int32)
    n = ox.size
    nt = tv.size // 3
    hit = np.empty(n, np.int32)
    t = np.empty(n, np.float32)
    steps = np.empty(n, np.int32)
    last = np.empty(n, np.int32) if want_last else None
    ms = nt + 8 if max_steps is None else int(max_steps)
    L.oracle_walk(nt, _p(vx), _p(vy), _p(tv), _p(tn), _p(ts), n, _p(ox), _p(oy), _p(dx), _p(dy), _p(start),
                  _p(hit), _p(t), _p(steps), _p(last) if want_last else None, ms, 1 if through else 0,
                  _nthreads(n_threads))
    return (hit, t, steps, last) if want_last else (hit, t, steps)


def steps_bruteforce(tri, ox, oy, dx, dy, hit, n_threads=None, mutant=0):
    """1 + interior edges crossed before the hit, by scanning all edges."""
    L = _load(mutant)
    vx, vy = _c(tri.vx, np.int32), _c(tri.vy, np.int32)
    tv, tn = _c(tri.tri_v, np.int32), _c(tri.tri_nb, np.int32)
    segs = _c(tri.segs, np.int32).reshape(-1, 4)
    ox, oy, dx, dy = _c(ox, np.int32), _c(oy, np.int32), _c(dx, np.float32), _c(dy, np.float32)
    hit = _c(hit, np.int32)
    n = ox.size
    steps = np.empty(n, np.int32)
    L.oracle_steps_bruteforce(tv.size // 3, _p(vx), _p(vy), _p(tv), _p(tn), segs.shape[0], _p(segs), n, _p(ox),
                              _p(oy), _p(dx), _p(dy), _p(hit), _p(steps), _nthreads(n_threads))
    return steps


def _bounce_out(n, n_bounce, with_steps):
    m = (n_bounce + 1) * n
    out = dict(hit=np.empty(m, np.int32), t=np.empty(m, np.float32), org_x=np.empty(m, np.int64),
               org_y=np.empty(m, np.int64), dir_x=np.empty(m, np.float32), dir_y=np.empty(m, np.float32))
    if with_steps:
        out["steps"] = np.empty(m, np.int32)
    return out


def _bounce_shape(out, n, n_bounce):
    return {k: v.reshape(n_bounce + 1, n) for k, v in out.items()}


def _frame(frame, n, n_bounce):
    if frame is None:
        return None
    f = _c(frame, np.float32).reshape(-1)
    if f.size != 2 * n * n_bounce:
        raise ValueError("frame must hold (c, s) for n_bounce x n secondary rays")
    return f


def bounce_walk(tri, ox, oy, dx, dy, start, n_bounce, max_steps=None, n_threads=None, mutant=0, frame=None):
    """Mirror paths (Sec. 5.2: each secondary ray starts in the final triangle
    of its parent's walk): dict of (1 + n_bounce, n) arrays hit, t, steps,
    org_x, org_y (origins in 2^-32 units), dir_x, dir_y.  frame (optional,
    (n_bounce, n, 2) float32): each secondary ray's direction (c, s) in the
    frame of its parent's hit edge instead of the mirror image."""
    L = _load(mutant)
    vx, vy = _c(tri.vx, np.int32), _c(tri.vy, np.int32)
    tv, tn, ts = _c(tri.tri_v, np.int32), _c(tri.tri_nb, np.int32), _c(tri.tri_seg, np.int32)
    ox, oy, dx, dy = _c(ox, np.int32), _c(oy, np.int32), _c(dx, np.float32), _c(dy, np.float32)
    start = _c(start, np.int32)
    n = ox.size
    nt = tv.size // 3
    o = _bounce_out(n, n_bounce, True)
    ms = nt + 8 if max_steps is None else int(max_steps)
    fr = _frame(frame, n, n_bounce)
    L.oracle_bounce_walk(nt, _p(vx), _p(vy), _p(tv), _p(tn), _p(ts), n, _p(ox), _p(oy), _p(dx), _p(dy), _p(start),
                         int(n_bounce), _p(o["hit"]), _p(o["t"]), _p(o["steps"]), _p(o["org_x"]), _p(o["org_y"]),
                         _p(o["dir_x"]), _p(o["dir_y"]), ms, _p(fr) if fr is not None else None, _nthreads(n_threads))
    return _bounce_shape(o, n, n_bounce)


def bounce_bruteforce(tri, ox, oy, dx, dy, n_bounce, n_threads=None, mutant=0, frame=None):
    """The same mirror paths by brute force over all segments (hit edges found
    by scanning the constrained edges): dict as bounce_walk without steps."""
    L = _load(mutant)
    vx, vy = _c(tri.vx, np.int32), _c(tri.vy, np.int32)
    tv, ts = _c(tri.tri_v, np.int32), _c(tri.tri_seg, np.int32)
    segs = _c(tri.segs, np.int32).reshape(-1, 4)
    ox, oy, dx, dy = _c(ox, np.int32), _c(oy, np.int32), _c(dx, np.float32), _c(dy, np.float32)
    n = ox.size
    o = _bounce_out(n, n_bounce, False)
    fr = _frame(frame, n, n_bounce)
    L.oracle_bounce_bruteforce(tv.size // 3, _p(vx), _p(vy), _p(tv), _p(ts), segs.shape[0], _p(segs), n, _p(ox),
                               _p(oy), _p(dx), _p(dy), int(n_bounce), _p(o["hit"]), _p(o["t"]), _p(o["org_x"]),
                               _p(o["org_y"]), _p(o["dir_x"]), _p(o["dir_y"]), _p(fr) if fr is not None else None,
                               _nthreads(n_threads))
    return _bounce_shape(o, n, n_bounce)


def locate_bruteforce(tri, px, py, n_threads=None):
    """Triangle strictly containing each point; -1 on an edge/vertex; -2 outside."""
    L = _load()
    vx, vy, tv = _c(tri.vx, np.int32), _c(tri.vy, np.int32), _c(tri.tri_v, np.int32)
    px, py = _c(px, np.int32), _c(py, np.int32)
    out = np.empty(px.size, np.int32)
    L.oracle_locate_bruteforce(tv.size // 3, _p(vx), _p(vy), _p(tv), px.size, _p(px), _p(py), _p(out),
                               _nthreads(n_threads))
    return out


def check_triangulation(tri, D, check_delaunay=False) -> int:
    """OR of failure bits (0 = every invariant holds); see oracle.c."""
    L = _load()
    vx, vy = _c(tri.vx, np.int32), _c(tri.vy, np.int32)
    tv, tn, ts = _c(tri.tri_v, np.int32), _c(tri.tri_nb, np.int32), _c(tri.tri_seg, np.int32)
    segs = _c(tri.segs, np.int32).reshape(-1, 4)
    return int(L.oracle_check_triangulation(D, vx.size, _p(vx), _p(vy), tv.size // 3, _p(tv), _p(tn), _p(ts),
                                            segs.shape[0], _p(segs), 1 if check_delaunay else 0))


def interior_length(tri) -> float:
    L = _load()
    vx, vy = _c(tri.vx, np.int32), _c(tri.vy, np.int32)
    tv, tn = _c(tri.tri_v, np.int32), _c(tri.tri_nb, np.int32)
    return float(L.oracle_interior_length(tv.size // 3, _p(vx), _p(vy), _p(tv), _p(tn)))


def line_crossings(tri, cx, cy, p):
    """Interior edges crossed by each line {x : (cx, cy).x = p} (brute force)."""
    L = _load()
    vx, vy = _c(tri.vx, np.int32), _c(tri.vy, np.int32)
    tv, tn = _c(tri.tri_v, np.int32), _c(tri.tri_nb, np.int32)
    cx, cy, p = _c(cx, np.float64), _c(cy, np.float64), _c(p, np.float64)
    out = np.empty(cx.size, np.int32)
    L.oracle_count_line_crossings(tv.size // 3, _p(vx), _p(vy), _p(tv), _p(tn), cx.size, _p(cx), _p(cy), _p(p),
                                  _p(out))
    return out


def crofton_lines(n, seed, D):
    """Isotropic, translation-invariant random lines meeting the square [0,D]^2,
    i.e. uniform in the line measure dp dtheta restricted to lines that meet it:
    the normal angle has density proportional to the square's width in that
    direction (D(|cos| + |sin|), sampled by rejection) and the offset is
    uniform over the square's projection."""
    rng = np.random.default_rng(seed)
    th = np.empty(0)
    while th.size < n:
        c = rng.uniform(0.0, np.pi, 2 * n)
        keep = rng.uniform(0.0, np.sqrt(2.0), 2 * n) < np.abs(np.cos(c)) + np.abs(np.sin(c))
        th = np.concatenate([th, c[keep]])
    th = th[:n]
    cx, cy = np.cos(th), np.sin(th)
    proj = np.stack([np.zeros(n), cx * D, cy * D, (cx + cy) * D])
    lo, hi = proj.min(0), proj.max(0)
    p = lo + (hi - lo) * rng.uniform(0.0, 1.0, n)
    return cx, cy, p


def bvh_trace(b, ox, oy, dx, dy, n_threads=None, mutant=0):
    """BVH traversal of Sec. 5.3.1: (hit, t, ops (n,2): AABB tests, segment tests)."""
    L = _load(mutant)
    box, c0, c1, pr = (_c(x, np.int32) for x in (b.box, b.child0, b.child1, b.prims))
    segs = _c(b.segs, np.int32)
    ox, oy, dx, dy = _c(ox, np.int32), _c(oy, np.int32), _c(dx, np.float32), _c(dy, np.float32)
    n = ox.size
    hit, t, ops = np.empty(n, np.int32), np.empty(n, np.float32), np.empty((n, 2), np.int32)
    L.oracle_bvh_trace(c0.size, _p(box), _p(c0), _p(c1), _p(pr), _p(segs), n, _p(ox), _p(oy), _p(dx), _p(dy),
                       _p(hit), _p(t), _p(ops), _nthreads(n_threads))
    return hit, t, ops


def kd_trace(k, ox, oy, dx, dy, n_threads=None, mutant=0):
    """Roped kd-tree traversal of Sec. 5.3.2: (hit, t, ops (n,6)): leaves,
    descent nodes, segment tests, distinct segments, rope search steps of an
    ideal rope tree (the rope counts found from the node boxes, not read from
    the tree's own table), 0."""
    L = _load(mutant)
    arrs = [_c(x, np.int32) for x in (k.axis, k.split, k.child, k.count, k.box, k.rope, k.refs, k.segs)]
    ox, oy, dx, dy = _c(ox, np.int32), _c(oy, np.int32), _c(dx, np.float32), _c(dy, np.float32)
    n = ox.size
    hit, t, ops = np.empty(n, np.int32), np.empty(n, np.float32), np.empty((n, 6), np.int32)
    L.oracle_kd_trace(arrs[0].size, *[_p(a) for a in arrs], n, _p(ox), _p(oy), _p(dx), _p(dy), _p(hit), _p(t),
                      _p(ops), _nthreads(n_threads))
    return hit, t, ops
