"""Seeded inputs: scenes of disjoint segments on the 2^20 integer grid, their
constrained Delaunay triangulation, a flip annealer (the paper's polishing
step with edge flips, Sec. 3.2.7 and 3.3), and ray batches with start cells.

This module only produces inputs.  Both the CUDA path (``paper_2112_05570_gb300``)
and the CPU oracle (``oracle``) consume what it returns; it holds none of the
walk / closest-hit arithmetic of Sec. 5.1.

Domain: integer points of [0, D]^2 with D = 2^20; the square's four corners are
vertices and its boundary is the triangulation hull.  Triangles are CCW and
edge i is the edge opposite vertex i.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

D = 1 << 20
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenegen.cpp")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libscenegen.so")
_lib = None
_lock = threading.Lock()  # the first use may come from several threads at once


def build(force: bool = False) -> str:
    """Compile the generator library in-tree with g++ (host code, any arch)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}.{threading.get_ident()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    with _lock:
        if _lib is not None:
            return _lib
        return _bind()


def _bind():
    global _lib
    L = ctypes.CDLL(_LIB)
    i64, i32, u64, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
    P = ctypes.POINTER
    L.sg_gen_random_segments.restype = i64
    L.sg_gen_random_segments.argtypes = [i64, u64, i32, dbl, dbl, dbl, dbl, vp, i64]
    L.sg_gen_clustered.restype = i64
    L.sg_gen_clustered.argtypes = [i64, u64, i32, dbl, dbl, dbl, i32, dbl, vp, i64]
    L.sg_gen_lines.restype = i64
    L.sg_gen_lines.argtypes = [i64, u64, i32, dbl, i32, dbl, dbl, vp, i64]
    L.sg_gen_circles.restype = i64
    L.sg_gen_circles.argtypes = [i64, u64, i32, i32, i32, vp, i64]
    L.sg_gen_dash_grid.restype = i64
    L.sg_gen_dash_grid.argtypes = [i64, dbl, i32, vp, i64]
    L.sg_gen_ring_of_circles.restype = i64
    L.sg_gen_ring_of_circles.argtypes = [i64, i32, vp, i64]
    L.sg_cdt_build.restype = vp
    L.sg_cdt_build.argtypes = [i64, vp, i32, P(i32)]
    L.sg_tri_import.restype = vp
    L.sg_tri_import.argtypes = [i32, i64, vp, vp, i64, vp, vp, vp]
    L.sg_tri_copy.restype = vp
    L.sg_tri_copy.argtypes = [vp]
    L.sg_tri_free.restype = None
    L.sg_tri_free.argtypes = [vp]
    L.sg_tri_status.restype = i32
    L.sg_tri_status.argtypes = [vp]
    L.sg_tri_sizes.restype = None
    L.sg_tri_sizes.argtypes = [vp, P(i64), P(i64)]
    L.sg_tri_export.restype = None
    L.sg_tri_export.argtypes = [vp, vp, vp, vp, vp, vp]
    L.sg_tri_length.restype = ctypes.c_float
    L.sg_tri_length.argtypes = [vp, i32]
    L.sg_anneal.restype = i64
    L.sg_anneal.argtypes = [vp, u64, dbl, dbl, dbl, dbl, dbl]
    L.sg_rays_isotropic.restype = i64
    L.sg_rays_isotropic.argtypes = [vp, i64, u64, vp, vp, vp, vp, vp, i32]
    L.sg_rays_pinhole.restype = i64
    L.sg_rays_pinhole.argtypes = [vp, i64, i64, dbl, u64, vp, vp, vp, vp, vp, i32]
    L.sg_refine.restype = i64
    L.sg_refine.argtypes = [vp, dbl, dbl, i64]
    L.sg_subdivide.restype = i64
    L.sg_subdivide.argtypes = [vp]
    L.sg_anneal_fuzzy.restype = i64
    L.sg_anneal_fuzzy.argtypes = [vp, ctypes.c_uint64, dbl, dbl, dbl, dbl, dbl, dbl]
    L.sg_contract_short_edges.restype = i64
    L.sg_contract_short_edges.argtypes = [vp, dbl]
    L.sg_fuzzy_check_group_deltas.restype = i64
    L.sg_fuzzy_check_group_deltas.argtypes = [vp, ctypes.c_uint64, i64, dbl, i32, dbl, P(dbl), P(i64)]
    L.sg_fuzzy_objective.restype = None
    L.sg_fuzzy_objective.argtypes = [vp, dbl, dbl, dbl, dbl, dbl, ctypes.c_int32, vp, vp]
    L.sg_refine_optimal.restype = vp
    L.sg_refine_optimal.argtypes = [vp, vp, i32, vp, i32, i64, i32, P(dbl), P(dbl)]
    L.sg_bvh_build.restype = vp
    L.sg_bvh_build.argtypes = [i64, vp, ctypes.c_float]
    L.sg_bvh_sizes.restype = None
    L.sg_bvh_sizes.argtypes = [vp, P(i64), P(i64)]
    L.sg_bvh_export.restype = None
    L.sg_bvh_export.argtypes = [vp, vp, vp, vp, vp]
    L.sg_bvh_free.restype = None
    L.sg_bvh_free.argtypes = [vp]
    L.sg_kd_build.restype = vp
    L.sg_kd_build.argtypes = [i64, vp, i32, ctypes.c_float, i32]
    L.sg_kd_sizes.restype = None
    L.sg_kd_sizes.argtypes = [vp, P(i64), P(i64)]
    L.sg_kd_export.restype = None
    L.sg_kd_export.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.sg_kd_free.restype = None
    L.sg_kd_free.argtypes = [vp]
    _lib = L
    return L


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _threads() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


# ----------------------------------------------------------------------------- scenes
def length_scale(n: int) -> float:
    """Segment lengths shrink as sqrt(200/N) above 200 segments, as the paper's
    line scenes scale their length with 1/sqrt(N) (Sec. 4.2)."""
    return 1.0 if n <= 200 else float(np.sqrt(200.0 / n))


def random_segments(n: int, seed: int, len_lo=0.005, len_hi=0.03, margin=0.01, scale=None) -> np.ndarray:
    """n pairwise-disjoint random segments, lengths U[len_lo, len_hi] of the
    domain side (times ``length_scale(n)``), endpoints >= margin from the border."""
    L = _load()
    out = np.zeros((n, 4), np.int32)
    s = length_scale(n) if scale is None else scale
    m = L.sg_gen_random_segments(n, seed, D, len_lo, len_hi, s, margin, _ptr(out), n)
    return out[:m].copy()


def clustered(n: int, seed: int, n_clusters=32, sigma=0.02, len_lo=0.005, len_hi=0.03) -> np.ndarray:
    L = _load()
    out = np.zeros((n, 4), np.int32)
    m = L.sg_gen_clustered(n, seed, D, len_lo, len_hi, length_scale(n), n_clusters, sigma, _ptr(out), n)
    return out[:m].copy()


LINE_ORIENTATIONS = {"uniform": 0, "vertical": 1, "diagonal": 2}


def lines(n: int, seed: int, factor: float = 1.0, orientation: str = "uniform", spread_deg: float = 10.0,
          margin: float = 0.01) -> np.ndarray:
    """The paper's `lines' scenes (Sec. 4.2): up to n pairwise-disjoint segments
    of length min(0.95, factor * 0.95 / sqrt(n)) of the domain side; orientation
    uniform, mostly vertical or mostly diagonal (normal spread of spread_deg
    degrees).  Dense scenes (factor 3, large n) may hold fewer than n."""
    L = _load()
    out = np.zeros((max(1, n), 4), np.int32)
    m = L.sg_gen_lines(n, seed, D, float(factor), LINE_ORIENTATIONS[orientation], float(spread_deg), float(margin),
                       _ptr(out), n)
    return out[:m].copy()


def circles(n_target: int, seed: int, min_sides=64, max_sides=1024) -> np.ndarray:
    L = _load()
    cap = n_target + max_sides + 8
    out = np.zeros((cap, 4), np.int32)
    m = L.sg_gen_circles(n_target, seed, D, min_sides, max_sides, _ptr(out), cap)
    return out[:m].copy()


def dash_grid(n_target: int, theta_deg: float) -> np.ndarray:
    L = _load()
    cap = 2 * n_target + 1024
    out = np.zeros((cap, 4), np.int32)
    m = L.sg_gen_dash_grid(n_target, theta_deg, D, _ptr(out), cap)
    return out[:m].copy()


def ring_of_circles(n_target: int) -> np.ndarray:
    L = _load()
    cap = n_target + 4096
    out = np.zeros((cap, 4), np.int32)
    m = L.sg_gen_ring_of_circles(n_target, D, _ptr(out), cap)
    if m < 0:
        raise RuntimeError("ring_of_circles: polygon rounding failed")
    return out[:m].copy()


def room(n_obstacles: int, seed: int, wall_margin: float = 0.005) -> np.ndarray:
    """A closed square room (four wall segments sharing their corners,
    wall_margin of the domain side from the border) around n_obstacles random
    segments (``random_segments``, 1% from the border, so inside the walls):
    mirror paths inside it end only by grazing or at the bounce limit."""
    m = int(round(wall_margin * D))
    walls = np.array([[m, m, D - m, m], [D - m, m, D - m, D - m], [D - m, D - m, m, D - m], [m, D - m, m, m]],
                     np.int32)
    if n_obstacles <= 0:
        return walls
    return np.concatenate([walls, random_segments(n_obstacles, seed)]).astype(np.int32)


# ----------------------------------------------------------------------------- triangulations
@dataclass
class Triangulation:
    """A triangulation of [0,D]^2 whose constrained edges cover the segments.

    vx, vy: int32 vertex coordinates; tri_v: (T,3) CCW vertex ids; tri_nb: (T,3)
    neighbour across edge i (opposite vertex i) or -1 on the hull; tri_seg: (T,3)
    scene segment id of a constrained edge or -1."""

    vx: np.ndarray
    vy: np.ndarray
    tri_v: np.ndarray
    tri_nb: np.ndarray
    tri_seg: np.ndarray
    segs: np.ndarray
    kind: str = "cdt"
    _h: int = field(default=0, repr=False)

    @property
    def n_tri(self) -> int:
        return int(self.tri_v.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.vx.shape[0])

    def length(self, interior_only=False) -> float:
        return float(_load().sg_tri_length(self._h, 1 if interior_only else 0))

    def save(self, path: str, domain: int = None) -> None:
        """Writes the triangulation in the file layout that cct_scene_load_file
        reads: the 8 bytes "CCTTRI1" + NUL, int32 n_vert, n_tri, n_seg, domain,
        then vx, vy, tri_v, tri_nb, tri_seg as little-endian int32."""
        d = D if domain is None else int(domain)
        n_seg = int(np.asarray(self.segs).reshape(-1, 4).shape[0])
        hdr = np.array([self.n_vert, self.n_tri, n_seg, d], "<i4")
        with open(path, "wb") as f:
            f.write(b"CCTTRI1\0")
            f.write(hdr.tobytes())
            for a in (self.vx, self.vy, self.tri_v, self.tri_nb, self.tri_seg):
                f.write(np.ascontiguousarray(a, "<i4").tobytes())

    def __del__(self):
        if self._h and _lib is not None:
            _lib.sg_tri_free(self._h)
            self._h = 0


def _export(h: int, segs: np.ndarray, kind: str) -> Triangulation:
    L = _load()
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    L.sg_tri_sizes(h, ctypes.byref(nv), ctypes.byref(nt))
    vx = np.zeros(nv.value, np.int32)
    vy = np.zeros(nv.value, np.int32)
    tv = np.zeros((nt.value, 3), np.int32)
    tn = np.zeros((nt.value, 3), np.int32)
    ts = np.zeros((nt.value, 3), np.int32)
    L.sg_tri_export(h, _ptr(vx), _ptr(vy), _ptr(tv), _ptr(tn), _ptr(ts))
    return Triangulation(vx, vy, tv, tn, ts, segs, kind, h)


def cdt(segs: np.ndarray) -> Triangulation:
    """Constrained Delaunay triangulation of the segments inside [0,D]^2."""
    L = _load()
    segs = np.ascontiguousarray(segs, np.int32).reshape(-1, 4)
    st = ctypes.c_int32(0)
    h = L.sg_cdt_build(segs.shape[0], _ptr(segs), D, ctypes.byref(st))
    if st.value < 0:
        L.sg_tri_free(h)
        raise RuntimeError(f"CDT construction failed with status {st.value}")
    return _export(h, segs, "cdt")


def load(path: str, segs: np.ndarray) -> Triangulation:
    """A triangulation written by Triangulation.save (the layout cct_scene_load_file
    reads), with the scene segments it was built for; checks the header, the
    size and the domain."""
    raw = open(path, "rb").read()
    if raw[:8] != b"CCTTRI1\0" or len(raw) < 24:
        raise ValueError(f"{path}: not a triangulation file")
    nv, nt, ns, dom = (int(x) for x in np.frombuffer(raw[8:24], "<i4"))
    if len(raw) != 24 + 4 * (2 * nv + 9 * nt) or dom != D or ns != np.asarray(segs).reshape(-1, 4).shape[0]:
        raise ValueError(f"{path}: size, domain or segment count does not match")
    a = np.frombuffer(raw[24:], "<i4")
    vx, vy = a[:nv].copy(), a[nv:2 * nv].copy()
    tv = a[2 * nv:2 * nv + 3 * nt].reshape(nt, 3).copy()
    tn = a[2 * nv + 3 * nt:2 * nv + 6 * nt].reshape(nt, 3).copy()
    ts = a[2 * nv + 6 * nt:].reshape(nt, 3).copy()
    return from_arrays(vx, vy, tv, tn, ts, segs, kind="loaded")


def anneal_resumable(tri: Triangulation, seed: int, checkpoint: str, sweeps: float = 20.0, chunks: int = 8,
                     T0: float = 0.02, T1: float = 1e-4, moves: float = 1.0, collapse: float = 0.5,
                     stop_after: int = None) -> Triangulation:
    """``anneal`` in ``chunks`` pieces of the exponential schedule T0 -> T1
    (piece k: sweeps / chunks sweeps from T0 (T1/T0)^(k/chunks) to
    T0 (T1/T0)^((k+1)/chunks), seed + k), checkpointing after each piece: the
    triangulation file ``checkpoint`` (replaced atomically) and a sidecar
    ``checkpoint + ".json"`` with the pieces done and the parameters.  A call
    with the same parameters and an existing checkpoint resumes after its last
    piece, so an interrupted run ends with the result of an uninterrupted one.
    stop_after (testing): return after that many pieces of this call."""
    import json
    import os

    params = dict(seed=int(seed), sweeps=float(sweeps), chunks=int(chunks), T0=float(T0), T1=float(T1),
                  moves=float(moves), collapse=float(collapse), n_vert=tri.n_vert, n_tri=tri.n_tri)
    side = checkpoint + ".json"
    start, cur = 0, tri
    if os.path.exists(side) and os.path.exists(checkpoint):
        st = json.load(open(side))
        if st.get("params") == params:
            start, cur = int(st["done"]), load(checkpoint, tri.segs)
    ran = 0
    for k in range(start, chunks):
        if stop_after is not None and ran >= stop_after:
            return cur
        ta = T0 * (T1 / T0) ** (k / chunks)
        tb = T0 * (T1 / T0) ** ((k + 1) / chunks)
        cur = anneal(cur, seed + k, sweeps=sweeps / chunks, T0=ta, T1=tb, moves=moves, collapse=collapse)
        tmp = checkpoint + ".tmp"
        cur.save(tmp)
        os.replace(tmp, checkpoint)
        # go on from the file's state, as a resumed run does (the in-memory
        # vertex-to-triangle map of a fresh import decides fan orders)
        cur = load(checkpoint, tri.segs)
        with open(side + ".tmp", "w") as f:
            json.dump({"done": k + 1, "params": params}, f)
        os.replace(side + ".tmp", side)
        ran += 1
    return cur


def anneal(tri: Triangulation, seed: int, sweeps=20.0, T0=0.02, T1=1e-4, moves=1.0, collapse=0.5) -> Triangulation:
    """A copy of ``tri`` annealed: greedy flips to shorter diagonals, then
    simulated annealing with temperature T0 -> T1 (units of the domain side,
    as the paper's unit-square schedule, Sec. 3.3) over edge flips (Sec. 3.2.7)
    and, with weight ``moves`` (0: flips only), the vertex perturbation and
    resampling of Sec. 3.2.2 and 3.2.4 on Steiner vertices -- free ones on the
    lattice, those inside a segment along it -- of which a share ``collapse``
    instead merges the vertex into a neighbour (contraction, Sec. 3.2.6 /
    3.4.1, as a discrete edge collapse); then greedy flips again; the shorter
    of (greedy only, annealed) is kept."""
    L = _load()
    h = L.sg_tri_copy(tri._h)
    L.sg_anneal(h, seed, float(sweeps), float(T0) * D, float(T1) * D, float(moves), float(collapse))
    return _export(h, tri.segs, "annealed")


FUZZY_DELTA = 1.0 + float(np.cos(np.deg2rad(179.0)))  # Sec. 2.2.3: the angle penalty acts above 179 degrees


def fuzzy_objective(tri: Triangulation, eps: float, delta: float = FUZZY_DELTA, eps0: float = 1e-10,
                    mu_angle: float = 1.0, mu_len: float = 10.0, polish: bool = False, per_edge: bool = False):
    """The objective f of Sec. 2.2 in unit-square units: dict with f, w_contr
    (the edge-length sum with fuzzy contraction at length scale eps), angle and
    length (the two penalty sums), and with per_edge the weight w(e) of every
    edge as an (n_tri, 3) array (edge i of triangle t, opposite vertex i)."""
    L = _load()
    terms = np.zeros(4, np.float64)
    w = np.zeros((tri.n_tri, 3), np.float64) if per_edge else None
    L.sg_fuzzy_objective(tri._h, float(eps), float(delta), float(eps0), float(mu_angle), float(mu_len),
                         1 if polish else 0, _ptr(terms), _ptr(w) if per_edge else None)
    out = dict(f=float(terms[0]), w_contr=float(terms[1]), angle=float(terms[2]), length=float(terms[3]))
    if per_edge:
        out["w"] = w
    return out


def anneal_fuzzy(tri: Triangulation, seed: int, sweeps: float = 20.0, T0: float = 0.02, T1: float = 1e-4,
                 eps_a: float = 0.05, eps_b: float = 1e-4, moves: float = 1.0):
    """A copy of ``tri`` annealed on the fuzzy objective (Sec. 2.2, 3.3: T and
    the contraction length eps decrease exponentially together, unit-square
    units), then with every contractible edge shorter than eps_b contracted
    (Sec. 3.4).  Returns (triangulation, contractions)."""
    L = _load()
    h = L.sg_tri_copy(tri._h)
    n = L.sg_anneal_fuzzy(h, int(seed), float(sweeps), float(T0), float(T1), float(eps_a), float(eps_b),
                          float(moves))
    return _export(h, tri.segs, "fuzzy"), int(n)


def _optimise_and_contract(tri: Triangulation, seed: int, sweeps: float, polish_sweeps: float, eps_a: float,
                           eps_b: float, T0: float, T1: float, max_rounds: int) -> Triangulation:
    """Fuzzy annealing with the contraction of edges shorter than eps_b, then
    the contract-and-polish loop of Sec. 3.4 (polish without contraction and
    greedy flips; the contraction length doubled per round until the total
    length stops decreasing)."""
    cur, _ = anneal_fuzzy(tri, seed, sweeps, T0, T1, eps_a, eps_b)
    best = anneal(cur, seed + 1, sweeps=polish_sweeps, T0=T1 * 10, T1=T1, moves=1.0, collapse=0.0)
    eps = eps_b
    for k in range(1, max_rounds):
        eps *= 2.0
        nxt, n = anneal_fuzzy(best, seed + 1 + k, 0.0, T0, T1, eps, eps)  # contraction only
        if n == 0:
            continue
        nxt = anneal(nxt, seed + 1 + k, sweeps=polish_sweeps, T0=T1 * 10, T1=T1, moves=1.0, collapse=0.0)
        if nxt.length(True) >= best.length(True):
            break
        best = nxt
    return best


def fuzzy_check_group_deltas(tri: Triangulation, seed: int, n: int, eps: float, init_bits: int = 12,
                             step: float = 0.01):
    """Test hook: n multi-vertex perturbations (Sec. 3.2.2's second variant) of
    a copy of ``tri`` at contraction length eps and vertex-move step factor
    ``step``, the annealer's region tables starting at 2^init_bits slots;
    returns (proposals compared, largest |region energy change - whole fuzzy
    objective change|, table growths)."""
    L = _load()
    err, grows = ctypes.c_double(), ctypes.c_int64()
    n_cmp = L.sg_fuzzy_check_group_deltas(tri._h, int(seed), int(n), float(eps), int(init_bits), float(step),
                                          ctypes.byref(err), ctypes.byref(grows))
    return int(n_cmp), float(err.value), int(grows.value)


def fuzzy_pipeline(segs: np.ndarray, seed: int, sweeps: float = 20.0, polish_sweeps: float = 10.0,
                   eps_a: float = 0.05, eps_b: float = 1e-4, T0: float = 0.02, T1: float = 1e-4,
                   max_rounds: int = 6, subdivisions: int = 0):
    """The optimisation of Sec. 3 with fuzzy contraction (the full pipeline of
    Sec. 3.5.3): the optimally refined CDT through optimisation and
    contraction (_optimise_and_contract), then, ``subdivisions`` times, a 1 -> 4
    subdivision of the result through the same process again, keeping the
    shortest triangulation.  Returns (refined CDT, result)."""
    r = refine_optimal(cdt(segs))
    args = (sweeps, polish_sweeps, eps_a, eps_b, T0, T1, max_rounds)
    best = _optimise_and_contract(r, seed, *args)
    for k in range(subdivisions):
        nxt = _optimise_and_contract(subdivide(best), seed + 100 * (k + 1), *args)
        if nxt.length(True) < best.length(True):
            best = nxt
    return r, best


def subdivide(tri: Triangulation) -> Triangulation:
    """A copy of ``tri`` with the lattice midpoint of every interior edge
    inserted (the 1 -> 4 subdivision of Sec. 3.5.2 on the lattice; constrained
    edges split along their segment), made constrained-Delaunay again."""
    L = _load()
    h = L.sg_tri_copy(tri._h)
    if L.sg_subdivide(h) < 0:
        L.sg_tri_free(h)
        raise RuntimeError("subdivision failed")
    return _export(h, tri.segs, "subdivided")


def refine(tri: Triangulation, min_angle_deg: float = 20.0, max_area: float = 0.0,
           max_insert: int | None = None) -> Triangulation:
    """A quality-refined copy of ``tri`` (Delaunay refinement on the integer
    grid: circumcentres of triangles with a smaller angle or a larger area,
    lattice midpoints of encroached constrained edges); max_area in grid units."""
    L = _load()
    h = L.sg_tri_copy(tri._h)
    cap = 4 * tri.n_vert + 1024 if max_insert is None else int(max_insert)
    if L.sg_refine(h, float(min_angle_deg), float(max_area), cap) < 0:
        L.sg_tri_free(h)
        raise RuntimeError("refinement failed")
    return _export(h, tri.segs, "refined")


OPT_ANGLES = (5.0, 10.0, 15.0, 20.0, 25.0)
OPT_AREA_FRACTIONS = (0.0, 4.0, 1.0, 0.25)  # max area = f * D^2 / n_segments (0 = no bound)


def refine_optimal(tri: Triangulation, angles=OPT_ANGLES, area_fractions=OPT_AREA_FRACTIONS,
                   max_insert: int | None = None, threads: int | None = None) -> Triangulation:
    """The optimally refined CDT (Sec. 3.5.1): of all (min angle, max area)
    refinements of the grid (and the unrefined CDT), the one with the shortest
    total edge length.  Sets .refine_params = (angle, max_area)."""
    L = _load()
    n_seg = max(1, int(np.asarray(tri.segs).reshape(-1, 4).shape[0]))
    ang = np.ascontiguousarray(angles, np.float64)
    areas = np.ascontiguousarray([0.0 if f == 0 else f * float(D) * D / n_seg for f in area_fractions], np.float64)
    cap = 4 * tri.n_vert + 1024 if max_insert is None else int(max_insert)
    ba, bA = ctypes.c_double(), ctypes.c_double()
    h = L.sg_refine_optimal(tri._h, _ptr(ang), ang.size, _ptr(areas), areas.size, cap, threads or _threads(),
                            ctypes.byref(ba), ctypes.byref(bA))
    out = _export(h, tri.segs, "refined")
    out.refine_params = (float(ba.value), float(bA.value))
    return out


def pipeline(segs: np.ndarray, seed: int, sweeps: float = 4.0, subdivisions: int = 1):
    """The offline build of the paper's triangulations: (unrefined CDT, optimally
    refined CDT (Sec. 3.5.1), annealed).  Annealed = the refined CDT optimised
    (greedy and simulated-annealing flips, Sec. 3.2.7, 3.3; vertex moves and
    contraction as discrete collapses), then, ``subdivisions`` times, the 1 -> 4
    subdivision of the result optimised again (the full pipeline of Sec. 3.5.3),
    keeping the shortest; its .route says which round won."""
    c = cdt(segs)
    r = refine_optimal(c)
    best = anneal(r, seed, sweeps=sweeps)
    best.route = "annealed"
    for k in range(subdivisions):
        nxt = anneal(subdivide(best), seed + 100 * (k + 1), sweeps=sweeps)
        if nxt.length(True) < best.length(True):
            best = nxt
            best.route = f"annealed after {k + 1} subdivision(s)"
    return c, r, best


def from_arrays(vx, vy, tri_v, tri_nb, tri_seg, segs, kind="given") -> Triangulation:
    """Wrap caller-made arrays (e.g. hand-written test triangulations)."""
    L = _load()
    vx = np.ascontiguousarray(vx, np.int32)
    vy = np.ascontiguousarray(vy, np.int32)
    tv = np.ascontiguousarray(tri_v, np.int32).reshape(-1, 3)
    tn = np.ascontiguousarray(tri_nb, np.int32).reshape(-1, 3)
    ts = np.ascontiguousarray(tri_seg, np.int32).reshape(-1, 3)
    h = L.sg_tri_import(D, vx.size, _ptr(vx), _ptr(vy), tv.shape[0], _ptr(tv), _ptr(tn), _ptr(ts))
    return Triangulation(vx, vy, tv, tn, ts, np.ascontiguousarray(segs, np.int32).reshape(-1, 4), kind, h)


# ----------------------------------------------------------------------------- rays
@dataclass
class Rays:
    """Ray batch: int32 origins, fp32 directions on the 2^-22 grid, and the
    triangle (export numbering) whose interior holds each origin."""

    ox: np.ndarray
    oy: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    start: np.ndarray

    def __len__(self):
        return int(self.ox.shape[0])

    def take(self, idx) -> "Rays":
        return Rays(self.ox[idx], self.oy[idx], self.dx[idx], self.dy[idx], self.start[idx])


def _alloc_rays(n):
    return Rays(np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.float32),
                np.zeros(n, np.float32), np.zeros(n, np.int32))


def rays_isotropic(tri: Triangulation, n: int, seed: int, threads: int | None = None) -> Rays:
    """Uniform, isotropic rays inside the domain (Sec. 5.4)."""
    L = _load()
    r = _alloc_rays(n)
    L.sg_rays_isotropic(tri._h, n, seed, _ptr(r.ox), _ptr(r.oy), _ptr(r.dx), _ptr(r.dy), _ptr(r.start),
                        threads or _threads())
    return r


def rays_pinhole(tri: Triangulation, n_eyes: int, rays_per_eye: int, seed: int, fov_deg=90.0,
                 threads: int | None = None) -> Rays:
    """Coherent pinhole fans: n_eyes eyes, rays_per_eye rays over fov_deg each."""
    L = _load()
    r = _alloc_rays(n_eyes * rays_per_eye)
    L.sg_rays_pinhole(tri._h, n_eyes, rays_per_eye, fov_deg, seed, _ptr(r.ox), _ptr(r.oy), _ptr(r.dx),
                      _ptr(r.dy), _ptr(r.start), threads or _threads())
    return r


# ----------------------------------------------------------------------------- baselines (Sec. 5.3)
@dataclass
class Bvh:
    """SAH BVH over segments: box (N,4) closed integer boxes; child0 >= 0 is an
    inner node's left child, child0 < 0 a leaf whose first primitive is
    -child0-1; child1 = right child or primitive count; prims = segment ids."""

    box: np.ndarray
    child0: np.ndarray
    child1: np.ndarray
    prims: np.ndarray
    segs: np.ndarray
    alpha: float

    @property
    def n_nodes(self):
        return int(self.child0.size)


def bvh(segs: np.ndarray, alpha: float = 1.0) -> Bvh:
    """Greedy top-down 2D SAH BVH (Sec. 5.3.1); alpha = AABB-test cost relative
    to a segment test (the per-scene tuned parameter)."""
    L = _load()
    segs = np.ascontiguousarray(segs, np.int32).reshape(-1, 4)
    h = L.sg_bvh_build(segs.shape[0], _ptr(segs), float(alpha))
    nn, npr = ctypes.c_int64(), ctypes.c_int64()
    L.sg_bvh_sizes(h, ctypes.byref(nn), ctypes.byref(npr))
    box = np.zeros((nn.value, 4), np.int32)
    c0 = np.zeros(nn.value, np.int32)
    c1 = np.zeros(nn.value, np.int32)
    pr = np.zeros(max(1, npr.value), np.int32)
    L.sg_bvh_export(h, _ptr(box), _ptr(c0), _ptr(c1), _ptr(pr))
    L.sg_bvh_free(h)
    return Bvh(box, c0, c1, pr[:npr.value].copy(), segs, float(alpha))


@dataclass
class KdTree:
    """Roped SAH kd-tree over segments in [0,D]^2: axis 0/1 split on x/y, 2 leaf;
    split coordinate; child = left child (right = left + 1) or first reference;
    count = references in a leaf; box (N,4); rope (N,4) node across faces
    x-min, x-max, y-min, y-max (-1 none); rope_log2 (N,4) = ceil(log2 of the
    leaves adjacent across that face); refs = segment ids."""

    axis: np.ndarray
    split: np.ndarray
    child: np.ndarray
    count: np.ndarray
    box: np.ndarray
    rope: np.ndarray
    rope_log2: np.ndarray
    refs: np.ndarray
    segs: np.ndarray
    lam: float

    @property
    def n_nodes(self):
        return int(self.axis.size)


def kdtree(segs: np.ndarray, lam: float = 1.0, max_depth: int = 40) -> KdTree:
    """Greedy top-down 2D SAH kd-tree with split candidates at every segment
    endpoint coordinate and ropes on leaf faces (Sec. 5.3.2); lam = traversal
    cost relative to a segment test (the per-scene tuned parameter)."""
    L = _load()
    segs = np.ascontiguousarray(segs, np.int32).reshape(-1, 4)
    h = L.sg_kd_build(segs.shape[0], _ptr(segs), D, float(lam), int(max_depth))
    nn, nr = ctypes.c_int64(), ctypes.c_int64()
    L.sg_kd_sizes(h, ctypes.byref(nn), ctypes.byref(nr))
    n = nn.value
    axis, split, child, count = (np.zeros(n, np.int32) for _ in range(4))
    box, rope, rl = np.zeros((n, 4), np.int32), np.zeros((n, 4), np.int32), np.zeros((n, 4), np.int32)
    refs = np.zeros(max(1, nr.value), np.int32)
    L.sg_kd_export(h, _ptr(axis), _ptr(split), _ptr(child), _ptr(count), _ptr(box), _ptr(rope), _ptr(rl),
                   _ptr(refs))
    L.sg_kd_free(h)
    return KdTree(axis, split, child, count, box, rope, rl, refs[:nr.value].copy(), segs, float(lam))
