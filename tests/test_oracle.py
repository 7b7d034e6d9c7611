"""Pins for the CPU oracle (no GPU): the oracle is checked against things other
than itself -- hand-derived worked cases, brute force vs walk vs brute-force
step counts, triangulation invariants with planted corruptions, the
Cauchy-Crofton identity (arXiv 2112.05570 Sec. 1.4), and planted mutations of
the oracle that these pins must catch.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_cases.json")
K = 1 << 22


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _scene_tri(segs):
    segs = np.asarray(segs, np.int32).reshape(-1, 4)
    return sg.cdt(segs)


def _exact_t(t):
    return np.float32(float(Fraction(t[0], t[1])))


def _golden_rays(cases):
    ox = np.array([c["o"][0] for c in cases], np.int32)
    oy = np.array([c["o"][1] for c in cases], np.int32)
    dx = np.array([c["k"][0] / K for c in cases], np.float32)
    dy = np.array([c["k"][1] / K for c in cases], np.float32)
    return ox, oy, dx, dy


def _check_golden(mutant=0):
    """Returns the list of mismatches of the oracle (or a mutant) on the golden cases."""
    g = _golden()
    bad = []
    for name, scene in g["scenes"].items():
        cases = [c for c in g["cases"] if c["scene"] == name]
        segs = np.asarray(scene["segs"], np.int32).reshape(-1, 4)
        tri = _scene_tri(segs)
        ox, oy, dx, dy = _golden_rays(cases)
        start = oracle.locate_bruteforce(tri, ox, oy)
        assert (start >= 0).all(), f"golden origin not strictly inside a triangle in {name}"
        hb, tb = oracle.closest_bruteforce(segs, ox, oy, dx, dy, mutant=mutant)
        hw, tw, sw = oracle.walk(tri, ox, oy, dx, dy, start, mutant=mutant)
        for i, c in enumerate(cases):
            exp_t = np.float32(np.inf) if c["t"] is None else _exact_t(c["t"])
            for tag, h, t in (("bruteforce", hb[i], tb[i]), ("walk", hw[i], tw[i])):
                if h != c["hit"]:
                    bad.append((name, i, tag, "hit", int(h), c["hit"]))
                elif not (t == exp_t or abs(float(t) - float(exp_t)) <= 2e-7 * abs(float(exp_t))):
                    bad.append((name, i, tag, "t", float(t), float(exp_t)))
            if "steps" in c and sw[i] != c["steps"]:
                bad.append((name, i, "walk", "steps", int(sw[i]), c["steps"]))
    return bad


def test_golden_worked_cases():
    assert _check_golden() == []


def _degenerate_rays(tri, n, seed):
    """Rays aimed exactly at vertices, rays collinear with triangulation edges,
    and axis-aligned rays: the degenerate cases of the side rule."""
    rng = np.random.default_rng(seed)
    vx, vy = tri.vx.astype(np.int64), tri.vy.astype(np.int64)
    ox, oy, kx, ky = [], [], [], []
    # aimed at a vertex
    for _ in range(n):
        v = rng.integers(0, vx.size)
        o = rng.integers(1, sg.D, 2)
        ux, uy = vx[v] - o[0], vy[v] - o[1]
        if ux == 0 and uy == 0:
            continue
        m = K // max(abs(ux), abs(uy))
        ox.append(o[0]); oy.append(o[1]); kx.append(ux * m); ky.append(uy * m)
    # along the line of an edge, starting beyond one of its endpoints
    tv = tri.tri_v
    for _ in range(n):
        t = rng.integers(0, tv.shape[0]); i = rng.integers(0, 3)
        a, b = tv[t, (i + 1) % 3], tv[t, (i + 2) % 3]
        ex, ey = vx[b] - vx[a], vy[b] - vy[a]
        g = np.gcd(abs(ex), abs(ey))
        ux, uy = ex // g, ey // g
        j = rng.integers(1, 50)
        o = (vx[a] - j * ux, vy[a] - j * uy)
        if not (0 < o[0] < sg.D and 0 < o[1] < sg.D):
            continue
        m = K // max(abs(ux), abs(uy))
        ox.append(o[0]); oy.append(o[1]); kx.append(ux * m); ky.append(uy * m)
    # axis-aligned
    for _ in range(n):
        o = rng.integers(1, sg.D, 2)
        d = [(K, 0), (-K, 0), (0, K), (0, -K)][rng.integers(0, 4)]
        ox.append(o[0]); oy.append(o[1]); kx.append(d[0]); ky.append(d[1])
    ox, oy = np.array(ox, np.int32), np.array(oy, np.int32)
    dx, dy = (np.array(kx, np.float64) / K).astype(np.float32), (np.array(ky, np.float64) / K).astype(np.float32)
    start = oracle.locate_bruteforce(tri, ox, oy)
    keep = start >= 0
    return ox[keep], oy[keep], dx[keep], dy[keep], start[keep]


def _random_checks(tri, segs, n_rays, seed, mutant=0):
    """Mismatch counts: (hit, t, steps) brute force vs walk vs brute-force steps."""
    r = sg.rays_isotropic(tri, n_rays, seed)
    dox, doy, ddx, ddy, dst = _degenerate_rays(tri, 300, seed + 1)
    ox = np.concatenate([r.ox, dox]); oy = np.concatenate([r.oy, doy])
    dx = np.concatenate([r.dx, ddx]); dy = np.concatenate([r.dy, ddy])
    st = np.concatenate([r.start, dst])
    hb, tb = oracle.closest_bruteforce(segs, ox, oy, dx, dy, mutant=mutant)
    hw, tw, sw = oracle.walk(tri, ox, oy, dx, dy, st, mutant=mutant)
    sb = oracle.steps_bruteforce(tri, ox, oy, dx, dy, hb, mutant=mutant)
    return int((hb != hw).sum()), int((~((tb == tw) | (np.isnan(tb) & np.isnan(tw)))).sum()), \
        int((sw != sb).sum()), int(len(ox))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bruteforce_walk_steps_agree(seed):
    segs = sg.random_segments(200, seed)
    assert segs.shape[0] == 200
    cdt = sg.cdt(segs)
    for tri in (cdt, sg.anneal(cdt, seed)):
        dh, dt, ds, n = _random_checks(tri, segs, 1 << 14, 100 + seed)
        assert n > (1 << 14)
        assert (dh, dt, ds) == (0, 0, 0)


def test_convex_polygon_from_inside_always_hits():
    """Special case: rays from inside one convex polygon all hit it (Sec. 5.1)."""
    segs = sg.circles(200, 5, min_sides=200, max_sides=200)
    assert segs.shape[0] == 200
    tri = sg.cdt(segs)
    xs = segs[:, 0].astype(np.int64); ys = segs[:, 1].astype(np.int64)
    cx, cy = int(xs.mean()), int(ys.mean())
    rng = np.random.default_rng(0)
    r = (xs.max() - xs.min()) // 5
    ox = (cx + rng.integers(-r, r, 4000)).astype(np.int32)
    oy = (cy + rng.integers(-r, r, 4000)).astype(np.int32)
    th = rng.uniform(0, 2 * np.pi, ox.size)
    dx = (np.rint(np.cos(th) * K) / K).astype(np.float32)
    dy = (np.rint(np.sin(th) * K) / K).astype(np.float32)
    st = oracle.locate_bruteforce(tri, ox, oy)
    k = st >= 0
    h, t, s = oracle.walk(tri, ox[k], oy[k], dx[k], dy[k], st[k])
    assert (h >= 0).all() and (h < 200).all()
    hb, _ = oracle.closest_bruteforce(segs, ox[k], oy[k], dx[k], dy[k])
    assert np.array_equal(h, hb)


def test_empty_scene_all_miss_two_triangles():
    D = sg.D
    tri = sg.cdt(np.zeros((0, 4), np.int32))
    assert tri.n_tri == 2
    r = sg.rays_isotropic(tri, 5000, 9)
    h, t, s = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    assert (h == -1).all() and np.isinf(t).all()
    assert ((s == 1) | (s == 2)).all()
    # closed form: steps == 2 exactly when the ray crosses the diagonal y = x ahead
    ox, oy = r.ox.astype(np.float64), r.oy.astype(np.float64)
    dx, dy = r.dx.astype(np.float64), r.dy.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        tc = (oy - ox) / (dx - dy)
    cross = (tc > 0) & (ox + tc * dx > 0) & (ox + tc * dx < D)
    assert np.array_equal(s == 2, cross)
    assert D == 1 << 20


def test_locate_bruteforce_matches_generator_and_rejects_edges():
    segs = sg.random_segments(200, 4)
    tri = sg.cdt(segs)
    r = sg.rays_isotropic(tri, 3000, 5)
    assert np.array_equal(oracle.locate_bruteforce(tri, r.ox, r.oy), r.start)
    # integer midpoints of edges lie on an edge -> -1; vertices -> -1
    tv = tri.tri_v
    a, b = tv[:, 1], tv[:, 2]
    mx, my = tri.vx[a].astype(np.int64) + tri.vx[b], tri.vy[a].astype(np.int64) + tri.vy[b]
    even = (mx % 2 == 0) & (my % 2 == 0)
    px, py = (mx[even] // 2).astype(np.int32), (my[even] // 2).astype(np.int32)
    assert px.size > 10
    assert (oracle.locate_bruteforce(tri, px, py) == -1).all()
    assert (oracle.locate_bruteforce(tri, tri.vx, tri.vy) == -1).all()


def _copy(tri, **kw):
    d = dict(vx=tri.vx.copy(), vy=tri.vy.copy(), tri_v=tri.tri_v.copy(), tri_nb=tri.tri_nb.copy(),
             tri_seg=tri.tri_seg.copy(), segs=tri.segs.copy())
    d.update(kw)
    return type("T", (), d)


def test_invariants_hold_and_corruptions_are_caught():
    D = sg.D
    segs = sg.random_segments(200, 6)
    cdt = sg.cdt(segs)
    ann = sg.anneal(cdt, 6)
    assert oracle.check_triangulation(cdt, D, check_delaunay=True) == 0
    assert oracle.check_triangulation(ann, D, check_delaunay=False) == 0
    # the annealer moved away from Delaunay and shortened the triangulation
    assert oracle.check_triangulation(ann, D, check_delaunay=True) == oracle.NOT_DELAUNAY
    assert oracle.interior_length(ann) < oracle.interior_length(cdt)
    # Euler: T = 2V - h - 2 with h = 4 corners (no other vertex on the hull)
    assert cdt.n_tri == 2 * cdt.n_vert - 4 - 2
    # planted corruptions
    t = cdt
    tv = t.tri_v.copy(); tv[5] = tv[5][[0, 2, 1]]
    assert oracle.check_triangulation(_copy(t, tri_v=tv), D) & oracle.NOT_CCW
    tn = t.tri_nb.copy(); j = np.argwhere(tn[7] >= 0)[0, 0]; tn[7, j] = (tn[7, j] + 1) % t.n_tri
    assert oracle.check_triangulation(_copy(t, tri_nb=tn), D) & oracle.NB_ASYM
    ts = t.tri_seg.copy(); tt, ti = np.argwhere(ts >= 0)[0]
    u = t.tri_nb[tt, ti]; uj = np.argwhere(t.tri_nb[u] == tt)[0, 0]
    ts[tt, ti] = -1; ts[u, uj] = -1
    assert oracle.check_triangulation(_copy(t, tri_seg=ts), D) & oracle.COVERAGE
    ts = t.tri_seg.copy(); ts[tt, ti] = -1
    assert oracle.check_triangulation(_copy(t, tri_seg=ts), D) & oracle.CONSTRAINT_ASYM
    ts = t.tri_seg.copy(); tt2, ti2 = np.argwhere((ts < 0) & (t.tri_nb >= 0))[0]
    u2 = t.tri_nb[tt2, ti2]; uj2 = np.argwhere(t.tri_nb[u2] == tt2)[0, 0]
    ts[tt2, ti2] = 0; ts[u2, uj2] = 0
    assert oracle.check_triangulation(_copy(t, tri_seg=ts), D) & oracle.COVERAGE
    vx = t.vx.copy(); vx[10] += 1  # moving one vertex breaks area and CCW/coverage/Delaunay somewhere
    assert oracle.check_triangulation(_copy(t, vx=vx), D, check_delaunay=True) != 0
    # a triangulation of a different domain size fails the area check
    assert oracle.check_triangulation(t, D // 2) & oracle.AREA


def _line_crossing_test(tri, n, seed):
    cx, cy, p = oracle.crofton_lines(n, seed, sg.D)
    c = oracle.line_crossings(tri, cx, cy, p).astype(np.float64)
    L = oracle.interior_length(tri)
    pred = L / (2.0 * sg.D)  # 2 L / perimeter, perimeter = 4 D
    return c, pred


def test_crofton_line_crossings():
    """Cauchy-Crofton: isotropic translation-invariant lines meeting a convex K
    cross curves of total length L on average 2 L / Per(K) times (Sec. 1.4)."""
    segs = sg.random_segments(200, 11)
    cdt = sg.cdt(segs)
    ann = sg.anneal(cdt, 11)
    n = 40000
    c1, p1 = _line_crossing_test(cdt, n, 21)
    c2, p2 = _line_crossing_test(ann, n, 21)
    for c, p in ((c1, p1), (c2, p2)):
        assert abs(c.mean() - p) <= 5.0 * c.std() / np.sqrt(n)
    # the shorter triangulation is crossed less often, paired on the same lines
    diff = c1 - c2
    assert p2 < p1 and diff.mean() > 5.0 * diff.std() / np.sqrt(n)
    assert abs(diff.mean() - (p1 - p2)) <= 5.0 * diff.std() / np.sqrt(n)


def test_crofton_through_walk():
    """The walk crossing constrained edges (until the hull) along a chord of a
    random line visits 1 + crossings triangles each way: per ray it matches the
    brute-force count, and the chord total matches 2 L / Per(K) on average."""
    D = sg.D
    segs = sg.random_segments(200, 12)
    tri = sg.anneal(sg.cdt(segs), 12)
    n = 6000
    cx, cy, p = oracle.crofton_lines(n, 31, D)
    rng = np.random.default_rng(32)
    # chord endpoints of each line inside the square, then a uniform point on it
    pts = []
    for i in range(n):
        ends = []
        for side in range(4):
            if side < 2:  # x = 0 or D
                x = 0.0 if side == 0 else float(D)
                if abs(cy[i]) < 1e-12:
                    continue
                y = (p[i] - cx[i] * x) / cy[i]
                if 0 <= y <= D:
                    ends.append((x, y))
            else:
                y = 0.0 if side == 2 else float(D)
                if abs(cx[i]) < 1e-12:
                    continue
                x = (p[i] - cy[i] * y) / cx[i]
                if 0 <= x <= D:
                    ends.append((x, y))
        (x0, y0), (x1, y1) = ends[0], ends[-1]
        u = rng.uniform()
        pts.append((x0 + u * (x1 - x0), y0 + u * (y1 - y0)))
    pts = np.array(pts)
    ox = np.clip(np.rint(pts[:, 0]), 1, D - 1).astype(np.int32)
    oy = np.clip(np.rint(pts[:, 1]), 1, D - 1).astype(np.int32)
    dx = (np.rint(-cy * K) / K).astype(np.float32)
    dy = (np.rint(cx * K) / K).astype(np.float32)
    st = oracle.locate_bruteforce(tri, ox, oy)
    k = st >= 0
    ox, oy, dx, dy, st = ox[k], oy[k], dx[k], dy[k], st[k]
    miss = np.full(ox.size, -1, np.int32)
    _, _, sf = oracle.walk(tri, ox, oy, dx, dy, st, through=True)
    _, _, sb = oracle.walk(tri, ox, oy, -dx, -dy, st, through=True)
    assert np.array_equal(sf, oracle.steps_bruteforce(tri, ox, oy, dx, dy, miss))
    assert np.array_equal(sb, oracle.steps_bruteforce(tri, ox, oy, -dx, -dy, miss))
    crossings = (sf - 1) + (sb - 1)
    pred = oracle.interior_length(tri) / (2.0 * D)
    # rounding the origin to the grid moves each line by <= 0.71 units: the bias
    # is at most (vertex degree sum) * 1.42 / D per unit of chord, far below the
    # statistical tolerance below.
    sd = crossings.std() / np.sqrt(crossings.size)
    assert abs(crossings.mean() - pred) <= 5.0 * sd + 0.05


@pytest.mark.parametrize("mutant", oracle.PRIMARY_MUTANTS)
def test_planted_mutations_are_caught(mutant):
    """Each planted mistake in the oracle (wrong sign, on-line side flipped,
    hits behind the origin accepted, entry edge taken for the exit) makes at
    least one pin fail."""
    bad_golden = _check_golden(mutant=mutant)
    segs = sg.random_segments(200, 3)
    tri = sg.cdt(segs)
    dh, dt, ds, _ = _random_checks(tri, segs, 4000, 77, mutant=mutant)
    assert bad_golden or dh or dt or ds


def test_generators_deterministic_and_disjoint():
    a = sg.random_segments(200, 42)
    b = sg.random_segments(200, 42)
    assert np.array_equal(a, b)
    # pairwise disjoint (exact, brute force)
    P = a[:, :2].astype(np.int64); Q = a[:, 2:].astype(np.int64)

    def orient(p, q, r):
        return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])

    n = a.shape[0]
    i, j = np.triu_indices(n, 1)
    o1 = np.sign(orient(P[i], Q[i], P[j])); o2 = np.sign(orient(P[i], Q[i], Q[j]))
    o3 = np.sign(orient(P[j], Q[j], P[i])); o4 = np.sign(orient(P[j], Q[j], Q[i]))
    proper = (o1 * o2 < 0) & (o3 * o4 < 0)
    assert not proper.any()
    assert not ((o1 == 0) & (o2 == 0)).any()
    lens = np.hypot(*(Q - P).T) / sg.D
    assert lens.min() >= 0.005 - 1e-6 and lens.max() <= 0.03 + 1e-6
    r1 = sg.rays_isotropic(sg.cdt(a), 1000, 3, threads=1)
    r2 = sg.rays_isotropic(sg.cdt(a), 1000, 3, threads=4)
    assert np.array_equal(r1.ox, r2.ox) and np.array_equal(r1.dx, r2.dx) and np.array_equal(r1.start, r2.start)
    k = r1.dx.astype(np.float64) * K
    assert np.array_equal(k, np.rint(k))


@pytest.mark.parametrize("gen", ["circles", "dash0", "dash45", "clustered", "ring"])
def test_scene_families_triangulate(gen):
    if gen == "circles":
        segs = sg.circles(3000, 1)
    elif gen == "dash0":
        segs = sg.dash_grid(3000, 0.0)
    elif gen == "dash45":
        segs = sg.dash_grid(3000, 45.0)
    elif gen == "clustered":
        segs = sg.clustered(3000, 1)
    else:
        segs = sg.ring_of_circles(3000)
    assert segs.shape[0] >= 2500
    tri = sg.cdt(segs)
    assert oracle.check_triangulation(tri, sg.D, check_delaunay=True) == 0
    ann = sg.anneal(tri, 1, sweeps=2)
    assert oracle.check_triangulation(ann, sg.D) == 0
    assert oracle.interior_length(ann) <= oracle.interior_length(tri) * (1 + 1e-9)
    r = sg.rays_isotropic(ann, 2000, 2)
    hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
    hw, tw, sw = oracle.walk(ann, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)


@pytest.mark.parametrize("gen", ["config1", "circles"])
def test_refined_cdt_is_valid_and_optimal(gen):
    """The optimally refined CDT (Sec. 3.5.1): still a valid constrained
    Delaunay triangulation covering every segment (constrained edges may be
    split at lattice midpoints), never longer than the unrefined CDT (which
    competes in the search), and the walk on it equals the brute force."""
    segs = sg.random_segments(200, 13) if gen == "config1" else sg.circles(3000, 13)
    cdt = sg.cdt(segs)
    ref = sg.refine_optimal(cdt)
    assert oracle.check_triangulation(ref, sg.D, check_delaunay=True) == 0
    assert oracle.interior_length(ref) <= oracle.interior_length(cdt) * (1 + 1e-6)
    for tri in (ref, sg.refine(cdt, 25.0), sg.anneal(ref, 13, sweeps=2)):
        assert oracle.check_triangulation(tri, sg.D) == 0
        r = sg.rays_isotropic(tri, 5000, 14)
        hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
        hw, tw, sw = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
        assert np.array_equal(hb, hw) and np.array_equal(tb, tw)
        assert np.array_equal(sw[:500], oracle.steps_bruteforce(tri, r.ox[:500], r.oy[:500], r.dx[:500],
                                                                 r.dy[:500], hb[:500]))
    if gen == "circles":
        # polygon interiors: refinement shortens the triangulation markedly
        assert oracle.interior_length(ref) < 0.5 * oracle.interior_length(cdt)


def test_lattice_fixture_valid_and_walk_matches_bruteforce(lattice):
    """The hand-made lattice triangulation (many collinear lattice points)
    passes every invariant, and on it the oracle walk from brute-force-located
    start triangles equals the all-segment closest-hit scan."""
    tri = lattice()
    assert oracle.check_triangulation(tri, tri.D) == 0
    g = np.arange(-1, tri.D + 2, dtype=np.int32)
    px, py = [a.ravel() for a in np.meshgrid(g, g)]
    start = oracle.locate_bruteforce(tri, px, py)
    ok = start >= 0
    # per square of side 4: 3 x 3 interior lattice points, 3 of them on the diagonal
    assert ok.sum() == 12 * 12 * 6
    rng = np.random.default_rng(3)
    ang = rng.uniform(0, 2 * np.pi, px.size)
    dx = (np.round(np.cos(ang) * K) / K).astype(np.float32)
    dy = (np.round(np.sin(ang) * K) / K).astype(np.float32)
    h, t, s = oracle.walk(tri, px, py, dx, dy, start)
    hb, tb = oracle.closest_bruteforce(tri.segs, px[ok], py[ok], dx[ok], dy[ok])
    assert np.array_equal(h[ok], hb)
    assert (s[~ok] == -1).all() and (s[ok] >= 1).all()


def test_vertex_moves_keep_the_scene_and_shorten():
    """Annealing with vertex perturbations (free Steiner vertices on the
    lattice, Steiner vertices inside a segment along it): the result is a valid
    triangulation of the same segments (every segment still covered by
    constrained edges, no other edge constrained), the segment endpoints and
    the hull stay where they were, it is no longer than flips alone on a scene
    with Steiner vertices, and the walk on it equals the brute force."""
    segs = sg.circles(3000, 21)
    ref = sg.refine_optimal(sg.cdt(segs))
    flips = sg.anneal(ref, 21, sweeps=4, moves=0.0)
    moved = sg.anneal(ref, 21, sweeps=4, moves=1.0)
    assert oracle.check_triangulation(moved, sg.D) == 0
    assert oracle.interior_length(moved) < oracle.interior_length(flips)
    # segment endpoints and hull corners are among the vertices, unmoved
    pts = set(zip(moved.vx.tolist(), moved.vy.tolist()))
    for x0, y0, x1, y1 in segs.tolist():
        assert (x0, y0) in pts and (x1, y1) in pts
    assert {(0, 0), (sg.D, 0), (sg.D, sg.D), (0, sg.D)} <= pts
    # some Steiner vertex did move (the refined CDT's vertex set is not kept)
    assert pts != set(zip(ref.vx.tolist(), ref.vy.tolist()))
    r = sg.rays_isotropic(moved, 4000, 22)
    hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
    hw, tw, sw = oracle.walk(moved, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)


def test_contraction_removes_steiner_vertices_and_keeps_the_scene():
    """The discrete contraction (a Steiner vertex merged into a neighbour, the
    two triangles on their edge deleted): still a valid triangulation of the
    same segments (Euler count, coverage, orientation, neighbours), with fewer
    vertices and no longer than without contraction, and the walk on it equals
    the brute force, steps included."""
    segs = sg.circles(3000, 23)
    ref = sg.refine_optimal(sg.cdt(segs))
    kept = sg.anneal(ref, 23, sweeps=4, collapse=0.0)
    merged = sg.anneal(ref, 23, sweeps=4, collapse=0.5)
    assert oracle.check_triangulation(merged, sg.D) == 0
    assert merged.n_vert < kept.n_vert and merged.n_tri < kept.n_tri
    assert oracle.interior_length(merged) < oracle.interior_length(kept)
    pts = set(zip(merged.vx.tolist(), merged.vy.tolist()))
    for x0, y0, x1, y1 in segs.tolist():
        assert (x0, y0) in pts and (x1, y1) in pts
    r = sg.rays_isotropic(merged, 4000, 24)
    hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
    hw, tw, sw = oracle.walk(merged, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)
    assert np.array_equal(sw[:500], oracle.steps_bruteforce(merged, r.ox[:500], r.oy[:500], r.dx[:500], r.dy[:500],
                                                             hb[:500]))


def test_subdivision_splits_edges_and_keeps_the_scene():
    """The 1 -> 4 subdivision (Sec. 3.5.2 on the lattice): every interior edge
    with a lattice midpoint gains that vertex, constrained edges are split
    along their segment, the result is a valid triangulation of the same
    segments, annealing it keeps it valid, and the walk on both equals the
    brute force."""
    segs = sg.random_segments(300, 31)
    base = sg.anneal(sg.refine_optimal(sg.cdt(segs)), 31, sweeps=2)
    sub = sg.subdivide(base)
    assert oracle.check_triangulation(sub, sg.D) == 0
    pts = set(zip(sub.vx.tolist(), sub.vy.tolist()))
    for t in range(base.n_tri):
        for i in range(3):
            u = base.tri_nb[t, i]
            if u < 0:
                continue
            p, q = base.tri_v[t, (i + 1) % 3], base.tri_v[t, (i + 2) % 3]
            mx, my = int(base.vx[p]) + int(base.vx[q]), int(base.vy[p]) + int(base.vy[q])
            if mx % 2 == 0 and my % 2 == 0:
                assert (mx // 2, my // 2) in pts
    assert sub.n_vert > base.n_vert and sub.n_tri > base.n_tri
    # constrained midpoints are vertices of constrained edges of the same segment
    for t in range(base.n_tri):
        for i in range(3):
            s = base.tri_seg[t, i]
            if s < 0:
                continue
            p, q = base.tri_v[t, (i + 1) % 3], base.tri_v[t, (i + 2) % 3]
            mx, my = int(base.vx[p]) + int(base.vx[q]), int(base.vy[p]) + int(base.vy[q])
            if mx % 2 or my % 2:
                continue
            m = int(np.argwhere((sub.vx == mx // 2) & (sub.vy == my // 2))[0, 0])
            inc = np.argwhere(sub.tri_v == m)
            labels = {int(sub.tri_seg[tt, k]) for tt, vi in inc for k in range(3) if k != vi}
            assert s in labels
    again = sg.anneal(sub, 32, sweeps=2)
    assert oracle.check_triangulation(again, sg.D) == 0
    for tri in (sub, again):
        r = sg.rays_isotropic(tri, 2000, 33)
        hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
        hw, tw, _ = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
        assert np.array_equal(hb, hw) and np.array_equal(tb, tw)


def test_annealer_checkpoint_resume(tmp_path):
    """The annealer checkpoints its triangulation after each piece of its
    schedule (a file cct_scene_load_file reads): a run stopped after three
    pieces and resumed from the checkpoint ends with exactly the triangulation
    of an uninterrupted run, which is valid and keeps the scene; a checkpoint
    of other parameters is not resumed."""
    segs = sg.circles(1500, 81)
    ref = sg.refine_optimal(sg.cdt(segs))
    full = sg.anneal_resumable(ref, 81, str(tmp_path / "a.cct"), sweeps=4, chunks=6)
    part = sg.anneal_resumable(ref, 81, str(tmp_path / "b.cct"), sweeps=4, chunks=6, stop_after=3)
    assert json.load(open(tmp_path / "b.cct.json"))["done"] == 3
    resumed = sg.anneal_resumable(ref, 81, str(tmp_path / "b.cct"), sweeps=4, chunks=6)
    for k in ("vx", "vy", "tri_v", "tri_nb", "tri_seg"):
        assert np.array_equal(getattr(full, k), getattr(resumed, k)), k
    assert oracle.check_triangulation(resumed, sg.D) == 0
    assert oracle.interior_length(resumed) < oracle.interior_length(ref)
    loaded = sg.load(str(tmp_path / "b.cct"), segs)
    assert np.array_equal(loaded.tri_v, resumed.tri_v)
    # other parameters: the checkpoint is ignored and the run starts over
    other = sg.anneal_resumable(ref, 82, str(tmp_path / "b.cct"), sweeps=4, chunks=6, stop_after=1)
    assert json.load(open(tmp_path / "b.cct.json"))["done"] == 1 and other.n_tri > 0
