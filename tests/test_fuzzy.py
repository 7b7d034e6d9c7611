"""Pins of the fuzzy objective of Sec. 2.2 (scenegen.fuzzy_objective): the
paper's worked example of fuzzy contraction (tests/golden/
fuzzy_contraction_figure.json), the planarity and degree-of-freedom rules of
contractibility, and closed forms (no contraction: plain length)."""
import json
import os

import numpy as np
import pytest

import oracle
import scenegen as sg

D = sg.D
HERE = os.path.dirname(os.path.abspath(__file__))
FIG = json.load(open(os.path.join(HERE, "golden", "fuzzy_contraction_figure.json")))


def _from_triangles(points, tris, segs=None, constrained=()):
    """Triangulation from named points (lattice) and CCW triangles; neighbours by edge matching."""
    names = list(points)
    idx = {n: i for i, n in enumerate(names)}
    vx = np.array([points[n][0] for n in names], np.int32)
    vy = np.array([points[n][1] for n in names], np.int32)
    tv = np.array([[idx[a] for a in t] for t in tris], np.int32)
    nt = len(tris)
    tn = np.full((nt, 3), -1, np.int32)
    ts = np.full((nt, 3), -1, np.int32)
    where = {}
    for t in range(nt):
        for i in range(3):
            a, b = tv[t, (i + 1) % 3], tv[t, (i + 2) % 3]
            where[(a, b)] = (t, i)
    for (a, b), (t, i) in where.items():
        if (b, a) in where:
            tn[t, i] = where[(b, a)][0]
    for s, (a, b) in enumerate(constrained):
        for key in ((idx[a], idx[b]), (idx[b], idx[a])):
            if key in where:
                t, i = where[key]
                ts[t, i] = s
    segs = np.zeros((0, 4), np.int32) if segs is None else np.asarray(segs, np.int32)
    return sg.from_arrays(vx, vy, tv, tn, ts, segs), idx


def _edge_weight(tri, w, idx, a, b):
    ia, ib = idx[a], idx[b]
    for t in range(tri.n_tri):
        for i in range(3):
            if {tri.tri_v[t, (i + 1) % 3], tri.tri_v[t, (i + 2) % 3]} == {ia, ib}:
                return w[t, i]
    raise KeyError((a, b))


def _lattice(case, shrink_units=4.0):
    """The figure's configuration on the lattice (square [-1, 1]^2 -> [0, 2^20]^2), the inner
    vertices pulled towards the contracted point so that contracted edges are a few units long."""
    h = D / 2
    cx, cy = FIG["contracted_point"]
    C = (round((cx + 1) * h), round((cy + 1) * h))
    pts = {k: (round((x + 1) * h), round((y + 1) * h)) for k, (x, y) in FIG["corners"].items()}
    for k, (x, y) in FIG[case]["inner"].items():
        pts[k] = (C[0] + round((x - cx) * shrink_units / 0.1 / 1), C[1] + round((y - cy) * shrink_units / 0.1 / 1))
    return pts, C


def _contracted_state_length(C):
    c = np.array(C, np.float64) / D
    corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
    return 4.0 + float(np.linalg.norm(corners - c, axis=1).sum())


@pytest.mark.parametrize("case", ["one_contracted_edge", "three_contracted_edges"])
def test_figure_worked_example(case):
    """The caption's weights: merging edges 1/2, the doubly merged edge 0, the
    contracted edges 0; the weighted sum equals the length of the contracted
    state (perimeter + four spokes) for both representations."""
    pts, C = _lattice(case)
    tri, idx = _from_triangles(pts, FIG[case]["triangles"])
    assert oracle.check_triangulation(tri, D) == 0
    eps = 0.05
    r = sg.fuzzy_objective(tri, eps, per_edge=True)
    for name, want in FIG[case]["expected_weight"].items():
        a, b = name.split("-")
        got = _edge_weight(tri, r["w"], idx, a, b)
        assert abs(got - want) < 2e-3, (case, name, got, want)
    assert abs(r["w_contr"] - _contracted_state_length(C)) < 2e-3
    assert r["angle"] == 0.0 and r["length"] == 0.0
    # without fuzzy contraction (eps -> 0) the weight is the plain length
    plain = sg.fuzzy_objective(tri, 1e-12)
    assert abs(plain["w_contr"] - tri.length(False) / D) < 1e-6 * plain["w_contr"]  # tri.length sums in fp32


def test_one_hop_connection_blocks_contraction():
    """A short edge A-B whose endpoints share a third neighbour H that is not
    an apex of its triangles (a nontrivial 1-hop connection), with both apexes
    farther than eps, is not contractible, so its neighbours keep weight 1;
    with H within eps of an apex it is, and they drop to 1/2."""
    pts = {"BL": (0, 0), "BR": (D, 0), "TR": (D, D), "TL": (0, D), "A": (500000, 500000), "B": (500010, 500000),
           "H": (500005, 700000), "I": (500005, 560000)}
    tris = [["A", "B", "I"], ["B", "H", "I"], ["H", "A", "I"], ["BL", "BR", "A"], ["A", "BR", "B"],
            ["B", "BR", "TR"], ["B", "TR", "H"], ["H", "TR", "TL"], ["A", "H", "TL"], ["A", "TL", "BL"]]
    tri, idx = _from_triangles(pts, tris)
    assert oracle.check_triangulation(tri, D) == 0
    w = sg.fuzzy_objective(tri, 0.05, per_edge=True)["w"]
    assert _edge_weight(tri, w, idx, "A", "BR") == 1.0  # A-B incontractible (H is 0.13 from I)
    w = sg.fuzzy_objective(tri, 0.5, per_edge=True)["w"]
    assert abs(_edge_weight(tri, w, idx, "A", "BR") - 0.5) < 1e-4  # H within eps of the apex I


def test_fixed_vertices_never_merge_and_free_ones_do():
    """A short segment (both endpoints fixed) is incontractible: the edges
    around it keep weight 1; the same short edge between two free vertices
    lowers them to 1/2."""
    h = D // 2
    pts = {"BL": (0, 0), "BR": (D, 0), "TR": (D, D), "TL": (0, D), "P": (h, h), "Q": (h + 6, h + 2)}
    tris = [["BL", "BR", "P"], ["P", "BR", "Q"], ["Q", "BR", "TR"], ["Q", "TR", "TL"], ["P", "Q", "TL"],
            ["BL", "P", "TL"]]
    seg = [[h, h, h + 6, h + 2]]
    fixed, idx = _from_triangles(pts, tris, segs=seg, constrained=[("P", "Q")])
    free, _ = _from_triangles(pts, tris)
    assert oracle.check_triangulation(fixed, D) == 0 and oracle.check_triangulation(free, D) == 0
    wf = sg.fuzzy_objective(fixed, 0.05, per_edge=True)["w"]
    wr = sg.fuzzy_objective(free, 0.05, per_edge=True)["w"]
    for a, b in (("P", "BR"), ("Q", "BR"), ("P", "TL"), ("Q", "TL")):
        assert _edge_weight(fixed, wf, idx, a, b) == 1.0
        assert abs(_edge_weight(free, wr, idx, a, b) - 0.5) < 1e-4


def test_polish_mode_and_penalties():
    """Polishing: every weight 1 (plain length) and the sharp-angle penalty;
    the obtuse-angle penalty counts angles above 179 degrees; the length
    penalty counts edges shorter than eps0."""
    segs = sg.random_segments(100, 3)
    tri = sg.pipeline(segs, 3, sweeps=1)[2]
    p = sg.fuzzy_objective(tri, 0.05, polish=True)
    assert abs(p["w_contr"] - tri.length(False) / D) < 1e-6 * p["w_contr"]
    # a triangle with an angle of about 179.5 degrees: the obtuse penalty is about 1/2 of its ramp
    import math
    a = math.radians(0.25)
    L = 400000
    pts = {"BL": (0, 0), "BR": (D, 0), "TR": (D, D), "TL": (0, D),
           "M": (D // 2, D // 2 + round(L * math.tan(a))), "L": (D // 2 - L, D // 2), "R": (D // 2 + L, D // 2)}
    tris = [["L", "R", "M"], ["BL", "BR", "L"], ["L", "BR", "R"], ["R", "BR", "TR"], ["R", "TR", "M"],
            ["M", "TR", "TL"], ["L", "M", "TL"], ["BL", "L", "TL"]]
    t2, _ = _from_triangles(pts, tris)
    assert oracle.check_triangulation(t2, D) == 0
    r = sg.fuzzy_objective(t2, 0.05)
    cosM = -math.cos(2 * a)
    want = max(0.0, -1 + sg.FUZZY_DELTA - cosM) / sg.FUZZY_DELTA
    assert 0.3 < want < 0.9 and abs(r["angle"] - want) < 0.02
    r = sg.fuzzy_objective(t2, 0.05, eps0=0.5)
    assert r["length"] > 0  # edges shorter than half the side


def test_fuzzy_annealing_and_contraction_keep_the_scene():
    """Annealing on the fuzzy objective (Sec. 3.3) and the contraction of
    short edges (Sec. 3.4) on a subdivided triangulation: a valid
    triangulation of the same segments with fewer vertices, on which the walk
    equals the brute force; after contraction no contractible edge shorter
    than eps_b is left whose collapse would keep the triangulation valid."""
    segs = sg.random_segments(120, 41)
    tri = sg.subdivide(sg.refine_optimal(sg.cdt(segs)))
    out, n = sg.anneal_fuzzy(tri, 41, sweeps=5, eps_b=2e-4)
    assert n > 0 and out.n_vert == tri.n_vert - n
    assert oracle.check_triangulation(out, D) == 0
    pts = set(zip(out.vx.tolist(), out.vy.tolist()))
    for x0, y0, x1, y1 in segs.tolist():
        assert (x0, y0) in pts and (x1, y1) in pts
    r = sg.rays_isotropic(out, 3000, 42)
    hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
    hw, tw, _ = oracle.walk(out, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)
    # a second contraction pass at the same length finds nothing more to do
    again, n2 = sg.anneal_fuzzy(out, 43, sweeps=0.0, eps_b=2e-4)
    assert n2 == 0 and again.n_vert == out.n_vert
    # the fuzzy objective at a small contraction length is the plain length of the result
    fz = sg.fuzzy_objective(out, 1e-12)
    assert abs(fz["w_contr"] - out.length(False) / D) < 1e-6 * fz["w_contr"]


def test_fuzzy_pipeline_contract_and_polish():
    """The full optimisation with fuzzy contraction (Sec. 3: fuzzy annealing,
    contraction, the contract-and-polish loop of Sec. 3.4, and a second round
    after a 1 -> 4 subdivision, Sec. 3.5.3): a valid
    triangulation of the same segments, shorter than the optimally refined
    CDT, on which the walk equals the brute force."""
    segs = sg.circles(600, 91)
    ref, out = sg.fuzzy_pipeline(segs, 91, sweeps=3, polish_sweeps=3, subdivisions=1)
    assert oracle.check_triangulation(out, D) == 0
    assert oracle.interior_length(out) < oracle.interior_length(ref)
    r = sg.rays_isotropic(out, 3000, 92)
    hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
    hw, tw, _ = oracle.walk(out, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)


def test_contraction_along_a_segment_and_fixed_vertices():
    """The contraction of short edges (Sec. 3.4): a Steiner vertex inside a
    segment, a few units from the segment's endpoint, merges into the endpoint
    along the segment (the segment stays covered by constrained edges and the
    walk equals the brute force); a short segment between two fixed vertices
    is never contracted."""
    h = D // 2
    # segment A-B with a Steiner vertex S 3 units from A; a short fixed segment P-Q elsewhere
    pts = {"BL": (0, 0), "BR": (D, 0), "TR": (D, D), "TL": (0, D),
           "A": (h - 200_000, h), "S": (h - 199_997, h), "B": (h + 200_000, h),
           "P": (h, h + 300_000), "Q": (h + 5, h + 300_001)}
    tris = [["BL", "BR", "A"], ["A", "BR", "S"], ["S", "BR", "B"], ["B", "BR", "TR"], ["B", "TR", "Q"],
            ["Q", "TR", "TL"], ["P", "Q", "TL"], ["A", "S", "P"], ["S", "B", "P"], ["B", "Q", "P"],
            ["A", "P", "TL"], ["BL", "A", "TL"]]
    segs = [[h - 200_000, h, h + 200_000, h], [h, h + 300_000, h + 5, h + 300_001]]
    tri, idx = _from_triangles(pts, tris, segs=segs, constrained=[("A", "S"), ("P", "Q")])
    # S-B carries segment 0 too
    ts = tri.tri_seg.copy()
    for t in range(tri.n_tri):
        for i in range(3):
            if {tri.tri_v[t, (i + 1) % 3], tri.tri_v[t, (i + 2) % 3]} == {idx["S"], idx["B"]}:
                ts[t, i] = 0
    tri = sg.from_arrays(tri.vx, tri.vy, tri.tri_v, tri.tri_nb, ts, np.asarray(segs, np.int32))
    assert oracle.check_triangulation(tri, D) == 0
    out, n = sg.anneal_fuzzy(tri, 5, sweeps=0.0, eps_b=1e-4)  # contraction only: edges < 105 units
    assert n == 1 and out.n_vert == tri.n_vert - 1
    assert oracle.check_triangulation(out, D) == 0
    pts_out = set(zip(out.vx.tolist(), out.vy.tolist()))
    assert pts["S"] not in pts_out and pts["A"] in pts_out and pts["P"] in pts_out and pts["Q"] in pts_out
    r = sg.rays_isotropic(out, 4000, 6)
    hb, tb = oracle.closest_bruteforce(np.asarray(segs, np.int32), r.ox, r.oy, r.dx, r.dy)
    hw, tw, _ = oracle.walk(out, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)


@pytest.mark.parametrize("init_bits", [3, 12])
def test_group_move_region_delta_equals_whole_objective(init_bits):
    """The annealer decides a multi-vertex perturbation (Sec. 3.2.2's second
    variant) on the energy change of a region (the stars of the moved vertices
    and of their neighbours).  For every proposal that change equals the change
    of the whole fuzzy objective -- also when the region's hash tables start at
    8 slots and must grow (rehash) during the evaluation."""
    segs = sg.circles(400, 5)
    tri = sg.refine_optimal(sg.cdt(segs))
    for eps in (0.02, 0.002):
        n, err, grows = sg.fuzzy_check_group_deltas(tri, 7, 300, eps, init_bits, step=0.003)
        assert n >= 100
        assert err <= 1e-9, (eps, err)
        if init_bits == 3:
            assert grows > 0


def test_pipeline_subdivision_round_keeps_the_shorter():
    """scenegen.pipeline: the optimised refined CDT, optimised again after a
    1 -> 4 subdivision (Sec. 3.5.3); the shorter is kept and is valid.  On the
    45-degree dash grid the subdivided round wins."""
    import oracle

    segs = sg.dash_grid(3000, 45.0)
    c, r, best = sg.pipeline(segs, 3, sweeps=4)
    plain = sg.anneal(r, 3, sweeps=4)
    assert oracle.check_triangulation(best, sg.D) == 0
    assert best.length(True) <= plain.length(True)
    assert best.route.startswith("annealed after 1 subdivision")
    assert best.length(True) < 0.97 * c.length(True)
    _, _, once = sg.pipeline(segs, 3, sweeps=4, subdivisions=0)
    assert once.route == "annealed" and once.length(True) == plain.length(True)
