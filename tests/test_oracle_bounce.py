"""Pins of the oracle's secondary rays (Sec. 5.2: a secondary ray starts where
its parent hit a segment, in the final triangle of the parent's walk; here the
mirror image of the parent).  The walk-chained paths are checked against the
same paths by brute force over all segments, and both against closed forms:
parallel mirrors, a 45-degree mirror, perpendicular incidence, the snapped
origin's exact position, and the reflected direction's length."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import scenegen as sg

D = sg.D
Q = 1 << 32
NONE = oracle.BOUNCE_NONE


def _locate(tri, ox, oy):
    st = oracle.locate_bruteforce(tri, ox, oy)
    assert (st >= 0).all(), "test origins must lie strictly inside a triangle"
    return st


def _rays(ox, oy, kx, ky):
    ox, oy = np.asarray(ox, np.int32), np.asarray(oy, np.int32)
    dx = (np.asarray(kx, np.float64) / 2 ** 22).astype(np.float32)
    dy = (np.asarray(ky, np.float64) / 2 ** 22).astype(np.float32)
    return ox, oy, dx, dy


def _k(d):
    return int(round(float(d) * 2 ** 22))


def _equal_paths(W, B):
    for key in ("hit", "org_x", "org_y", "dir_x", "dir_y"):
        assert np.array_equal(W[key], B[key]), key
    assert np.array_equal(W["t"], B["t"], equal_nan=True)


def _path_ok(W, nb):
    """Record structure: once a path ends, every later entry is 'no ray';
    a path continues only after a hit."""
    st, hit = W["steps"], W["hit"]
    for b in range(1, nb + 1):
        cont = st[b] != NONE
        assert (hit[b - 1][cont] >= 0).all()
        assert (st[b - 1][cont] > 0).all()
        assert (st[b][st[b - 1] == NONE] == NONE).all()


@pytest.mark.parametrize("scene", ["random", "room", "circles"])
def test_bounce_walk_equals_bruteforce(scene):
    """Walks chained through their final triangles give, ray by ray and
    bounce by bounce, the paths found by brute force over all segments (hit,
    t, snapped origin, mirror direction); the first ray of each path is the
    primary walk of oracle.walk."""
    if scene == "random":
        segs = sg.random_segments(200, 5)
    elif scene == "room":
        segs = sg.room(150, 6)
    else:
        segs = sg.circles(3000, 7)
    for tri in (sg.cdt(segs), sg.anneal(sg.refine_optimal(sg.cdt(segs)), 8, sweeps=2)):
        r = sg.rays_isotropic(tri, 3000, 9)
        nb = 8
        W = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb)
        B = oracle.bounce_bruteforce(tri, r.ox, r.oy, r.dx, r.dy, nb)
        _equal_paths(W, B)
        _path_ok(W, nb)
        h, t, s = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
        assert np.array_equal(W["hit"][0], h) and np.array_equal(W["steps"][0], s)
        assert np.array_equal(W["t"][0], t, equal_nan=True)
        assert np.array_equal(W["org_x"][0], r.ox.astype(np.int64) << 32)
        if scene == "room":
            # closed room: most paths use every bounce
            assert (W["steps"][nb] > 0).mean() > 0.5
        assert (W["steps"][1] > 0).sum() > 300


def _mirrors(y1=400_000, y2=600_000, m=1000):
    return np.array([[m, y1, D - m, y1], [D - m, y2, m, y2]], np.int32)


@pytest.mark.parametrize("refined", [False, True])
def test_parallel_mirrors_closed_form(refined):
    """Between two horizontal mirrors y = y1, y2 the path alternates between
    them, the direction's vertical component flips exactly, every origin after
    the first lies exactly on a mirror, each secondary ray's t is
    (y2 - y1) / |d_y|, and the origins follow the exact zig-zag within the
    snapping error."""
    y1, y2 = 400_000, 600_000
    segs = _mirrors(y1, y2)
    tri = sg.cdt(segs)
    if refined:
        tri = sg.anneal(sg.refine_optimal(tri), 3, sweeps=2)
    rng = np.random.default_rng(11)
    n, nb = 64, 8
    th = np.deg2rad(rng.uniform(78, 102, n)) * np.where(rng.random(n) < 0.5, 1, -1)
    kx = np.array([_k(np.cos(a)) for a in th])
    ky = np.array([_k(np.sin(a)) for a in th])
    ox = rng.integers(480_000, 560_000, n)
    oy = rng.integers(450_000, 550_000, n) | 1
    ox, oy, dx, dy = _rays(ox, oy, kx, ky)
    st = _locate(tri, ox, oy)
    W = oracle.bounce_walk(tri, ox, oy, dx, dy, st, nb)
    _equal_paths(W, oracle.bounce_bruteforce(tri, ox, oy, dx, dy, nb))
    for i in range(n):
        up = ky[i] > 0
        x_exact = Fraction(int(ox[i]))
        y_prev = int(oy[i])
        for b in range(nb + 1):
            assert W["steps"][b, i] > 0
            sign = 1 if (b % 2 == 0) == up else -1
            assert W["dir_x"][b, i] == dx[i] and W["dir_y"][b, i] == np.float32(sign * abs(dy[i]))
            target = y2 if sign > 0 else y1
            assert W["hit"][b, i] == (1 if sign > 0 else 0)
            dist = abs(target - y_prev)
            t_exact = Fraction(dist * 2 ** 22, abs(int(ky[i])))
            assert abs(Fraction(float(W["t"][b, i])) - t_exact) <= t_exact * Fraction(1, 2 ** 23)
            if b > 0:
                assert W["org_y"][b, i] == y_prev * Q
                err = abs(Fraction(int(W["org_x"][b, i]), Q) - x_exact)
                assert err <= Fraction(b * (D - 2000), Q)
            x_exact += t_exact * Fraction(int(kx[i]), 2 ** 22)
            y_prev = target


def test_diagonal_mirror_swaps_the_direction():
    """A mirror along (1, 1) maps k = (kx, ky) to (ky, kx) exactly."""
    segs = np.array([[300_000, 300_000, 700_000, 700_000]], np.int32)
    tri = sg.cdt(segs)
    rng = np.random.default_rng(12)
    n = 400
    ox = rng.integers(420_000, 620_000, n)
    oy = ox - rng.integers(20_000, 100_000, n)
    th = rng.uniform(0, 2 * np.pi, n)
    kx = np.array([_k(np.cos(a)) for a in th])
    ky = np.array([_k(np.sin(a)) for a in th])
    ox, oy, dx, dy = _rays(ox, oy, kx, ky)
    W = oracle.bounce_walk(tri, ox, oy, dx, dy, _locate(tri, ox, oy), 1)
    on = W["hit"][0] == 0
    assert on.sum() > 50
    assert np.array_equal(W["dir_x"][1][on], dy[on]) and np.array_equal(W["dir_y"][1][on], dx[on])
    # the mirror image travels away from the mirror: no second hit on it
    assert (W["hit"][1][on] == -1).all()


def test_perpendicular_incidence_returns_along_the_ray():
    """A ray meeting a mirror at right angles comes back along itself (k' =
    -k exactly) and then hits what the reversed primary ray hits, at the sum
    of the two distances."""
    segs = np.concatenate([_mirrors(), sg.random_segments(60, 13)[:, :]])
    segs = segs[(np.minimum(segs[:, 1], segs[:, 3]) > 620_000) | (np.maximum(segs[:, 1], segs[:, 3]) < 380_000)
                | (np.arange(len(segs)) < 2)]
    tri = sg.cdt(segs)
    n = 64
    rng = np.random.default_rng(14)
    ox = rng.integers(5000, D - 5000, n)
    oy = rng.integers(410_000, 590_000, n) | 1
    k = 1 << 22
    ky = np.where(rng.random(n) < 0.5, k, -k)
    ox, oy, dx, dy = _rays(ox, oy, np.zeros(n, int), ky)
    W = oracle.bounce_walk(tri, ox, oy, dx, dy, _locate(tri, ox, oy), 2)
    assert np.array_equal(W["dir_y"][1], -dy) and (W["dir_x"][1] == 0).all()
    hb, tb = oracle.closest_bruteforce(segs, ox, oy, -dx, -dy)
    assert np.array_equal(W["hit"][1], hb)
    np.testing.assert_allclose(W["t"][1], W["t"][0] + tb, rtol=1e-6)
    # the snapped origin: a dyadic parameter of the mirror, within |e| / 2 units of 2^-32
    assert (np.abs(W["org_x"][1] - ox.astype(np.int64) * Q) <= (D - 2000) // 2).all()


def test_snapped_origins_lie_on_the_hit_segment():
    """Each secondary origin lies exactly on the hit segment, strictly between
    its endpoints, within |segment| 2^-32 of the exact hit point of its
    parent; the reflected direction keeps the length of k within rounding."""
    segs = sg.room(100, 15)
    tri = sg.anneal(sg.refine_optimal(sg.cdt(segs)), 15, sweeps=2)
    r = sg.rays_isotropic(tri, 400, 16)
    nb = 6
    W = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb)
    checked = 0
    for b in range(nb):
        for i in np.nonzero(W["steps"][b + 1] > 0)[0]:
            s = int(W["hit"][b, i])
            ax, ay, bx, by = (int(v) for v in segs[s])
            X, Y = Fraction(int(W["org_x"][b, i]), Q), Fraction(int(W["org_y"][b, i]), Q)
            kx, ky = _k(W["dir_x"][b, i]), _k(W["dir_y"][b, i])
            ex, ey = bx - ax, by - ay
            t = Fraction(ex * (ay - Y) - ey * (ax - X)) / Fraction(ex * ky - ey * kx)
            hx, hy = X + t * kx, Y + t * ky  # exact hit point (t in units of k)
            X2, Y2 = Fraction(int(W["org_x"][b + 1, i]), Q), Fraction(int(W["org_y"][b + 1, i]), Q)
            assert ex * (Y2 - ay) - ey * (X2 - ax) == 0
            lam = ((X2 - ax) * ex + (Y2 - ay) * ey) / (ex * ex + ey * ey)
            assert 0 < lam < 1
            bound = Fraction(ex * ex + ey * ey) / Fraction(Q * Q)
            assert (X2 - hx) ** 2 + (Y2 - hy) ** 2 <= bound
            k2x, k2y = _k(W["dir_x"][b + 1, i]), _k(W["dir_y"][b + 1, i])
            assert abs(np.hypot(k2x, k2y) - np.hypot(kx, ky)) <= 1.0
            # the mirror image points back to the parent's side
            assert (ex * ky - ey * kx) * (ex * k2y - ey * k2x) < 0
            checked += 1
    assert checked > 500


@pytest.mark.parametrize("mutant", oracle.BOUNCE_MUTANTS)
def test_planted_bounce_mutations_are_caught(mutant):
    """Each planted mistake in the secondary-ray construction (the incoming
    direction added instead of subtracted; the snapped parameter measured from
    the wrong endpoint; the frame's normal on the far side) fails a
    closed-form pin."""
    failed = []
    for fn in (test_parallel_mirrors_closed_form, test_snapped_origins_lie_on_the_hit_segment,
               test_frame_directions_on_parallel_mirrors_closed_form):
        real = oracle._libs.get(0)
        try:
            oracle._libs[0] = oracle._load(mutant)
            if fn is test_parallel_mirrors_closed_form:
                fn(False)
            else:
                fn()
        except AssertionError:
            failed.append(fn.__name__)
        finally:
            if real is not None:
                oracle._libs[0] = real
            else:
                oracle._libs.pop(0, None)
    assert failed


def _frames(rng, n, nb, grazing=0.0):
    """Random frame directions (c, s): s > 0, |(c, s)| <= 1, on the 2^-22 grid."""
    th = rng.uniform(0.02, np.pi - 0.02, (nb, n))
    if grazing:
        th = np.where(rng.random((nb, n)) < grazing, rng.choice([1e-7, np.pi - 1e-7], (nb, n)), th)
    c = np.round(np.cos(th) * 2 ** 22) / 2 ** 22
    s = np.maximum(np.round(np.sin(th) * 2 ** 22), 0) / 2 ** 22
    return np.stack([c, s], -1).astype(np.float32)


@pytest.mark.parametrize("scene", ["room", "circles"])
def test_frame_directions_walk_equals_bruteforce(scene):
    """Secondary rays with the caller's directions in the hit edges' frames:
    the chained walks equal the brute-force paths; every secondary direction
    points back to its parent's side."""
    segs = sg.room(150, 61) if scene == "room" else sg.circles(3000, 62)
    tri = sg.anneal(sg.refine_optimal(sg.cdt(segs)), 63, sweeps=2)
    r = sg.rays_isotropic(tri, 3000, 64)
    nb = 6
    fr = _frames(np.random.default_rng(65), r.ox.size, nb, grazing=0.05)
    W = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb, frame=fr)
    B = oracle.bounce_bruteforce(tri, r.ox, r.oy, r.dx, r.dy, nb, frame=fr)
    _equal_paths(W, B)
    assert (W["steps"][nb] > 0).sum() > 200
    # the invalid frame direction case: s = 0 (along the edge) makes the next ray invalid
    bad = fr.copy()
    bad[0, :, 1] = 0.0
    Wb = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb, frame=bad)
    hit0 = W["hit"][0] >= 0
    assert (Wb["steps"][1][hit0] == -1).all() and (Wb["steps"][2:][:, hit0] == NONE).all()


def test_frame_directions_on_parallel_mirrors_closed_form():
    """On horizontal mirrors the frame is axis-aligned: the direction (c, s)
    becomes exactly (+-c, s) or (-c, -s) in grid units (the normal points back
    to the parent's side), each secondary ray travels y2 - y1 with
    t = (y2 - y1) / s, and a perpendicular direction (0, 1) leaves straight
    back."""
    y1, y2 = 400_000, 600_000
    segs = _mirrors(y1, y2)
    tri = sg.cdt(segs)
    rng = np.random.default_rng(66)
    n, nb = 64, 6
    ox = rng.integers(480_000, 560_000, n)
    oy = rng.integers(450_000, 550_000, n) | 1
    ky = np.where(rng.random(n) < 0.5, 1, -1) * (1 << 22)
    ox, oy, dx, dy = _rays(ox, oy, np.zeros(n, int), ky)
    st = _locate(tri, ox, oy)
    th = rng.uniform(np.deg2rad(86), np.deg2rad(94), (nb, n))
    fr = np.stack([np.round(np.cos(th) * 2 ** 22) / 2 ** 22, np.round(np.sin(th) * 2 ** 22) / 2 ** 22], -1)
    fr = fr.astype(np.float32)
    W = oracle.bounce_walk(tri, ox, oy, dx, dy, st, nb, frame=fr)
    _equal_paths(W, oracle.bounce_bruteforce(tri, ox, oy, dx, dy, nb, frame=fr))
    # mirror 0 (y1) runs +x, mirror 1 (y2) runs -x: u = (+-1, 0) * length
    for i in range(n):
        for b in range(1, nb + 1):
            assert W["steps"][b, i] > 0
            on_top = W["hit"][b - 1, i] == 1  # parent hit the upper mirror: u points -x, normal -y
            c, s = float(fr[b - 1, i, 0]), float(fr[b - 1, i, 1])
            ex_dx, ex_dy = (-c, -s) if on_top else (c, s)
            assert W["dir_x"][b, i] == np.float32(ex_dx) and W["dir_y"][b, i] == np.float32(ex_dy)
            t_exact = Fraction(y2 - y1) / Fraction(abs(float(W["dir_y"][b, i])))
            assert abs(Fraction(float(W["t"][b, i])) - t_exact) <= t_exact * Fraction(1, 2 ** 23)
    perp = np.zeros_like(fr)
    perp[..., 1] = 1.0
    Wp = oracle.bounce_walk(tri, ox, oy, dx, dy, st, nb, frame=perp)
    assert np.array_equal(Wp["dir_y"][1], -dy) and (Wp["dir_x"][1] == 0).all()


def _two_mirror_room(split_top: bool):
    """Lower mirror y = 100000 and upper mirror y = 500000 (x from 100000 to
    900000); the upper one either one segment with a Steiner vertex at x =
    500000 (split_top) or two collinear segments meeting there."""
    import test_fuzzy as tf

    pts = {"BL": (0, 0), "BR": (D, 0), "TR": (D, D), "TL": (0, D),
           "L0": (100_000, 100_000), "L1": (900_000, 100_000),
           "U0": (100_000, 500_000), "UM": (500_000, 500_000), "U1": (900_000, 500_000)}
    tris = [["BL", "BR", "L1"], ["BL", "L1", "L0"], ["BL", "L0", "U0"], ["BL", "U0", "TL"],
            ["L1", "BR", "U1"], ["BR", "TR", "U1"], ["U1", "TR", "TL"], ["UM", "U1", "TL"], ["U0", "UM", "TL"],
            ["L0", "L1", "UM"], ["L0", "UM", "U0"], ["L1", "U1", "UM"]]
    if split_top:
        segs = [[100_000, 100_000, 900_000, 100_000], [100_000, 500_000, 900_000, 500_000]]
        cons = [("L0", "L1"), ("U0", "UM"), ("UM", "U1")]
        labels = {("L0", "L1"): 0, ("U0", "UM"): 1, ("UM", "U1"): 1}
    else:
        segs = [[100_000, 100_000, 900_000, 100_000], [100_000, 500_000, 500_000, 500_000],
                [500_000, 500_000, 900_000, 500_000]]
        cons = [("L0", "L1"), ("U0", "UM"), ("UM", "U1")]
        labels = {("L0", "L1"): 0, ("U0", "UM"): 1, ("UM", "U1"): 2}
    tri, idx = tf._from_triangles(pts, tris, segs=segs, constrained=cons)
    ts = tri.tri_seg.copy()
    for t in range(tri.n_tri):
        for i in range(3):
            e = {tri.tri_v[t, (i + 1) % 3], tri.tri_v[t, (i + 2) % 3]}
            for (a, b), lab in labels.items():
                if e == {idx[a], idx[b]}:
                    ts[t, i] = lab
    tri = sg.from_arrays(tri.vx, tri.vy, tri.tri_v, tri.tri_nb, ts, np.asarray(segs, np.int32))
    assert oracle.check_triangulation(tri, D) == 0
    return tri, np.asarray(segs, np.int32)


@pytest.mark.parametrize("split_top", [True, False])
def test_secondary_ray_from_a_vertex_hit(split_top):
    """A ray straight up through the vertex (500000, 500000) of the upper
    mirror: the ray, shifted infinitesimally to its right, hits the part of the
    mirror on its right (the sub-edge towards x = 900000, or the right-hand
    segment when two segments meet there); the secondary origin is snapped to
    i = 2^32 - 1 on that edge, just right of the vertex, and the mirror image
    goes straight down to the lower mirror at t = 400000.  Walk = brute force."""
    tri, segs = _two_mirror_room(split_top)
    ox, oy, dx, dy = _rays([500_000], [300_001], [0], [1 << 22])
    st = _locate(tri, ox, oy)
    W = oracle.bounce_walk(tri, ox, oy, dx, dy, st, 2)
    _equal_paths(W, oracle.bounce_bruteforce(tri, ox, oy, dx, dy, 2))
    right = 1 if split_top else 2
    assert W["hit"][0, 0] == right and W["t"][0, 0] == np.float32(199_999)
    # snapped on the edge (U1 -> UM): a = U1 (right of the upward ray), b = UM on its line: mu = 1 -> i = 2^32 - 1
    X, Y = int(W["org_x"][1, 0]), int(W["org_y"][1, 0])
    assert Y == 500_000 * Q and X == 900_000 * Q + (Q - 1) * (500_000 - 900_000)
    assert X > 500_000 * Q  # just right of the vertex
    assert W["dir_x"][1, 0] == 0 and W["dir_y"][1, 0] == -1.0
    assert W["hit"][1, 0] == 0 and W["t"][1, 0] == np.float32(400_000)
