"""The `lines' scenes of Sec. 4.2 (the workload of the ops-vs-N comparison of
Sec. 6.1): generator properties, and the whole CPU pipeline on them -- CDT,
refinement, annealing, the walk, and the BVH / kd-tree traversals -- against
the brute-force closest hit."""
import numpy as np
import pytest

import oracle
import scenegen as sg


def _orient(p, q, r):
    return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])


@pytest.mark.parametrize("factor,orientation,n", [(0.1, "uniform", 300), (1.0, "vertical", 100),
                                                  (3.0, "diagonal", 300), (3.0, "uniform", 1000)])
def test_lines_generator(factor, orientation, n):
    a = sg.lines(n, 5, factor, orientation)
    assert np.array_equal(a, sg.lines(n, 5, factor, orientation))
    assert a.shape[0] == n  # every requested line fits at these densities
    P = a[:, :2].astype(np.int64)
    Q = a[:, 2:].astype(np.int64)
    # one length, min(0.95, factor * 0.95 / sqrt(n)) of the side, up to the endpoints' rounding
    want = min(0.95, factor * 0.95 / np.sqrt(n)) * sg.D
    lens = np.hypot(*(Q - P).T)
    assert np.all(np.abs(lens - want) <= 1.5)
    # pairwise disjoint, exactly (no proper crossing, no shared or collinear-overlapping points)
    i, j = np.triu_indices(a.shape[0], 1)
    o1 = np.sign(_orient(P[i], Q[i], P[j]))
    o2 = np.sign(_orient(P[i], Q[i], Q[j]))
    o3 = np.sign(_orient(P[j], Q[j], P[i]))
    o4 = np.sign(_orient(P[j], Q[j], Q[i]))
    assert not ((o1 * o2 <= 0) & (o3 * o4 <= 0) & ~((o1 == 0) & (o2 == 0) & (o3 == 0) & (o4 == 0))).any()
    assert np.all(a >= 0.01 * sg.D - 1) and np.all(a <= 0.99 * sg.D + 1)
    # orientation: the angle mod 180 degrees
    ang = np.degrees(np.arctan2(Q[:, 1] - P[:, 1], Q[:, 0] - P[:, 0])) % 180.0
    if orientation == "vertical":
        assert abs(np.median(ang) - 90.0) < 3.0 and np.mean(np.abs(ang - 90.0) < 30.0) > 0.95
    elif orientation == "diagonal":
        assert abs(np.median(ang) - 45.0) < 3.0 and np.mean(np.abs(ang - 45.0) < 30.0) > 0.95
    else:
        hist = np.histogram(ang, bins=6, range=(0, 180))[0]
        assert hist.min() > 0.5 * n / 6


@pytest.mark.parametrize("factor,orientation", [(1.0, "uniform"), (3.0, "diagonal"), (3.0, "vertical")])
def test_lines_pipeline_matches_bruteforce(factor, orientation):
    segs = sg.lines(100, 9, factor, orientation)
    cdt, ref, tri = sg.pipeline(segs, 9, sweeps=2)
    for t in (cdt, ref, tri):
        assert oracle.check_triangulation(t, sg.D) == 0
    assert oracle.interior_length(tri) <= oracle.interior_length(cdt) * (1 + 1e-9)
    r = sg.rays_isotropic(tri, 3000, 10)
    hb, tb = oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy)
    hw, tw, sw = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(hb, hw) and np.array_equal(tb, tw)
    # the comparison structures find the same closest hits
    hbv, tbv, _ = oracle.bvh_trace(sg.bvh(segs, 1.0), r.ox, r.oy, r.dx, r.dy)
    hkd, tkd, _ = oracle.kd_trace(sg.kdtree(segs, 1.0), r.ox, r.oy, r.dx, r.dy)
    assert np.array_equal(hbv, hb) and np.array_equal(hkd, hb)
