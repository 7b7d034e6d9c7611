"""Comparison structures of Sec. 5.3 (SAH BVH, roped kd-tree).

CPU: the oracle's traversals return the brute-force closest hit (the plain
definition) on random and degenerate rays; closed forms for single-leaf
trees; op-count invariants; the library rejects malformed structures.
GPU: the kernels equal the oracle's traversals element by element -- hit ids,
t and every operation count (the traversal order is fixed by the stated rules,
so counts are deterministic)."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from test_oracle import _degenerate_rays


@pytest.fixture(scope="module")
def scene_rays():
    segs = sg.random_segments(200, 8)
    tri = sg.cdt(segs)
    r = sg.rays_isotropic(tri, 20000, 9)
    ox, oy, dx, dy, _ = _degenerate_rays(tri, 500, 10)
    ox = np.concatenate([r.ox, ox]); oy = np.concatenate([r.oy, oy])
    dx = np.concatenate([r.dx, dx]); dy = np.concatenate([r.dy, dy])
    return segs, tri, (ox, oy, dx, dy)


@pytest.mark.parametrize("alpha", [0.25, 1.0, 4.0])
def test_bvh_oracle_equals_bruteforce(scene_rays, alpha):
    segs, tri, rays = scene_rays
    hb, tb = oracle.closest_bruteforce(segs, *rays)
    b = sg.bvh(segs, alpha)
    h, t, ops = oracle.bvh_trace(b, *rays)
    assert np.array_equal(h, hb) and np.array_equal(t, tb)
    assert (ops[:, 0] >= 1).all() and (ops[:, 0] % 2 == 1).all()  # root + pairs of children
    assert (ops[:, 1] >= (h >= 0)).all()


@pytest.mark.parametrize("lam", [0.25, 1.0, 4.0])
def test_kd_oracle_equals_bruteforce(scene_rays, lam):
    segs, tri, rays = scene_rays
    hb, tb = oracle.closest_bruteforce(segs, *rays)
    k = sg.kdtree(segs, lam)
    h, t, ops = oracle.kd_trace(k, *rays)
    assert np.array_equal(h, hb) and np.array_equal(t, tb)
    assert (ops[:, 0] >= 1).all() and (ops[:, 3] <= ops[:, 2]).all() and (ops[:, 5] == 0).all()
    # every leaf a ray crosses but the last is left through a rope
    assert (ops[:, 4] >= 0).all()


def test_single_leaf_closed_forms(scene_rays):
    """A BVH that is one leaf costs 1 AABB test + all N segment tests for rays
    whose origin lies inside the scene's box; a kd-tree that is one leaf visits
    one leaf and tests all N segments once."""
    segs, tri, (ox, oy, dx, dy) = scene_rays
    n = segs.shape[0]
    b = sg.bvh(segs, alpha=1e9)
    assert b.n_nodes == 1
    h, t, ops = oracle.bvh_trace(b, ox, oy, dx, dy)
    x0, y0 = segs[:, [0, 2]].min(), segs[:, [1, 3]].min()
    x1, y1 = segs[:, [0, 2]].max(), segs[:, [1, 3]].max()
    inside = (ox >= x0) & (ox <= x1) & (oy >= y0) & (oy <= y1)
    assert (ops[inside, 0] == 1).all() and (ops[inside, 1] == n).all()
    k = sg.kdtree(segs, lam=1e9)
    assert k.n_nodes == 1
    h2, t2, ops2 = oracle.kd_trace(k, ox, oy, dx, dy)
    assert (ops2[:, 0] == 1).all() and (ops2[:, 2] == n).all() and (ops2[:, 3] == n).all()
    assert (ops2[:, 1] == 0).all() and (ops2[:, 4] == 0).all()
    assert np.array_equal(h, h2)


def test_kd_ropes_point_across_faces():
    segs = sg.random_segments(200, 12)
    k = sg.kdtree(segs, 1.0)
    leaves = np.flatnonzero(k.axis == 2)
    for L in leaves[:200]:
        b = k.box[L]
        for f in range(4):
            r = k.rope[L, f]
            on_border = (f == 0 and b[0] == 0) or (f == 1 and b[2] == sg.D) or (f == 2 and b[1] == 0) or \
                        (f == 3 and b[3] == sg.D)
            assert (r < 0) == on_border
            if r < 0:
                continue
            rb = k.box[r]
            a = f // 2
            plane = b[a] if f % 2 == 0 else b[2 + a]
            # the rope node touches the face plane and covers the face's extent
            assert rb[a] <= plane <= rb[2 + a]
            assert rb[1 - a] <= b[1 - a] and rb[3 - a] >= b[3 - a]


def test_library_rejects_malformed_structures():
    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    segs = sg.random_segments(50, 3)
    b = sg.bvh(segs, 1.0)
    c0 = b.child0.copy()
    c0[0] = 0  # a node that is its own child
    with pytest.raises(cct.CctError) as e:
        cct.cct_bvh_load(b.box, c0, b.child1, b.prims, segs)
    assert e.value.code == cct.CCT_ERR_INVALID_ARGUMENT
    pr = b.prims.copy()
    pr[0] = 999
    with pytest.raises(cct.CctError) as e:
        cct.cct_bvh_load(b.box, b.child0, b.child1, pr, segs)
    assert e.value.code == cct.CCT_ERR_INVALID_ARGUMENT
    k = sg.kdtree(segs, 1.0)
    rope = k.rope.copy()
    rope[np.argmax(k.axis == 2), 0] = k.n_nodes + 4
    with pytest.raises(cct.CctError) as e:
        cct.cct_kdtree_load(k.axis, k.split, k.child, k.count, k.box, rope, k.rope_log2, k.refs, segs, sg.D)
    assert e.value.code == cct.CCT_ERR_INVALID_ARGUMENT


# ------------------------------------------------------------------------------------------------ GPU
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    return torch, cct


def _run_gpu(torch, struct, rays):
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in rays]
    h, t, ops = struct.trace(*d)
    torch.cuda.synchronize()
    return h.cpu().numpy(), t.cpu().numpy(), ops.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("param", [0.25, 1.0, 4.0])
def test_gpu_bvh_and_kd_equal_oracle(scene_rays, param):
    torch, cct = _gpu()
    segs, tri, rays = scene_rays
    b = sg.bvh(segs, param)
    eh, et, eops = oracle.bvh_trace(b, *rays)
    g = cct.Bvh(b)
    h, t, ops = _run_gpu(torch, g, rays)
    assert np.array_equal(h, eh) and np.array_equal(ops, eops)
    fin = np.isfinite(et)
    assert np.array_equal(np.isfinite(t), fin) and np.all(np.abs(t[fin] - et[fin]) <= 1e-6 * np.abs(et[fin]))
    g.free()
    k = sg.kdtree(segs, param)
    eh, et, eops = oracle.kd_trace(k, *rays)
    g = cct.KdTree(k, sg.D)
    h, t, ops = _run_gpu(torch, g, rays)
    assert (ops[:, 5] == 0).all()
    assert np.array_equal(h, eh) and np.array_equal(ops[:, :5], eops[:, :5])
    fin = np.isfinite(et)
    assert np.array_equal(np.isfinite(t), fin) and np.all(np.abs(t[fin] - et[fin]) <= 1e-6 * np.abs(et[fin]))
    g.free()


@pytest.mark.gpu
@pytest.mark.parametrize("family", ["dash45", "clustered"])
def test_gpu_baselines_config2_scale(family):
    """3e4-segment scenes, 2^18 rays: every output against the oracle."""
    torch, cct = _gpu()
    segs = sg.dash_grid(30000, 45.0) if family == "dash45" else sg.clustered(30000, 4)
    tri = sg.cdt(segs)
    r = sg.rays_isotropic(tri, 1 << 18, 5)
    rays = (r.ox, r.oy, r.dx, r.dy)
    hw, tw, sw = oracle.walk(tri, *rays, r.start)
    for name, build, tr in (("bvh", lambda: sg.bvh(segs, 1.0), oracle.bvh_trace),
                            ("kd", lambda: sg.kdtree(segs, 1.0), oracle.kd_trace)):
        s = build()
        eh, et, eops = tr(s, *rays)
        assert np.array_equal(eh, hw)  # the same closest hits as the walk
        g = cct.Bvh(s) if name == "bvh" else cct.KdTree(s, sg.D)
        h, t, ops = _run_gpu(torch, g, rays)
        assert np.array_equal(h, eh)
        if name == "kd":
            ok = ops[:, 5] == 0
            assert ok.mean() > 0.999
            assert np.array_equal(ops[ok, :5], eops[ok, :5])
        else:
            assert np.array_equal(ops, eops)
        g.free()


@pytest.mark.gpu
@pytest.mark.parametrize("factor,orientation,n", [(3.0, "diagonal", 30), (1.0, "vertical", 300),
                                                  (0.1, "uniform", 1000)])
def test_gpu_lines_scenes_walk_kd_bvh_equal_oracle(factor, orientation, n):
    """The lines scenes (Sec. 4.2): the walk (start cells given and located),
    the kd-tree and the BVH on the GPU give the oracle's hits, steps and
    operation counts; the diagonal case is the one whose best kd-tree is a
    single leaf (Sec. 6.1)."""
    torch, cct = _gpu()
    segs = sg.lines(n, 31, factor, orientation)
    tri = sg.pipeline(segs, 31, sweeps=2)[2]
    r = sg.rays_isotropic(tri, 50_000, 32)
    rays = (r.ox, r.oy, r.dx, r.dy)
    hw, tw, sw = oracle.walk(tri, *rays, r.start)
    hb, tb = oracle.closest_bruteforce(segs, *rays)
    assert np.array_equal(hw, hb) and np.array_equal(tw, tb)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in rays]
    for start in (torch.from_numpy(r.start).cuda(), None):
        h, t, s = scene.trace(*d, start)
        torch.cuda.synchronize()
        assert np.array_equal(h.cpu().numpy(), hw) and np.array_equal(s.cpu().numpy(), sw)
        t = t.cpu().numpy()
        fin = np.isfinite(tw)
        assert np.array_equal(np.isfinite(t), fin) and np.all(np.abs(t[fin] - tw[fin]) <= 1e-6 * np.abs(tw[fin]))
    scene.free()
    for name, s, tr in (("bvh", sg.bvh(segs, 1.0), oracle.bvh_trace), ("kd", sg.kdtree(segs, 1.0), oracle.kd_trace)):
        eh, et, eops = tr(s, *rays)
        assert np.array_equal(eh, hw)
        g = cct.Bvh(s) if name == "bvh" else cct.KdTree(s, sg.D)
        h, t, ops = _run_gpu(torch, g, rays)
        assert np.array_equal(h, eh)
        if name == "kd":
            ok = ops[:, 5] == 0
            assert ok.mean() > 0.999
            assert np.array_equal(ops[ok, :5], eops[ok, :5])
        else:
            assert np.array_equal(ops, eops)
        g.free()
