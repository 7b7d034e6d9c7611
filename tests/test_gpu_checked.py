"""The checked build (libcct_checked.so): every index a kernel reads out of a
device table is range-checked, and a ray that meets one out of range ends with
CCT_RAY_BAD_INDEX instead of reading it.

In the normal test process (bound to libcct.so) this file runs two tests:
the unchecked library refuses to corrupt a table, and
`test_checked_build_suite` re-runs, in a child process bound to the checked
build (CCT_LIBRARY=checked), the GPU parity tests of the walk, locate and
binning, the batched launch, the secondary-ray paths, the fuzzy optimiser's
triangulations and the comparison structures -- the checked kernels must equal
the oracle wherever the unchecked ones do -- together with the fault-injection
tests below, which run only in that child.

Fault injection: out-of-range words are planted in one device table at a
time with the checked build's poke calls.  Every ray either reads a planted
word and is reported CCT_RAY_BAD_INDEX (hit -1, t NaN), or equals the oracle
(or the same library's result on the clean table).  The planted values lie
just past the end of each table (the bound + a few entries), so that even a
kernel missing a check would read inside the same allocation and show up here
as a wrong result rather than touch memory outside the scene.
"""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import oracle
import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.environ.get("CCT_LIBRARY") == "checked"
SUITE = ["tests/test_gpu_walk.py", "tests/test_gpu_batched.py", "tests/test_gpu_bounce.py",
         "tests/test_gpu_fuzzy.py", "tests/test_baselines.py", "tests/test_gpu_checked.py"]


@pytest.fixture(scope="module")
def cct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct as c

    _build.build()
    return c


def _only_checked():
    if not CHECKED:
        pytest.skip("fault injection runs in the child process bound to libcct_checked.so")


def test_unchecked_library_refuses_pokes(cct):
    """libcct.so's kernels do not check, so its poke calls refuse with
    CCT_ERR_UNSUPPORTED and write nothing."""
    if CHECKED:
        pytest.skip("the unchecked library's behaviour")
    assert not cct.cct_is_checked()
    tri = sg.cdt(sg.random_segments(50, 3))
    scene = cct.Scene.from_triangulation(tri, sg.D)
    r = sg.rays_isotropic(tri, 4096, 4)
    d = [torch.from_numpy(a).cuda() for a in (r.ox, r.oy, r.dx, r.dy, r.start)]
    before = [x.cpu() for x in scene.trace(*d)]
    for table in (cct.CCT_TABLE_HALF_EDGE_EXIT, cct.CCT_TABLE_SEED, cct.CCT_TABLE_USER_TO_RECORD):
        with pytest.raises(cct.CctError) as e:
            cct.cct_scene_poke(scene.handle, table, 0, 3 * tri.n_tri)
        assert e.value.code == cct.CCT_ERR_UNSUPPORTED
    after = [x.cpu() for x in scene.trace(*d)]
    assert all(torch.equal(a, b) for a, b in zip(before, after))
    scene.free()


def test_checked_build_suite(cct):
    """The GPU parity tests and this file's fault-injection tests, in a child
    process bound to libcct_checked.so."""
    if CHECKED:
        pytest.skip("this is the child")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    env = dict(os.environ, CCT_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-rs", "-m", "gpu", "-p", "no:cacheprovider",
                        *SUITE], cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 60, tail
    # every fault-injection test ran in the child (none skipped)
    assert not re.search(r"SKIPPED.*test_gpu_checked.py:\d+: fault injection", r.stdout), tail


# ----------------------------------------------------------------------------- fault injection (child only)
@pytest.fixture(scope="module")
def base():
    """A random-segment scene (constrained edges everywhere), rays with their
    start cells, and the oracle's results."""
    segs = sg.random_segments(400, 71)
    tri = sg.cdt(segs)
    r = sg.rays_isotropic(tri, (1 << 16) + 77, 72)
    eh, et, es = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    return segs, tri, r, (eh, et, es)


def _plant(cct, handle, poke, table_len, table, bound, frac, seed, lo=0, spread=61):
    """Writes bound + (k % spread) at a random `frac` of the table's entries
    from `lo` on (all when frac >= 1); returns how many."""
    n = table_len(handle, table)
    rng = np.random.default_rng(seed)
    idx = np.arange(lo, n) if frac >= 1 else lo + rng.choice(n - lo, size=max(1, int((n - lo) * frac)),
                                                              replace=False)
    for k, i in enumerate(idx):
        poke(handle, table, int(i), int(bound + k % spread))
    return len(idx)


def _check_rays(cct, h, t, s, ref):
    """Every ray is either reported bad (hit -1, t NaN) or equals the
    reference; returns the number of bad rays."""
    import bench

    eh, et, es = ref
    bad = s == cct.CCT_RAY_BAD_INDEX
    assert (h[bad] == -1).all() and np.isnan(t[bad]).all()
    mism = bench.parity_mismatches(h[~bad], t[~bad], s[~bad], eh[~bad], et[~bad], es[~bad])
    assert not mism, mism
    return int(bad.sum())


# which ray paths read each table: given start cells (user ids), located
PATHS = {  # name: (start given, flags)
    "given": (True, 0), "given_exact": (True, 1), "given_binned": (True, 2), "given_staged": (True, 8),
    "located": (False, 0), "located_split": (False, 4), "located_binned": (False, 2),
}


@pytest.mark.parametrize("table,frac,reads", [
    ("NEIGHBOUR", 0.1, "all"), ("HALF_EDGE_EXIT", 0.1, "all"), ("CONSTRAINED", 1.0, "located"),
    ("SEED", 0.1, "located"), ("USER_TO_RECORD", 0.1, "given")])
def test_planted_scene_indices_are_reported(cct, base, table, frac, reads):
    """One scene table corrupted at a time, every trace path: rays that read a
    planted word are reported, all others equal the oracle; paths that never
    read the table are unaffected."""
    _only_checked()
    assert cct.cct_is_checked()
    segs, tri, r, ref = base
    tid = getattr(cct, "CCT_TABLE_" + table)
    bound = tri.n_tri if table in ("SEED", "USER_TO_RECORD") else 3 * tri.n_tri
    scene = cct.Scene.from_triangulation(tri, sg.D)
    scene.set_tuning({"block_threads": 64, "refill_min": 16, "chunk": 256, "bin_shift": -1, "trace_flags": 0})
    planted = _plant(cct, scene.handle, cct.cct_scene_poke, cct.cct_scene_table_len, tid, bound, frac, 5)
    assert planted > 0
    d = [torch.from_numpy(a).cuda() for a in (r.ox, r.oy, r.dx, r.dy, r.start)]
    for name, (given, flags) in PATHS.items():
        h, t, s = scene.trace(*d[:4], d[4] if given else None, flags=flags)
        torch.cuda.synchronize()
        n_bad = _check_rays(cct, h.cpu().numpy(), t.cpu().numpy(), s.cpu().numpy(), ref)
        affected = reads == "all" or reads == ("given" if given else "located")
        assert (n_bad > 0) == affected, (table, name, n_bad)
    if table == "SEED":
        # cct_locate reports the origins whose seed cell was planted
        st = scene.locate(d[0], d[1]).cpu().numpy()
        bad = st == cct.CCT_RAY_BAD_INDEX
        assert 0 < bad.sum() < len(st)
        assert (st[~bad] == r.start[~bad]).all()
    scene.free()


def test_planted_two_step_exits_are_reported(cct, base):
    """A scene with two-step records, 10 % of their exit words planted: the
    path kernel, which walks them, reports the paths that read one (at most
    one bad ray per path, the others of the path equal to the oracle's chained
    walk up to it); the walks of cct_trace and the batched launch read the
    16-byte records and equal the oracle, as do paths with CCT_TRACE_ONE_STEP."""
    _only_checked()
    segs, tri, r, ref = base
    scene = cct.Scene.from_triangulation(tri, sg.D, flags=cct.CCT_LOAD_TWO_STEP)
    # the two-step table ends just before the scene's counters: plant exactly one past its end
    _plant(cct, scene.handle, cct.cct_scene_poke, cct.cct_scene_table_len, cct.CCT_TABLE_TWO_STEP_EXIT,
           3 * tri.n_tri, 0.1, 11, spread=1)
    d = [torch.from_numpy(a).cuda() for a in (r.ox, r.oy, r.dx, r.dy, r.start)]
    for given in (True, False):
        for flags in (0, 1, 4, 2):
            h, t, s = scene.trace(*d[:4], d[4] if given else None, flags=flags)
            torch.cuda.synchronize()
            assert _check_rays(cct, h.cpu().numpy(), t.cpu().numpy(), s.cpu().numpy(), ref) == 0, (given, flags)
    n = d[0].numel()
    o = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda"),
         torch.empty(n, dtype=torch.int32, device="cuda"))
    cct.cct_trace_batched([scene], [(0, *d[:4], None, *o)], cct.CCT_TRACE_EXACT_ONLY)
    assert _check_rays(cct, o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy(), ref) == 0
    for flags, affected in ((0, True), (cct.CCT_TRACE_ONE_STEP, False)):
        paths = scene.trace_bounces(*d[:4], 2, start=d[4], flags=flags)
        torch.cuda.synchronize()
        p0 = [paths[k][0].cpu().numpy() for k in ("hit", "t", "steps")]
        assert (_check_rays(cct, *p0, ref) > 0) == affected
        assert (paths["steps"].cpu().numpy() == cct.CCT_RAY_BAD_INDEX).sum(axis=0).max() <= int(affected)
    scene.free()


def test_planted_indices_in_a_batched_launch(cct, base):
    """The multi-scene launch: a half-edge-corrupted and a seed-corrupted scene
    beside a clean one; items with and without start cells."""
    _only_checked()
    segs, tri, r, ref = base
    scenes = [cct.Scene.from_triangulation(tri, sg.D) for _ in range(3)]
    _plant(cct, scenes[0].handle, cct.cct_scene_poke, cct.cct_scene_table_len, cct.CCT_TABLE_HALF_EDGE_EXIT,
           3 * tri.n_tri, 0.1, 6)
    _plant(cct, scenes[1].handle, cct.cct_scene_poke, cct.cct_scene_table_len, cct.CCT_TABLE_SEED, tri.n_tri,
           0.1, 7)
    d = [torch.from_numpy(a).cuda() for a in (r.ox, r.oy, r.dx, r.dy, r.start)]
    n = d[0].numel()
    cases = [(0, True), (0, False), (1, True), (1, False), (2, True), (2, False)]
    outs = [(torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda"),
             torch.empty(n, dtype=torch.int32, device="cuda")) for _ in cases]
    items = [(sc, *d[:4], d[4] if given else None, *o) for (sc, given), o in zip(cases, outs)]
    for flags in (0, cct.CCT_TRACE_EXACT_ONLY):
        cct.cct_trace_batched(scenes, items, flags)
        for (sc, given), (h, t, s) in zip(cases, outs):
            n_bad = _check_rays(cct, h.cpu().numpy(), t.cpu().numpy(), s.cpu().numpy(), ref)
            expect = sc == 0 or (sc == 1 and not given)
            assert (n_bad > 0) == expect, (sc, given, flags, n_bad)
    for s_ in scenes:
        s_.free()


def test_planted_indices_in_secondary_ray_paths(cct, base):
    """Mirror paths on a half-edge-corrupted scene: a path equals the clean
    one up to its first reported ray, which is bad, and has no ray after it;
    paths that meet no planted word equal the clean ones."""
    _only_checked()
    segs, tri, r, _ = base
    scene = cct.Scene.from_triangulation(tri, sg.D)
    d = [torch.from_numpy(a).cuda() for a in (r.ox, r.oy, r.dx, r.dy, r.start)]
    clean = {k: v.cpu().numpy() for k, v in scene.trace_bounces(*d[:4], 4, start=d[4]).items()}
    _plant(cct, scene.handle, cct.cct_scene_poke, cct.cct_scene_table_len, cct.CCT_TABLE_HALF_EDGE_EXIT,
           3 * tri.n_tri, 0.05, 8)
    got = {k: v.cpu().numpy() for k, v in scene.trace_bounces(*d[:4], 4, start=d[4]).items()}
    bad = got["steps"] == cct.CCT_RAY_BAD_INDEX  # (5, n)
    assert bad.any() and (bad.sum(axis=0) <= 1).all()
    first = np.where(bad.any(axis=0), bad.argmax(axis=0), 5)
    for b in range(5):
        before, at, after = first > b, first == b, first < b
        for k in ("hit", "steps", "org_x", "org_y", "dir_x", "dir_y"):
            assert np.array_equal(got[k][b][before], clean[k][b][before]), (b, k)
        assert np.array_equal(got["t"][b][before], clean["t"][b][before], equal_nan=True)
        assert (got["hit"][b][at] == -1).all() and np.isnan(got["t"][b][at]).all()
        assert (got["steps"][b][after] == cct.CCT_RAY_NONE).all()
    scene.free()


@pytest.mark.parametrize("table", ["KD_CHILD", "KD_ROPE", "KD_REF", "BVH_CHILD0", "BVH_CHILD1", "BVH_PRIM"])
def test_planted_indices_in_the_comparison_structures(cct, base, table):
    """The kd-tree and the BVH: rays that meet a planted child, rope,
    reference or primitive are reported (every op count CCT_RAY_BAD_INDEX),
    all others equal the clean structure's results."""
    _only_checked()
    segs, tri, r, _ = base
    kd = table.startswith("KD")
    if kd:
        s = sg.kdtree(segs, 1.0)
        g = cct.KdTree(s, sg.D)
        poke, tlen = cct.cct_kdtree_poke, cct.cct_kdtree_table_len
        nodes, items = len(s.axis), len(s.refs)
    else:
        s = sg.bvh(segs, 1.0)
        g = cct.Bvh(s)
        poke, tlen = cct.cct_bvh_poke, cct.cct_bvh_table_len
        nodes, items = len(s.child0), len(s.prims)
    n_seg = len(segs)
    d = [torch.from_numpy(a).cuda() for a in (r.ox, r.oy, r.dx, r.dy)]
    ch, ct, co = (x.cpu().numpy() for x in g.trace(*d))
    tid = getattr(cct, "CCT_TABLE_" + table)
    if table in ("KD_REF", "BVH_PRIM"):
        # the segment table ends its allocation: plant exactly one past its end
        n = tlen(g.handle, tid)
        for i in np.random.default_rng(9).choice(n, size=max(1, n // 10), replace=False):
            poke(g.handle, tid, int(i), n_seg)
    else:
        bound = {"KD_CHILD": max(nodes, items), "KD_ROPE": nodes, "BVH_CHILD0": nodes,
                 "BVH_CHILD1": max(nodes, items + 1)}[table]
        _plant(cct, g.handle, poke, tlen, tid, bound, 0.1, 10, lo=1)  # the root's entry stays: not every ray
    h, t, o = (x.cpu().numpy() for x in g.trace(*d))
    bad = (o == cct.CCT_RAY_BAD_INDEX).all(axis=1)
    assert bad.any() and not bad.all()
    assert not ((o == cct.CCT_RAY_BAD_INDEX).any(axis=1) & ~bad).any()
    assert (h[bad] == -1).all() and np.isnan(t[bad]).all()
    ok = ~bad
    assert np.array_equal(h[ok], ch[ok]) and np.array_equal(o[ok], co[ok])
    assert np.array_equal(t[ok], ct[ok], equal_nan=True)
    g.free()
