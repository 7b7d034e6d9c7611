"""GPU parity of the walk, locate and binning kernels against the CPU oracle,
through the C ABI.  Bar: hit ids and step counts bit-exact; t within 1e-6
relative (fp32 division of exact int64 numerator and denominator, <= 4 ulp).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_RTOL = 1e-6
K = 1 << 22


@pytest.fixture(scope="module")
def cct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct as c

    _build.build()
    return c


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _trace(scene, ox, oy, dx, dy, start, flags=0):
    h, t, s = scene.trace(_dev(ox), _dev(oy), _dev(dx), _dev(dy), None if start is None else _dev(start), flags)
    torch.cuda.synchronize()
    return h.cpu().numpy(), t.cpu().numpy(), s.cpu().numpy()


def _assert_parity(got, exp):
    h, t, s = got
    eh, et, es = exp
    assert np.array_equal(h, eh), f"hit ids differ at {np.flatnonzero(h != eh)[:10]}"
    assert np.array_equal(s, es), f"steps differ at {np.flatnonzero(s != es)[:10]}"
    fin = np.isfinite(et)
    assert np.array_equal(np.isfinite(t), fin)
    assert np.array_equal(np.isnan(t), np.isnan(et))
    rel = np.abs(t[fin].astype(np.float64) - et[fin]) / np.abs(et[fin].astype(np.float64))
    assert rel.size == 0 or rel.max() <= T_RTOL, f"t rel err {rel.max()}"


@pytest.fixture(scope="module")
def scenes():
    out = []
    for seed in (1, 2):
        segs = sg.random_segments(200, seed)
        cdt = sg.cdt(segs)
        out.append(("cdt", seed, cdt))
        out.append(("annealed", seed, sg.anneal(cdt, seed)))
    return out


@pytest.mark.parametrize("flags_name", ["filtered", "exact", "binned", "binned_exact"])
def test_config1_given_start_bit_exact(cct, scenes, flags_name):
    flags = {"filtered": 0, "exact": cct.CCT_TRACE_EXACT_ONLY, "binned": cct.CCT_TRACE_BIN,
             "binned_exact": cct.CCT_TRACE_BIN | cct.CCT_TRACE_EXACT_ONLY}[flags_name]
    for kind, seed, tri in scenes:
        r = sg.rays_isotropic(tri, 65536, 10 + seed)
        exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
        scene = cct.Scene.from_triangulation(tri, sg.D)
        _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, r.start, flags), exp)
        # closest hit also equals the brute-force definition
        hb, tb = oracle.closest_bruteforce(tri.segs, r.ox, r.oy, r.dx, r.dy)
        assert np.array_equal(exp[0], hb)
        scene.free()


def test_config1_locate_then_walk(cct, scenes):
    for kind, seed, tri in scenes:
        r = sg.rays_isotropic(tri, 65536 + 37, 20 + seed)  # ragged tail
        exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
        scene = cct.Scene.from_triangulation(tri, sg.D)
        for flags in (0, cct.CCT_TRACE_BIN, cct.CCT_TRACE_SPLIT_LOCATE):
            _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, None, flags), exp)
        st = scene.locate(_dev(r.ox), _dev(r.oy))
        torch.cuda.synchronize()
        assert np.array_equal(st.cpu().numpy(), r.start)
        stats = scene.stats()
        assert stats["located"] == 3 * len(r) + len(r)
        scene.free()


def test_locate_edges_vertices_and_outside(cct, scenes):
    kind, seed, tri = scenes[1]
    tv = tri.tri_v
    a, b = tv[:, 1], tv[:, 2]
    mx = tri.vx[a].astype(np.int64) + tri.vx[b]
    my = tri.vy[a].astype(np.int64) + tri.vy[b]
    even = (mx % 2 == 0) & (my % 2 == 0)
    px = np.concatenate([(mx[even] // 2), tri.vx, [-5, sg.D + 1, 100]]).astype(np.int32)
    py = np.concatenate([(my[even] // 2), tri.vy, [10, 10, -1]]).astype(np.int32)
    rng = np.random.default_rng(5)
    qx = rng.integers(0, sg.D + 1, 20000).astype(np.int32)
    qy = rng.integers(0, sg.D + 1, 20000).astype(np.int32)
    px, py = np.concatenate([px, qx]), np.concatenate([py, qy])
    exp = oracle.locate_bruteforce(tri, px, py)
    exp = np.where(exp < 0, -1, exp)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    got = scene.locate(_dev(px), _dev(py))
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), exp)
    scene.free()


@pytest.mark.parametrize("density", [0, 2, 5, 8])
def test_locate_seed_ties_on_lattice(cct, lattice, density):
    """Seed points (cell centres) that fall on vertices and edges, and origins
    collinear with seed points and vertices: every integer point of a small
    lattice triangulation, located and traced from no start cell, equals the
    brute-force location and the oracle walk.  Density 8 gives cells of side 1,
    so every seed point is a lattice point."""
    tri = lattice()
    g = np.arange(-1, tri.D + 2, dtype=np.int32)
    px, py = [np.ascontiguousarray(a.ravel()) for a in np.meshgrid(g, g)]
    exp = oracle.locate_bruteforce(tri, px, py)
    exp = np.where(exp < 0, -1, exp)
    scene = cct.Scene.from_triangulation(tri, tri.D, flags=cct.CCT_LOAD_SEED_DENSITY(density))
    got = scene.locate(_dev(px), _dev(py))
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), exp)
    rng = np.random.default_rng(density)
    ang = rng.uniform(0, 2 * np.pi, px.size)
    dx = (np.round(np.cos(ang) * K) / K).astype(np.float32)
    dy = (np.round(np.sin(ang) * K) / K).astype(np.float32)
    ref = oracle.walk(tri, px, py, dx, dy, exp)
    for flags in (0, cct.CCT_TRACE_EXACT_ONLY, cct.CCT_TRACE_BIN, cct.CCT_TRACE_SPLIT_LOCATE):
        _assert_parity(_trace(scene, px, py, dx, dy, None, flags), ref)
    scene.free()


def test_golden_worked_cases_gpu(cct):
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_cases.json")))
    for name, scene_def in g["scenes"].items():
        cases = [c for c in g["cases"] if c["scene"] == name]
        segs = np.asarray(scene_def["segs"], np.int32).reshape(-1, 4)
        tri = sg.cdt(segs)
        ox = np.array([c["o"][0] for c in cases], np.int32)
        oy = np.array([c["o"][1] for c in cases], np.int32)
        dx = np.array([c["k"][0] / K for c in cases], np.float32)
        dy = np.array([c["k"][1] / K for c in cases], np.float32)
        scene = cct.Scene.from_triangulation(tri, sg.D)
        for start in (oracle.locate_bruteforce(tri, ox, oy), None):
            h, t, s = _trace(scene, ox, oy, dx, dy, start)
            for i, c in enumerate(cases):
                assert h[i] == c["hit"], (name, i)
                if c["t"] is None:
                    assert np.isinf(t[i])
                else:
                    et = float(Fraction(c["t"][0], c["t"][1]))
                    assert abs(float(t[i]) - et) <= T_RTOL * et
                if "steps" in c:
                    assert s[i] == c["steps"]
        scene.free()


def test_degenerate_rays_bit_exact(cct, scenes):
    from test_oracle import _degenerate_rays

    for kind, seed, tri in scenes:
        ox, oy, dx, dy, st = _degenerate_rays(tri, 2000, 40 + seed)
        exp = oracle.walk(tri, ox, oy, dx, dy, st)
        scene = cct.Scene.from_triangulation(tri, sg.D)
        for flags in (0, cct.CCT_TRACE_EXACT_ONLY):
            _assert_parity(_trace(scene, ox, oy, dx, dy, st, flags), exp)
        scene.free()


def test_invalid_rays_and_edge_sizes(cct, scenes):
    kind, seed, tri = scenes[0]
    r = sg.rays_isotropic(tri, 64, 3)
    ox, oy, dx, dy, st = r.ox.copy(), r.oy.copy(), r.dx.copy(), r.dy.copy(), r.start.copy()
    dx[0] = np.float32(0.1)             # off the 2^-22 grid
    dx[1] = 0.0; dy[1] = 0.0            # zero direction
    dx[2] = 2.0                          # |component| > 1
    st[3] = -5                           # start out of range
    st[4] = tri.n_tri + 3
    st[5] = (st[5] + 1) % tri.n_tri      # start triangle does not hold the origin
    dy[6] = np.float32(np.nan)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    h, t, s = _trace(scene, ox, oy, dx, dy, st)
    bad = np.zeros(64, bool)
    bad[:7] = True
    if oracle.locate_bruteforce(tri, ox[5:6], oy[5:6])[0] == st[5]:
        bad[5] = False
    assert (s[bad] == cct.CCT_RAY_INVALID).all() and (h[bad] == -1).all() and np.isnan(t[bad]).all()
    exp = oracle.walk(tri, ox, oy, dx, dy, st)
    _assert_parity((h, t, s), exp)
    # n = 0 is a no-op, n = 1 works
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    ef = torch.empty(0, dtype=torch.float32, device="cuda")
    cct.cct_trace(scene.handle, e, e, ef, ef, e, e, ef, e)
    _assert_parity(_trace(scene, ox[10:11], oy[10:11], dx[10:11], dy[10:11], st[10:11]),
                   tuple(a[10:11] for a in exp))
    scene.free()


def test_walk_limit_on_corrupt_triangulation(cct, scenes):
    """A triangulation whose triangle 0 names itself as every neighbour (loaded
    without validation): the walk circles inside it and must stop at the step
    limit with CCT_RAY_WALK_LIMIT instead of hanging."""
    kind, seed, tri = scenes[0]
    tn = tri.tri_nb.copy()
    ts = tri.tri_seg.copy()
    tn[0] = [0, 0, 0]
    ts[0] = [-1, -1, -1]
    # rays that start in triangle 0
    vx, vy = tri.vx[tri.tri_v[0]].astype(np.int64), tri.vy[tri.tri_v[0]].astype(np.int64)
    cx, cy = int(vx.sum() // 3), int(vy.sum() // 3)
    n = 64
    ox = np.full(n, cx, np.int32)
    oy = np.full(n, cy, np.int32)
    assert oracle.locate_bruteforce(tri, ox[:1], oy[:1])[0] == 0
    th = np.linspace(0, 2 * np.pi, n, endpoint=False)
    dx = (np.rint(np.cos(th) * K) / K).astype(np.float32)
    dy = (np.rint(np.sin(th) * K) / K).astype(np.float32)
    st = np.zeros(n, np.int32)
    scene = cct.Scene(tri.vx, tri.vy, tri.tri_v, tn, ts, tri.segs.shape[0], sg.D,
                      flags=cct.CCT_LOAD_NO_VALIDATE | cct.CCT_LOAD_NO_REORDER)
    h, t, s = _trace(scene, ox, oy, dx, dy, st)
    assert (s == cct.CCT_RAY_WALK_LIMIT).all() and (h == -1).all()
    assert scene.stats()["walk_limit_rays"] == n
    scene.free()


def test_stats_counters(cct, scenes):
    kind, seed, tri = scenes[2]
    r = sg.rays_isotropic(tri, 100000, 7)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    h, t, s = _trace(scene, r.ox, r.oy, r.dx, r.dy, r.start)
    st = scene.stats(reset=True)
    assert st["rays"] == len(r) and st["steps"] == int(s.sum())
    assert st["side_tests"] == int(s.sum()) + len(r)  # 2 in the first triangle, 1 per later step
    assert st["exact_fallbacks"] < st["side_tests"] * 1e-3
    h, t, s = _trace(scene, r.ox, r.oy, r.dx, r.dy, r.start, cct.CCT_TRACE_EXACT_ONLY)
    st2 = scene.stats()
    assert st2["exact_fallbacks"] == 0 and st2["steps"] == st["steps"]
    scene.free()


def test_empty_scene_and_tiny_domain(cct):
    tri = sg.cdt(np.zeros((0, 4), np.int32))
    r = sg.rays_isotropic(tri, 10000, 1)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, None), exp)
    assert (exp[0] == -1).all()
    scene.free()


@pytest.mark.parametrize("family", ["circles", "circles_refined", "dash22", "clustered"])
def test_config2_scale_full_parity(cct, family):
    """Config-2-sized scenes (3e4 segments), 2^20 rays: every output checked.
    circles_refined: the optimally refined + annealed pipeline, whose
    constrained edges are split at Steiner points."""
    segs = {"circles": lambda: sg.circles(30000, 3), "circles_refined": lambda: sg.circles(30000, 3),
            "dash22": lambda: sg.dash_grid(30000, 22.5), "clustered": lambda: sg.clustered(30000, 3)}[family]()
    if family == "circles_refined":
        tri = sg.pipeline(segs, 3, sweeps=2)[2]
    else:
        tri = sg.anneal(sg.cdt(segs), 3, sweeps=2)
    r = sg.rays_isotropic(tri, 1 << 20, 4)
    exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    for flags in (0, cct.CCT_TRACE_BIN):
        _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, None, flags), exp)
    # the brute-force definition on a sample
    idx = np.random.default_rng(0).choice(len(r), 2000, replace=False)
    hb, tb = oracle.closest_bruteforce(segs, r.ox[idx], r.oy[idx], r.dx[idx], r.dy[idx])
    assert np.array_equal(hb, exp[0][idx]) and np.array_equal(tb, exp[1][idx])
    scene.free()


def test_scene_with_two_step_records_walks_identically(cct, scenes):
    """A scene loaded with two-step records (CCT_LOAD_TWO_STEP, for the path
    kernel) walks on its 16-byte records as before: every path -- start cells
    given or located (fused and split), fp32-filtered and exact-only, binned,
    degenerate rays -- equals the oracle, and the counters are unchanged."""
    from test_oracle import _degenerate_rays

    for kind, seed, tri in scenes:
        r = sg.rays_isotropic(tri, 65536 + 37, 60 + seed)
        exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
        ox, oy, dx, dy, st = _degenerate_rays(tri, 2000, 70 + seed)
        dexp = oracle.walk(tri, ox, oy, dx, dy, st)
        scene = cct.Scene.from_triangulation(tri, sg.D, flags=cct.CCT_LOAD_TWO_STEP)
        for flags in (0, cct.CCT_TRACE_EXACT_ONLY, cct.CCT_TRACE_SPLIT_LOCATE, cct.CCT_TRACE_BIN):
            for start in (r.start, None):
                _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, start, flags), exp)
        for flags in (0, cct.CCT_TRACE_EXACT_ONLY):
            _assert_parity(_trace(scene, ox, oy, dx, dy, st, flags), dexp)
        scene.stats(reset=True)
        h, t, s = _trace(scene, r.ox, r.oy, r.dx, r.dy, r.start)
        st2 = scene.stats()
        assert st2["steps"] == int(s.sum()) and st2["side_tests"] == int(s.sum()) + len(r)
        scene.free()


def test_results_independent_of_tuning(cct, scenes):
    """Block size, refill threshold, chunk and binning granularity change the
    schedule only: results stay bit-identical to the oracle."""
    kind, seed, tri = scenes[3]
    r = sg.rays_isotropic(tri, 50000 + 13, 77)
    exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    for tu in ({"block_threads": 32, "refill_min": 1, "chunk": 32},
               {"block_threads": 512, "refill_min": 32, "chunk": 4096},
               {"block_threads": 128, "refill_min": 4, "chunk": 64, "bin_shift": 0},
               {"block_threads": 96, "refill_min": 16, "chunk": 200, "bin_shift": 5,
                "trace_flags": cct.CCT_TRACE_EXACT_ONLY},
               {"block_threads": 64, "refill_min": 24, "chunk": 64, "trace_flags": cct.CCT_TRACE_SPLIT_LOCATE}):
        scene.set_tuning(tu)
        assert all(scene.tuning()[k] == v for k, v in tu.items())
        for start in (r.start, None):
            for flags in (0, cct.CCT_TRACE_BIN):
                _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, start, flags), exp)
    scene.set_tuning(None)
    with pytest.raises(cct.CctError):
        scene.set_tuning({"block_threads": 33})
    scene.free()


def test_scene_from_file_traces_identically(cct, scenes, tmp_path):
    """A scene loaded by cct_scene_load_file gives the same results as one
    loaded from the arrays (and as the oracle)."""
    kind, seed, tri = scenes[1]
    path = tmp_path / "scene.cct"
    tri.save(str(path))
    r = sg.rays_isotropic(tri, 20000, 91)
    exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    from_file = cct.Scene.from_file(str(path))
    assert from_file.n_tri == tri.n_tri
    for start in (r.start, None):
        _assert_parity(_trace(from_file, r.ox, r.oy, r.dx, r.dy, start), exp)
    from_file.free()


@pytest.mark.parametrize("N", [100_000, 1_000_000])
def test_config3_ring_of_circles_sampled(cct, N):
    """The scaling workload (ring of circles in a fixed domain, built as the
    scaling run builds it) at 10^5 and 10^6 segments, where the tables outgrow
    L2: 2^22 isotropic rays and 1024 pinhole fans of 4096 rays, start cells from
    the fused locate and with binning; 4096 sampled rays of each equal the
    oracle (start cells from the CPU)."""
    segs = sg.ring_of_circles(N)
    tri = sg.pipeline(segs, 3, sweeps=1)[2]
    scene = cct.Scene.from_triangulation(tri, sg.D)
    try:
        for name, r in (("iso", sg.rays_isotropic(tri, 1 << 22, 11)), ("fans", sg.rays_pinhole(tri, 1024, 4096, 12))):
            idx = np.sort(np.random.default_rng(13).choice(len(r), 4096, replace=False))
            exp = oracle.walk(tri, r.ox[idx], r.oy[idx], r.dx[idx], r.dy[idx], r.start[idx])
            for flags in (0, cct.CCT_TRACE_BIN):
                h, t, s = _trace(scene, r.ox, r.oy, r.dx, r.dy, None, flags)
                _assert_parity((h[idx], t[idx], s[idx]), exp)
    finally:
        scene.free()


@pytest.mark.parametrize("block", [64, 512])
@pytest.mark.parametrize("exact", [0, 1])
def test_staged_half_edge_table_bit_exact(cct, scenes, block, exact):
    """CCT_TRACE_STAGE (the half-edge table copied into each block's shared
    memory): start cells given, located in the walk kernel, and located by the
    split locate kernel, on the config-1 scenes with a ragged ray count and
    degenerate rays; every output equals the oracle."""
    from test_oracle import _degenerate_rays

    fl = cct.CCT_TRACE_STAGE | (cct.CCT_TRACE_EXACT_ONLY if exact else 0)
    for kind, seed, tri in scenes:
        r = sg.rays_isotropic(tri, 65536 + 77, 30 + seed)
        ox, oy, dx, dy, _ = _degenerate_rays(tri, 300, 40 + seed)
        st = oracle.locate_bruteforce(tri, ox, oy)
        ok = st >= 0
        cat = lambda a, b: np.ascontiguousarray(np.concatenate([a, b[ok]]))
        ox, oy, dx, dy, st = cat(r.ox, ox), cat(r.oy, oy), cat(r.dx, dx), cat(r.dy, dy), cat(r.start, st)
        exp = oracle.walk(tri, ox, oy, dx, dy, st)
        scene = cct.Scene.from_triangulation(tri, sg.D)
        scene.set_tuning({"block_threads": block, "refill_min": 16, "chunk": 256})
        for start, extra in ((st, 0), (None, 0), (None, cct.CCT_TRACE_SPLIT_LOCATE)):
            _assert_parity(_trace(scene, ox, oy, dx, dy, start, fl | extra), exp)
        scene.free()


def test_stage_flag_ignored_where_the_table_does_not_fit(cct):
    """A scene whose half-edge table does not fit in shared memory beside the
    stacks walks from global memory under CCT_TRACE_STAGE: same results."""
    segs = sg.random_segments(3000, 9)
    tri = sg.cdt(segs)
    assert tri.n_tri * 48 > 227 * 1024
    r = sg.rays_isotropic(tri, 100_000, 11)
    exp = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, r.start, cct.CCT_TRACE_STAGE), exp)
    _assert_parity(_trace(scene, r.ox, r.oy, r.dx, r.dy, None, cct.CCT_TRACE_STAGE), exp)
    scene.free()
