"""GPU parity of the mirror paths (cct_trace_bounces: secondary rays that start
in the final triangle of their parent's walk, Sec. 5.2) against the oracle's
walk-chained paths, through the C ABI.  Bar: hit ids, step counts, snapped
origins and reflected directions bit-exact; t within 1e-6 relative (fp32
division of an exact int128 numerator and int64 denominator)."""
import numpy as np
import pytest

import oracle
import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_RTOL = 1e-6
NONE = -3


@pytest.fixture(scope="module")
def cct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct as c

    _build.build()
    return c


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_paths(scene, r, nb, start=True, flags=0):
    out = scene.trace_bounces(_dev(r.ox), _dev(r.oy), _dev(r.dx), _dev(r.dy), nb,
                              start=_dev(r.start) if start else None, flags=flags)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _assert_paths(got, exp):
    for k in ("hit", "steps", "org_x", "org_y", "dir_x", "dir_y"):
        if k in got:
            bad = np.argwhere(got[k] != exp[k])
            assert bad.size == 0, f"{k} differs at (bounce, ray) {bad[:8].tolist()}"
    t, et = got["t"], exp["t"]
    fin = np.isfinite(et)
    assert np.array_equal(np.isfinite(t), fin)
    assert np.array_equal(np.isnan(t), np.isnan(et))
    rel = np.abs(t[fin].astype(np.float64) - et[fin]) / np.maximum(np.abs(et[fin].astype(np.float64)), 1e-30)
    assert rel.size == 0 or rel.max() <= T_RTOL, f"t rel err {rel.max()}"


def _scene_cases():
    return [("random", lambda: sg.random_segments(200, 21)), ("room", lambda: sg.room(300, 22)),
            ("circles", lambda: sg.circles(6000, 23)), ("dash45", lambda: sg.dash_grid(4000, 45.0))]


@pytest.mark.parametrize("name,gen", _scene_cases(), ids=[c[0] for c in _scene_cases()])
def test_bounce_paths_equal_oracle(cct, name, gen):
    """Paths of 9 rays (8 bounces) on the CDT and on the annealed
    triangulation, start cells given and located: bit-exact against the
    oracle's walk-chained paths; the scene counters count every ray of a path
    and every step."""
    segs = gen()
    for tri in (sg.cdt(segs), sg.pipeline(segs, 24, sweeps=2)[2]):
        scene = cct.Scene.from_triangulation(tri, sg.D)
        try:
            r = sg.rays_isotropic(tri, 20_000 + 77, 25)  # several chunks and a ragged tail
            nb = 8
            exp = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb)
            scene.stats(reset=True)
            got = _gpu_paths(scene, r, nb)
            _assert_paths(got, exp)
            st = scene.stats(reset=True)
            walked = exp["steps"] != NONE
            assert st["rays"] == int(walked.sum())
            assert st["steps"] == int(exp["steps"][exp["steps"] > 0].sum())
            _assert_paths(_gpu_paths(scene, r, nb, start=False), exp)
            if name == "room":
                assert (exp["steps"][nb] > 0).mean() > 0.5
        finally:
            scene.free()


@pytest.mark.parametrize("name,gen", _scene_cases(), ids=[c[0] for c in _scene_cases()])
def test_bounce_paths_on_two_step_records(cct, name, gen):
    """Scenes loaded with two-step records: mirror paths and paths of
    caller-given directions (two triangles per iteration) equal the oracle's,
    start cells given and located, and so do the paths that keep the 16-byte
    records (CCT_TRACE_ONE_STEP)."""
    segs = gen()
    tri = sg.pipeline(segs, 24, sweeps=2)[2]
    scene = cct.Scene.from_triangulation(tri, sg.D, flags=cct.CCT_LOAD_TWO_STEP)
    try:
        r = sg.rays_isotropic(tri, 20_000 + 77, 29)
        nb = 8
        exp = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb)
        for flags in (0, cct.CCT_TRACE_ONE_STEP):
            _assert_paths(_gpu_paths(scene, r, nb, flags=flags), exp)
        _assert_paths(_gpu_paths(scene, r, nb, start=False), exp)
        fr = _frames(30, r.ox.size, nb)
        efr = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb, frame=fr)
        out = scene.trace_bounces(_dev(r.ox), _dev(r.oy), _dev(r.dx), _dev(r.dy), nb, start=_dev(r.start),
                                  frame=_dev(fr))
        torch.cuda.synchronize()
        _assert_paths({k: v.cpu().numpy() for k, v in out.items()}, efr)
    finally:
        scene.free()


def test_zero_bounces_equal_cct_trace(cct):
    """n_bounce = 0: one record per ray, equal to cct_trace's results."""
    segs = sg.circles(3000, 26)
    tri = sg.pipeline(segs, 27, sweeps=2)[2]
    scene = cct.Scene.from_triangulation(tri, sg.D)
    try:
        r = sg.rays_isotropic(tri, 5000, 28)
        got = _gpu_paths(scene, r, 0)
        h, t, s = scene.trace(_dev(r.ox), _dev(r.oy), _dev(r.dx), _dev(r.dy), _dev(r.start))
        assert np.array_equal(got["hit"][0], h.cpu().numpy()) and np.array_equal(got["steps"][0], s.cpu().numpy())
        np.testing.assert_allclose(got["t"][0], t.cpu().numpy(), rtol=T_RTOL)
    finally:
        scene.free()


def test_invalid_primaries_and_optional_outputs(cct):
    """Invalid primary rays (direction off the grid, zero direction, origin
    on an edge, start triangle out of range) give CCT_RAY_INVALID and then no
    rays; the optional outputs may be omitted; n = 0 is a no-op and
    out-of-range arguments are errors."""
    segs = sg.room(50, 29)
    tri = sg.cdt(segs)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    try:
        r = sg.rays_isotropic(tri, 256, 30)
        r.dx[0] = np.float32(0.1)  # off the 2^-22 grid
        r.dx[1] = 0.0
        r.dy[1] = 0.0
        r.start[2] = tri.n_tri + 3
        # an origin on a triangulation edge: the midpoint of an even edge
        tv = tri.tri_v
        for t_ in range(tri.n_tri):
            a, b = tv[t_, 1], tv[t_, 2]
            if (tri.vx[a] + tri.vx[b]) % 2 == 0 and (tri.vy[a] + tri.vy[b]) % 2 == 0:
                r.ox[3] = (tri.vx[a] + tri.vx[b]) // 2
                r.oy[3] = (tri.vy[a] + tri.vy[b]) // 2
                r.start[3] = t_
                break
        nb = 3
        exp = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb)
        got = _gpu_paths(scene, r, nb)
        _assert_paths(got, exp)
        assert (got["steps"][0, :4] == -1).all() and (got["steps"][1:, :4] == NONE).all()
        assert (got["org_x"][:, :4] == 0).all()
        lean = scene.trace_bounces(_dev(r.ox), _dev(r.oy), _dev(r.dx), _dev(r.dy), nb, start=_dev(r.start),
                                   with_rays=False)
        assert np.array_equal(lean["hit"].cpu().numpy(), exp["hit"])
        e = torch.empty(0, dtype=torch.int32, device="cuda")
        ef = torch.empty(0, dtype=torch.float32, device="cuda")
        cct.cct_trace_bounces(scene.handle, e, e, ef, ef, None, 5, e, ef, e)  # n = 0
        o = _dev(r.ox)
        with pytest.raises(cct.CctError):
            scene.trace_bounces(o, _dev(r.oy), _dev(r.dx), _dev(r.dy), cct.CCT_MAX_BOUNCES + 1)
        with pytest.raises(cct.CctError):
            scene.trace_bounces(o, _dev(r.oy), _dev(r.dx), _dev(r.dy), 2, flags=2)
    finally:
        scene.free()


def test_parallel_mirrors_long_paths(cct):
    """Between two long horizontal mirrors every path uses all its bounces;
    1024 bounces (CCT_MAX_BOUNCES) on a few rays match the oracle."""
    D = sg.D
    segs = np.array([[1000, 400_000, D - 1000, 400_000], [D - 1000, 600_000, 1000, 600_000]], np.int32)
    tri = sg.pipeline(segs, 31, sweeps=2)[2]
    scene = cct.Scene.from_triangulation(tri, sg.D)
    try:
        rng = np.random.default_rng(32)
        n = 96
        th = np.deg2rad(rng.uniform(89.9, 90.1, n)) * np.where(rng.random(n) < 0.5, 1, -1)
        r = sg.Rays(ox=rng.integers(500_000, 548_000, n).astype(np.int32),
                    oy=(rng.integers(450_000, 550_000, n) | 1).astype(np.int32),
                    dx=(np.round(np.cos(th) * 2 ** 22) / 2 ** 22).astype(np.float32),
                    dy=(np.round(np.sin(th) * 2 ** 22) / 2 ** 22).astype(np.float32),
                    start=np.zeros(n, np.int32))
        r.start = oracle.locate_bruteforce(tri, r.ox, r.oy).astype(np.int32)
        assert (r.start >= 0).all()
        nb = cct.CCT_MAX_BOUNCES
        exp = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb)
        got = _gpu_paths(scene, r, nb)
        _assert_paths(got, exp)
        assert (got["steps"][nb] > 0).mean() > 0.9
    finally:
        scene.free()


@pytest.mark.parametrize("family", ["circles", "dash45"])
def test_bench_size_paths_sampled(cct, family):
    """The bench's secondary-ray workload at full size (the bench's scene,
    2^22 paths, up to 8 bounces, start cells given): 4096 randomly sampled
    paths equal the oracle's chained walks; every path's record structure is
    consistent (a path continues only after a hit) and the counters count every
    walked ray."""
    import bench

    k = bench.FAMILIES.index(family)
    segs = bench.family_segments(family)
    tri = sg.pipeline(segs, bench.SCENE_SEED + k, sweeps=4)[2]
    r = sg.rays_isotropic(tri, bench.N_BOUNCE_RAYS, 100 + k)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    try:
        nb = bench.N_BOUNCE
        scene.stats(reset=True)
        got = _gpu_paths(scene, r, nb)
        st = scene.stats(reset=True)
        idx = np.sort(np.random.default_rng(50 + k).choice(r.ox.size, 4096, replace=False))
        exp = oracle.bounce_walk(tri, r.ox[idx], r.oy[idx], r.dx[idx], r.dy[idx], r.start[idx], nb)
        _assert_paths({key: v[:, idx] for key, v in got.items()}, exp)
        steps, hit = got["steps"], got["hit"]
        for b in range(1, nb + 1):
            cont = steps[b] != NONE
            assert (hit[b - 1][cont] >= 0).all() and (steps[b - 1][cont] > 0).all()
        assert st["rays"] == int((steps != NONE).sum())
        assert st["steps"] == int(steps[steps > 0].sum())
    finally:
        scene.free()


def _frames(seed, n, nb):
    """Frame directions (c, s) for secondary rays: mostly valid, some grazing,
    some invalid (s = 0, a component off the 2^-22 grid)."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.02, np.pi - 0.02, (nb, n))
    th = np.where(rng.random((nb, n)) < 0.03, rng.choice([1e-7, np.pi - 1e-7], (nb, n)), th)
    c = np.round(np.cos(th) * 2 ** 22) / 2 ** 22
    s = np.maximum(np.round(np.sin(th) * 2 ** 22), 0) / 2 ** 22
    fr = np.stack([c, s], -1).astype(np.float32)
    bad = rng.random((nb, n))
    fr[..., 1][bad < 0.01] = 0.0
    fr[..., 0][(bad >= 0.01) & (bad < 0.02)] = np.float32(0.1)
    return fr


@pytest.mark.parametrize("name,gen", _scene_cases()[1:3], ids=[c[0] for c in _scene_cases()[1:3]])
def test_frame_direction_paths_equal_oracle(cct, name, gen):
    """Secondary rays with the caller's directions in the hit edges' frames
    (diffuse-style bounces, some grazing, some invalid): bit-exact against the
    oracle's chained walks, start cells given and located; the counters count
    every walked ray, the invalid secondary ones included."""
    segs = gen()
    tri = sg.pipeline(segs, 71, sweeps=2)[2]
    scene = cct.Scene.from_triangulation(tri, sg.D)
    try:
        r = sg.rays_isotropic(tri, 20_000 + 33, 72)
        nb = 6
        fr = _frames(73, r.ox.size, nb)
        exp = oracle.bounce_walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, nb, frame=fr)
        assert (exp["steps"][1:] == -1).sum() > 100 and (exp["steps"][nb] > 0).sum() > 1000
        scene.stats(reset=True)
        out = scene.trace_bounces(_dev(r.ox), _dev(r.oy), _dev(r.dx), _dev(r.dy), nb, start=_dev(r.start),
                                  frame=_dev(fr))
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        _assert_paths(got, exp)
        st = scene.stats(reset=True)
        assert st["rays"] == int((exp["steps"] != NONE).sum())
        assert st["invalid_rays"] == int((exp["steps"] == -1).sum())
        out = scene.trace_bounces(_dev(r.ox), _dev(r.oy), _dev(r.dx), _dev(r.dy), nb, frame=_dev(fr))
        torch.cuda.synchronize()
        _assert_paths({k: v.cpu().numpy() for k, v in out.items()}, exp)
        with pytest.raises(ValueError):
            scene.trace_bounces(_dev(r.ox), _dev(r.oy), _dev(r.dx), _dev(r.dy), nb, frame=_dev(fr[:-1]))
    finally:
        scene.free()


@pytest.mark.parametrize("load_flags", [0, 4])  # 4: CCT_LOAD_TWO_STEP
def test_walk_limit_on_corrupt_triangulation(cct, load_flags):
    """Mirror paths in a triangulation whose triangle 0 names itself as every
    neighbour (loaded without validation): the primary rays starting in it stop
    at the step limit with CCT_RAY_WALK_LIMIT, the rest of each path is 'no
    ray', and the kernel returns instead of hanging."""
    K = 1 << 22
    segs = sg.random_segments(200, 1)
    tri = sg.cdt(segs)
    tn = tri.tri_nb.copy()
    ts = tri.tri_seg.copy()
    tn[0] = [0, 0, 0]
    ts[0] = [-1, -1, -1]
    vx, vy = tri.vx[tri.tri_v[0]].astype(np.int64), tri.vy[tri.tri_v[0]].astype(np.int64)
    n = 64
    ox = np.full(n, int(vx.sum() // 3), np.int32)
    oy = np.full(n, int(vy.sum() // 3), np.int32)
    assert oracle.locate_bruteforce(tri, ox[:1], oy[:1])[0] == 0
    th = np.linspace(0, 2 * np.pi, n, endpoint=False)
    dx = (np.rint(np.cos(th) * K) / K).astype(np.float32)
    dy = (np.rint(np.sin(th) * K) / K).astype(np.float32)
    scene = cct.Scene(tri.vx, tri.vy, tri.tri_v, tn, ts, tri.segs.shape[0], sg.D,
                      flags=cct.CCT_LOAD_NO_VALIDATE | cct.CCT_LOAD_NO_REORDER | load_flags)
    try:
        r = sg.Rays(ox=ox, oy=oy, dx=dx, dy=dy, start=np.zeros(n, np.int32))
        got = _gpu_paths(scene, r, 3)
        assert (got["steps"][0] == cct.CCT_RAY_WALK_LIMIT).all() and (got["hit"][0] == -1).all()
        assert (got["steps"][1:] == NONE).all()
        assert scene.stats()["walk_limit_rays"] == n
    finally:
        scene.free()
