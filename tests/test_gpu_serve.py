"""Continuous-batching server: every request's result in the mix (fused
batched ticks, graph replays, overlapping uploads and downloads, admission by
a memory budget) equals the same request traced alone: hit ids and step
counts bit for bit, t within the 1e-6 relative tolerance; and a sample of
every request equals the oracle."""
import numpy as np
import pytest

import oracle
import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct, serve

    _build.build()
    tris, scenes, rays = [], [], []
    for k, n in enumerate((150, 900, 4000)):
        tri = sg.anneal(sg.cdt(sg.random_segments(n, 60 + k)), k, sweeps=1)
        tris.append(tri)
        scenes.append(cct.Scene.from_triangulation(tri, sg.D))
        rays.append(sg.rays_isotropic(tri, 200_000, 70 + k))
    return cct, serve, tris, scenes, rays


@pytest.mark.parametrize("batched,ahead", [(True, None), (False, None), (True, 4096)])
def test_each_result_equals_alone(env, batched, ahead):
    """ahead: a small upload window (Server.AHEAD_RAYS), so that admission also
    waits for the ticks to take what was uploaded."""
    cct, serve, tris, scenes, rays = env
    pool = serve.RayPool(rays, capacity_out=1 << 24)
    sched = serve.poisson_schedule(3000.0, 0.25, len(scenes), 50, 20000, seed=3)
    budget = 28 * 60_000  # small: forces admission to wait for memory
    srv = serve.Server(scenes, budget_bytes=budget, max_items=256)
    if ahead is not None:
        srv.AHEAD_RAYS = ahead
    res, reqs = srv.run(sched, pool, batched=batched, seed=4, keep_requests=True)
    assert res.completed == res.offered == len(sched) and res.queue_depth_end == 0
    assert np.isfinite(res.p50_ms) and res.p99_ms >= res.p50_ms
    for r in reqs:
        src = torch.cat([aos for aos, soa in r.src], dim=0).cuda()  # (n, 4) interleaved ray records
        ox, oy = src[:, 0].contiguous(), src[:, 1].contiguous()
        dx, dy = src[:, 2].contiguous().view(torch.float32), src[:, 3].contiguous().view(torch.float32)
        h, t, s = scenes[r.scene].trace(ox, oy, dx, dy)
        torch.cuda.synchronize()
        out = r.out.numpy()
        assert np.array_equal(out[0], h.cpu().numpy())
        assert np.array_equal(out[2], s.cpu().numpy())
        ta, tb = out[1].view(np.float32), t.cpu().numpy()
        fin = np.isfinite(tb)
        assert np.array_equal(np.isfinite(ta), fin)
        assert np.all(np.abs(ta[fin] - tb[fin]) <= 1e-6 * np.abs(tb[fin]))  # the stated t tolerance
        # a sample of the request (both ends included) against the oracle, through the pool's indices
        m = out.shape[1]
        idx = np.unique(np.concatenate([np.linspace(0, m - 1, min(m, 512)).astype(np.int64), [0, m - 1]]))
        pr = rays[r.scene]
        pi = (r.pool_lo + idx) % pr.ox.shape[0]
        eh, et, es = oracle.walk(tris[r.scene], pr.ox[pi], pr.oy[pi], pr.dx[pi], pr.dy[pi], pr.start[pi])
        assert np.array_equal(out[0][idx], eh) and np.array_equal(out[2][idx], es)
        fo = np.isfinite(et)
        assert np.array_equal(np.isfinite(ta[idx]), fo)
        assert np.all(np.abs(ta[idx][fo] - et[fo]) <= 1e-6 * np.abs(et[fo]))


def test_copies_async_moves_every_piece():
    """cct_copies_async: pieces of a pinned host buffer to scattered device
    offsets and back, on one stream, in order (the later copy into a range wins)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    src = torch.arange(1 << 16, dtype=torch.int32).pin_memory()
    dev = torch.full((1 << 17,), -1, dtype=torch.int32, device="cuda")
    back = torch.zeros(1 << 17, dtype=torch.int32).pin_memory()
    s = torch.cuda.Stream()
    pieces = [(0, 100, 7), (100, 5000, 3), (60000, 70000, 5536), (10, 10, 0), (0, 100, 20)]  # (src, dst, n) words
    cct.cct_copies_async([dev.data_ptr() + 4 * d for _, d, _ in pieces], [src.data_ptr() + 4 * a for a, _, _ in pieces],
                         [4 * n for *_, n in pieces], s)
    cct.cct_copies_async([back.data_ptr()], [dev.data_ptr()], [4 * (1 << 17)], s)
    s.synchronize()
    exp = np.full(1 << 17, -1, np.int32)
    for a, d, n in pieces:
        exp[d:d + n] = np.arange(a, a + n)
    assert np.array_equal(back.numpy(), exp)
