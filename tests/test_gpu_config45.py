"""Oracle parity of the batched and served forms at the scale they are measured.

The batching workload itself: 512 scenes from the random-segment generator,
segment counts log-uniform over 100-200,000 (about 1.3e7 segments), each with
its own isotropic batch of 1k-1M rays (about 7.4e7 rays), all triangulations
resident, start cells found on the GPU.  One CUDA-graph-replayed persistent
launch walks every item; 4096 sampled rays of every item (all rays of the
small ones) equal the oracle: hit ids and steps exactly, t within 1e-6
relative.  Both predicate modes (fp32 filter, exact-only) run, at a tuned
configuration (128 threads, refill 16, chunk 512) and with 32-ray chunks
(about 2.3e6 chunks: the chunk and item index arithmetic at its largest).

The continuous-batching server (serve.py) at the same scale: requests naming
scenes of all sizes, each request's results sampled against the oracle.
"""
import numpy as np
import pytest

import bench
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SAMPLE = 4096


@pytest.fixture(scope="module")
def config4():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    import scenegen as sg

    work = bench.config4_scenes(n_scenes=512)
    scenes = [cct.Scene.from_triangulation(tri, sg.D) for segs, tri, r, _ in work]
    dev = torch.device("cuda")
    items = []
    for k, (segs, tri, r, _) in enumerate(work):
        n = len(r)
        items.append((k, torch.from_numpy(r.ox).to(dev), torch.from_numpy(r.oy).to(dev),
                      torch.from_numpy(r.dx).to(dev), torch.from_numpy(r.dy).to(dev), None,
                      torch.full((n,), -9, dtype=torch.int32, device=dev),
                      torch.full((n,), -9.0, dtype=torch.float32, device=dev),
                      torch.full((n,), -9, dtype=torch.int32, device=dev)))
    yield cct, work, scenes, items
    for s in scenes:
        s.free()


def _samples(n, k):
    if n <= N_SAMPLE:
        return np.arange(n)
    rng = np.random.default_rng(1000 + k)
    idx = rng.choice(n, N_SAMPLE - 2, replace=False)
    return np.unique(np.concatenate([idx, [0, n - 1]]))  # both ends of every item


def _check_items(work, items, label):
    checked = 0
    for k, ((segs, tri, r, _), it) in enumerate(zip(work, items)):
        n = len(r)
        idx = _samples(n, k)
        eh, et, es = oracle.walk(tri, r.ox[idx], r.oy[idx], r.dx[idx], r.dy[idx], r.start[idx])
        h, t, s = (it[j].cpu().numpy()[idx] for j in (6, 7, 8))
        bad = bench.parity_mismatches(h, t, s, eh, et, es)
        assert not bad, f"{label}: item {k} ({segs.shape[0]} segments, {n} rays): {bad}"
        checked += idx.size
    return checked


def test_config4_scale_is_what_it_claims(config4):
    cct, work, scenes, items = config4
    nseg = np.array([w[0].shape[0] for w in work])
    nray = np.array([len(w[2]) for w in work])
    assert len(work) == 512 and nseg.min() >= 100 and nseg.max() > 100_000 and nseg.max() <= 200_000
    assert nray.min() >= 1000 and nray.max() > 500_000 and nray.sum() > 5e7


@pytest.mark.parametrize("flags_name", ["filtered", "exact"])
@pytest.mark.parametrize("tuning", [{"block_threads": 128, "refill_min": 16, "chunk": 512},
                                    {"block_threads": 64, "refill_min": 24, "chunk": 32}],
                         ids=["tuned", "chunk32"])
def test_config4_graph_replay_equals_oracle(config4, flags_name, tuning):
    cct, work, scenes, items = config4
    flags = cct.CCT_TRACE_EXACT_ONLY if flags_name == "exact" else 0
    b = cct.Batch(scenes, len(items), flags)
    b.set_tuning(tuning)
    for it in items:  # results of an earlier run must not survive into this one
        it[6].fill_(-9)
        it[7].fill_(-9.0)
        it[8].fill_(-9)
    b.stage(items)
    b.capture()  # one warm-up enqueue, then the captured one
    b.stats(reset=True)
    b.replay()
    torch.cuda.synchronize()
    st = b.stats(reset=True)
    total = sum(len(w[2]) for w in work)
    assert st["rays"] == total and st["invalid_rays"] == 0 and st["walk_limit_rays"] == 0
    assert st["located"] == total
    if flags:
        assert st["exact_fallbacks"] == 0
    checked = _check_items(work, items, f"{flags_name}/{tuning}")
    assert checked > 1_500_000
    b.free()


def test_served_requests_equal_oracle():
    """Config-5 requests (1k-4M rays, log-uniform; scenes of the batching
    workload's generator, 100-200,000 segments, the largest included) through
    the continuous-batching loop with the 60 GB budget: a sample of every
    completed request equals the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct, serve

    _build.build()
    import scenegen as sg

    work = bench.config4_scenes(n_scenes=24, seed=9, pool_rays=1 << 20)
    big = int(np.argmax([w[0].shape[0] for w in work]))
    assert work[big][0].shape[0] > 50_000
    scenes = [cct.Scene.from_triangulation(tri, sg.D) for segs, tri, r, pool in work]
    pools = [w[3] for w in work]
    sched = serve.poisson_schedule(200.0, 0.2, len(scenes), 1000, 4_000_000, seed=11)
    sched.append((0.2, big, 4_000_000))  # the largest request on the largest scene
    # a result ring that holds every request's results at once (none overwritten before the check)
    pool = serve.RayPool(pools, capacity_out=sum(n for _, _, n in sched) + 1)
    srv = serve.Server(scenes, budget_bytes=60 << 30, max_items=4096)
    res, reqs = srv.run(sched, pool, batched=True, seed=12, keep_requests=True)
    assert res.completed == res.offered == len(sched) and len(sched) >= 20
    for q, r in enumerate(reqs):
        out = r.out.numpy()
        m = out.shape[1]
        idx = _samples(m, q)
        pr = pools[r.scene]
        pi = (r.pool_lo + idx) % pr.ox.shape[0]
        eh, et, es = oracle.walk(work[r.scene][1], pr.ox[pi], pr.oy[pi], pr.dx[pi], pr.dy[pi], pr.start[pi])
        bad = bench.parity_mismatches(out[0][idx], out[1].view(np.float32)[idx], out[2][idx], eh, et, es)
        assert not bad, f"request {q} (scene {r.scene}, {r.n} rays): {bad}"
    for s in scenes:
        s.free()
