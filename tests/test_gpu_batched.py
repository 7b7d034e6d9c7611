"""The multi-scene persistent launch (cct_batch_*): every item's results equal
the single-scene cct_trace results and the oracle, bit for bit (ids, steps) and
within 1e-6 (t); a captured CUDA graph replays correctly after re-staging."""
import numpy as np
import pytest

import oracle
import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    rng = np.random.default_rng(5)
    tris, scenes = [], []
    for k, n in enumerate((100, 700, 3000, 12000)):
        segs = sg.random_segments(n, 40 + k)
        tri = sg.anneal(sg.cdt(segs), k, sweeps=1)
        tris.append(tri)
        scenes.append(cct.Scene.from_triangulation(tri, sg.D))
    items = []
    for k in range(13):  # several items per scene, ragged sizes, one empty item
        si = int(rng.integers(0, len(tris)))
        n = [0, 1, 31, 500, 4097, 20000, 70001][k % 7]
        r = sg.rays_isotropic(tris[si], max(n, 1), 100 + k)
        items.append((si, r, n))
    return cct, tris, scenes, items


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _make(items, with_start):
    out = []
    for k, (si, r, n) in enumerate(items):
        st = _dev(r.start[:n]) if (with_start and k % 2 == 0) else None
        out.append((si, _dev(r.ox[:n]), _dev(r.oy[:n]), _dev(r.dx[:n]), _dev(r.dy[:n]), st,
                    torch.full((n,), -9, dtype=torch.int32, device="cuda"),
                    torch.full((n,), -9.0, dtype=torch.float32, device="cuda"),
                    torch.full((n,), -9, dtype=torch.int32, device="cuda")))
    return out


def _check(setup, dev_items):
    cct, tris, scenes, items = setup
    for (si, r, n), it in zip(items, dev_items):
        eh, et, es = oracle.walk(tris[si], r.ox[:n], r.oy[:n], r.dx[:n], r.dy[:n], r.start[:n])
        h, t, s = it[6].cpu().numpy(), it[7].cpu().numpy(), it[8].cpu().numpy()
        assert np.array_equal(h, eh) and np.array_equal(s, es)
        fin = np.isfinite(et)
        assert np.array_equal(np.isfinite(t), fin)
        assert np.all(np.abs(t[fin] - et[fin]) <= 1e-6 * np.abs(et[fin]))


@pytest.mark.parametrize("flags", [0, 1])
def test_batched_equals_oracle(setup, flags):
    cct, tris, scenes, items = setup
    dev_items = _make(items, with_start=True)
    cct.cct_trace_batched(scenes, dev_items, flags=flags)
    torch.cuda.synchronize()
    _check(setup, dev_items)


def test_batch_tunings_and_graph_replay(setup):
    cct, tris, scenes, items = setup
    b = cct.Batch(scenes, max_items=64)
    for tu in ({"block_threads": 64, "refill_min": 1, "chunk": 32}, {"block_threads": 512, "refill_min": 16,
                                                                     "chunk": 1024}):
        b.set_tuning(tu)
        dev_items = _make(items, with_start=False)
        b.stage(dev_items)
        b.enqueue()
        torch.cuda.synchronize()
        _check(setup, dev_items)
    b.set_tuning(None)
    first = _make(items, with_start=True)
    b.stage(first)
    b.capture()
    torch.cuda.synchronize()
    for rep in range(2):  # replay with a different staged work list each time
        dev_items = _make(items[rep::2], with_start=(rep == 0))
        b.stage(dev_items)
        b.replay()
        torch.cuda.synchronize()
        _check((cct, tris, scenes, items[rep::2]), dev_items)
    st = b.stats()
    assert st["rays"] > 0 and st["invalid_rays"] == 0
    b.free()


def test_batched_scenes_with_two_step_records(setup):
    """Scenes loaded with two-step records (for the path kernel), some of them,
    in one batch: every item equals the oracle, graph replay included."""
    cct, tris, _, items = setup
    scenes2 = [cct.Scene.from_triangulation(t, sg.D, flags=0 if k == 1 else cct.CCT_LOAD_TWO_STEP)
               for k, t in enumerate(tris)]
    for flags in (0, cct.CCT_TRACE_EXACT_ONLY):
        dev_items = _make(items, with_start=True)
        cct.cct_trace_batched(scenes2, dev_items, flags=flags)
        torch.cuda.synchronize()
        _check((cct, tris, scenes2, items), dev_items)
    b = cct.Batch(scenes2, max_items=64, flags=cct.CCT_TRACE_EXACT_ONLY)
    with pytest.raises(cct.CctError):
        cct.Batch(scenes2, max_items=64, flags=cct.CCT_TRACE_ONE_STEP)  # a path-kernel flag
    b.set_tuning({"block_threads": 64, "refill_min": 16, "chunk": 512})
    dev_items = _make(items, with_start=False)
    b.stage(dev_items)
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    _check((cct, tris, scenes2, items), dev_items)
    b.free()
    for sc in scenes2:
        sc.free()


def test_batch_rejects_bad_items(setup):
    cct, tris, scenes, items = setup
    b = cct.Batch(scenes, max_items=2)
    dev_items = _make(items[:3], with_start=False)
    with pytest.raises(cct.CctError):
        b.stage(dev_items)  # more than max_items
    bad = list(dev_items[0])
    bad[0] = 99
    with pytest.raises(cct.CctError):
        b.stage([tuple(bad)])
    b.free()
