"""cct_trace_noalloc, the entry point for callers that cannot allocate device
memory during a query (a process whose memory is reserved by its own pool, a
latency-critical loop that must not enter an allocator): through the C ABI it
must give the same results as cct_trace, call after call, although all calls
share one static scratch array.  Collected last on purpose (file name)."""
import ctypes

import numpy as np
import pytest

import oracle
import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cct():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct as c

    _build.build()
    return c


def _p(x):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def test_noalloc_matches_cct_trace_two_calls_in_a_row(cct):
    segs = sg.random_segments(200, 31)
    tri = sg.anneal(sg.cdt(segs), 31)
    n = 300_001  # ragged; below CCT_NOALLOC_MAX_RAYS
    r = sg.rays_isotropic(tri, n, 32)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    dev = torch.device("cuda")
    ox, oy = torch.from_numpy(r.ox).to(dev), torch.from_numpy(r.oy).to(dev)
    dx, dy = torch.from_numpy(r.dx).to(dev), torch.from_numpy(r.dy).to(dev)
    start = torch.from_numpy(r.start).to(dev)
    L = cct.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for start_arg in (None, start):
        ref = scene.trace(ox, oy, dx, dy, start_arg)
        torch.cuda.synchronize()
        ref = tuple(x.cpu().numpy() for x in ref)
        for call in range(2):
            hit = torch.full((n,), -7, dtype=torch.int32, device=dev)
            t = torch.full((n,), -7.0, dtype=torch.float32, device=dev)
            steps = torch.full((n,), -7, dtype=torch.int32, device=dev)
            rc = L.cct_trace_noalloc(ctypes.c_void_p(scene.handle), _p(ox), _p(oy), _p(dx), _p(dy), _p(start_arg),
                                     n, _p(hit), _p(t), _p(steps), 0, stream)
            assert rc == cct.CCT_OK, cct.cct_error_string(rc)
            torch.cuda.synchronize()
            h, tt, s = hit.cpu().numpy(), t.cpu().numpy(), steps.cpu().numpy()
            assert np.array_equal(h, ref[0]), f"call {call}: hit ids differ"
            assert np.array_equal(s, ref[2]), f"call {call}: steps differ"
            fin = np.isfinite(ref[1])
            assert np.array_equal(np.isfinite(tt), fin)
            rel = np.abs(tt[fin].astype(np.float64) - ref[1][fin]) / np.abs(ref[1][fin].astype(np.float64))
            assert rel.max() <= 1e-6
    # and both equal the oracle
    eh, et, es = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    assert np.array_equal(h, eh) and np.array_equal(s, es)
    scene.free()


def test_noalloc_rejects_sizes_beyond_its_limit(cct):
    tri = sg.cdt(sg.random_segments(50, 33))
    scene = cct.Scene.from_triangulation(tri, sg.D)
    L = cct.lib()
    dev = torch.device("cuda")
    big = cct.CCT_NOALLOC_MAX_RAYS + 1
    bi = torch.zeros(big, dtype=torch.int32, device=dev)
    bf = torch.zeros(big, dtype=torch.float32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.cct_trace_noalloc(ctypes.c_void_p(scene.handle), _p(bi), _p(bi), _p(bf), _p(bf), None, big, _p(bi),
                             _p(bf), _p(bi), 0, stream)
    assert rc == cct.CCT_ERR_INVALID_ARGUMENT
    rc = L.cct_trace_noalloc(ctypes.c_void_p(scene.handle), _p(bi), _p(bi), _p(bf), _p(bf), None, 16, _p(bi),
                             _p(bf), _p(bi), cct.CCT_TRACE_BIN, stream)
    assert rc == cct.CCT_ERR_INVALID_ARGUMENT
    scene.free()


def test_noalloc_follows_the_scenes_tuning(cct):
    """The scene's launch configuration and predicate choice apply to the
    allocation-free call as to cct_trace: under an exact-only tuning it takes
    no int64 fallbacks of the fp32 filter (there is no filter), and its
    results still equal cct_trace's, located and with start cells."""
    segs = sg.random_segments(200, 35)
    tri = sg.anneal(sg.cdt(segs), 35)
    n = 100_003
    r = sg.rays_isotropic(tri, n, 36)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    dev = torch.device("cuda")
    ox, oy = torch.from_numpy(r.ox).to(dev), torch.from_numpy(r.oy).to(dev)
    dx, dy = torch.from_numpy(r.dx).to(dev), torch.from_numpy(r.dy).to(dev)
    start = torch.from_numpy(r.start).to(dev)
    L = cct.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for tune in ({"block_threads": 64, "refill_min": 16, "chunk": 512, "trace_flags": cct.CCT_TRACE_EXACT_ONLY},
                 {"block_threads": 128, "refill_min": 24, "chunk": 256,
                  "trace_flags": cct.CCT_TRACE_EXACT_ONLY | cct.CCT_TRACE_SPLIT_LOCATE | cct.CCT_TRACE_BIN}):
        scene.set_tuning(tune)
        for start_arg in (None, start):
            ref = tuple(x.cpu().numpy() for x in scene.trace(ox, oy, dx, dy, start_arg))
            scene.stats(reset=True)
            hit = torch.empty(n, dtype=torch.int32, device=dev)
            t = torch.empty(n, dtype=torch.float32, device=dev)
            steps = torch.empty(n, dtype=torch.int32, device=dev)
            rc = L.cct_trace_noalloc(ctypes.c_void_p(scene.handle), _p(ox), _p(oy), _p(dx), _p(dy), _p(start_arg),
                                     n, _p(hit), _p(t), _p(steps), 0, stream)
            assert rc == cct.CCT_OK, cct.cct_error_string(rc)
            torch.cuda.synchronize()
            st = scene.stats(reset=True)
            assert st["rays"] == n and st["side_tests"] > 0 and st["exact_fallbacks"] == 0
            assert np.array_equal(hit.cpu().numpy(), ref[0]) and np.array_equal(steps.cpu().numpy(), ref[2])
            assert np.array_equal(t.cpu().numpy(), ref[1])
    scene.free()


def test_noalloc_on_two_step_records(cct):
    """On a scene loaded with two-step records (which only the path kernel
    reads) the allocation-free entry point gives the oracle's results as
    cct_trace does (fused and split locate, start cells given)."""
    tri = sg.anneal(sg.cdt(sg.random_segments(300, 35)), 35)
    n = 200_003
    r = sg.rays_isotropic(tri, n, 36)
    scene = cct.Scene.from_triangulation(tri, sg.D, flags=cct.CCT_LOAD_TWO_STEP)
    dev = torch.device("cuda")
    ox, oy = torch.from_numpy(r.ox).to(dev), torch.from_numpy(r.oy).to(dev)
    dx, dy = torch.from_numpy(r.dx).to(dev), torch.from_numpy(r.dy).to(dev)
    start = torch.from_numpy(r.start).to(dev)
    L = cct.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    eh, et, es = oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start)
    for start_arg, flags in ((None, 0), (None, cct.CCT_TRACE_SPLIT_LOCATE), (start, cct.CCT_TRACE_EXACT_ONLY)):
        hit = torch.full((n,), -7, dtype=torch.int32, device=dev)
        t = torch.full((n,), -7.0, dtype=torch.float32, device=dev)
        steps = torch.full((n,), -7, dtype=torch.int32, device=dev)
        rc = L.cct_trace_noalloc(ctypes.c_void_p(scene.handle), _p(ox), _p(oy), _p(dx), _p(dy), _p(start_arg), n,
                                 _p(hit), _p(t), _p(steps), flags, stream)
        assert rc == cct.CCT_OK, cct.cct_error_string(rc)
        torch.cuda.synchronize()
        h, tt, s = hit.cpu().numpy(), t.cpu().numpy(), steps.cpu().numpy()
        assert np.array_equal(h, eh) and np.array_equal(s, es), flags
        fin = np.isfinite(et)
        assert np.array_equal(np.isfinite(tt), fin)
        assert np.all(np.abs(tt[fin].astype(np.float64) - et[fin]) <= 1e-6 * np.abs(et[fin].astype(np.float64)))
    scene.free()
