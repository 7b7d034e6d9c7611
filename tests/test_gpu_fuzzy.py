"""The walk on the fuzzy-contraction optimiser's triangulations.

The paper's own optimiser (fuzzy contraction, Sec. 2.2, 3.3, 3.4, and the full
pipeline of Sec. 3.5.3 with its 1 -> 4 subdivision round) produces topologies
the discrete optimiser does not: subdivided and partly re-contracted edges,
Steiner vertices moved along segments, contracted groups.  On four scene
families the GPU walk (start cells given, and located by the fused seed walk;
fp32-filtered and exact-only predicates) equals the oracle on every output:
hit ids and step counts exactly, t within 1e-6 relative, including rays aimed
at vertices and along edges.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import scenegen as sg
from test_oracle import _degenerate_rays

torch = pytest.importorskip("torch")

CASES = (("random200", lambda: sg.random_segments(200, 41)), ("clustered1k", lambda: sg.clustered(1000, 42)),
         ("circles1k", lambda: sg.circles(1000, 43)), ("dash45_1k", lambda: sg.dash_grid(1000, 45.0)))


@pytest.fixture(scope="module")
def fuzzy_tris():
    def one(case):
        name, mk = case
        segs = mk()
        _, tri = sg.fuzzy_pipeline(segs, 44, sweeps=10, polish_sweeps=4, subdivisions=1)
        return name, segs, tri

    with ThreadPoolExecutor(len(CASES)) as ex:
        return list(ex.map(one, CASES))


def test_fuzzy_outputs_are_valid_and_not_longer(fuzzy_tris):
    """CPU: every output is a valid constrained triangulation of its segments
    (all invariants) and no longer than the CDT."""
    for name, segs, tri in fuzzy_tris:
        assert oracle.check_triangulation(tri, sg.D) == 0, name
        assert tri.length(True) <= sg.cdt(segs).length(True) * (1 + 1e-9), name


def _rays(tri, seed):
    r = sg.rays_isotropic(tri, (1 << 17) + 333, seed)  # several chunks and a ragged tail
    ox, oy, dx, dy, _ = _degenerate_rays(tri, 400, seed + 1)
    cat = lambda a, b: np.ascontiguousarray(np.concatenate([a, b]))
    sx, sy = cat(r.ox, ox), cat(r.oy, oy)
    # start cells of the degenerate rays by brute-force location (-1 marks an origin on an edge)
    st = oracle.locate_bruteforce(tri, ox, oy)
    return sx, sy, cat(r.dx, dx), cat(r.dy, dy), cat(r.start, st)


@pytest.mark.gpu
def test_gpu_walk_on_fuzzy_triangulations_equals_oracle(fuzzy_tris):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    import bench

    for k, (name, segs, tri) in enumerate(fuzzy_tris):
        ox, oy, dx, dy, start = _rays(tri, 100 + k)
        ok = start >= 0
        eh, et, es = oracle.walk(tri, ox[ok], oy[ok], dx[ok], dy[ok], start[ok])
        scene = cct.Scene.from_triangulation(tri, sg.D)
        d = [torch.from_numpy(a).cuda() for a in (ox, oy, dx, dy, start)]
        for flags in (0, cct.CCT_TRACE_EXACT_ONLY):
            for given in (True, False):
                h, t, s = scene.trace(*d[:4], d[4] if given else None, flags=flags)
                torch.cuda.synchronize()
                h, t, s = h.cpu().numpy(), t.cpu().numpy(), s.cpu().numpy()
                bad = bench.parity_mismatches(h[ok], t[ok], s[ok], eh, et, es)
                assert not bad, f"{name} flags={flags} given={given}: {bad}"
                # origins on an edge or a vertex are invalid rays, located or given
                assert (s[~ok] == cct.CCT_RAY_INVALID).all() and (h[~ok] == -1).all()
        scene.free()
