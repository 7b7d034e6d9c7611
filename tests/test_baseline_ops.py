"""Operation counts of the comparison structures, pinned by hand.

The kd-tree and BVH traversals of the oracle (Sec. 5.3.1, 5.3.2, counted as
Sec. 5.4 states) are checked against counts derived by hand on small trees
built directly from arrays (``tests/golden/baseline_op_cases.json``, each case
with its derivation), not by the scene generator's builders.  Planted oracle
mistakes in the counting (a rope search charged for every leaf, floor instead
of ceil of log2, a BVH that opens nodes entered beyond the best hit, a BVH
that ignores the nearer-child order) each fail a case.  The builder's own
rope-count table (``rope_log2``, read by the GPU kernel) is checked against a
brute-force count of the leaves adjacent across each face.  On the GPU the
kernels give the hand-derived counts too.
"""
import json
import os

import numpy as np
import pytest

import oracle
import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "baseline_op_cases.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)


def _kd(c):
    a = lambda k: np.asarray(c[k], np.int32)
    return sg.KdTree(a("axis"), a("split"), a("child"), a("count"), a("box").reshape(-1, 4),
                     a("rope").reshape(-1, 4), a("rope_log2").reshape(-1, 4), a("refs"),
                     a("segs").reshape(-1, 4), 1.0)


def _bvh(c):
    a = lambda k: np.asarray(c[k], np.int32)
    return sg.Bvh(a("box").reshape(-1, 4), a("child0"), a("child1"), a("prims"), a("segs").reshape(-1, 4), 1.0)


def _rays(c):
    o = np.asarray([r["o"] for r in c["rays"]], np.int32)
    k = np.asarray([r["k"] for r in c["rays"]], np.float64)
    d = (k / 2.0 ** 22).astype(np.float32)
    return o[:, 0].copy(), o[:, 1].copy(), d[:, 0].copy(), d[:, 1].copy()


def _expect(c):
    hit = np.asarray([r["hit"] for r in c["rays"]], np.int32)
    t = np.asarray([np.inf if r["t"] is None else r["t"] for r in c["rays"]], np.float32)
    ops = np.asarray([r["ops"] for r in c["rays"]], np.int32)
    return hit, t, ops


def _check(c, got, label):
    hit, t, ops = got
    eh, et, eops = _expect(c)
    for i, r in enumerate(c["rays"]):
        assert hit[i] == eh[i], f"{label} ray {i}: hit {hit[i]} != {eh[i]} ({r['derivation']})"
        assert t[i] == et[i], f"{label} ray {i}: t {t[i]} != {et[i]}"
        assert np.array_equal(ops[i, :eops.shape[1]], eops[i]), f"{label} ray {i}: ops {ops[i]} != {eops[i]}"


def _fails(c, got):
    try:
        _check(c, got, "")
    except AssertionError:
        return True
    return False


def test_golden_cases_are_consistent():
    """The hand-made structures are well formed: child links in range, every
    leaf's box inside its parent's, refs of a leaf touch its box, hits agree
    with brute force over the segments."""
    g = _cases()
    for c in g["kd"]:
        k = _kd(c)
        for n in range(k.n_nodes):
            if k.axis[n] != 2:
                for ch in (k.child[n], k.child[n] + 1):
                    assert 0 < ch < k.n_nodes
                    assert (k.box[ch, :2] >= k.box[n, :2]).all() and (k.box[ch, 2:] <= k.box[n, 2:]).all()
        hb, tb = oracle.closest_bruteforce(k.segs, *_rays(c))
        assert np.array_equal(hb, _expect(c)[0]) and np.array_equal(tb, _expect(c)[1])
    for c in g["bvh"]:
        b = _bvh(c)
        hb, tb = oracle.closest_bruteforce(b.segs, *_rays(c))
        assert np.array_equal(hb, _expect(c)[0]) and np.array_equal(tb, _expect(c)[1])


def test_oracle_kd_counts_equal_hand_derived():
    for c in _cases()["kd"]:
        _check(c, oracle.kd_trace(_kd(c), *_rays(c)), c["name"])


def test_oracle_bvh_counts_equal_hand_derived():
    for c in _cases()["bvh"]:
        _check(c, oracle.bvh_trace(_bvh(c), *_rays(c)), c["name"])


def test_oracle_kd_ignores_the_trees_own_rope_counts():
    """The oracle counts a face's ropes from the node boxes: a wrong rope_log2
    table in the tree changes nothing."""
    for c in _cases()["kd"]:
        k = _kd(c)
        k.rope_log2 = np.full_like(k.rope_log2, 7)
        _check(c, oracle.kd_trace(k, *_rays(c)), c["name"])


@pytest.mark.parametrize("mutant", oracle.KD_MUTANTS)
def test_planted_kd_count_mistakes_fail_a_case(mutant):
    cases = _cases()["kd"]
    assert any(_fails(c, oracle.kd_trace(_kd(c), *_rays(c), mutant=mutant)) for c in cases)


@pytest.mark.parametrize("mutant", oracle.BVH_MUTANTS)
def test_planted_bvh_count_mistakes_fail_a_case(mutant):
    cases = _cases()["bvh"]
    assert any(_fails(c, oracle.bvh_trace(_bvh(c), *_rays(c), mutant=mutant)) for c in cases)


@pytest.mark.parametrize("mutant", oracle.KD_MUTANTS + oracle.BVH_MUTANTS)
def test_planted_count_mistakes_keep_the_hits(mutant):
    """The count mutants change no hit: only the count pins can catch them."""
    segs = sg.random_segments(100, 21)
    tri = sg.cdt(segs)
    r = sg.rays_isotropic(tri, 3000, 22)
    rays = (r.ox, r.oy, r.dx, r.dy)
    hb, tb = oracle.closest_bruteforce(segs, *rays)
    tr = oracle.kd_trace if mutant in oracle.KD_MUTANTS else oracle.bvh_trace
    s = sg.kdtree(segs, 0.5) if mutant in oracle.KD_MUTANTS else sg.bvh(segs, 0.5)
    h, t, ops = tr(s, *rays, mutant=mutant)
    assert np.array_equal(h, hb) and np.array_equal(t, tb)
    _, _, ops0 = tr(s, *rays)
    assert not np.array_equal(ops, ops0)


def _adjacent_leaves_bruteforce(k, L, f):
    a = f // 2
    B = k.box
    plane = B[L, a] if f % 2 == 0 else B[L, 2 + a]
    leaves = np.flatnonzero(k.axis == 2)
    touch = (B[leaves, 2 + a] == plane) if f % 2 == 0 else (B[leaves, a] == plane)
    ov = np.minimum(B[L, 3 - a], B[leaves, 3 - a]) - np.maximum(B[L, 1 - a], B[leaves, 1 - a])
    return int((touch & (ov > 0)).sum())


@pytest.mark.parametrize("lam", [0.25, 1.0])
def test_builder_rope_log2_is_ceil_log2_of_adjacent_leaves(lam):
    """The builder's rope-count table (what the GPU kernel adds per rope) is
    ceil(log2 n) of the leaves adjacent across each face, n counted here by
    brute force over all leaves."""
    segs = sg.random_segments(200, 12)
    k = sg.kdtree(segs, lam)
    for L in np.flatnonzero(k.axis == 2):
        for f in range(4):
            if k.rope[L, f] < 0:
                continue
            n = _adjacent_leaves_bruteforce(k, L, f)
            assert n >= 1
            assert k.rope_log2[L, f] == int(np.ceil(np.log2(n))), (L, f, n)


# ------------------------------------------------------------------------------------------------ GPU
@pytest.mark.gpu
def test_gpu_kernels_give_the_hand_derived_counts():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    g = _cases()
    for kind, cases in (("kd", g["kd"]), ("bvh", g["bvh"])):
        for c in cases:
            host = _kd(c) if kind == "kd" else _bvh(c)
            dev = cct.KdTree(host, 16) if kind == "kd" else cct.Bvh(host)
            d = [torch.from_numpy(a).cuda() for a in _rays(c)]
            h, t, ops = dev.trace(*d)
            torch.cuda.synchronize()
            _check(c, (h.cpu().numpy(), t.cpu().numpy(), ops.cpu().numpy()), f"GPU {c['name']}")
            dev.free()
