import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def D():
    import scenegen

    return scenegen.D


def lattice_triangulation(n: int = 12, step: int = 4):
    """Hand-made triangulation of [0, n step]^2: n x n squares of side `step`,
    each cut by a diagonal (alternating direction), a band of diagonals and a
    horizontal run of edges constrained (one segment each).  Vertices at
    multiples of `step` put many integer points on edges and on lines through
    vertices: the degenerate cases of point location."""
    import types

    import numpy as np

    D = n * step
    vid = lambda i, j: j * (n + 1) + i  # noqa: E731
    vx = np.array([i * step for j in range(n + 1) for i in range(n + 1)], np.int32)
    vy = np.array([j * step for j in range(n + 1) for i in range(n + 1)], np.int32)
    tris = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris += [(a, b, c), (a, c, d)] if (i + j) % 2 == 0 else [(a, b, d), (b, c, d)]
    tv = np.array(tris, np.int32)
    edge = {}
    for t in range(len(tv)):
        for k in range(3):
            edge[(int(tv[t, (k + 1) % 3]), int(tv[t, (k + 2) % 3]))] = (t, k)
    nb = -np.ones_like(tv)
    seg = -np.ones_like(tv)
    seg_id, segs = {}, []
    for (u, v), (t, k) in edge.items():
        if (v, u) in edge:
            nb[t, k] = edge[(v, u)][0]
        x0, y0, x1, y1 = int(vx[u]), int(vy[u]), int(vx[v]), int(vy[v])
        i0, j0 = min(x0, x1) // step, min(y0, y1) // step
        diag = x0 != x1 and y0 != y1 and i0 % 3 == 1 and j0 % 2 == 0
        run = y0 == y1 == D // 2 and max(x0, x1) <= D - 2 * step
        if diag or run:
            key = (min(u, v), max(u, v))
            if key not in seg_id:
                seg_id[key] = len(segs)
                segs.append((int(vx[key[0]]), int(vy[key[0]]), int(vx[key[1]]), int(vy[key[1]])))
            seg[t, k] = seg_id[key]
    return types.SimpleNamespace(vx=vx, vy=vy, tri_v=tv, tri_nb=nb, tri_seg=seg,
                                 segs=np.array(segs, np.int32).reshape(-1, 4), D=D)


@pytest.fixture(scope="session")
def lattice():
    return lattice_triangulation
