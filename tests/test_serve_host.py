"""Host logic of the serving loop, without a GPU: the memory arena that
stands for the device-memory budget (a ring of blocks taken in admission
order and returned in completion order)."""
import pytest

from paper_2112_05570_gb300 import serve


class _FakeTorch:
    """Just enough of torch for DeviceArena: a buffer whose slices are (start, stop)."""
    int32 = None

    @staticmethod
    def empty(n, dtype=None, device=None):
        class Buf:
            def numel(self):
                return n

            def __getitem__(self, sl):
                return (sl.start, sl.stop)

        return Buf()


def _arena(words):
    return serve.DeviceArena(_FakeTorch, words)


def test_blocks_are_aligned_disjoint_and_come_back_in_order():
    a = _arena(1024)
    b1, v1 = a.alloc(300)
    b2, v2 = a.alloc(300)
    b3, v3 = a.alloc(300)
    assert v1 == (0, 300) and v2 == (320, 620) and v3 == (640, 940)  # 64-word aligned starts
    assert a.alloc(200) is None  # full: admission waits
    a.free(b1)
    _, v4 = a.alloc(200)  # wraps into the freed front
    assert v4 == (0, 200)
    assert a.alloc(100) is None  # [256, 320) is too small
    a.free(b3)  # out of order: reclaimed only once b2 is
    assert a.alloc(100) is None
    a.free(b2)
    _, v5 = a.alloc(600)
    assert v5 == (256, 856)


def test_empty_ring_restarts_at_zero_and_oversized_requests_raise():
    a = _arena(1024)
    b, _ = a.alloc(1000)
    a.free(b)
    assert a.alloc(1024)[1] == (0, 1024)
    with pytest.raises(ValueError):
        _arena(1024).alloc(1025)


def test_fifo_traffic_never_overlaps():
    """Random sizes, freed in admission order with a lag: live blocks never overlap."""
    import random

    rng = random.Random(3)
    a = _arena(10_000)
    live = []
    for _ in range(5000):
        n = rng.randint(1, 3000)
        got = a.alloc(n)
        if got is None:
            a.free(live.pop(0)[0])
            continue
        live.append((got[0], got[1]))
        spans = sorted(v for _, v in live)
        assert all(s1[1] <= s2[0] for s1, s2 in zip(spans, spans[1:]))
        assert all(0 <= s[0] and s[1] <= a.cap for s in spans)
        if len(live) > 4 and rng.random() < 0.5:
            a.free(live.pop(0)[0])


def test_reset_returns_every_block():
    a = _arena(1024)
    a.alloc(500)
    a.alloc(500)
    assert a.alloc(100) is None
    a.reset()  # a run that stopped early gives its abandoned blocks back
    assert a.alloc(1024)[1] == (0, 1024)
