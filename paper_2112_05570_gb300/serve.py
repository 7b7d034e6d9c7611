"""Continuous-batching request server over device-resident scenes.

Host orchestration of the batched walk (cct_batch_*, include/cct.h): no
counterpart in the paper, whose Sec. 5 traces rays one query at a time.

Requests (scene, n rays) arrive on an open-loop schedule.  Each tick:
  1. arrivals join the pending queue;
  2. admission: pending requests are admitted in arrival order while the
     device-memory budget (28 bytes per ray: rays in, results out) has room --
     the budget is one device buffer handed out as a ring (DeviceArena), so
     admitting a request calls no allocator; admitted rays are copied to the
     device on the upload stream, in rounds of up to 2^24 rays that share one
     completion event;
  3. uploaded rounds (up to 2^25 rays) form this tick's work list, staged
     into a free one of three cct_batch objects and launched by replaying that
     batch's captured CUDA graph on the compute stream -- requests that arrive
     while others are on the GPU are admitted into later ticks, so work from
     different ticks overlaps on the device;
  4. finished ticks copy their results back on the download stream (uploads
     and downloads run on separate copy engines, both overlapping the walks);
     a request is done when its results are on the host, and its block returns
     to the arena.
Latency of a request = its results on the host - its arrival.  The same loop
with one plain cct_trace launch per request gives the unbatched comparison.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import cct

BYTES_PER_RAY = 28  # ox, oy, dx, dy (16 B) + hit, t, steps (12 B)


@dataclass
class Request:
    rid: int
    scene: int
    n: int
    arrival: float          # seconds, relative to the start of the run
    src: list               # pinned host slices of the scene's pool (wrapping around): ((k, 4) records, (4, k) arrays)
    out: object = None      # pinned host (3, n) view: hit, t bits, steps, filled on completion
    admitted: float = -1.0
    done: float = -1.0
    dev: object = None      # device int32 buffer of 7 n words while in flight: rays (n, 4), then results (3, n)
    blk: object = None      # its block of the server's memory arena while in flight
    upload: object = None   # CUDA event: rays on the device
    tick: int = -1
    pool_lo: int = 0        # index of the request's first ray in its scene's pool (the rays wrap around it)
    ranges: list = None     # its pieces of the pool: (first ray, count), wrapping around


@dataclass
class ServeResult:
    completed: int
    offered: int
    rays_completed: int
    wall_s: float
    latency_s: np.ndarray = field(repr=False)
    queue_depth_end: int = 0
    ticks: int = 0

    @property
    def p50_ms(self):
        return float(np.percentile(self.latency_s, 50) * 1e3) if self.latency_s.size else float("nan")

    @property
    def p99_ms(self):
        return float(np.percentile(self.latency_s, 99) * 1e3) if self.latency_s.size else float("nan")

    @property
    def rays_per_s(self):
        return self.rays_completed / self.wall_s if self.wall_s > 0 else 0.0

    def as_dict(self):
        return {"completed": self.completed, "offered": self.offered, "rays_completed": self.rays_completed,
                "wall_s": self.wall_s, "p50_ms": self.p50_ms, "p99_ms": self.p99_ms, "rays_per_s": self.rays_per_s,
                "queue_depth_end": self.queue_depth_end, "ticks": self.ticks}


def poisson_schedule(rate_hz: float, duration_s: float, n_scenes: int, min_rays: int, max_rays: int, seed: int):
    """Open-loop arrivals: exponential gaps of mean 1/rate, a uniform scene and a
    log-uniform ray count per request."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n = int(np.exp(rng.uniform(np.log(min_rays), np.log(max_rays))))
        out.append((t, int(rng.integers(0, n_scenes)), n))
    return out


class RayPool:
    """Per scene, one pinned host pool of rays as interleaved 16-byte records
    (ox, oy, dx bits, dy bits: an (m, 4) int32 array); a request takes
    contiguous slices of it (wrapping around), and its results land in a
    contiguous region of a pinned 1-D result ring (3 n int32: hit, t bits,
    steps)."""

    def __init__(self, rays_per_scene, capacity_out: int):
        import torch

        self.src, self.soa = [], []
        for r in rays_per_scene:
            a = np.stack([r.ox.astype(np.int32), r.oy.astype(np.int32), r.dx.view(np.int32), r.dy.view(np.int32)], 1)
            self.src.append(torch.from_numpy(np.ascontiguousarray(a)).pin_memory())
            # the same rays as four separate arrays (the layout cct_trace takes)
            self.soa.append(torch.from_numpy(np.ascontiguousarray(a.T)).pin_memory())
        self.n = [int(r.ox.shape[0]) for r in rays_per_scene]
        self.src_ptr = [t.data_ptr() for t in self.src]  # 16 bytes per ray
        self.soa_ptr = [t.data_ptr() for t in self.soa]  # 4 rows of n[scene] words
        self.out = torch.empty(3 * capacity_out, dtype=torch.int32).pin_memory()
        self.out_cap = capacity_out
        self.out_pos = 0

    def take(self, scene: int, n: int, rng):
        """n rays of `scene`: a list of (k, 4) pool slices (wrapping around the
        pool when n exceeds it), a (3, n') view of the result ring (n' = n, or
        the ring's capacity if smaller), the first ray's pool index, and the
        pieces as (first ray, count)."""
        m = self.n[scene]
        lo = int(rng.integers(0, m))
        parts, ranges, left, pos = [], [], n, lo
        while left > 0:
            k = min(left, m - pos)
            parts.append((self.src[scene][pos:pos + k], self.soa[scene][:, pos:pos + k]))
            ranges.append((pos, k))
            left -= k
            pos = 0
        n_out = min(n, self.out_cap)
        if self.out_pos + n_out > self.out_cap:
            self.out_pos = 0
        out = self.out[3 * self.out_pos:3 * (self.out_pos + n_out)].view(3, n_out)
        self.out_pos += n_out
        return parts, out, lo, ranges


class DeviceArena:
    """The memory budget as one device buffer of int32 words, handed out as a
    ring: blocks are taken in admission order and come back in (nearly)
    completion order, so a request needs no allocator call.  A block that is
    freed out of order is reclaimed when the blocks before it are."""

    ALIGN = 64  # words: 256-byte aligned blocks

    def __init__(self, torch, words: int):
        self.buf = torch.empty(max(self.ALIGN, int(words)), dtype=torch.int32, device="cuda")
        self.cap = int(self.buf.numel())
        self.head = 0                    # next free word
        self.live = collections.deque()  # [start, size, freed] in allocation order

    def alloc(self, words: int):
        """A block of `words` words (a tensor view), or None while the ring is full."""
        n = -(-int(words) // self.ALIGN) * self.ALIGN
        if n > self.cap:
            raise ValueError(f"a request of {words} words exceeds the memory budget ({self.cap} words)")
        if not self.live:
            self.head = 0
            start = 0
        else:
            tail = self.live[0][0]
            if self.head > tail:  # free: [head, cap) and [0, tail)
                start = self.head if self.cap - self.head >= n else (0 if tail >= n else -1)
            else:  # free: [head, tail)
                start = self.head if tail - self.head >= n else -1
        if start < 0:
            return None
        blk = [start, n, False]
        self.live.append(blk)
        self.head = start + n
        return blk, self.buf[start:start + int(words)]

    def free(self, blk):
        blk[2] = True
        while self.live and self.live[0][2]:
            self.live.popleft()

    def reset(self):
        """Every block back (the caller has synchronised: nothing on the GPU uses them)."""
        self.live.clear()
        self.head = 0


class Server:
    """The continuous-batching loop over loaded cct.Scene objects."""

    ROUND_RAYS = 1 << 24  # rays uploaded between two upload events (one tick takes whole rounds)
    STALL_S = 60.0        # no admission, tick or completion for this long: the loop raises
    TICK_RAYS = 1 << 25   # rays per tick (a burst is cut into ticks that overlap each other's copies)
    TICK_MIN_RAYS = 1 << 22  # while a tick runs, the next starts only with this many rays ready: a
                             # launch has a fixed ramp-up and drain, so many small ticks waste the GPU
    AHEAD_RAYS = 1 << 27     # admitted rays that no tick has taken yet, at most (None: up to the
                             # memory budget).  With every request of a deep queue admitted at once
                             # the upload stream holds gigabytes of copies ahead of the walks and the
                             # whole burst ran at 5.9e9 rays/s (1024 requests of 2^20 rays); a window
                             # of 2^26..2^28 rays: 8.4e9

    def __init__(self, scenes, budget_bytes: int, max_items: int = 4096, flags: int = 0, use_graph: bool = True,
                 tuning: dict | None = None, n_batches: int = 3):
        import torch

        self.torch = torch
        self.scenes = scenes
        self.budget = int(budget_bytes)
        self.flags = flags
        self.max_items = max_items
        self.batches = [cct.Batch(scenes, max_items, flags) for _ in range(n_batches)]
        if tuning:
            for b in self.batches:
                b.set_tuning(tuning)
        # uploads, walks and downloads on three streams: the copy engines move rays in and
        # results out at the same time, both overlapping the walks
        self.compute = torch.cuda.Stream()
        self.h2d = torch.cuda.Stream()
        self.d2h = torch.cuda.Stream()
        self.arena = DeviceArena(torch, self.budget // 4)
        self.use_graph = use_graph
        self._graphs_ready = False

    def _capture(self, probe):
        torch = self.torch
        for b in self.batches:
            b.stage_raw([probe], ray_stride=4)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(self.compute):
                b.enqueue(self.compute)  # warm-up outside capture
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=self.compute):
                b.enqueue()
            b.graph = g
        torch.cuda.synchronize()
        self._graphs_ready = True

    def _alloc(self, n: int):
        return self.torch.empty(7 * n, dtype=self.torch.int32, device="cuda")  # the capture probe only

    @staticmethod
    def _item(r, interleaved: bool = True):
        """(scene, n, ox, oy, dx, dy, start, hit, t, steps) raw addresses of a
        request: the rays (interleaved records, or four arrays), then the three
        result rows."""
        base, res, n = r.dev.data_ptr(), r.dev.data_ptr() + 16 * r.n, r.n
        if interleaved:
            return (r.scene, n, base, base + 4, base + 8, base + 12, 0, res, res + 4 * n, res + 8 * n)
        return (r.scene, n, base, base + 4 * n, base + 8 * n, base + 12 * n, 0, res, res + 4 * n, res + 8 * n)

    def run(self, schedule, pool: RayPool, batched: bool = True, seed: int = 0, drain: bool = True,
            max_wall_s: float | None = None, keep_requests: bool = False):
        """Serves the (arrival, scene, n) schedule; returns a ServeResult (and the
        requests when keep_requests)."""
        torch = self.torch
        rng = np.random.default_rng(seed)
        reqs = []
        for k, (t, sc, n) in enumerate(schedule):
            parts, out, lo, ranges = pool.take(sc, n, rng)
            reqs.append(Request(k, sc, int(n), t, parts, out, pool_lo=lo, ranges=ranges))
        if batched and self.use_graph and not self._graphs_ready and reqs:
            probe = Request(-1, reqs[0].scene, 1, 0.0, [(reqs[0].src[0][0][:1], None)])
            probe.dev = self._alloc(1)
            probe.dev[:4].copy_(probe.src[0][0].reshape(-1))
            self._capture_item = self._item(probe)
            self._capture(self._capture_item)
            self._probe = probe
        for r in reqs:  # a request larger than the whole budget could never be admitted
            if -(-7 * r.n // DeviceArena.ALIGN) * DeviceArena.ALIGN > self.arena.cap:
                raise ValueError(f"request {r.rid}: {r.n} rays exceed the memory budget")
        arena = self.arena
        pending = collections.deque()
        admitted = collections.deque()  # upload rounds: (event, requests)
        ticks_in_flight = collections.deque()  # (event, batch index, requests)
        downloads = collections.deque()  # (event, requests)
        nxt = 0
        done_lat, done_rays = [], 0
        free_batch = [True] * len(self.batches)
        ahead = 0  # rays uploaded or uploading that no tick has taken yet
        tick = 0
        start = time.perf_counter()
        deadline = None if max_wall_s is None else start + max_wall_s
        horizon = schedule[-1][0] if schedule else 0.0
        last_progress = start
        while True:
            now = time.perf_counter() - start
            rounds_before, done_before = len(admitted), len(done_lat)
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            # admission by memory budget, in arrival order: blocks of the arena, uploads in rounds
            if pending:
                while pending:
                    rnd, rays, dst, src, nb = [], 0, [], [], []
                    while pending and len(rnd) < self.max_items and rays < self.ROUND_RAYS:
                        r = pending[0]
                        if self.AHEAD_RAYS is not None and ahead + rays >= self.AHEAD_RAYS:
                            break
                        got = arena.alloc(7 * r.n)
                        if got is None:
                            break
                        pending.popleft()
                        r.blk, r.dev = got
                        r.admitted = now
                        base, off = r.dev.data_ptr(), 0
                        for pos, k in r.ranges:
                            if batched:  # interleaved records: one contiguous piece
                                dst.append(base + 16 * off)
                                src.append(pool.src_ptr[r.scene] + 16 * pos)
                                nb.append(16 * k)
                            else:  # four arrays
                                m = pool.n[r.scene]
                                for q in range(4):
                                    dst.append(base + 4 * (q * r.n + off))
                                    src.append(pool.soa_ptr[r.scene] + 4 * (q * m + pos))
                                    nb.append(4 * k)
                            off += k
                        rnd.append(r)
                        rays += r.n
                    if not rnd:
                        break
                    # the round's copies in one call, then one event for all of them
                    cct.cct_copies_async(dst, src, nb, self.h2d)
                    ev = torch.cuda.Event()
                    ev.record(self.h2d)
                    admitted.append((ev, rnd))
                    ahead += rays
            # completed downloads: the requests are done, their blocks return to the arena
            while downloads and downloads[0][0].query():
                _, rs = downloads.popleft()
                t_done = time.perf_counter() - start
                for r in rs:
                    r.done = t_done
                    done_lat.append(t_done - r.arrival)
                    done_rays += r.n
                    arena.free(r.blk)
                    r.dev = r.blk = None
            # finished ticks -> download their results
            while ticks_in_flight and ticks_in_flight[0][0].query():
                ev, bi, rs = ticks_in_flight.popleft()
                free_batch[bi] = True
                self.d2h.wait_event(ev)
                dst, src, nb = [], [], []
                for r in rs:
                    m, res, out = r.out.shape[1], r.dev.data_ptr() + 16 * r.n, r.out.data_ptr()
                    if m == r.n:  # the three result rows in one piece
                        dst.append(out)
                        src.append(res)
                        nb.append(12 * m)
                    else:  # the ring holds only the first m results of each row
                        for q in range(3):
                            dst.append(out + 4 * q * m)
                            src.append(res + 4 * q * r.n)
                            nb.append(4 * m)
                cct.cct_copies_async(dst, src, nb, self.d2h)
                dev = torch.cuda.Event()
                dev.record(self.d2h)
                downloads.append((dev, rs))
            # a tick: uploaded rounds, on a free batch
            ready = []
            bi = free_batch.index(True) if (batched and True in free_batch) else (0 if not batched else -1)
            if bi >= 0:
                # the uploaded rounds at the front, up to a tick's size
                k, rays, items = 0, 0, 0
                while (k < len(admitted) and admitted[k][0].query() and items + len(admitted[k][1]) <= self.max_items
                       and rays < self.TICK_RAYS):
                    items += len(admitted[k][1])
                    rays += sum(r.n for r in admitted[k][1])
                    k += 1
                if k and (not ticks_in_flight or rays >= self.TICK_MIN_RAYS):
                    for _ in range(k):
                        ready.extend(admitted.popleft()[1])
                    ahead -= rays
            if ready:
                if batched:
                    b = self.batches[bi]
                    b.stage_raw([self._item(r) for r in ready], ray_stride=4)
                    with torch.cuda.stream(self.compute):
                        if self.use_graph:
                            b.graph.replay()
                        else:
                            b.enqueue(self.compute)
                        ev = torch.cuda.Event()
                        ev.record(self.compute)
                    free_batch[bi] = False
                    ticks_in_flight.append((ev, bi, ready))
                    tick += 1
                else:
                    L = cct.lib()
                    sp = cct._stream_ptr(self.compute)
                    with torch.cuda.stream(self.compute):
                        for r in ready:
                            it = [ctypes.c_void_p(x) if x else None for x in self._item(r, interleaved=False)[2:]]
                            rc = L.cct_trace(ctypes.c_void_p(self.scenes[r.scene].handle), *it[:5], r.n, *it[5:],
                                             self.flags, sp)
                            if rc != cct.CCT_OK:
                                raise cct.CctError(rc, "cct_trace")
                        ev = torch.cuda.Event()
                        ev.record(self.compute)
                    ticks_in_flight.append((ev, 0, ready))
                    tick += 1
            finished = nxt >= len(reqs) and not pending and not admitted and not ticks_in_flight and not downloads
            if finished:
                break
            t_now = time.perf_counter()
            if not drain and (t_now - start) > horizon:
                break
            if deadline is not None and t_now > deadline:
                break
            busy = pending or admitted or ticks_in_flight or downloads
            if not busy or ready or rounds_before != len(admitted) or done_before != len(done_lat):
                last_progress = t_now
            elif t_now - last_progress > self.STALL_S:
                torch.cuda.synchronize()
                arena.reset()
                raise RuntimeError(f"serving loop made no progress for {self.STALL_S} s "
                                   f"({len(pending)} pending, {len(admitted)} upload rounds, "
                                   f"{len(ticks_in_flight)} ticks, {len(downloads)} downloads)")
            if not busy:
                # nothing in flight: wait for the next arrival (a short sleep); with work on the
                # GPU the loop keeps polling, so a finished tick is followed at once by the next
                time.sleep(0.0002)
        torch.cuda.synchronize()
        # requests still in flight when the run stopped early (drain=False, max_wall_s) are
        # abandoned: their blocks go back to the arena for the next run
        arena.reset()
        wall = time.perf_counter() - start
        res = ServeResult(len(done_lat), len(reqs), done_rays, wall, np.asarray(done_lat),
                          len(pending) + len(admitted), tick)
        return (res, reqs) if keep_requests else res
