"""Autotuner for the walk's launch configuration (cct_tuning, include/cct.h).

No counterpart in the paper.  Knobs: threads per block, the refill threshold
(idle lanes a warp collects before serving new rays), the chunk of rays a warp
takes from the work counter ("rays per warp"), ray binning and its
granularity, where start cells are found when none are given (inside the walk
kernel, or by a separate locate kernel first), the side test (fp32-filtered vs
exact int64), and on small scenes the half-edge table staged in shared memory.  Coordinate
descent from the defaults: each knob in turn takes the value with the lowest
median CUDA-event time on a ray sample, others fixed; two passes.  Results are
cached per (GPU, triangle-count class, ray-count class, start cells given)
in a JSON file next to this module.
"""
from __future__ import annotations

import json
import math
import os

from . import cct

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning_cache.json")

KNOBS = {
    "block_threads": (64, 128, 256, 512),
    "refill_min": (4, 8, 16, 24, 32),
    "chunk": (64, 128, 512, 2048),
    "path": ("plain", "split", "bin", "bin-coarse", "bin-fine"),
    "exact": (0, 1),
}
# the half-edge table staged in shared memory (CCT_TRACE_STAGE) is tried on scenes up to this size
STAGE_MAX_TRI = 1000


def _key(n_tri: int, n_rays: int, has_start: bool) -> str:
    import torch

    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|tri2^{int(math.log2(max(1, n_tri)))}|rays2^{int(math.log2(max(1, n_rays)))}|start{int(has_start)}"


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _to_tuning(cfg: dict, n_tri: int, n_rays: int) -> dict:
    flags = cct.CCT_TRACE_EXACT_ONLY if cfg["exact"] else 0
    if cfg.get("stage"):
        flags |= cct.CCT_TRACE_STAGE
    shift = -1
    if cfg["path"] == "split":
        flags |= cct.CCT_TRACE_SPLIT_LOCATE
    elif cfg["path"] != "plain":
        flags |= cct.CCT_TRACE_BIN
        target = max(1024, n_rays // 64)
        auto = 0
        while (n_tri >> auto) > target and auto < 30:
            auto += 1
        shift = {"bin": auto, "bin-coarse": min(30, auto + 3), "bin-fine": max(0, auto - 3)}[cfg["path"]]
    return {"block_threads": cfg["block_threads"], "refill_min": cfg["refill_min"], "chunk": cfg["chunk"],
            "bin_shift": shift, "trace_flags": flags}


def tune_scene(scene: "cct.Scene", ox, oy, dx, dy, start=None, reps: int = 3, passes: int = 2,
               use_cache: bool = True, apply: bool = True) -> dict:
    """Tunes `scene` for rays like (ox, oy, dx, dy[, start]) (device tensors, a
    representative sample).  Sets the scene's tuning when `apply`; returns
    {"tuning": ..., "ms": best time, "tried": {...}}."""
    import torch

    n = ox.numel()
    key = _key(scene.n_tri, n, start is not None)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        if apply:
            scene.set_tuning(cache[key]["tuning"])
        return cache[key]
    hit = torch.empty(n, dtype=torch.int32, device=ox.device)
    t = torch.empty(n, dtype=torch.float32, device=ox.device)
    steps = torch.empty(n, dtype=torch.int32, device=ox.device)
    stream = torch.cuda.current_stream()

    def time_cfg(cfg):
        scene.set_tuning(_to_tuning(cfg, scene.n_tri, n))
        cct.cct_trace(scene.handle, ox, oy, dx, dy, start, hit, t, steps, 0, stream)  # warm-up
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cct.cct_trace(scene.handle, ox, oy, dx, dy, start, hit, t, steps, 0, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return sorted(times)[len(times) // 2]

    cfg = {"block_threads": 256, "refill_min": 8, "chunk": 128, "path": "plain", "exact": 0, "stage": 0}
    knobs = dict(KNOBS, stage=(0, 1)) if scene.n_tri <= STAGE_MAX_TRI else KNOBS
    tried = {}
    best_ms = time_cfg(cfg)
    tried[json.dumps(cfg, sort_keys=True)] = best_ms
    for _ in range(passes):
        for knob, values in knobs.items():
            for v in values:
                if v == cfg[knob]:
                    continue
                c = dict(cfg, **{knob: v})
                k = json.dumps(c, sort_keys=True)
                ms = tried[k] if k in tried else time_cfg(c)
                tried[k] = ms
                if ms < best_ms:
                    best_ms, cfg = ms, c
    tuning = _to_tuning(cfg, scene.n_tri, n)
    out = {"tuning": tuning, "config": cfg, "ms": best_ms, "rays": n, "n_tried": len(tried)}
    if apply:
        scene.set_tuning(tuning)
    else:
        scene.set_tuning(None)
    if use_cache:
        cache = _load_cache()
        cache[key] = out
        _save_cache(cache)
    return out


def tune_batch(batch: "cct.Batch", items, reps: int = 3) -> dict:
    """Tunes a multi-scene batch (block size, refill threshold, chunk) on a
    staged work list; leaves the best tuning set."""
    import torch

    stream = torch.cuda.current_stream()
    best, best_ms, tried = None, float("inf"), {}
    for bt in KNOBS["block_threads"]:
        for rm in (8, 16, 24, 32):
            for ch in KNOBS["chunk"]:
                tu = {"block_threads": bt, "refill_min": rm, "chunk": ch}
                batch.set_tuning(tu)
                batch.stage(items)
                batch.enqueue(stream)
                times = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    batch.enqueue(stream)
                    e1.record(stream)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = sorted(times)[len(times) // 2]
                tried[json.dumps(tu, sort_keys=True)] = ms
                if ms < best_ms:
                    best, best_ms = tu, ms
    batch.set_tuning(best)
    batch.stage(items)
    return {"tuning": best, "ms": best_ms, "n_tried": len(tried)}
