"""Closest-hit ray throughput on one GB300 (and N replicas under torchrun).

Workload (the paper-shaped scenes, Sec. 4 / 6): 30,000-segment scenes of
polygonal circles with 64-1024 sides, annealed triangulation, 2^24 isotropic
rays (origins uniform on the integer grid, angles uniform), start cells found
on the GPU.  One step = the whole query path on one batch: locate (Sec. 5.2)
+ walk (Sec. 5.1) of all 2^24 rays through ``cct_trace``.  Inputs (2^24 rays,
320 MB with results) are larger than L2; the 2 MB triangle table stays
L2-resident across steps as an acceleration structure would.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead (the baseline arm).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SEGMENTS = 30000
N_RAYS = 1 << 24
SCENE_SEED = 2
RAY_SEED = 7
WORKLOAD = "config2-circles-30k-annealed-2^24-isotropic"


def build_workload(n_rays=N_RAYS):
    import scenegen as sg

    segs = sg.circles(N_SEGMENTS, SCENE_SEED)
    cdt = sg.cdt(segs)
    tri = sg.anneal(cdt, SCENE_SEED, sweeps=4)
    rays = sg.rays_isotropic(tri, n_rays, RAY_SEED)
    return segs, cdt, tri, rays


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(tri, rays, seconds_target=4.0, max_rays=1 << 22):
    """Oracle walk (given start cells) on the host cores: rays/s over a bounded sample."""
    import oracle

    threads = os.cpu_count() or 1
    n = 1 << 16
    t0 = time.perf_counter()
    oracle.walk(tri, rays.ox[:n], rays.oy[:n], rays.dx[:n], rays.dy[:n], rays.start[:n], n_threads=threads)
    dt = time.perf_counter() - t0
    n2 = int(min(max_rays, len(rays), max(n, n * seconds_target / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.walk(tri, rays.ox[:n2], rays.oy[:n2], rays.dx[:n2], rays.dy[:n2], rays.start[:n2], n_threads=threads)
    dt = time.perf_counter() - t0
    return n2 / dt, threads, n2, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    segs, cdt, tri, rays = build_workload()
    import oracle

    threads = os.cpu_count() or 1
    sample = 1 << 20
    for _ in range(args.warmup):
        oracle.walk(tri, rays.ox[:4096], rays.oy[:4096], rays.dx[:4096], rays.dy[:4096], rays.start[:4096],
                    n_threads=threads)
    times = []
    for k in range(args.steps):
        lo = (k * sample) % (len(rays) - sample + 1)
        sl = slice(lo, lo + sample)
        t0 = time.perf_counter()
        oracle.walk(tri, rays.ox[sl], rays.oy[sl], rays.dx[sl], rays.dy[sl], rays.start[sl], n_threads=threads)
        times.append(time.perf_counter() - t0)
    value = sample * len(times) / sum(times)
    line = {"impl": "reference", "metric": "closest-hit rays/s", "value": value, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_step": sample, "segments": int(segs.shape[0]),
                       "triangles": tri.n_tri},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": threads, "kind": "oracle",
                             "sample": f"oracle walk from given start cells, {sample} rays per step"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--flags", default="auto", help="auto | plain | bin")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2112_05570_gb300 import _build, cct

    _build.build()
    import scenegen as sg

    segs, cdt, tri, rays = build_workload()
    scene = cct.Scene.from_triangulation(tri, sg.D)
    n = len(rays)
    ox, oy = torch.from_numpy(rays.ox).to(dev), torch.from_numpy(rays.oy).to(dev)
    dx, dy = torch.from_numpy(rays.dx).to(dev), torch.from_numpy(rays.dy).to(dev)
    start = torch.from_numpy(rays.start).to(dev)
    hit = torch.empty(n, dtype=torch.int32, device=dev)
    t = torch.empty(n, dtype=torch.float32, device=dev)
    steps = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(flags):
        cct.cct_trace(scene.handle, ox, oy, dx, dy, None, hit, t, steps, flags, stream)

    # path choice: plain vs binned (a short measurement; "auto" keeps the faster)
    def time_loop(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    choice = {"plain": 0, "bin": cct.CCT_TRACE_BIN}
    if args.flags == "auto":
        for f in choice.values():
            step(f)
        tried = {k: time_loop(lambda f=f: step(f), 3) for k, f in choice.items()}
        path = min(tried, key=tried.get)
    else:
        path, tried = args.flags, {}
    flags = choice[path]
    kernels_per_step = 2 + (5 if flags & cct.CCT_TRACE_BIN else 0)

    for _ in range(max(3, args.warmup)):
        step(flags)
    torch.cuda.synchronize(dev)
    scene.stats(reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(flags)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        dist.barrier()
        m = torch.tensor([ms], device=dev)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
        ms = float(m.item())
    stats = scene.stats(reset=True)
    value = n * world / (ms * 1e-3)
    steps_per_ray = stats["steps"] / max(1, stats["rays"])

    # ---- roofline of the dominant kernel (the walk), start cells given
    torch.cuda.synchronize(dev)
    for _ in range(3):
        cct.cct_trace(scene.handle, ox, oy, dx, dy, start, hit, t, steps, 0, stream)
    k_rep = max(5, args.steps // 2)
    walk_ms = time_loop(lambda: cct.cct_trace(scene.handle, ox, oy, dx, dy, start, hit, t, steps, 0, stream), k_rep)
    st_walk = scene.stats(reset=True)
    walk_steps = st_walk["steps"] / (k_rep + 3)  # steps per launch (warm-up launches included in the counters)
    alg_bytes = walk_steps * 32.0 + n * 32.0
    achieved_gbs = alg_bytes / (walk_ms * 1e-3) / 1e9
    table_bytes = tri.n_tri * 32
    _, l2_bps = cct.cct_measure_gather(table_bytes, 1 << 27, 5, stream)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = None
    if os.path.exists(peaks_path):
        hbm_peak = json.load(open(peaks_path)).get("hbm_gbs")
    hbm_src = "MEASURED_PEAKS.json" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    l2_peak = l2_bps / 1e9
    roofline = {"bound": "l2", "achieved": achieved_gbs, "peak": l2_peak, "unit": "GB/s",
                "frac": achieved_gbs / l2_peak, "traffic": None,
                "kernel": "walk_kernel (start cells given)",
                "peak_source": f"measured in this run: random 32-byte sector gathers over a {table_bytes} B table "
                               "(cct_measure_gather)",
                "algorithmic_bytes_per_launch": alg_bytes,
                "ms_per_launch": walk_ms,
                "hbm": {"peak": hbm_peak, "frac": achieved_gbs / hbm_peak, "source": hbm_src}}

    # ---- end to end through the public API with host buffers
    pin = {k: torch.from_numpy(getattr(rays, k)).pin_memory() for k in ("ox", "oy", "dx", "dy")}
    out_h = (torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory(),
             torch.empty(n, dtype=torch.int32).pin_memory())

    def e2e_step():
        dox = pin["ox"].to(dev, non_blocking=True)
        doy = pin["oy"].to(dev, non_blocking=True)
        ddx = pin["dx"].to(dev, non_blocking=True)
        ddy = pin["dy"].to(dev, non_blocking=True)
        cct.cct_trace(scene.handle, dox, doy, ddx, ddy, None, hit, t, steps, flags, stream)
        out_h[0].copy_(hit, non_blocking=True)
        out_h[1].copy_(t, non_blocking=True)
        out_h[2].copy_(steps, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
    k_e2e = max(3, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / k_e2e
    e2e = {"value": n * world / e2e_s, "unit": "rays/s", "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 12 * n}

    line = {"metric": "closest-hit rays/s", "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64+fp32-filter", "data": "synthetic",
            "config": {"workload": WORKLOAD, "segments": int(segs.shape[0]), "triangles": tri.n_tri,
                       "rays_per_step": n, "path": path, "path_ms_tried": tried,
                       "l2": "inputs larger than L2 (rays + results 512 MB); triangle table L2-resident",
                       "parallelism": f"replicas x{world}"},
            "steps_per_ray": steps_per_ray,
            "fallback_rate": stats["exact_fallbacks"] / max(1, stats["side_tests"]),
            "locate_steps_per_ray": stats["locate_steps"] / max(1, stats["located"]),
            "roofline": roofline, "e2e": e2e, "gpu_launches": kernels_per_step * args.steps}
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, sample_n, dt = cpu_oracle_rate(tri, rays)
        line["cpu_baseline"] = {"value": rate, "unit": "rays/s", "cores": cores, "kind": "oracle",
                                "sample": f"oracle walk from given start cells over the first {sample_n} rays "
                                          f"({dt:.1f} s wall)"}
    if rank == 0:
        line["clocks"] = clk.summary()
        print(json.dumps(line))
    scene.free()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
