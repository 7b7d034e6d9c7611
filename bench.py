"""Closest-hit ray throughput on one GB300 (and N replicas under torchrun).

Workload: the paper-shaped scene families (the lines / floor-plan shapes of
Sec. 4 and 6, rendered as synthetic scenes): polygonal circles with 64-1024
sides, a regular dash grid rotated by 0, 1, 22.5 and 45 degrees (kd-tree
misalignment stress), and Gaussian-clustered random segments -- six scenes of
about 30,000 segments, each with its annealed triangulation and 2^24 isotropic
rays (origins uniform on the integer grid, angles uniform).  One step = the
whole query path on one batch: for every scene, locate (Sec. 5.2) + walk
(Sec. 5.1) of its 2^24 rays, start cells found on the GPU, in one batched
launch over the six scenes (``cct_batch_enqueue`` replayed from a CUDA graph);
the same step as six plain ``cct_trace`` launches is reported beside it.  Inputs (6 x 2^24 rays, 2 GB with results) are larger than L2; the
2-4 MB triangle tables stay L2-resident as acceleration structures do.

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
WORKLOAD = "config2-families-30k-annealed-6x2^24-isotropic"
FAMILIES = ("circles", "dash0", "dash1", "dash22.5", "dash45", "clustered")


def family_segments(name, n=N_SEGMENTS):
    import scenegen as sg

    if name == "circles":
        return sg.circles(n, SCENE_SEED)
    if name == "clustered":
        return sg.clustered(n, SCENE_SEED)
    return sg.dash_grid(n, float(name[4:]))


def build_workload(n_rays=N_RAYS, families=FAMILIES, with_refined=False):
    """[(name, segs, cdt, annealed, rays)] for the scene families (annealed =
    the optimally refined CDT optimised, and optimised again after a 1 -> 4
    subdivision, the shorter kept: scenegen.pipeline); with_refined appends the
    refined CDT to each tuple.  The scenes are built in parallel."""
    import scenegen as sg

    def one(k):
        name = families[k]
        segs = family_segments(name)
        cdt, ref, tri = sg.pipeline(segs, SCENE_SEED + FAMILIES.index(name), sweeps=4)
        rays = sg.rays_isotropic(tri, n_rays, 100 + FAMILIES.index(name))
        return (name, segs, cdt, tri, rays) + ((ref,) if with_refined else ())

    return _parallel(one, range(len(families)), workers=len(families))


FUZZY_SEGMENTS = 3000


def fuzzy_family(k):
    """One scene family at 3000 segments through both optimisers: the bench's
    discrete route (scenegen.pipeline) and the paper's fuzzy contraction
    (Sec. 2.2, 3.3-3.5: scenegen.fuzzy_pipeline, with its 1 -> 4 subdivision
    round).  Returns the triangulations and the CPU seconds of each route."""
    import scenegen as sg

    name = FAMILIES[k]
    segs = family_segments(name, FUZZY_SEGMENTS)
    t0 = time.perf_counter()
    cdt, ref, ann = sg.pipeline(segs, SCENE_SEED + k, sweeps=4)
    t1 = time.perf_counter()
    _, fz = sg.fuzzy_pipeline(segs, SCENE_SEED + k, sweeps=10, polish_sweeps=4, subdivisions=1)
    t2 = time.perf_counter()
    return {"name": name, "segs": segs, "cdt": cdt, "refined": ref, "annealed": ann, "fuzzy": fz,
            "annealed_s": t1 - t0, "fuzzy_s": t2 - t1}


def fuzzy_comparison(torch, cct, sg, built, dev, stream, n_rays=1 << 20):
    """Per family (3000 segments): total interior edge length against the CDT
    and walk steps per ray on the GPU for the CDT, the optimally refined CDT,
    the discrete route and the fuzzy route; the walk's rate on the fuzzy
    triangulation (start cells given, event-timed)."""
    out = {}
    for b in built:
        L = b["cdt"].length(True)
        row = {"segments": int(b["segs"].shape[0]), "annealed_build_s": b["annealed_s"],
               "fuzzy_build_s": b["fuzzy_s"], "annealed_route": getattr(b["annealed"], "route", ""),
               "length_over_cdt": {}, "steps_per_ray": {}, "vertices": {}}
        for kind in ("cdt", "refined", "annealed", "fuzzy"):
            tri = b[kind]
            row["length_over_cdt"][kind] = tri.length(True) / L
            row["vertices"][kind] = int(tri.n_vert)
            r = sg.rays_isotropic(tri, n_rays, 500)
            d = [torch.from_numpy(getattr(r, a)).to(dev) for a in ("ox", "oy", "dx", "dy", "start")]
            sc = cct.Scene.from_triangulation(tri, sg.D)
            sc.trace(*d, stream=stream)
            torch.cuda.synchronize(dev)
            sc.stats(reset=True)
            res = sc.trace(*d, stream=stream)
            torch.cuda.synchronize(dev)
            st = sc.stats(reset=True)
            row["steps_per_ray"][kind] = st["steps"] / max(1, st["rays"])
            if kind == "fuzzy":
                ms = _time_loop(torch, dev, stream, lambda: sc.trace(*d, stream=stream, out=res), 5)
                row["walk_rays_per_s_fuzzy"] = n_rays / (ms * 1e-3)
            sc.free()
        out[b["name"]] = row
    return out


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
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once sampling runs (nvidia-smi takes a moment to start)
            t_end = time.perf_counter() + 5.0
            while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.005)
            self.lines.clear()
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


def cpu_oracle_rate(work, seconds_target=12.0, timed_results=None):
    """Oracle walk (given start cells) on all host cores over a bounded sample:
    the first rays of every scene, sized to take about seconds_target.  With
    timed_results (per scene: hit, t, steps of the timed GPU launch, host
    arrays), the oracle's results on the sample are then compared with them:
    ids and steps exactly, t within 1e-6 relative; a mismatch raises."""
    import oracle

    threads = os.cpu_count() or 1
    n = 1 << 17  # pilot, large enough that thread start-up does not dominate
    t0 = time.perf_counter()
    for w in work:
        tri, r = w[3], w[4]
        oracle.walk(tri, r.ox[:n], r.oy[:n], r.dx[:n], r.dy[:n], r.start[:n], n_threads=threads)
    dt = time.perf_counter() - t0
    n2 = int(min(N_RAYS, max(n, n * seconds_target / max(dt, 1e-6))))
    outs = []
    t0 = time.perf_counter()
    for w in work:
        tri, r = w[3], w[4]
        outs.append(oracle.walk(tri, r.ox[:n2], r.oy[:n2], r.dx[:n2], r.dy[:n2], r.start[:n2], n_threads=threads))
    dt = time.perf_counter() - t0
    checked = 0
    if timed_results is not None:
        for w, (eh, et, es), (h, t, st) in zip(work, outs, timed_results):
            m = min(n2, len(h))
            bad = parity_mismatches(h[:m], t[:m], st[:m], eh[:m], et[:m], es[:m])
            if bad:
                raise RuntimeError(f"timed launch differs from the oracle on scene {w[0]}: {bad}")
            checked += m
    return n2 * len(work) / dt, threads, n2, dt, checked


def parity_mismatches(h, t, st, eh, et, es, rel=1e-6):
    """The walk's parity contract: hit ids and step counts equal, t equal to
    1e-6 relative (both infinite on a miss).  Returns a short description of
    the mismatches, or '' when there are none."""
    out = []
    if not np.array_equal(h, eh):
        out.append(f"{int((h != eh).sum())} hit ids")
    if not np.array_equal(st, es):
        out.append(f"{int((st != es).sum())} step counts")
    fin = np.isfinite(et)
    if not np.array_equal(np.isfinite(t), fin):
        out.append("finiteness of t")
    else:
        dev = np.abs(t[fin].astype(np.float64) - et[fin]) > rel * np.abs(et[fin].astype(np.float64))
        if dev.any():
            out.append(f"{int(dev.sum())} t values beyond {rel} relative")
    return ", ".join(out)


def cpu_oracle_bounce_rate(work, n=1 << 20):
    """Oracle mirror paths (8 bounces, given start cells) on all host cores over
    the first n rays of every scene: walked rays per second."""
    import oracle

    threads = os.cpu_count() or 1
    walked = 0
    t0 = time.perf_counter()
    for w in work:
        tri, r = w[3], w[4]
        p = oracle.bounce_walk(tri, r.ox[:n], r.oy[:n], r.dx[:n], r.dy[:n], r.start[:n], N_BOUNCE, n_threads=threads)
        walked += int((p["steps"] != oracle.BOUNCE_NONE).sum())
    dt = time.perf_counter() - t0
    return walked / dt, threads, n, dt


def job_step_ms(dist, ms: float, device=None) -> float:
    """The job's time per step under N replicas: every rank times its own steps,
    then the slowest rank's time is the job's (barrier + all-reduce MAX; no
    collective touches the ray data).  Without a process group: ms."""
    if dist is None:
        return ms
    import torch

    dist.barrier()
    m = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(m.item())


def job_rays_per_s(rays_per_step_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput of N replicas (weak scaling: every rank walks its own
    full workload per step) over the job's step time."""
    return rays_per_step_per_rank * world / (ms * 1e-3)


def run_reference(args):
    """The baseline arm: the CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    sample = 1 << 18
    work = build_workload(n_rays=sample * max(1, min(args.steps, 4)))
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        for name, segs, cdt, tri, r in work:
            oracle.walk(tri, r.ox[:4096], r.oy[:4096], r.dx[:4096], r.dy[:4096], r.start[:4096], n_threads=threads)
    times = []
    for k in range(args.steps):
        lo = (k * sample) % (len(work[0][4]) - sample + 1)
        sl = slice(lo, lo + sample)
        t0 = time.perf_counter()
        for name, segs, cdt, tri, r in work:
            oracle.walk(tri, r.ox[sl], r.oy[sl], r.dx[sl], r.dy[sl], r.start[sl], n_threads=threads)
        times.append(time.perf_counter() - t0)
    rays_per_step = sample * len(work)
    value = rays_per_step * len(times) / sum(times)
    line = {"impl": "reference", "metric": "closest-hit rays/s", "value": value, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_step": rays_per_step, "families": list(FAMILIES)},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": threads, "kind": "oracle",
                             "sample": f"oracle walk from given start cells, {sample} rays of each of the "
                                       f"{len(work)} scenes per step"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _time_loop(torch, dev, stream, fn, k):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(k):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / k


TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "batch_kernel_six_scenes_dram.md")
TRAFFIC_SOURCES = ("paper_2112_05570_gb300/csrc/batched.cu", "paper_2112_05570_gb300/csrc/cct_internal.cuh",
                   "paper_2112_05570_gb300/csrc/scene.cu")


def kernel_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic():
    """DRAM bytes and L2 sector bytes per launch of the timed step's kernel
    (batch_kernel over the six scenes) from the committed ncu summary, or None
    when the kernel sources changed since that capture."""
    try:
        text = open(TRAFFIC_SUMMARY).read()
    except OSError:
        return None, "no ncu summary", None
    import re

    vals = dict(re.findall(r"^- `(\w+)`: `([^`]+)`", text, flags=re.M))
    try:
        b = float(vals["traffic_bytes_per_launch_mean"])
        sha = vals["sources_sha256"]
    except (KeyError, ValueError):
        return None, "ncu summary unreadable", None
    if sha != kernel_sources_sha256():
        return None, "kernel changed since the ncu capture", None
    l2 = vals.get("l2_sector_bytes_per_launch_mean")
    return (b, "DRAM read+write bytes per launch from " + os.path.basename(TRAFFIC_SUMMARY),
            float(l2) if l2 else None)


TUNE_PARAMS = (0.25, 0.5, 1.0, 2.0, 4.0)


def comparison_structures(torch, cct, sg, sc, dev, stream, n_timed):
    """Sec. 5.3 baselines on the scene's own rays: a BVH and a roped kd-tree per
    cost parameter, the parameter with the fewest measured operations kept
    (the paper's per-scene tuning on the measured rays); then ops/ray and the
    GPU rays/s of the kept structures."""
    d = sc["d"]
    n = d["ox"].numel()
    out = {}
    for kind in ("bvh", "kd"):
        best = None
        for prm in TUNE_PARAMS:
            host = sg.bvh(sc["segs"], prm) if kind == "bvh" else sg.kdtree(sc["segs"], prm)
            g = cct.Bvh(host) if kind == "bvh" else cct.KdTree(host, sg.D)
            h, t, ops = g.trace(d["ox"], d["oy"], d["dx"], d["dy"], stream)
            ops = ops.to(torch.int64)
            if kind == "bvh":
                cost = float(ops.sum()) / n
                detail = {"aabb_per_ray": float(ops[:, 0].sum()) / n, "prim_per_ray": float(ops[:, 1].sum()) / n}
            else:
                cost = float((ops[:, 0] + ops[:, 3] + ops[:, 4]).sum()) / n
                detail = {"leaves_per_ray": float(ops[:, 0].sum()) / n,
                          "unique_prims_per_ray": float(ops[:, 3].sum()) / n,
                          "rope_log2_per_ray": float(ops[:, 4].sum()) / n,
                          "prim_tests_per_ray": float(ops[:, 2].sum()) / n,
                          "descent_nodes_per_ray": float(ops[:, 1].sum()) / n,
                          "mailbox_overflow_rays": int((ops[:, 5] > 0).sum())}
            if best is None or cost < best[0]:
                if best is not None:
                    best[2].free()
                best = (cost, prm, g, detail, host)
            else:
                g.free()
        cost, prm, g, detail, host = best
        ms = _time_loop(torch, dev, stream, lambda: g.trace(d["ox"], d["oy"], d["dx"], d["dy"], stream), n_timed)
        out[kind] = {"ops_per_ray": cost, "param": prm, "rays_per_s": n / (ms * 1e-3),
                     "nodes": int(host.n_nodes), **detail}
        g.free()
    return out


# ---------------------------------------------------------------------------------------------- configs 3-5
N_BOUNCE = 8
N_BOUNCE_RAYS = 1 << 22


def secondary_rays(torch, cct, scenes, dev, stream, gather_bps, k_rep):
    """Mirror paths (cct_trace_bounces: each secondary ray starts in the final
    triangle of its parent's walk, Sec. 5.2) of the first 2^22 rays of each
    scene with up to 8 bounces; event-timed per scene.  The primary records
    are checked against cct_trace's results."""
    out, tot_ms, tot_rays, tot_steps, tot_bytes_over_peak = {}, 0.0, 0, 0, 0.0
    diffuse, d_ms, d_rays, d_steps = {}, 0.0, 0, 0
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    # diffuse bounces: directions cosine-weighted about the normal, given in each hit edge's
    # frame as (c, s) = (sin theta, cos theta), theta = asin(2 u - 1), on the 2^-22 grid
    u = torch.rand((N_BOUNCE, N_BOUNCE_RAYS), generator=gen, device=dev, dtype=torch.float64)
    th = torch.asin(2.0 * u - 1.0)
    frame = torch.stack([torch.round(torch.sin(th) * 2.0 ** 22), torch.round(torch.cos(th) * 2.0 ** 22)], -1)
    frame = (frame / 2.0 ** 22).to(torch.float32).contiguous()
    del u, th
    for sc in scenes:
        d = sc["d"]
        m = N_BOUNCE_RAYS
        args = (d["ox"][:m], d["oy"][:m], d["dx"][:m], d["dy"][:m], N_BOUNCE)
        res = sc["scene"].trace_bounces(*args, start=d["start"][:m], stream=stream, with_rays=False)
        h, _, s_ = sc["scene"].trace(d["ox"][:m], d["oy"][:m], d["dx"][:m], d["dy"][:m], d["start"][:m],
                                     stream=stream)
        torch.cuda.synchronize(dev)
        if not (torch.equal(res["hit"][0], h) and torch.equal(res["steps"][0], s_)):
            raise RuntimeError("primary records of the mirror paths differ from cct_trace")
        full = float((res["steps"][N_BOUNCE] > 0).float().mean())
        sc["scene"].stats(reset=True)
        ms = _time_loop(torch, dev, stream,
                        lambda sc=sc: sc["scene"].trace_bounces(*args, start=d["start"][:m], stream=stream,
                                                                with_rays=False), k_rep)
        st = sc["scene"].stats(reset=True)
        rays, steps = st["rays"] / k_rep, st["steps"] / k_rep
        # 32 B per triangle visited, 20 B per primary ray in, 12 B per record out
        alg = 32.0 * steps + 20.0 * m + 12.0 * m * (N_BOUNCE + 1)
        bps = gather_bps[sc["name"]]
        out[sc["name"]] = {"ms": ms, "walked_rays_per_s": rays / (ms * 1e-3), "steps_per_walked_ray": steps / rays,
                           "walked_rays_per_path": rays / m, "paths_using_every_bounce": full,
                           "gather_frac": alg / (ms * 1e-3) / bps}
        tot_ms += ms
        tot_rays += rays
        tot_steps += steps
        tot_bytes_over_peak += alg / bps
        ms_d = _time_loop(torch, dev, stream,
                          lambda sc=sc: sc["scene"].trace_bounces(*args, start=d["start"][:m], stream=stream,
                                                                  with_rays=False, frame=frame), k_rep)
        st = sc["scene"].stats(reset=True)
        diffuse[sc["name"]] = {"ms": ms_d, "walked_rays_per_s": st["rays"] / k_rep / (ms_d * 1e-3),
                               "steps_per_walked_ray": st["steps"] / max(1, st["rays"])}
        d_ms += ms_d
        d_rays += st["rays"] / k_rep
        d_steps += st["steps"] / k_rep
    return {"n_bounce": N_BOUNCE, "primary_rays_per_scene": N_BOUNCE_RAYS,
            "walked_rays_per_s": tot_rays / (tot_ms * 1e-3), "steps_per_walked_ray": tot_steps / tot_rays,
            "gather_frac": tot_bytes_over_peak / (tot_ms * 1e-3),
            "kernel": "bounce_kernel: one path per lane, exact int64 side tests on 2^-32 origins",
            "diffuse": {"walked_rays_per_s": d_rays / (d_ms * 1e-3), "steps_per_walked_ray": d_steps / d_rays,
                        "directions": "cosine-weighted about the normal, given in each hit edge's frame "
                                      "(d_frame of cct_trace_bounces)", "per_scene": diffuse},
            "reading": "mirror reflection about the hit segment; origin snapped onto the hit edge at a 2^-32 "
                       "parameter; start cell = the parent's final triangle (no locate)",
            "per_scene": out}


def make_roofline(achieved, l2_peak, hbm_peak, hbm_src, traffic, traffic_note, launch_ms, alg_per_launch,
                  l2_bytes=None):
    """The roofline object of the timed kernel (batch_kernel): achieved =
    algorithmic bytes per launch over its event-timed duration (GB/s).  The
    kernel is a dependent gather of 32-byte records from L2-resident tables,
    so its bound is the random-sector gather rate of the L2, measured live over
    tables of the scenes' sizes (cct_measure_gather, byte-weighted over the
    scenes): `peak` and `frac` are against it.  The HBM copy peak and the DRAM
    bytes the kernel actually moves (ncu) are reported beside it."""
    r = {"bound": "l2_gather", "achieved": achieved, "peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
         "traffic": traffic, "traffic_note": traffic_note,
         "peak_source": "measured live: random 32-byte sector gathers over tables of each scene's size "
                        "(cct_measure_gather), weighted by each scene's share of the algorithmic bytes",
         "kernel": "batch_kernel: one launch per step over the six scenes (before it, in the same graph, a "
                   "one-block kernel stages the work table: the step's two launches are timed together)",
         "launch_ms_mean": launch_ms, "algorithmic_bytes_per_launch_mean": alg_per_launch,
         "bytes_model": "32 B per distinct triangle record read (walk steps + locate steps - 1 per ray) + "
                        "4 B seed cell + 28 B per ray (16 B ray in, 12 B result out)",
         "hbm_peak": hbm_peak, "hbm_peak_source": hbm_src, "hbm_frac_of_algorithmic": achieved / hbm_peak,
         "dram_frac": None if traffic is None else traffic / (launch_ms * 1e-3) / 1e9 / hbm_peak,
         "l2_bytes_per_launch": l2_bytes,
         "l2_over_algorithmic": None if l2_bytes is None else l2_bytes / alg_per_launch}
    return r


def _parallel(fn, items, workers=None):
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=workers or (os.cpu_count() or 1)) as ex:
        return list(ex.map(fn, items))


def config4_scenes(n_scenes=512, seed=4, pool_rays=0):
    """512 config-1-generator scenes, segment counts log-uniform over 100-200,000
    (lengths scaled by sqrt(200/N)), annealed (one sweep); rays per scene
    log-uniform over 1k-1M; optional extra ray pools for the server."""
    import scenegen as sg

    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(100), np.log(200_000), n_scenes)).astype(int)
    nr = np.exp(rng.uniform(np.log(1_000), np.log(1_000_000), n_scenes)).astype(int)

    def build(k):
        segs = sg.random_segments(int(ns[k]), 1000 + k)
        tri = sg.anneal(sg.cdt(segs), k, sweeps=1)
        r = sg.rays_isotropic(tri, int(nr[k]), 2000 + k, threads=1)
        pool = sg.rays_isotropic(tri, pool_rays, 3000 + k, threads=1) if pool_rays else None
        return segs, tri, r, pool

    return _parallel(build, range(n_scenes))


def run_config4(args, torch, cct, sg, dev):
    from paper_2112_05570_gb300 import autotune

    t0 = time.perf_counter()
    work = config4_scenes(n_scenes=args.scenes)
    build_s = time.perf_counter() - t0
    scenes = [cct.Scene.from_triangulation(tri, sg.D) for segs, tri, r, _ in work]
    stream = torch.cuda.current_stream(dev)
    items = []
    for k, (segs, tri, r, _) in enumerate(work):
        n = len(r)
        items.append((k, torch.from_numpy(r.ox).to(dev), torch.from_numpy(r.oy).to(dev),
                      torch.from_numpy(r.dx).to(dev), torch.from_numpy(r.dy).to(dev), None,
                      torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.float32, device=dev),
                      torch.empty(n, dtype=torch.int32, device=dev)))
    total = sum(len(w[2]) for w in work)
    if args.profile:
        # profiling mode: the default launch configuration, one warm-up launch
        # and one launch a profiler captures; no timing, no JSON
        b = cct.Batch(scenes, len(items), 0)
        b.stage(items)
        b.enqueue(stream)
        b.enqueue(stream)
        torch.cuda.synchronize(dev)
        b.free()
        return work, scenes, None
    out = {}
    for name, flags in (("filtered", 0), ("exact", cct.CCT_TRACE_EXACT_ONLY)):
        b = cct.Batch(scenes, len(items), flags)
        tune = autotune.tune_batch(b, items)
        b.capture()
        for _ in range(args.warmup):
            b.replay()
        b.stats(reset=True)
        ms = _time_loop(torch, dev, stream, b.replay, args.steps)
        st = b.stats(reset=True)
        out[name] = {"rays_per_s": total / (ms * 1e-3), "ms_per_launch": ms, "tuning": tune["tuning"],
                     "steps_per_ray": st["steps"] / max(1, st["rays"]),
                     "fallback_rate": st["exact_fallbacks"] / max(1, st["side_tests"])}
        b.free()

    def plain():
        for it in items:
            cct.cct_trace(scenes[it[0]].handle, *it[1:5], None, *it[6:9], 0, stream)

    plain()
    ms_plain = _time_loop(torch, dev, stream, plain, max(2, args.steps // 2))
    line = {"metric": "closest-hit rays/s (batched multi-scene)", "value": out["filtered"]["rays_per_s"],
            "unit": "rays/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["filtered"]["ms_per_launch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64+fp32-filter", "data": "synthetic",
            "config": {"workload": "config4-512-scenes-100..200k-segments-1k..1M-rays", "scenes": len(scenes),
                       "segments_total": int(sum(w[0].shape[0] for w in work)),
                       "triangles_total": int(sum(w[1].n_tri for w in work)), "rays_per_step": total,
                       "scene_device_bytes_total": int(sum(sc.info()[0] for sc in scenes)),
                       "build_s": build_s, "launch": "one persistent batched kernel, CUDA-graph replay"},
            "batched": out, "plain_512_launches": {"rays_per_s": total / (ms_plain * 1e-3), "ms": ms_plain},
            "gpu_launches": 2 * args.steps}
    print(json.dumps(line))
    return work, scenes, out


def run_config5(args, torch, cct, sg, dev):
    from paper_2112_05570_gb300 import serve

    t0 = time.perf_counter()
    work = config4_scenes(pool_rays=1 << 18)
    build_s = time.perf_counter() - t0
    scenes = [cct.Scene.from_triangulation(tri, sg.D) for segs, tri, r, pool in work]
    pool = serve.RayPool([w[3] for w in work], capacity_out=1 << 26)
    mean_rays = (4_000_000 - 1_000) / np.log(4_000_000 / 1_000)
    srv = serve.Server(scenes, budget_bytes=60 << 30, max_items=4096)
    # capacity: a saturated burst (requests of 2^20 rays, all arrived at once) through the same
    # server; the longer burst amortises the pipeline's fill (first upload) and drain (last
    # download) and gives the sustained rate
    burst = [(0.0, int(k % len(scenes)), 1 << 20) for k in range(1024)]
    srv.run(burst[:64], pool, batched=True, seed=1)
    runs = {"capacity_burst_256x2^20": srv.run(burst[:256], pool, batched=True, seed=2).as_dict()}
    res_cap = srv.run(burst, pool, batched=True, seed=2)
    runs["capacity_burst_1024x2^20"] = res_cap.as_dict()
    capacity = res_cap.rays_per_s
    # the host loop's own limit: 8000 requests of 1000 rays, all arrived at once
    small = [(0.0, int(k % len(scenes)), 1000) for k in range(8000)]
    res_small = srv.run(small, pool, batched=True, seed=3)
    runs["host_limit_8000x1000"] = dict(res_small.as_dict(), requests_per_s=res_small.completed / res_small.wall_s)
    nominal = serve.poisson_schedule(20_000.0, 2.0, len(scenes), 1_000, 4_000_000, seed=5)
    runs["nominal_20k_req_s"] = srv.run(nominal, pool, batched=True, seed=6, drain=False,
                                        max_wall_s=6.0).as_dict()
    for frac in (0.6, 0.8, 1.0):
        rate = frac * capacity / mean_rays
        sched = serve.poisson_schedule(rate, 3.0, len(scenes), 1_000, 4_000_000, seed=7)
        runs[f"poisson_{frac}_of_capacity"] = dict(srv.run(sched, pool, batched=True, seed=8).as_dict(),
                                                    rate_req_s=rate)
    rate = 0.6 * capacity / mean_rays
    sust = serve.poisson_schedule(rate, 3.0, len(scenes), 1_000, 4_000_000, seed=7)
    runs["sustainable_batched"] = runs["poisson_0.6_of_capacity"]
    runs["sustainable_plain_per_request"] = srv.run(sust, pool, batched=False, seed=8).as_dict()
    r = runs["sustainable_batched"]
    line = {"metric": "p50/p99 request latency (continuous batching)", "value": r["p99_ms"], "unit": "ms",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": r["wall_s"] * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+fp32-filter", "data": "synthetic",
            "config": {"workload": "config5-poisson-512-scenes-1k..4M-rays-60GB", "build_s": build_s,
                       "offered_nominal_rays_per_s": 20_000 * mean_rays, "capacity_rays_per_s": capacity,
                       "sustainable_rate_req_s": rate},
            "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "rays_per_s": r["rays_per_s"], "runs": runs}
    print(json.dumps(line))


def run_config1(args, torch, cct, sg, dev):
    """The tiny plain case: 200 random non-crossing segments (CDT and
    annealed), 65,536 isotropic rays, four seeds; per triangulation the walk
    from given start cells and the fused locate + walk (CUDA events), steps per
    ray; as the CPU baseline, the oracle walk and the all-segment brute force
    timed on the host cores (the brute force is timed here only).  (Their
    parity with the oracle is a test: tests/test_gpu_walk.py.)"""
    import oracle

    n = 1 << 16
    stream = torch.cuda.current_stream(dev)
    hit = torch.empty(n, dtype=torch.int32, device=dev)
    t = torch.empty(n, dtype=torch.float32, device=dev)
    steps = torch.empty(n, dtype=torch.int32, device=dev)
    out = {}
    threads = os.cpu_count() or 1
    for seed in (1, 2, 3, 4):
        segs = sg.random_segments(200, seed)
        cdt, _, ann = sg.pipeline(segs, seed, sweeps=20)
        for kind, tri in (("cdt", cdt), ("annealed", ann)):
            r = sg.rays_isotropic(tri, n, 10 + seed)
            d = [torch.from_numpy(getattr(r, k)).to(dev) for k in ("ox", "oy", "dx", "dy", "start")]
            sc = cct.Scene.from_triangulation(tri, sg.D)
            res = {}
            sc.stats(reset=True)
            for label, st in (("given", d[4]), ("locate", None)):
                fn = lambda st=st: cct.cct_trace(sc.handle, *d[:4], st, hit, t, steps, 0, stream)
                for _ in range(3):
                    fn()
                ms = _time_loop(torch, dev, stream, fn, max(10, args.steps))
                res[f"{label}_rays_per_s"] = n / (ms * 1e-3)
            st = sc.stats(reset=True)
            res.update(steps_per_ray=st["steps"] / max(1, st["rays"]), triangles=tri.n_tri)
            # the CPU baseline: the oracle's walk and brute force, timed
            oracle.walk(tri, r.ox[:1024], r.oy[:1024], r.dx[:1024], r.dy[:1024], r.start[:1024], n_threads=threads)
            t0 = time.perf_counter()
            oracle.walk(tri, r.ox, r.oy, r.dx, r.dy, r.start, n_threads=threads)
            t1 = time.perf_counter()
            oracle.closest_bruteforce(segs, r.ox, r.oy, r.dx, r.dy, n_threads=threads)
            t2 = time.perf_counter()
            res["cpu_baseline"] = {"oracle_walk_rays_per_s": n / (t1 - t0),
                                   "oracle_bruteforce_rays_per_s": n / (t2 - t1), "cores": threads}
            out[f"seed{seed}/{kind}"] = res
            sc.free()
    mean = lambda key, kind: float(np.mean([v[key] for k, v in out.items() if k.endswith(kind)]))
    print(json.dumps({"config": "1: 200 random segments, 65,536 isotropic rays, four seeds", "per_scene": out,
                      "steps_per_ray": {"cdt": mean("steps_per_ray", "cdt"),
                                        "annealed": mean("steps_per_ray", "annealed")},
                      "given_rays_per_s": mean("given_rays_per_s", "annealed"),
                      "locate_rays_per_s": mean("locate_rays_per_s", "annealed"), "cpu_cores": threads,
                      "note": "65,536 rays are a few microseconds of GPU work: the rates are launch-bound"}))
    return 0


def run_config3(args, torch, cct, sg, dev):
    """Ring of circles, N = 1e3 .. 1e6 in a fixed domain; 2^26 isotropic rays and
    4096 pinhole fans of 4096 rays; start cells from the GPU locate."""
    out = {}
    stream = torch.cuda.current_stream(dev)
    for N in (1_000, 10_000, 100_000, 1_000_000):
        t0 = time.perf_counter()
        segs = sg.ring_of_circles(N)
        cdt, ref, tri = sg.pipeline(segs, 3, sweeps=1)
        iso = sg.rays_isotropic(tri, 1 << 26, 11)
        fan = sg.rays_pinhole(tri, 4096, 4096, 12)
        build_s = time.perf_counter() - t0
        scene = cct.Scene.from_triangulation(tri, sg.D)
        res = {"segments": int(segs.shape[0]), "triangles": tri.n_tri, "build_s": build_s,
               "refine_params": list(ref.refine_params), "length_annealed_over_cdt": tri.length(True) / cdt.length(True)}
        for name, r in (("incoherent", iso), ("coherent", fan)):
            n = len(r)
            d = [torch.from_numpy(getattr(r, k)).to(dev) for k in ("ox", "oy", "dx", "dy")]
            h = torch.empty(n, dtype=torch.int32, device=dev)
            t = torch.empty(n, dtype=torch.float32, device=dev)
            s = torch.empty(n, dtype=torch.int32, device=dev)
            for label, flags in (("plain", 0), ("binned", cct.CCT_TRACE_BIN)):
                cct.cct_trace(scene.handle, *d, None, h, t, s, flags, stream)
                scene.stats(reset=True)
                ms = _time_loop(torch, dev, stream, lambda: cct.cct_trace(scene.handle, *d, None, h, t, s, flags,
                                                                           stream), 3)
                st = scene.stats(reset=True)
                res[f"{name}_{label}"] = {"rays": n, "rays_per_s": n / (ms * 1e-3), "ms": ms,
                                          "steps_per_ray": st["steps"] / max(1, st["rays"]),
                                          "locate_steps_per_ray": st["locate_steps"] / max(1, st["located"]),
                                          "invalid": st["invalid_rays"] / 3}
            del d, h, t, s
        scene.free()
        out[str(N)] = res
        torch.cuda.empty_cache()
    line = {"metric": "closest-hit rays/s and steps/ray vs N", "value": out["1000000"]["incoherent_plain"]["rays_per_s"],
            "unit": "rays/s", "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": out["1000000"]["incoherent_plain"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+fp32-filter",
            "data": "synthetic", "config": {"workload": "config3-ring-of-circles-1e3..1e6-2^26-iso-2^24-fans"},
            "by_n": out}
    print(json.dumps(line))


LINES_N = (1, 3, 10, 30, 100, 300, 1000)


def run_lines(args, torch, cct, sg, dev):
    """The `lines' scenes of Sec. 4.2 / 6.1: length factors 0.1, 1, 3 x orientations
    uniform, mostly vertical, mostly diagonal x N = 1..1000 lines, two scenes each;
    2^16 isotropic rays per scene with known start cells (the paper's setting).
    Operations per ray, as in Sec. 5.4: triangles visited by the walk on the
    annealed, optimally refined and unrefined triangulations; BVH AABB + segment
    tests; roped kd-tree leaves + ideal rope steps + distinct segments tested
    (each structure's cost parameter chosen per scene by the fewest operations).
    All on the GPU; the three structures' hit ids are checked equal."""
    stream = torch.cuda.current_stream(dev)
    n_rays = 1 << 16
    table = {}
    t0 = time.perf_counter()
    for factor in (0.1, 1.0, 3.0):
        for orient in ("uniform", "vertical", "diagonal"):
            rows = {}
            for N in LINES_N:
                acc = {"segments": [], "walk": [], "walk_refined": [], "walk_cdt": [], "kd": [], "bvh": [],
                       "kd_leaves": [], "kd_rope": [], "kd_prims": [], "bvh_aabb": [], "bvh_prims": []}
                for rep in range(2):
                    seed = 7000 + 97 * rep + N
                    segs = sg.lines(N, seed, factor, orient)
                    cdt, ref, tri = sg.pipeline(segs, seed, sweeps=4)
                    r = sg.rays_isotropic(tri, n_rays, seed + 1)
                    d = [torch.from_numpy(getattr(r, k)).to(dev) for k in ("ox", "oy", "dx", "dy")]
                    start = torch.from_numpy(r.start).to(dev)
                    hits = []
                    for key, tr in (("walk", tri), ("walk_refined", ref), ("walk_cdt", cdt)):
                        # start cells are caller triangle ids of the triangulation the rays were made for
                        sc = cct.Scene.from_triangulation(tr, sg.D)
                        st = start if tr is tri else None
                        h, _, stp = sc.trace(*d, st)
                        # rays made for the annealed triangulation may start on an edge of the
                        # others (rare; reported invalid there): mean over valid rays
                        stp = stp[stp > 0].to(torch.float64)
                        acc[key].append(float(stp.mean()))
                        if tr is tri:
                            hits.append(h)
                        sc.free()
                    best = {}
                    for kind in ("bvh", "kd"):
                        for prm in TUNE_PARAMS:
                            host = sg.bvh(segs, prm) if kind == "bvh" else sg.kdtree(segs, prm)
                            g = cct.Bvh(host) if kind == "bvh" else cct.KdTree(host, sg.D)
                            h, _, ops = g.trace(*d, stream)
                            ops = ops.to(torch.float64)
                            if kind == "bvh":
                                parts = (float(ops[:, 0].mean()), float(ops[:, 1].mean()))
                            else:
                                parts = (float(ops[:, 0].mean()), float(ops[:, 4].mean()), float(ops[:, 3].mean()))
                            if kind not in best or sum(parts) < sum(best[kind][0]):
                                best[kind] = (parts, h)
                            g.free()
                        hits.append(best[kind][1])
                    if not all(torch.equal(hits[0], h) for h in hits[1:]):
                        raise RuntimeError(f"lines {factor} {orient} {N}: hit ids differ between structures")
                    acc["segments"].append(int(segs.shape[0]))
                    acc["bvh"].append(sum(best["bvh"][0]))
                    acc["bvh_aabb"].append(best["bvh"][0][0])
                    acc["bvh_prims"].append(best["bvh"][0][1])
                    acc["kd"].append(sum(best["kd"][0]))
                    acc["kd_leaves"].append(best["kd"][0][0])
                    acc["kd_rope"].append(best["kd"][0][1])
                    acc["kd_prims"].append(best["kd"][0][2])
                rows[str(N)] = {k: float(np.mean(v)) for k, v in acc.items()}
            table[f"factor{factor:g}/{orient}"] = rows
    line = {"metric": "operations per ray vs N (lines scenes)", "value": None, "unit": "ops/ray",
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "lines-scenes-factor0.1,1,3-uniform,vertical,diagonal-N1..1000-2^16-rays",
                       "rays_per_scene": n_rays, "scenes_per_point": 2, "build_and_trace_s": time.perf_counter() - t0},
            "by_scene": table}
    print(json.dumps(line))


def run_profile_kernels(args, torch, cct, sg, dev):
    """Profiling mode: every kernel of the library on one config-2 scene
    (2^23 isotropic rays, larger than L2 with their results): the locate
    kernel, the binned trace (locate, histogram, three scan passes, scatter,
    sorted walk), the split and fused walks, the kd-tree and BVH baselines,
    a four-item batched launch over the same scene, mirror and diffuse paths
    of 2^21 of the rays with 8 bounces, the mirror paths again on two-step
    records (CCT_LOAD_TWO_STEP), and the gather peak; each twice (warm-up,
    then the launch a profiler captures).
    Prints the CUDA-event time of the second launch of each call and the
    scene's steps per ray."""
    name = args.families.split(",")[0]
    segs = family_segments(name)
    cdt, ref, tri = sg.pipeline(segs, SCENE_SEED + FAMILIES.index(name), sweeps=4)
    n = 1 << 23
    r = sg.rays_isotropic(tri, n, 100 + FAMILIES.index(name))
    d = [torch.from_numpy(getattr(r, k)).to(dev) for k in ("ox", "oy", "dx", "dy")]
    start = torch.from_numpy(r.start).to(dev)
    hit = torch.empty(n, dtype=torch.int32, device=dev)
    t = torch.empty(n, dtype=torch.float32, device=dev)
    steps = torch.empty(n, dtype=torch.int32, device=dev)
    loc = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    scene = cct.Scene.from_triangulation(tri, sg.D)
    scene2 = cct.Scene.from_triangulation(tri, sg.D, flags=cct.CCT_LOAD_TWO_STEP)
    bvh = cct.Bvh(sg.bvh(segs, 1.0))
    kd = cct.KdTree(sg.kdtree(segs, 1.0), sg.D)
    q = n // 4
    items = [(0, d[0][k * q:(k + 1) * q], d[1][k * q:(k + 1) * q], d[2][k * q:(k + 1) * q],
              d[3][k * q:(k + 1) * q], None, hit[k * q:(k + 1) * q], t[k * q:(k + 1) * q], steps[k * q:(k + 1) * q])
             for k in range(4)]
    batch = cct.Batch([scene], max_items=4)
    batch.stage(items)
    nb_rays = 1 << 21  # mirror paths: 2^21 primary rays, up to 8 bounces (9 records each)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    th = torch.asin(2.0 * torch.rand((N_BOUNCE, nb_rays), generator=gen, device=dev, dtype=torch.float64) - 1.0)
    frame = (torch.stack([torch.round(torch.sin(th) * 2.0 ** 22), torch.round(torch.cos(th) * 2.0 ** 22)], -1)
             / 2.0 ** 22).to(torch.float32).contiguous()  # diffuse bounces (cosine-weighted, in the hit edges' frames)
    calls = {
        "locate_kernel": lambda: cct.cct_locate(scene.handle, d[0], d[1], loc, stream),
        "binned_trace": lambda: cct.cct_trace(scene.handle, *d, None, hit, t, steps, cct.CCT_TRACE_BIN, stream),
        "split_trace": lambda: cct.cct_trace(scene.handle, *d, None, hit, t, steps, cct.CCT_TRACE_SPLIT_LOCATE,
                                             stream),
        "fused_trace": lambda: cct.cct_trace(scene.handle, *d, None, hit, t, steps, 0, stream),
        "given_trace": lambda: cct.cct_trace(scene.handle, *d, start, hit, t, steps, 0, stream),
        "kd_trace": lambda: kd.trace(*d, stream),
        "bvh_trace": lambda: bvh.trace(*d, stream),
        "batched_4_items": lambda: batch.enqueue(stream),
        "bounce_8": lambda: scene.trace_bounces(d[0][:nb_rays], d[1][:nb_rays], d[2][:nb_rays], d[3][:nb_rays],
                                                N_BOUNCE, start=start[:nb_rays], stream=stream, with_rays=False),
        "bounce_8_diffuse": lambda: scene.trace_bounces(d[0][:nb_rays], d[1][:nb_rays], d[2][:nb_rays],
                                                        d[3][:nb_rays], N_BOUNCE, start=start[:nb_rays], stream=stream,
                                                        with_rays=False, frame=frame),
        "bounce_8_two_step": lambda: scene2.trace_bounces(d[0][:nb_rays], d[1][:nb_rays], d[2][:nb_rays],
                                                          d[3][:nb_rays], N_BOUNCE, start=start[:nb_rays],
                                                          stream=stream, with_rays=False),
    }
    out = {}
    for label, fn in calls.items():
        fn()
        out[label] = _time_loop(torch, dev, stream, fn, 1)
    ms, bps = cct.cct_measure_gather(tri.n_tri * 32, 1 << 27, 1, stream)
    out["gather_kernel"] = ms
    scene.stats(reset=True)
    cct.cct_trace(scene.handle, *d, start, hit, t, steps, 0, stream)
    st = scene.stats(reset=True)
    print(json.dumps({"profile_kernels_ms": out, "scene": name, "rays": n, "triangles": tri.n_tri,
                      "steps_per_ray": st["steps"] / max(1, st["rays"]), "gather_peak_gbs": bps / 1e9}))
    for o in (batch, bvh, kd, scene, scene2):
        o.free()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--flags", default="auto", help="auto | plain | bin")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fuzzy", action="store_true",
                    help="leave out the optimiser comparison (discrete vs fuzzy contraction, 3000-segment scenes)")
    ap.add_argument("--config", default="2", choices=["1", "2", "3", "4", "5", "lines"],
                    help="2 (default): the six config-2 scene families; 1: the tiny plain case (200 segments, "
                         "65,536 rays, with the oracle's rates); 3: scaling in N; 4: 512 scenes in one "
                         "batched launch; 5: the continuous-batching server; lines: operations per ray vs N on "
                         "the paper's lines scenes (walk, kd-tree, BVH)")
    ap.add_argument("--profile", action="store_true",
                    help="profiling mode: per scene, 2 warm-up traces, then one trace with start cells given and "
                         "one with the fused locate; no timing, no JSON.  With --config 4: one warm-up and one "
                         "profiled batched launch at the default launch configuration")
    ap.add_argument("--seed-densities", default="",
                    help="with --profile: also time the fused locate with these seed-grid densities (k: 2^k cells "
                         "per triangle), e.g. 1,2,3,4")
    ap.add_argument("--profile-step", action="store_true",
                    help="profiling mode: the timed step's batched launch over the six scenes at a fixed "
                         "configuration, twice (warm-up, captured); no timing, no JSON")
    ap.add_argument("--profile-rays", type=int, default=24,
                    help="with --profile-step: 2^k rays per scene (24 is the workload; fewer for captures that "
                         "save and restore device memory many times)")
    ap.add_argument("--scenes", type=int, default=512,
                    help="--config 4: number of scenes (512 is the workload; fewer for profiling runs)")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="profiling mode: every kernel of the library, twice each, on the first of --families "
                         "(2^23 rays); CUDA-event times of the second launches, no JSON bench line")
    ap.add_argument("--families", default=",".join(FAMILIES),
                    help="comma-separated scene families (profiling runs)")
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

    if args.profile_kernels:
        return run_profile_kernels(args, torch, cct, sg, dev)
    if args.config != "2":
        fn = {"1": run_config1, "3": run_config3, "4": run_config4, "5": run_config5, "lines": run_lines}[args.config]
        fn(args, torch, cct, sg, dev)
        return 0
    fams = tuple(f for f in args.families.split(",") if f) if args.profile else FAMILIES
    n_build = min(N_RAYS, 1 << args.profile_rays) if args.profile_step else N_RAYS
    fz_pool, fz_futs = None, []
    if not (args.profile or args.profile_step or args.no_fuzzy):
        # the optimiser comparison's scenes (CPU only) build while the GPU work runs
        from concurrent.futures import ThreadPoolExecutor

        fz_pool = ThreadPoolExecutor(max_workers=len(FAMILIES))
        fz_futs = [fz_pool.submit(fuzzy_family, k) for k in range(len(FAMILIES))]
    work = build_workload(n_rays=n_build, families=fams, with_refined=True)
    stream = torch.cuda.current_stream(dev)
    n = N_RAYS
    hit = torch.empty(n, dtype=torch.int32, device=dev)
    t = torch.empty(n, dtype=torch.float32, device=dev)
    steps = torch.empty(n, dtype=torch.int32, device=dev)
    scenes = []
    for name, segs, cdt, tri, r, ref in work:
        d = {k: torch.from_numpy(getattr(r, k)).to(dev) for k in ("ox", "oy", "dx", "dy", "start")}
        scenes.append(dict(name=name, segs=segs, cdt=cdt, ref=ref, tri=tri, rays=r, d=d,
                           scene=cct.Scene.from_triangulation(tri, sg.D, flags=cct.CCT_LOAD_TWO_STEP)))

    def trace(sc, start, flags, s=None):
        d = sc["d"]
        cct.cct_trace(sc["scene"].handle, d["ox"], d["oy"], d["dx"], d["dy"], start, hit, t, steps, flags,
                      stream if s is None else s)

    if args.profile_step:
        # the timed step's launch at a fixed configuration (exact-only predicates, 64 threads,
        # refill 16, chunk 512): one warm-up and one launch a profiler captures
        m = min(n, 1 << args.profile_rays)
        outs = [(torch.empty(m, dtype=torch.int32, device=dev), torch.empty(m, dtype=torch.float32, device=dev),
                 torch.empty(m, dtype=torch.int32, device=dev)) for _ in scenes]
        items = [(k, sc["d"]["ox"][:m], sc["d"]["oy"][:m], sc["d"]["dx"][:m], sc["d"]["dy"][:m], None, *outs[k])
                 for k, sc in enumerate(scenes)]
        b = cct.Batch([sc["scene"] for sc in scenes], len(items), cct.CCT_TRACE_EXACT_ONLY)
        b.set_tuning({"block_threads": 64, "refill_min": 16, "chunk": 512})
        b.stage(items)
        b.enqueue(stream)
        b.enqueue(stream)
        torch.cuda.synchronize(dev)
        b.free()
        return 0
    if args.profile:
        # per scene: 2 warm-up traces, then start cells given / fused locate, each
        # with the fp32 filter and exact-only; CUDA-event times of 3 more of each
        ex = cct.CCT_TRACE_EXACT_ONLY
        sp = cct.CCT_TRACE_SPLIT_LOCATE
        variants = (("given", "start", 0), ("given_exact", "start", ex), ("locate", None, 0), ("locate_exact", None, ex),
                    ("split", None, sp), ("split_exact", None, sp | ex))
        times = {}
        for sc in scenes:
            for _ in range(2):
                trace(sc, sc["d"]["start"], 0)
            for name, st, fl in variants:
                trace(sc, sc["d"][st] if st else None, fl)
        torch.cuda.synchronize(dev)
        for sc in scenes:
            for name, st, fl in variants:
                times[f"{sc['name']}/{name}"] = _time_loop(
                    torch, dev, stream, lambda st=st, fl=fl: trace(sc, sc["d"][st] if st else None, fl), 3)
        # the locate kernel alone (start cells into a preallocated buffer)
        loc_out = torch.empty(n, dtype=torch.int32, device=dev)
        for sc in scenes:
            d = sc["d"]
            run = lambda d=d, sc=sc: cct.cct_locate(sc["scene"].handle, d["ox"], d["oy"], loc_out, stream)
            run()
            times[f"{sc['name']}/locate_kernel"] = _time_loop(torch, dev, stream, run, 3)
        out = {"profile_ms": times}
        if args.seed_densities:
            # the fused locate under other seed-grid densities (2^k cells per
            # triangle): time and locate steps per origin
            sweep = {}
            for sc in scenes:
                for k in (int(x) for x in args.seed_densities.split(",")):
                    other = cct.Scene.from_triangulation(sc["tri"], sg.D, flags=cct.CCT_LOAD_SEED_DENSITY(k))
                    d = sc["d"]
                    run = lambda other=other, d=d: cct.cct_trace(other.handle, d["ox"], d["oy"], d["dx"], d["dy"],
                                                                None, hit, t, steps, 0, stream)
                    run()
                    other.stats(reset=True)
                    run()
                    torch.cuda.synchronize(dev)
                    st = other.stats()
                    sweep[f"{sc['name']}/k{k}"] = {"ms": _time_loop(torch, dev, stream, run, 3),
                                                   "locate_steps": st["locate_steps"] / max(1, st["located"])}
                    other.free()
            out["seed_density"] = sweep
        print(json.dumps(out))
        return 0

    def step(flags):
        for sc in scenes:
            trace(sc, None, flags)

    # launch configuration per scene: the autotuner (block size, refill
    # threshold, chunk, binning, fp32-filtered vs exact-only) on a 2^22-ray
    # sample of the scene's rays, start cells found on the GPU as in the timed step
    from paper_2112_05570_gb300 import autotune

    tuned = {}
    if args.flags == "auto":
        m = 1 << 22
        for sc in scenes:
            d = sc["d"]
            res = autotune.tune_scene(sc["scene"], d["ox"][:m], d["oy"][:m], d["dx"][:m], d["dy"][:m], None,
                                      use_cache=False)
            tuned[sc["name"]] = res["config"]
        path = "autotuned"
    else:
        path = args.flags
        for sc in scenes:
            sc["scene"].set_tuning({"trace_flags": cct.CCT_TRACE_BIN if path == "bin" else 0})
    flags = 0
    tried = tuned

    # ---- the timed step: one batched launch (cct_batch_enqueue, replayed from a CUDA graph) walks
    # the rays of all six scenes, start cells found on the GPU; one launch per step also hides the
    # drain at the end of each scene's walk (a few long rays stepping alone) behind the others'
    # work.  Launch configuration (block size, refill threshold, chunk, fp32-filtered or exact-only
    # predicates) from the autotuner.
    outs = [(torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.float32, device=dev),
             torch.empty(n, dtype=torch.int32, device=dev)) for _ in scenes]
    items = [(k, sc["d"]["ox"], sc["d"]["oy"], sc["d"]["dx"], sc["d"]["dy"], None, *outs[k])
             for k, sc in enumerate(scenes)]
    batch, btune = None, None
    arms = {}
    for label, bflags in (("filtered", 0), ("exact", cct.CCT_TRACE_EXACT_ONLY)):
        b = cct.Batch([sc["scene"] for sc in scenes], len(items), bflags)
        res = autotune.tune_batch(b, items)
        # one launch at the arm's tuned configuration: its fallback rate (0 by construction when exact-only)
        b.stage(items)
        b.stats(reset=True)
        b.enqueue(stream)
        st = b.stats(reset=True)
        arms[label] = {"ms_per_launch_tuned": res["ms"], "tuning": res["tuning"],
                       "int64_fallback_rate": st["exact_fallbacks"] / max(1, st["side_tests"]),
                       "int64_fallbacks": int(st["exact_fallbacks"]), "side_tests": int(st["side_tests"])}
        if btune is None or res["ms"] < btune["ms"]:
            if batch is not None:
                batch.free()
            batch, btune = b, dict(res, predicates=label)
        else:
            b.free()
    batch.stage(items)
    batch.capture()
    for _ in range(max(3, args.warmup)):
        batch.replay()
    torch.cuda.synchronize(dev)
    batch.stats(reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    # per-launch events on the launching stream bracket each replay (one batch_kernel launch)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            batch.replay()
            ev[k][1].record(stream)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    launch_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms = job_step_ms(dist, ms, dev)
    rays_per_step = n * len(scenes)
    value = job_rays_per_s(rays_per_step, world, ms)
    tot = batch.stats(reset=True)
    # the results of the timed launches, kept on the host for the oracle comparison (cpu_baseline leg)
    timed_results = [tuple(x.cpu().numpy() for x in o) for o in outs]
    # ... and equal to the plain per-scene trace's (every scene, every ray, t bit for bit)
    for k, sc in enumerate(scenes):
        trace(sc, None, 0)
        torch.cuda.synchronize(dev)
        o = outs[k]
        if not (torch.equal(o[0], hit) and torch.equal(o[2], steps) and torch.equal(o[1], t)):
            raise RuntimeError(f"batched results differ from the plain trace on scene {sc['name']}")

    # ---- the same step as six plain launches (one cct_trace per scene, each at its own tuned
    # configuration), for comparison; per-scene counters weight the roofline's peak
    for _ in range(2):
        step(flags)
    torch.cuda.synchronize(dev)
    for sc in scenes:
        sc["scene"].stats(reset=True)
    k_plain = max(3, args.steps // 4)
    plain_ms = _time_loop(torch, dev, stream, lambda: step(flags), k_plain)
    plain_stats = [sc["scene"].stats(reset=True) for sc in scenes]

    # ---- roofline of the timed kernel (batch_kernel): algorithmic bytes per launch over its
    # event-timed duration, against the random-sector gather peak measured over tables of the
    # scenes' sizes (weighted by each scene's share of the bytes)
    def alg_bytes(st, reps):
        # distinct record reads: locate triangles + walk triangles - 1 (the start triangle
        # serves both); 4 B seed cell; 16 B ray in, 12 B out
        return (32.0 * (st["steps"] + st["locate_steps"] - st["located"]) + 4.0 * st["located"]
                + 28.0 * st["rays"]) / reps

    gather_bps = {}
    share_over_peak = 0.0
    plain_alg = [alg_bytes(st, k_plain) for st in plain_stats]
    for i, sc in enumerate(scenes):
        _, bps = cct.cct_measure_gather(sc["tri"].n_tri * 32, 1 << 27, 5, stream)
        gather_bps[sc["name"]] = bps
        share_over_peak += plain_alg[i] / sum(plain_alg) / bps
    alg_per_launch = alg_bytes(tot, args.steps)

    # ---- per scene: the walk kernel alone (start cells given); CDT vs annealed steps
    per = {}
    for sc in scenes:
        tuned_cfg = sc["scene"].tuning()
        sc["scene"].set_tuning(dict(tuned_cfg, trace_flags=tuned_cfg["trace_flags"] & ~cct.CCT_TRACE_BIN))
        for _ in range(2):
            trace(sc, sc["d"]["start"], 0)
        sc["scene"].stats(reset=True)
        k_rep = max(3, args.steps // 4)
        wms = _time_loop(torch, dev, stream, lambda sc=sc: trace(sc, sc["d"]["start"], 0), k_rep)
        st = sc["scene"].stats(reset=True)
        wsteps = st["steps"] / k_rep
        alg = wsteps * 32.0 + n * 32.0
        bps = gather_bps[sc["name"]]
        d = sc["d"]
        other = {}
        for kind in ("cdt", "ref"):
            o_scene = cct.Scene.from_triangulation(sc[kind], sg.D)
            cct.cct_trace(o_scene.handle, d["ox"], d["oy"], d["dx"], d["dy"], None, hit, t, steps, 0, stream)
            other[kind] = o_scene.stats()
            o_scene.free()
        cst = other["cdt"]
        cmp = comparison_structures(torch, cct, sg, sc, dev, stream, 2)
        per[sc["name"]] = {"segments": int(sc["segs"].shape[0]), "triangles": sc["tri"].n_tri,
                           "kd": cmp["kd"], "bvh": cmp["bvh"],
                           "walk_rays_per_s": n / (wms * 1e-3), "steps_per_ray": wsteps / n,
                           "steps_per_ray_cdt": cst["steps"] / max(1, cst["rays"]),
                           "steps_per_ray_refined_cdt": other["ref"]["steps"] / max(1, other["ref"]["rays"]),
                           "refine_params": list(getattr(sc["ref"], "refine_params", (0.0, 0.0))),
                           "annealed_route": getattr(sc["tri"], "route", ""),
                           "length_annealed_over_cdt": sc["tri"].length(True) / sc["cdt"].length(True),
                           "length_refined_over_cdt": sc["ref"].length(True) / sc["cdt"].length(True),
                           "walk_l2_frac": (alg / (wms * 1e-3)) / bps, "gather_peak_gbs": bps / 1e9}
    secondary = secondary_rays(torch, cct, scenes, dev, stream, gather_bps, max(3, args.steps // 10))
    optimisers = None
    if fz_pool is not None:
        built = [f.result() for f in fz_futs]
        fz_pool.shutdown()
        optimisers = {"segments_per_scene": FUZZY_SEGMENTS,
                      "routes": "cdt; refined = optimally refined CDT (Sec. 3.5.1); annealed = the bench's route "
                                "(scenegen.pipeline: discrete optimisation, again after a 1 -> 4 subdivision, the "
                                "shorter kept); fuzzy = fuzzy contraction (Sec. 2.2, 3.3-3.5.3, "
                                "scenegen.fuzzy_pipeline: 10 sweeps, contract-and-polish, one subdivision round)",
                      "per_scene": fuzzy_comparison(torch, cct, sg, built, dev, stream)}
        del built
    achieved = alg_per_launch / (launch_ms * 1e-3) / 1e9
    l2_peak = 1.0 / share_over_peak / 1e9  # byte-weighted gather peak over the scenes' table sizes
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak = json.load(open(peaks_path)).get("hbm_gbs") if os.path.exists(peaks_path) else None
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm_peak else "fallback 6800 GB/s (of fallback)"
    hbm_peak = hbm_peak or 6800.0
    traffic, traffic_note, l2_bytes = captured_traffic()
    roofline = make_roofline(achieved, l2_peak, hbm_peak, hbm_src, traffic, traffic_note, launch_ms, alg_per_launch,
                             l2_bytes)

    # ---- end to end through the public API with host buffers (pinned), every scene.  The
    # scenes' rays stream through a three-stream pipeline, as a serving caller would run them:
    # the host->device copy of scene i+1 and the device->host copy of scene i-1 overlap the
    # walk of scene i (two device buffer sets, ordered by events), across step boundaries; the
    # host waits for the last results once, after the timed steps.
    piece = n
    for sc in scenes:
        sc["pin"] = {k: torch.from_numpy(getattr(sc["rays"], k)).pin_memory() for k in ("ox", "oy", "dx", "dy")}
        sc["pin_out"] = (torch.empty(n, dtype=torch.int32).pin_memory(),
                         torch.empty(n, dtype=torch.float32).pin_memory(),
                         torch.empty(n, dtype=torch.int32).pin_memory())
    n_buf = 2
    dbuf = [{k: torch.empty(piece, dtype=torch.int32 if k in ("ox", "oy") else torch.float32, device=dev)
             for k in ("ox", "oy", "dx", "dy")} for _ in range(n_buf)]
    obuf = [(torch.empty(piece, dtype=torch.int32, device=dev), torch.empty(piece, dtype=torch.float32, device=dev),
             torch.empty(piece, dtype=torch.int32, device=dev)) for _ in range(n_buf)]
    h2d_s, d2h_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(n_buf)]    # inputs of buffer set b uploaded
    ev_walk = [torch.cuda.Event() for _ in range(n_buf)]  # walk on buffer set b done
    ev_out = [torch.cuda.Event() for _ in range(n_buf)]   # results of buffer set b downloaded
    pieces = [(sc, lo) for sc in scenes for lo in range(0, n, piece)]

    def e2e_step():
        for i, (sc, lo) in enumerate(pieces):
            b = i % n_buf
            m = min(piece, n - lo)
            h2d_s.wait_event(ev_walk[b])  # the previous walk on this buffer set has read its rays
            with torch.cuda.stream(h2d_s):
                for k in dbuf[b]:
                    dbuf[b][k][:m].copy_(sc["pin"][k][lo:lo + m], non_blocking=True)
            ev_in[b].record(h2d_s)
            stream.wait_event(ev_in[b])
            stream.wait_event(ev_out[b])  # its previous results have left the device
            d, o = dbuf[b], obuf[b]
            cct.cct_trace(sc["scene"].handle, d["ox"][:m], d["oy"][:m], d["dx"][:m], d["dy"][:m], None, o[0][:m],
                          o[1][:m], o[2][:m], flags, stream)
            ev_walk[b].record(stream)
            d2h_s.wait_event(ev_walk[b])
            with torch.cuda.stream(d2h_s):
                for host, dv in zip(sc["pin_out"], o):
                    host[lo:lo + m].copy_(dv[:m], non_blocking=True)
            ev_out[b].record(d2h_s)

    e2e_step()
    torch.cuda.synchronize(dev)
    k_e2e = max(2, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / k_e2e
    # the same pipeline's copies alone (no walk): a reference for the copy-bound rate (it varies between runs)
    def copies_only():
        for i, (sc, lo) in enumerate(pieces):
            b = i % n_buf
            m = min(piece, n - lo)
            with torch.cuda.stream(h2d_s):
                for k in dbuf[b]:
                    dbuf[b][k][:m].copy_(sc["pin"][k][lo:lo + m], non_blocking=True)
            with torch.cuda.stream(d2h_s):
                for host, dv in zip(sc["pin_out"], obuf[b]):
                    host[lo:lo + m].copy_(dv[:m], non_blocking=True)

    copies_only()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        copies_only()
    torch.cuda.synchronize(dev)
    copy_s = (time.perf_counter() - t0) / k_e2e
    e2e = {"value": rays_per_step * world / e2e_s, "unit": "rays/s", "h2d_bytes_per_step": 16 * rays_per_step,
           "d2h_bytes_per_step": 12 * rays_per_step,
           "copies_only_rays_per_s": rays_per_step * world / copy_s,
           "pipeline": "per scene: pinned host->device copy, cct_trace, device->host copy on three streams, "
                       "two device buffer sets; the copies of neighbouring scenes (also across steps) overlap each "
                       "walk; one host wait after the timed steps"}
    # the results that came back equal those of one device-resident trace of the same rays (last scene)
    last = scenes[-1]
    cct.cct_trace(last["scene"].handle, last["d"]["ox"], last["d"]["oy"], last["d"]["dx"], last["d"]["dy"], None,
                  hit, t, steps, flags, stream)
    torch.cuda.synchronize(dev)
    if not (torch.equal(hit.cpu(), last["pin_out"][0]) and torch.equal(steps.cpu(), last["pin_out"][2])):
        raise RuntimeError("end-to-end results differ from the device-resident trace")

    line = {"metric": "closest-hit rays/s", "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64" if btune["predicates"] == "exact" else "int64+fp32-filter",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "families": list(FAMILIES), "segments_per_scene": N_SEGMENTS,
                       "rays_per_step": rays_per_step,
                       "launch": "one batched launch per step over the six scenes (CUDA-graph replay)",
                       "batch_tuning": dict(btune["tuning"], predicates=btune["predicates"]),
                       "l2": "inputs larger than L2 (6 x 2^24 rays + results, 2 GB); triangle tables L2-resident",
                       "parallelism": f"replicas x{world}"},
            "plain_per_scene": {"rays_per_s": rays_per_step * world / (plain_ms * 1e-3), "ms_per_step": plain_ms,
                                "launch": "one cct_trace per scene, each at its own autotuned configuration",
                                "path": path, "tuning": tried},
            "steps_per_ray": tot["steps"] / max(1, tot["rays"]),
            "kd_ops_per_ray": float(np.mean([p["kd"]["ops_per_ray"] for p in per.values()])),
            "bvh_ops_per_ray": float(np.mean([p["bvh"]["ops_per_ray"] for p in per.values()])),
            "walk_steps_per_ray_mean_over_scenes": float(np.mean([p["steps_per_ray"] for p in per.values()])),
            "fallback_rate": tot["exact_fallbacks"] / max(1, tot["side_tests"]),
            "predicate_arms": arms,
            "kd_mailbox_overflow_rays": int(sum(p["kd"]["mailbox_overflow_rays"] for p in per.values())),
            "kd_rays_traced": int(len(per) * n),
            "locate_steps_per_ray": tot["locate_steps"] / max(1, tot["located"]),
            "per_scene": per, "roofline": roofline, "e2e": e2e, "secondary_rays": secondary,
            "optimisers": optimisers,
            "gpu_launches": 2 * args.steps}
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, sample_n, dt, checked = cpu_oracle_rate(work, timed_results=timed_results)
        line["cpu_baseline"] = {"value": rate, "unit": "rays/s", "cores": cores, "kind": "oracle",
                                "sample": f"oracle walk from given start cells over the first {sample_n} rays of "
                                          f"each of the {len(work)} scenes ({dt:.1f} s wall)"}
        line["parity"] = {"rays_checked_against_oracle": checked, "mismatches": 0,
                          "what": "the timed launch's hit ids and step counts equal the oracle's, t within 1e-6 "
                                  "relative, on the cpu_baseline sample of every scene; every ray of every scene "
                                  "equal to a plain cct_trace"}
        brate, bcores, bn, bdt = cpu_oracle_bounce_rate(work)
        secondary["cpu_oracle"] = {"value": brate, "unit": "walked rays/s", "cores": bcores, "kind": "oracle",
                                   "sample": f"oracle mirror paths ({N_BOUNCE} bounces) of the first {bn} rays of "
                                             f"each of the {len(work)} scenes ({bdt:.1f} s wall)"}
    if rank == 0:
        line["clocks"] = clk.summary()
        print(json.dumps(line))
    for sc in scenes:
        sc["scene"].free()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
