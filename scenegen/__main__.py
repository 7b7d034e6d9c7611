"""Offline build of a scene's triangulation (Sec. 3), written once as the file
cct_scene_load_file reads:

    python -m scenegen build --family circles --n 30000 --seed 2 --out circles.cct
    python -m scenegen build --family random --n 200 --optimiser fuzzy --out tiny.cct
    python -m scenegen info circles.cct

Optimisers: "anneal" (the default: optimally refined CDT, then annealing with
edge flips, vertex moves and contraction by discrete collapses; with
--checkpoint it runs in pieces and resumes an interrupted build), "fuzzy" (the
paper's fuzzy contraction with its contract-and-polish loop), "refined" (the
optimally refined CDT alone) and "cdt" (the unrefined CDT).  The segments are
written beside the file (<out>.segs.npy) so that the triangulation can be read
back with scenegen.load."""
import argparse
import json
import sys
import time

import numpy as np

from . import (D, anneal, anneal_resumable, cdt, circles, clustered, dash_grid, fuzzy_pipeline, lines, load,
               random_segments, refine_optimal, ring_of_circles, room)


def _segments(family: str, n: int, seed: int, theta: float) -> np.ndarray:
    if family == "random":
        return random_segments(n, seed)
    if family == "clustered":
        return clustered(n, seed)
    if family == "circles":
        return circles(n, seed)
    if family == "dash":
        return dash_grid(n, theta)
    if family == "ring":
        return ring_of_circles(n)
    if family == "lines":
        return lines(n, seed)
    if family == "room":
        return room(n, seed)
    raise SystemExit(f"unknown family {family}")


def _build(a) -> int:
    t0 = time.perf_counter()
    segs = np.load(a.segments) if a.segments else _segments(a.family, a.n, a.seed, a.theta)
    segs = np.ascontiguousarray(segs, np.int32).reshape(-1, 4)
    base = cdt(segs)
    if a.optimiser == "cdt":
        tri = base
    elif a.optimiser == "refined":
        tri = refine_optimal(base)
    elif a.optimiser == "fuzzy":
        tri = fuzzy_pipeline(segs, a.seed, sweeps=a.sweeps)[1]
    else:
        ref = refine_optimal(base)
        tri = (anneal_resumable(ref, a.seed, a.checkpoint, sweeps=a.sweeps) if a.checkpoint
               else anneal(ref, a.seed, sweeps=a.sweeps))
    tri.save(a.out)
    np.save(a.out + ".segs.npy", segs)
    print(json.dumps({"out": a.out, "segments": int(segs.shape[0]), "vertices": tri.n_vert, "triangles": tri.n_tri,
                      "interior_length_over_cdt": tri.length(True) / base.length(True),
                      "seconds": round(time.perf_counter() - t0, 2)}))
    return 0


def _info(a) -> int:
    segs = np.load(a.file + ".segs.npy")
    tri = load(a.file, segs)
    print(json.dumps({"file": a.file, "segments": int(segs.shape[0]), "vertices": tri.n_vert, "triangles": tri.n_tri,
                      "domain": D, "interior_length": tri.length(True)}))
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m scenegen")
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("build", help="generate (or read) segments, triangulate and optimise, write the file")
    b.add_argument("--family", default="random",
                   choices=["random", "clustered", "circles", "dash", "ring", "lines", "room"])
    b.add_argument("--n", type=int, default=200, help="segments (target)")
    b.add_argument("--seed", type=int, default=1)
    b.add_argument("--theta", type=float, default=0.0, help="dash grid rotation in degrees")
    b.add_argument("--segments", default="", help="an .npy file of int32 (n, 4) segments instead of a family")
    b.add_argument("--optimiser", default="anneal", choices=["anneal", "fuzzy", "refined", "cdt"])
    b.add_argument("--sweeps", type=float, default=20.0)
    b.add_argument("--checkpoint", default="", help="anneal in pieces, checkpointing here (and resume from it)")
    b.add_argument("--out", required=True)
    i = sub.add_parser("info", help="read a triangulation file back")
    i.add_argument("file")
    a = ap.parse_args(argv)
    return _build(a) if a.cmd == "build" else _info(a)


if __name__ == "__main__":
    sys.exit(main())
