"""Builds libcct.so and libcct_checked.so in-tree from csrc/*.cu with nvcc for
sm_103a (GB300).

libcct_checked.so is the same sources compiled with -DCCT_CHECKED: every index
its kernels read out of a device table is range-checked, and the poke calls
that corrupt a table for fault-injection tests are enabled (include/cct.h).
Translation units of both libraries compile in parallel; each library links
the CUDA runtime statically, so it loads next to any PyTorch build without a
second copy of libcudart on the library path.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libcct.so")
LIB_CHECKED = os.path.join(LIBDIR, "libcct_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libcct needs the CUDA toolkit to build")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds both libraries (only what is stale unless `force`); returns the
    path of libcct.so."""
    srcs = sources()
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    variants = [(LIB, LIBDIR, []), (LIB_CHECKED, os.path.join(LIBDIR, "checked"), ["-DCCT_CHECKED"])]
    todo = [(lib, d, defs) for lib, d, defs in variants if force or _stale(lib, srcs + headers)]
    if not todo:
        return LIB
    cc = nvcc()
    jobs = []
    for lib, d, defs in todo:
        os.makedirs(d, exist_ok=True)
        for src in srcs:
            obj = os.path.join(d, os.path.basename(src)[:-3] + ".o")
            if force or _stale(obj, [src] + headers):
                jobs.append((src, obj, defs))

    def compile_one(job):
        src, obj, defs = job
        cmd = [cc, *ARCH, *NVCC_FLAGS, *defs, "-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)} {' '.join(defs)}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1, len(jobs)))) as ex:
        list(ex.map(compile_one, jobs))
    for lib, d, _ in todo:
        objs = [os.path.join(d, os.path.basename(s)[:-3] + ".o") for s in srcs]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed for {os.path.basename(lib)}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
