"""Thin Python binding of libcct (include/cct.h): the same entry points, with
torch CUDA tensors for device buffers and torch streams.  Argument marshalling
only -- every step of the ray query runs in the library's CUDA kernels.  There
is no CPU fallback: if libcct.so is missing or no GPU is present, calls raise.

With the environment variable CCT_LIBRARY=checked set before the first call,
the process binds libcct_checked.so instead: the same entry points with every
device-table index range-checked in the kernels, and the poke calls of the
fault-injection tests enabled.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

CCT_OK = 0
CCT_ERR_INVALID_ARGUMENT = -1
CCT_ERR_BAD_TRIANGULATION = -2
CCT_ERR_OUT_OF_MEMORY = -3
CCT_ERR_CUDA = -4
CCT_ERR_WALK_LIMIT = -5
CCT_ERR_NO_DEVICE = -6
CCT_ERR_IO = -7
CCT_ERR_UNSUPPORTED = -8
CCT_RAY_INVALID = -1
CCT_RAY_WALK_LIMIT = -2
CCT_RAY_NONE = -3
CCT_RAY_BAD_INDEX = -4
CCT_MAX_BOUNCES = 1024
CCT_LOAD_NO_REORDER = 1
CCT_LOAD_NO_VALIDATE = 2
CCT_LOAD_TWO_STEP = 4


def CCT_LOAD_SEED_DENSITY(k: int) -> int:
    """Load flag: about 2^k locate seed cells per triangle (k in [0, 8])."""
    return (int(k) + 1) << 8


CCT_TRACE_EXACT_ONLY = 1
CCT_TRACE_BIN = 2
CCT_TRACE_SPLIT_LOCATE = 4
CCT_TRACE_STAGE = 8
CCT_TRACE_ONE_STEP = 16
CCT_NOALLOC_MAX_RAYS = 1 << 20
CCT_TABLE_NEIGHBOUR = 1
CCT_TABLE_HALF_EDGE_EXIT = 2
CCT_TABLE_CONSTRAINED = 3
CCT_TABLE_SEED = 4
CCT_TABLE_USER_TO_RECORD = 5
CCT_TABLE_KD_CHILD = 6
CCT_TABLE_KD_ROPE = 7
CCT_TABLE_KD_REF = 8
CCT_TABLE_BVH_CHILD0 = 9
CCT_TABLE_BVH_CHILD1 = 10
CCT_TABLE_BVH_PRIM = 11
CCT_TABLE_TWO_STEP_EXIT = 12


class CctError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {cct_error_string(code)} ({code})")
        self.code = code


class _TriDesc(ctypes.Structure):
    _fields_ = [("n_vert", ctypes.c_int32), ("n_tri", ctypes.c_int32), ("n_seg", ctypes.c_int32),
                ("domain", ctypes.c_int32), ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p),
                ("tri_v", ctypes.c_void_p), ("tri_nb", ctypes.c_void_p), ("tri_seg", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    """cct_tuning (include/cct.h): the walk's launch configuration of a scene."""
    _fields_ = [("block_threads", ctypes.c_int32), ("refill_min", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("bin_shift", ctypes.c_int32), ("trace_flags", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class _BvhDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_prims", ctypes.c_int32), ("n_seg", ctypes.c_int32),
                ("box", ctypes.c_void_p), ("child0", ctypes.c_void_p), ("child1", ctypes.c_void_p),
                ("prims", ctypes.c_void_p), ("seg", ctypes.c_void_p)]


class _KdDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_refs", ctypes.c_int32), ("n_seg", ctypes.c_int32),
                ("domain", ctypes.c_int32)] + [(k, ctypes.c_void_p) for k in
                                                ("axis", "split", "child", "count", "box", "rope", "rope_log2",
                                                 "refs", "seg")]


class _BatchItem(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_int32), ("ray_stride", ctypes.c_int32), ("n", ctypes.c_int64)] + [
        (k, ctypes.c_void_p) for k in ("d_ox", "d_oy", "d_dx", "d_dy", "d_start_tri", "d_hit_seg", "d_t", "d_steps")]


class _Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("rays", "steps", "side_tests", "exact_fallbacks", "invalid_rays",
                                               "walk_limit_rays", "located", "locate_steps")]


_lib = None


def library_path() -> str:
    """libcct.so, or libcct_checked.so when CCT_LIBRARY=checked."""
    which = os.environ.get("CCT_LIBRARY", "")
    if which not in ("", "checked"):
        raise RuntimeError(f"CCT_LIBRARY={which!r}: expected 'checked' or unset")
    return _build.LIB_CHECKED if which == "checked" else _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded library (library_path()); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not built at {path}: call __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    L.cct_copies_async.restype = ctypes.c_int
    L.cct_copies_async.argtypes = [i32, vp, vp, vp, vp]
    L.cct_scene_load.restype = ctypes.c_int
    L.cct_scene_load.argtypes = [ctypes.POINTER(_TriDesc), u32, vp, ctypes.POINTER(vp)]
    L.cct_scene_free.restype = ctypes.c_int
    L.cct_scene_free.argtypes = [vp]
    L.cct_scene_load_file.restype = ctypes.c_int
    L.cct_scene_load_file.argtypes = [ctypes.c_char_p, u32, vp, ctypes.POINTER(vp)]
    L.cct_scene_info.restype = ctypes.c_int
    L.cct_scene_info.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i32)]
    L.cct_locate.restype = ctypes.c_int
    L.cct_locate.argtypes = [vp, vp, vp, i64, vp, vp]
    L.cct_trace.restype = ctypes.c_int
    L.cct_trace.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, u32, vp]
    L.cct_scene_set_tuning.restype = ctypes.c_int
    L.cct_scene_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.cct_scene_get_tuning.restype = ctypes.c_int
    L.cct_scene_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.cct_batch_create.restype = ctypes.c_int
    L.cct_batch_create.argtypes = [ctypes.POINTER(vp), i32, i32, u32, ctypes.POINTER(vp)]
    L.cct_batch_free.restype = ctypes.c_int
    L.cct_batch_free.argtypes = [vp]
    L.cct_batch_set_tuning.restype = ctypes.c_int
    L.cct_batch_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.cct_batch_stage.restype = ctypes.c_int
    L.cct_batch_stage.argtypes = [vp, ctypes.POINTER(_BatchItem), i32]
    L.cct_batch_enqueue.restype = ctypes.c_int
    L.cct_batch_enqueue.argtypes = [vp, vp]
    L.cct_batch_get_stats.restype = ctypes.c_int
    L.cct_batch_get_stats.argtypes = [vp, ctypes.POINTER(_Stats), ctypes.c_int, vp]
    L.cct_trace_batched.restype = ctypes.c_int
    L.cct_trace_batched.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(_BatchItem), i32, u32, vp]
    L.cct_bvh_load.restype = ctypes.c_int
    L.cct_bvh_load.argtypes = [ctypes.POINTER(_BvhDesc), vp, ctypes.POINTER(vp)]
    L.cct_bvh_free.restype = ctypes.c_int
    L.cct_bvh_free.argtypes = [vp]
    L.cct_trace_bvh.restype = ctypes.c_int
    L.cct_trace_bvh.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp, vp]
    L.cct_kdtree_load.restype = ctypes.c_int
    L.cct_kdtree_load.argtypes = [ctypes.POINTER(_KdDesc), vp, ctypes.POINTER(vp)]
    L.cct_kdtree_free.restype = ctypes.c_int
    L.cct_kdtree_free.argtypes = [vp]
    L.cct_trace_kdtree.restype = ctypes.c_int
    L.cct_trace_kdtree.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp, vp]
    L.cct_trace_bounces.restype = ctypes.c_int
    L.cct_trace_bounces.argtypes = [vp, vp, vp, vp, vp, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, u32, vp]
    L.cct_trace_noalloc.restype = ctypes.c_int
    L.cct_trace_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, u32, vp]
    L.cct_get_stats.restype = ctypes.c_int
    L.cct_get_stats.argtypes = [vp, ctypes.POINTER(_Stats), ctypes.c_int, vp]
    L.cct_error_string.restype = ctypes.c_char_p
    L.cct_error_string.argtypes = [ctypes.c_int]
    L.cct_version.restype = ctypes.c_int
    L.cct_is_checked.restype = ctypes.c_int
    for name in ("cct_scene_poke", "cct_kdtree_poke", "cct_bvh_poke"):
        f = getattr(L, name)
        f.restype = ctypes.c_int
        f.argtypes = [vp, i32, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.cct_measure_gather.restype = ctypes.c_int
    L.cct_measure_gather.argtypes = [ctypes.c_size_t, i64, i32, vp, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_double)]
    _lib = L
    return L


def cct_error_string(code: int) -> str:
    return lib().cct_error_string(int(code)).decode()


def cct_copies_async(dst, src, nbytes, stream=None) -> None:
    """Enqueues len(dst) copies on `stream` in one call (include/cct.h): dst,
    src and nbytes are equal-length sequences of addresses and byte counts."""
    n = len(dst)
    if n == 0:
        return
    d = np.ascontiguousarray(dst, dtype=np.uint64)
    s_ = np.ascontiguousarray(src, dtype=np.uint64)
    b = np.ascontiguousarray(nbytes, dtype=np.uint64)
    if not (d.size == s_.size == b.size == n):
        raise ValueError("cct_copies_async: dst, src and nbytes differ in length")
    _check(lib().cct_copies_async(n, d.ctypes.data, s_.ctypes.data, b.ctypes.data, _stream_ptr(stream)),
           "cct_copies_async")


def _check(code: int, what: str):
    if code != CCT_OK:
        raise CctError(code, what)


def _stream_ptr(stream):
    """A cudaStream_t: an int handle, a torch stream, or None for torch's
    current stream (the legacy default stream when CUDA is unavailable)."""
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    import torch

    if stream is None:
        if not torch.cuda.is_available():
            return ctypes.c_void_p(0)
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name):
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------- entry points
def cct_scene_load(vx, vy, tri_v, tri_nb, tri_seg, n_seg: int, domain: int, flags: int = 0, stream=None) -> int:
    """Validate and upload a triangulation (host arrays); returns the scene handle."""
    arrs = [np.ascontiguousarray(a, np.int32).ravel() for a in (vx, vy, tri_v, tri_nb, tri_seg)]
    d = _TriDesc(arrs[0].size, arrs[2].size // 3, int(n_seg), int(domain),
                 *[ctypes.c_void_p(a.ctypes.data) for a in arrs])
    h = ctypes.c_void_p()
    _check(lib().cct_scene_load(ctypes.byref(d), flags, _stream_ptr(stream), ctypes.byref(h)), "cct_scene_load")
    return h.value


def cct_scene_load_file(path: str, flags: int = 0, stream=None) -> int:
    """Load a triangulation file (include/cct.h for the layout); returns the scene handle."""
    h = ctypes.c_void_p()
    _check(lib().cct_scene_load_file(os.fsencode(path), flags, _stream_ptr(stream), ctypes.byref(h)),
           "cct_scene_load_file")
    return h.value


def cct_scene_free(scene: int) -> None:
    _check(lib().cct_scene_free(ctypes.c_void_p(scene)), "cct_scene_free")


def cct_scene_info(scene: int):
    b, n = ctypes.c_size_t(), ctypes.c_int32()
    _check(lib().cct_scene_info(ctypes.c_void_p(scene), ctypes.byref(b), ctypes.byref(n)), "cct_scene_info")
    return int(b.value), int(n.value)


def cct_scene_set_tuning(scene: int, tuning: "Tuning | dict | None") -> None:
    if tuning is None:
        _check(lib().cct_scene_set_tuning(ctypes.c_void_p(scene), None), "cct_scene_set_tuning")
        return
    if isinstance(tuning, dict):
        tu = cct_scene_get_tuning(scene)
        for k, v in tuning.items():
            setattr(tu, k, int(v))
        tuning = tu
    _check(lib().cct_scene_set_tuning(ctypes.c_void_p(scene), ctypes.byref(tuning)), "cct_scene_set_tuning")


def cct_scene_get_tuning(scene: int) -> Tuning:
    tu = Tuning()
    _check(lib().cct_scene_get_tuning(ctypes.c_void_p(scene), ctypes.byref(tu)), "cct_scene_get_tuning")
    return tu


def cct_locate(scene: int, ox, oy, start, stream=None) -> None:
    import torch

    n = ox.numel()
    _check(lib().cct_locate(ctypes.c_void_p(scene), _dev(ox, torch.int32, "ox"), _dev(oy, torch.int32, "oy"), n,
                            _dev(start, torch.int32, "start"), _stream_ptr(stream)), "cct_locate")


def cct_trace(scene: int, ox, oy, dx, dy, start, hit, t, steps, flags: int = 0, stream=None) -> None:
    import torch

    n = ox.numel()
    for a in (oy, dx, dy, hit, t, steps) + ((start,) if start is not None else ()):
        if a.numel() != n:
            raise ValueError("all ray and result tensors must have the same length")
    _check(lib().cct_trace(ctypes.c_void_p(scene), _dev(ox, torch.int32, "ox"), _dev(oy, torch.int32, "oy"),
                           _dev(dx, torch.float32, "dx"), _dev(dy, torch.float32, "dy"),
                           _dev(start, torch.int32, "start"), n, _dev(hit, torch.int32, "hit"),
                           _dev(t, torch.float32, "t"), _dev(steps, torch.int32, "steps"), flags,
                           _stream_ptr(stream)), "cct_trace")


def cct_trace_noalloc(scene: int, ox, oy, dx, dy, start, hit, t, steps, flags: int = 0, stream=None) -> None:
    """cct_trace without any allocation (include/cct.h): at most
    CCT_NOALLOC_MAX_RAYS rays, no binning; calls on one GPU must not overlap."""
    import torch

    n = ox.numel()
    for a in (oy, dx, dy, hit, t, steps) + ((start,) if start is not None else ()):
        if a.numel() != n:
            raise ValueError("all ray and result tensors must have the same length")
    _check(lib().cct_trace_noalloc(ctypes.c_void_p(scene), _dev(ox, torch.int32, "ox"), _dev(oy, torch.int32, "oy"),
                                   _dev(dx, torch.float32, "dx"), _dev(dy, torch.float32, "dy"),
                                   _dev(start, torch.int32, "start"), n, _dev(hit, torch.int32, "hit"),
                                   _dev(t, torch.float32, "t"), _dev(steps, torch.int32, "steps"), flags,
                                   _stream_ptr(stream)), "cct_trace_noalloc")


def cct_trace_bounces(scene: int, ox, oy, dx, dy, start, n_bounce: int, hit, t, steps, org_x=None, org_y=None,
                      dir_x=None, dir_y=None, flags: int = 0, stream=None, frame=None) -> None:
    """Mirror paths (include/cct.h): outputs hold (1 + n_bounce) * n entries,
    entry b * n + r for ray b of path r; org_*, dir_* are optional; frame
    (optional, 2 * n_bounce * n floats): the secondary rays' directions (c, s)
    in their hit edges' frames instead of mirror images."""
    import torch

    n = ox.numel()
    for a in (oy, dx, dy) + ((start,) if start is not None else ()):
        if a.numel() != n:
            raise ValueError("all ray tensors must have the same length")
    m = (int(n_bounce) + 1) * n
    if frame is not None and frame.numel() != 2 * int(n_bounce) * n:
        raise ValueError("frame must hold 2 * n_bounce * n floats")
    for a in (hit, t, steps, org_x, org_y, dir_x, dir_y):
        if a is not None and a.numel() != m:
            raise ValueError("result tensors must hold (1 + n_bounce) * n entries")
    _check(lib().cct_trace_bounces(ctypes.c_void_p(scene), _dev(ox, torch.int32, "ox"), _dev(oy, torch.int32, "oy"),
                                   _dev(dx, torch.float32, "dx"), _dev(dy, torch.float32, "dy"),
                                   _dev(start, torch.int32, "start"), n, int(n_bounce),
                                   _dev(frame, torch.float32, "frame"), _dev(hit, torch.int32, "hit"), _dev(t, torch.float32, "t"),
                                   _dev(steps, torch.int32, "steps"), _dev(org_x, torch.int64, "org_x"),
                                   _dev(org_y, torch.int64, "org_y"), _dev(dir_x, torch.float32, "dir_x"),
                                   _dev(dir_y, torch.float32, "dir_y"), flags, _stream_ptr(stream)),
           "cct_trace_bounces")


def cct_get_stats(scene: int, reset: bool = False, stream=None) -> dict:
    s = _Stats()
    _check(lib().cct_get_stats(ctypes.c_void_p(scene), ctypes.byref(s), 1 if reset else 0, _stream_ptr(stream)),
           "cct_get_stats")
    return {k: int(getattr(s, k)) for k, _ in _Stats._fields_}


def cct_version() -> int:
    return int(lib().cct_version())


def cct_measure_gather(table_bytes: int, loads: int, reps: int = 5, stream=None):
    """Random 32-byte sector gather rate over a table of table_bytes
    (include/cct_measure.h): (ms per launch, bytes per second)."""
    ms, bps = ctypes.c_float(), ctypes.c_double()
    _check(lib().cct_measure_gather(int(table_bytes), int(loads), int(reps), _stream_ptr(stream), ctypes.byref(ms),
                                    ctypes.byref(bps)), "cct_measure_gather")
    return float(ms.value), float(bps.value)


# ----------------------------------------------------------------------------- convenience
class Scene:
    """A device-resident triangulation (owns its handle)."""

    def __init__(self, vx, vy, tri_v, tri_nb, tri_seg, n_seg: int, domain: int, flags: int = 0, stream=None):
        self.handle = cct_scene_load(vx, vy, tri_v, tri_nb, tri_seg, n_seg, domain, flags, stream)
        self.n_tri = int(np.asarray(tri_v).size // 3)
        self.load_flags = int(flags)

    @classmethod
    def from_triangulation(cls, tri, domain: int, flags: int = 0, stream=None) -> "Scene":
        n_seg = int(np.asarray(tri.segs).reshape(-1, 4).shape[0])
        return cls(tri.vx, tri.vy, tri.tri_v, tri.tri_nb, tri.tri_seg, n_seg, domain, flags, stream)

    @classmethod
    def from_file(cls, path: str, flags: int = 0, stream=None) -> "Scene":
        """A scene loaded by cct_scene_load_file."""
        self = cls.__new__(cls)
        self.handle = cct_scene_load_file(path, flags, stream)
        self.n_tri = cct_scene_info(self.handle)[1]
        self.load_flags = int(flags)
        return self

    def trace(self, ox, oy, dx, dy, start=None, flags: int = 0, stream=None, out=None):
        """Closest hits of the rays (device tensors): (hit, t, steps) tensors."""
        import torch

        n = ox.numel()
        if out is None:
            out = (torch.empty(n, dtype=torch.int32, device=ox.device),
                   torch.empty(n, dtype=torch.float32, device=ox.device),
                   torch.empty(n, dtype=torch.int32, device=ox.device))
        cct_trace(self.handle, ox, oy, dx, dy, start, out[0], out[1], out[2], flags, stream)
        return out

    def trace_bounces(self, ox, oy, dx, dy, n_bounce: int, start=None, flags: int = 0, stream=None,
                      with_rays: bool = True, frame=None):
        """Mirror paths: dict of (1 + n_bounce, n) tensors hit, t, steps (and
        org_x, org_y, dir_x, dir_y when with_rays); frame (optional, a
        (n_bounce, n, 2) float32 device tensor): the secondary rays' directions
        in their hit edges' frames."""
        import torch

        n, dev = ox.numel(), ox.device
        shape = (int(n_bounce) + 1, n)
        out = dict(hit=torch.empty(shape, dtype=torch.int32, device=dev),
                   t=torch.empty(shape, dtype=torch.float32, device=dev),
                   steps=torch.empty(shape, dtype=torch.int32, device=dev))
        if with_rays:
            out.update(org_x=torch.empty(shape, dtype=torch.int64, device=dev),
                       org_y=torch.empty(shape, dtype=torch.int64, device=dev),
                       dir_x=torch.empty(shape, dtype=torch.float32, device=dev),
                       dir_y=torch.empty(shape, dtype=torch.float32, device=dev))
        cct_trace_bounces(self.handle, ox, oy, dx, dy, start, n_bounce, out["hit"], out["t"], out["steps"],
                          out.get("org_x"), out.get("org_y"), out.get("dir_x"), out.get("dir_y"), flags, stream,
                          frame)
        return out

    def locate(self, ox, oy, stream=None):
        import torch

        start = torch.empty(ox.numel(), dtype=torch.int32, device=ox.device)
        cct_locate(self.handle, ox, oy, start, stream)
        return start

    def set_tuning(self, tuning=None):
        cct_scene_set_tuning(self.handle, tuning)

    def tuning(self) -> dict:
        return cct_scene_get_tuning(self.handle).as_dict()

    def stats(self, reset: bool = False, stream=None) -> dict:
        return cct_get_stats(self.handle, reset, stream)

    def info(self):
        return cct_scene_info(self.handle)

    def free(self):
        if self.handle:
            cct_scene_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ----------------------------------------------------------------------------- checked build
def cct_is_checked() -> bool:
    """True when the bound library is libcct_checked.so."""
    return bool(lib().cct_is_checked())


def _poke(fn: str, handle: int, table: int, index: int, value: int) -> int:
    old = ctypes.c_int32()
    _check(getattr(lib(), fn)(ctypes.c_void_p(handle), int(table), int(index), int(value), ctypes.byref(old), None),
           fn)
    return int(old.value)


def _table_len(fn: str, handle: int, table: int) -> int:
    n = ctypes.c_int64()
    _check(getattr(lib(), fn)(ctypes.c_void_p(handle), int(table), -1, 0, None, ctypes.byref(n)), fn)
    return int(n.value)


def cct_scene_poke(scene: int, table: int, index: int, value: int) -> int:
    """Checked build only: overwrite entry `index` of a scene table
    (CCT_TABLE_*), returning the old word (include/cct.h)."""
    return _poke("cct_scene_poke", scene, table, index, value)


def cct_scene_table_len(scene: int, table: int) -> int:
    return _table_len("cct_scene_poke", scene, table)


def cct_kdtree_poke(h: int, table: int, index: int, value: int) -> int:
    return _poke("cct_kdtree_poke", h, table, index, value)


def cct_kdtree_table_len(h: int, table: int) -> int:
    return _table_len("cct_kdtree_poke", h, table)


def cct_bvh_poke(h: int, table: int, index: int, value: int) -> int:
    return _poke("cct_bvh_poke", h, table, index, value)


def cct_bvh_table_len(h: int, table: int) -> int:
    return _table_len("cct_bvh_poke", h, table)


# ----------------------------------------------------------------------------- comparison structures (Sec. 5.3)
def _i32(a):
    return np.ascontiguousarray(a, np.int32).ravel()


def cct_bvh_load(box, child0, child1, prims, segs, stream=None) -> int:
    arrs = [_i32(a) for a in (box, child0, child1, prims, segs)]
    d = _BvhDesc(arrs[1].size, arrs[3].size, arrs[4].size // 4, *[ctypes.c_void_p(a.ctypes.data) for a in arrs])
    h = ctypes.c_void_p()
    _check(lib().cct_bvh_load(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)), "cct_bvh_load")
    return h.value


def cct_bvh_free(h: int) -> None:
    _check(lib().cct_bvh_free(ctypes.c_void_p(h)), "cct_bvh_free")


def cct_trace_bvh(h: int, ox, oy, dx, dy, hit, t, ops, stream=None) -> None:
    import torch

    _check(lib().cct_trace_bvh(ctypes.c_void_p(h), _dev(ox, torch.int32, "ox"), _dev(oy, torch.int32, "oy"),
                               _dev(dx, torch.float32, "dx"), _dev(dy, torch.float32, "dy"), ox.numel(),
                               _dev(hit, torch.int32, "hit"), _dev(t, torch.float32, "t"),
                               _dev(ops, torch.int32, "ops"), _stream_ptr(stream)), "cct_trace_bvh")


def cct_kdtree_load(axis, split, child, count, box, rope, rope_log2, refs, segs, domain: int, stream=None) -> int:
    arrs = [_i32(a) for a in (axis, split, child, count, box, rope, rope_log2, refs, segs)]
    d = _KdDesc(arrs[0].size, arrs[7].size, arrs[8].size // 4, int(domain),
                *[ctypes.c_void_p(a.ctypes.data) for a in arrs])
    h = ctypes.c_void_p()
    _check(lib().cct_kdtree_load(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)), "cct_kdtree_load")
    return h.value


def cct_kdtree_free(h: int) -> None:
    _check(lib().cct_kdtree_free(ctypes.c_void_p(h)), "cct_kdtree_free")


def cct_trace_kdtree(h: int, ox, oy, dx, dy, hit, t, ops, stream=None) -> None:
    import torch

    _check(lib().cct_trace_kdtree(ctypes.c_void_p(h), _dev(ox, torch.int32, "ox"), _dev(oy, torch.int32, "oy"),
                                  _dev(dx, torch.float32, "dx"), _dev(dy, torch.float32, "dy"), ox.numel(),
                                  _dev(hit, torch.int32, "hit"), _dev(t, torch.float32, "t"),
                                  _dev(ops, torch.int32, "ops"), _stream_ptr(stream)), "cct_trace_kdtree")


class Bvh:
    """A device-resident BVH (owns its handle); built by scenegen.bvh."""

    def __init__(self, b, stream=None):
        self.handle = cct_bvh_load(b.box, b.child0, b.child1, b.prims, b.segs, stream)

    def trace(self, ox, oy, dx, dy, stream=None):
        import torch

        n = ox.numel()
        hit = torch.empty(n, dtype=torch.int32, device=ox.device)
        t = torch.empty(n, dtype=torch.float32, device=ox.device)
        ops = torch.empty((n, 2), dtype=torch.int32, device=ox.device)
        cct_trace_bvh(self.handle, ox, oy, dx, dy, hit, t, ops, stream)
        return hit, t, ops

    def free(self):
        if self.handle:
            cct_bvh_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class KdTree:
    """A device-resident roped kd-tree (owns its handle); built by scenegen.kdtree."""

    def __init__(self, k, domain: int, stream=None):
        self.handle = cct_kdtree_load(k.axis, k.split, k.child, k.count, k.box, k.rope, k.rope_log2, k.refs,
                                      k.segs, domain, stream)

    def trace(self, ox, oy, dx, dy, stream=None):
        import torch

        n = ox.numel()
        hit = torch.empty(n, dtype=torch.int32, device=ox.device)
        t = torch.empty(n, dtype=torch.float32, device=ox.device)
        ops = torch.empty((n, 6), dtype=torch.int32, device=ox.device)
        cct_trace_kdtree(self.handle, ox, oy, dx, dy, hit, t, ops, stream)
        return hit, t, ops

    def free(self):
        if self.handle:
            cct_kdtree_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ----------------------------------------------------------------------------- many scenes per launch
def _items(items):
    """items: sequence of (scene_index, ox, oy, dx, dy, start | None, hit, t, steps) with CUDA tensors."""
    import torch

    arr = (_BatchItem * max(1, len(items)))()
    for k, (sc, ox, oy, dx, dy, st, hit, t, steps) in enumerate(items):
        arr[k] = _BatchItem(int(sc), 0, int(ox.numel()), _dev(ox, torch.int32, "ox"), _dev(oy, torch.int32, "oy"),
                            _dev(dx, torch.float32, "dx"), _dev(dy, torch.float32, "dy"),
                            _dev(st, torch.int32, "start"), _dev(hit, torch.int32, "hit"),
                            _dev(t, torch.float32, "t"), _dev(steps, torch.int32, "steps"))
    return arr


def cct_trace_batched(scenes, items, flags: int = 0, stream=None) -> None:
    """One-shot batched trace (synchronises the stream): scenes = handles or Scene
    objects; items as in Batch.stage."""
    hs = [s.handle if isinstance(s, Scene) else s for s in scenes]
    harr = (ctypes.c_void_p * len(hs))(*hs)
    arr = _items(items)
    _check(lib().cct_trace_batched(harr, len(hs), arr, len(items), flags, _stream_ptr(stream)), "cct_trace_batched")


class Batch:
    """A reusable multi-scene launch (include/cct.h, cct_batch_*): stage a work
    list on the host, enqueue (or replay a captured CUDA graph of the enqueue)."""

    def __init__(self, scenes, max_items: int, flags: int = 0):
        hs = [s.handle if isinstance(s, Scene) else s for s in scenes]
        self._harr = (ctypes.c_void_p * len(hs))(*hs)
        h = ctypes.c_void_p()
        _check(lib().cct_batch_create(self._harr, len(hs), int(max_items), flags, ctypes.byref(h)), "cct_batch_create")
        self.handle = h.value
        self._keep = None
        self.graph = None

    def set_tuning(self, tuning=None):
        if tuning is None:
            _check(lib().cct_batch_set_tuning(ctypes.c_void_p(self.handle), None), "cct_batch_set_tuning")
            return
        tu = Tuning(256, 8, 128, -1, 0)
        for k, v in dict(tuning).items():
            setattr(tu, k, int(v))
        _check(lib().cct_batch_set_tuning(ctypes.c_void_p(self.handle), ctypes.byref(tu)), "cct_batch_set_tuning")

    def stage(self, items):
        arr = _items(items)
        _check(lib().cct_batch_stage(ctypes.c_void_p(self.handle), arr, len(items)), "cct_batch_stage")
        self._keep = items  # the tensors must outlive the launch

    def stage_raw(self, items, ray_stride: int = 1):
        """items: (scene, n, ox, oy, dx, dy, start, hit, t, steps) with raw device
        addresses (ints, start may be 0 for none); ray_stride 4 for interleaved
        ray records.  The caller keeps the memory alive."""
        arr = (_BatchItem * max(1, len(items)))()
        for k, it in enumerate(items):
            arr[k] = _BatchItem(int(it[0]), int(ray_stride), int(it[1]),
                                *[ctypes.c_void_p(x) if x else None for x in it[2:]])
        _check(lib().cct_batch_stage(ctypes.c_void_p(self.handle), arr, len(items)), "cct_batch_stage")

    def enqueue(self, stream=None):
        _check(lib().cct_batch_enqueue(ctypes.c_void_p(self.handle), _stream_ptr(stream)), "cct_batch_enqueue")

    def capture(self):
        """Captures one enqueue in a CUDA graph (stage something first); replay()
        then re-runs it with whatever is staged at that time."""
        import torch

        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.enqueue(s)  # warm-up launch outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            self.enqueue()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def stats(self, reset: bool = False, stream=None) -> dict:
        st = _Stats()
        _check(lib().cct_batch_get_stats(ctypes.c_void_p(self.handle), ctypes.byref(st), 1 if reset else 0,
                                         _stream_ptr(stream)), "cct_batch_get_stats")
        return {k: int(getattr(st, k)) for k, _ in _Stats._fields_}

    def free(self):
        if self.handle:
            self.graph = None
            cct_batch_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cct_batch_free(h: int) -> None:
    _check(lib().cct_batch_free(ctypes.c_void_p(h)), "cct_batch_free")
