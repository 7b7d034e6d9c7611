"""C-ABI library checks that need no GPU: libcct.so (and its checked build,
libcct_checked.so) loads, exports every symbol include/ declares, and its
host-side validation returns status codes."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import scenegen as sg
from paper_2112_05570_gb300 import _build, cct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(cct_\w+)\s*\(", txt, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(_build.LIB)


@pytest.fixture(scope="module")
def checked_lib():
    _build.build()
    return ctypes.CDLL(_build.LIB_CHECKED)


def test_every_declared_symbol_is_exported(lib, checked_lib):
    names = _declared()
    assert "cct_trace" in names and "cct_scene_load" in names and len(names) >= 8
    assert {"cct_is_checked", "cct_scene_poke", "cct_kdtree_poke", "cct_bvh_poke"} <= set(names)
    for L in (lib, checked_lib):
        for n in names:
            assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_checked_build_identifies_itself(lib, checked_lib):
    """libcct.so is the unchecked build and libcct_checked.so the checked one;
    both refuse a poke of no object, and the binding picks the library from
    CCT_LIBRARY."""
    assert lib.cct_is_checked() == 0 and checked_lib.cct_is_checked() == 1
    for L in (lib, checked_lib):
        for fn in ("cct_scene_poke", "cct_kdtree_poke", "cct_bvh_poke"):
            f = getattr(L, fn)
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                          ctypes.c_void_p]
            assert f(None, cct.CCT_TABLE_SEED, 0, 0, None, None) == cct.CCT_ERR_INVALID_ARGUMENT
    assert "checked" in cct.cct_error_string(cct.CCT_ERR_UNSUPPORTED)
    old = os.environ.get("CCT_LIBRARY")
    try:
        os.environ["CCT_LIBRARY"] = "checked"
        assert cct.library_path() == _build.LIB_CHECKED
        os.environ["CCT_LIBRARY"] = "other"
        with pytest.raises(RuntimeError):
            cct.library_path()
    finally:
        if old is None:
            os.environ.pop("CCT_LIBRARY", None)
        else:
            os.environ["CCT_LIBRARY"] = old
    assert cct.library_path() == (_build.LIB_CHECKED if old == "checked" else _build.LIB)


def test_status_strings_and_version():
    assert cct.cct_error_string(cct.CCT_OK) == "ok"
    assert "validation" in cct.cct_error_string(cct.CCT_ERR_BAD_TRIANGULATION)
    assert cct.cct_version() >= 1


def _tri(n=60, seed=3):
    return sg.cdt(sg.random_segments(n, seed))


@pytest.mark.parametrize("corrupt", ["orientation", "neighbour", "label", "index", "area", "hull"])
def test_load_rejects_corrupt_triangulations(corrupt):
    t = _tri()
    vx, vy, tv, tn, ts = t.vx.copy(), t.vy.copy(), t.tri_v.copy(), t.tri_nb.copy(), t.tri_seg.copy()
    n_seg = t.segs.shape[0]
    if corrupt == "orientation":
        tv[4] = tv[4][[0, 2, 1]]
    elif corrupt == "neighbour":
        i = np.argwhere(tn[5] >= 0)[0, 0]
        tn[5, i] = (tn[5, i] + 1) % t.n_tri
    elif corrupt == "label":
        tt, ti = np.argwhere(ts >= 0)[0]
        ts[tt, ti] = -1
    elif corrupt == "index":
        tv[2, 1] = t.n_vert + 5
    elif corrupt == "area":
        vx = vx.copy()
        vx[vx == sg.D] = sg.D - 1  # the hull no longer spans the domain
    elif corrupt == "hull":
        i = np.argwhere(tn[0] >= 0)[0, 0]
        tn = tn.copy()
        u = tn[0, i]
        j = np.argwhere(tn[u] == 0)[0, 0]
        tn[0, i] = -1
        tn[u, j] = -1
    with pytest.raises(cct.CctError) as e:
        cct.cct_scene_load(vx, vy, tv, tn, ts, n_seg, sg.D)
    assert e.value.code == cct.CCT_ERR_BAD_TRIANGULATION


def test_load_argument_errors():
    t = _tri()
    with pytest.raises(cct.CctError) as e:
        cct.cct_scene_load(t.vx, t.vy, t.tri_v, t.tri_nb, t.tri_seg, t.segs.shape[0], (1 << 20) + 1)
    assert e.value.code == cct.CCT_ERR_INVALID_ARGUMENT
    with pytest.raises(cct.CctError) as e:
        cct.cct_scene_load(t.vx, t.vy, t.tri_v[:0], t.tri_nb[:0], t.tri_seg[:0], 0, sg.D)
    assert e.value.code == cct.CCT_ERR_INVALID_ARGUMENT
    L = cct.lib()
    assert L.cct_trace(None, None, None, None, None, None, 0, None, None, None, 0, None) == cct.CCT_ERR_INVALID_ARGUMENT
    assert L.cct_locate(None, None, None, 0, None, None) == cct.CCT_ERR_INVALID_ARGUMENT
    assert L.cct_scene_free(None) == cct.CCT_OK
    # cct_trace_bounces: a null scene, n < 0, n_bounce outside [0, CCT_MAX_BOUNCES], other flags
    args = [None, None, None, None, None, None, 0, 0, None, None, None, None, None, None, None, None, 0, None]
    assert L.cct_trace_bounces(*args) == cct.CCT_ERR_INVALID_ARGUMENT
    fake = ctypes.c_void_p(1)  # never dereferenced: the checks come first
    for n, nb, fl in ((-1, 0, 0), (1, -1, 0), (1, cct.CCT_MAX_BOUNCES + 1, 0), (1, 2, cct.CCT_TRACE_BIN)):
        a = list(args)
        a[0], a[6], a[7], a[16] = fake, n, nb, fl
        assert L.cct_trace_bounces(*a) == cct.CCT_ERR_INVALID_ARGUMENT, (n, nb, fl)
    a = list(args)
    a[0] = fake
    assert L.cct_trace_bounces(*a) == cct.CCT_OK  # n = 0: a no-op before any pointer is read
    # cct_copies_async: n < 0 or missing arrays; n = 0 is a no-op
    assert L.cct_copies_async(-1, None, None, None, None) == cct.CCT_ERR_INVALID_ARGUMENT
    assert L.cct_copies_async(2, None, None, None, None) == cct.CCT_ERR_INVALID_ARGUMENT
    assert L.cct_copies_async(0, None, None, None, None) == cct.CCT_OK
    with pytest.raises(ValueError):
        cct.cct_copies_async([1, 2], [3], [4, 5])


def test_valid_triangulation_passes_validation_without_gpu():
    """Without a GPU a valid triangulation gets past validation and stops at the
    device check; with a GPU it loads."""
    import torch

    t = _tri()
    if torch.cuda.is_available():
        s = cct.Scene.from_triangulation(t, sg.D)
        s.free()
        return
    with pytest.raises(cct.CctError) as e:
        cct.Scene.from_triangulation(t, sg.D)
    assert e.value.code == cct.CCT_ERR_NO_DEVICE


def test_scene_file_round_trip_and_malformed_files(tmp_path):
    """cct_scene_load_file: a file written by the offline build gets past the
    header checks and validation (and loads where a GPU is present); a missing
    file, a wrong magic, counts out of range, a size that does not match the
    counts and a truncated array are CCT_ERR_IO; corrupt arrays are
    CCT_ERR_BAD_TRIANGULATION (the validation of cct_scene_load)."""
    import torch

    t = _tri()
    good = tmp_path / "scene.cct"
    t.save(str(good))
    raw = good.read_bytes()
    assert raw[:8] == b"CCTTRI1\0"
    hdr = np.frombuffer(raw[8:24], "<i4")
    assert list(hdr) == [t.n_vert, t.n_tri, t.segs.shape[0], sg.D]
    assert len(raw) == 24 + 4 * (2 * t.n_vert + 9 * t.n_tri)
    if torch.cuda.is_available():
        s = cct.Scene.from_file(str(good))
        assert s.n_tri == t.n_tri
        s.free()
    else:
        with pytest.raises(cct.CctError) as e:
            cct.cct_scene_load_file(str(good))
        assert e.value.code == cct.CCT_ERR_NO_DEVICE

    def expect(data, code, name):
        p = tmp_path / name
        p.write_bytes(data)
        with pytest.raises(cct.CctError) as e:
            cct.cct_scene_load_file(str(p))
        assert e.value.code == code, name

    with pytest.raises(cct.CctError) as e:
        cct.cct_scene_load_file(str(tmp_path / "missing.cct"))
    assert e.value.code == cct.CCT_ERR_IO
    expect(b"CCTTRI2\0" + raw[8:], cct.CCT_ERR_IO, "magic")
    expect(raw[:-4], cct.CCT_ERR_IO, "truncated")
    expect(raw + b"\0\0\0\0", cct.CCT_ERR_IO, "trailing")
    bad = bytearray(raw)
    bad[12:16] = np.array([1 << 29], "<i4").tobytes()  # n_tri out of range
    expect(bytes(bad), cct.CCT_ERR_IO, "count")
    bad = bytearray(raw)
    bad[8:12] = np.array([t.n_vert + 1], "<i4").tobytes()  # size no longer matches
    expect(bytes(bad), cct.CCT_ERR_IO, "size")
    # a neighbour index out of range: the arrays reach cct_scene_load's checks
    off = 24 + 4 * (2 * t.n_vert + 3 * t.n_tri)  # start of tri_nb
    bad = bytearray(raw)
    bad[off:off + 4] = np.array([t.n_tri + 7], "<i4").tobytes()
    expect(bytes(bad), cct.CCT_ERR_BAD_TRIANGULATION, "arrays")
    assert "file" in cct.cct_error_string(cct.CCT_ERR_IO)


def test_binding_constants_match_the_header():
    """Every integer constant include/cct.h defines (status codes, per-ray
    statuses, load and trace flags, limits) has the same value in the Python
    binding."""
    txt = open(os.path.join(ROOT, "include", "cct.h")).read()
    defs = dict(re.findall(r"^#define (CCT_[A-Z0-9_]+) \(?([-0-9<> ]+?)u?\)?\s*(?:/\*|$)", txt, re.M))
    defs = {k: eval(v.replace("u", "")) for k, v in defs.items() if k != "CCT_H"}  # noqa: S307 (integer literals)
    assert {"CCT_OK", "CCT_ERR_IO", "CCT_RAY_NONE", "CCT_MAX_BOUNCES", "CCT_TRACE_BIN",
            "CCT_NOALLOC_MAX_RAYS"} <= set(defs)
    for name, value in defs.items():
        assert getattr(cct, name) == value, name
    assert cct.CCT_LOAD_SEED_DENSITY(3) == (3 + 1) << 8


def test_offline_build_command(tmp_path):
    """python -m scenegen build writes a triangulation file (with its segments)
    that reads back valid and passes cct_scene_load_file's header checks; the
    checkpointed build resumes to the same file."""
    import subprocess
    import sys

    import oracle

    out = str(tmp_path / "s.cct")
    cmd = [sys.executable, "-m", "scenegen", "build", "--family", "circles", "--n", "800", "--seed", "3",
           "--sweeps", "2", "--checkpoint", str(tmp_path / "ck.cct"), "--out", out]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, check=True)
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["triangles"] > 0 and rep["interior_length_over_cdt"] < 1.0
    segs = np.load(out + ".segs.npy")
    tri = sg.load(out, segs)
    assert oracle.check_triangulation(tri, sg.D) == 0
    info = subprocess.run([sys.executable, "-m", "scenegen", "info", out], cwd=ROOT, capture_output=True, text=True,
                          check=True)
    assert json.loads(info.stdout)["triangles"] == tri.n_tri
    again = subprocess.run(cmd[:-1] + [str(tmp_path / "t.cct")], cwd=ROOT, capture_output=True, text=True, check=True)
    assert open(str(tmp_path / "t.cct"), "rb").read() == open(out, "rb").read()
    import torch

    if not torch.cuda.is_available():
        with pytest.raises(cct.CctError) as e:
            cct.cct_scene_load_file(out)
        assert e.value.code == cct.CCT_ERR_NO_DEVICE  # past the header and size checks
