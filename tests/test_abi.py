"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every function include/*.h declares, carries no oracle code, and rejects bad
arguments on the host before touching a device."""
import ctypes
import glob
import math
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1809_04424_b300 as vr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(vr_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("vr_build", "vr_complex_dim", "vr_complex_free", "vr_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = vr.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", vr.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(L, n)


def test_library_carries_no_oracle_code():
    out = subprocess.run(["nm", "-D", vr.LIB_PATH], capture_output=True, text=True).stdout
    assert "vro_" not in out


def test_library_targets_sm_103a():
    """The build compiles every source for sm_103a only (one -gencode pair,
    real architecture sm_103a, virtual compute_103a)."""
    from paper_1809_04424_b300 import build as b
    pairs = [b.FLAGS[i + 1] for i, f in enumerate(b.FLAGS) if f == "-gencode"]
    assert pairs == ["arch=compute_103a,code=sm_103a"]
    assert not any(f.startswith(("-arch", "--gpu-architecture")) for f in b.FLAGS)


@pytest.mark.parametrize("args,status", [
    (dict(n=0), vr.VR_ERR_RANGE), (dict(n=8193), vr.VR_ERR_RANGE), (dict(d=0), vr.VR_ERR_ARG),
    (dict(maxdim=4), vr.VR_ERR_UNSUPPORTED), (dict(maxdim=-1), vr.VR_ERR_ARG),
    (dict(maxrad=-1.0), vr.VR_ERR_ARG), (dict(maxrad=math.nan), vr.VR_ERR_ARG), (dict(dtype=9), vr.VR_ERR_ARG)])
def test_host_argument_checks(args, status):
    """These are rejected before any CUDA call, so they run without a GPU."""
    a = dict(n=4, d=3, dtype=vr.VR_I8, maxdim=2, maxrad=math.inf)
    a.update(args)
    buf = np.zeros(64, np.int8)
    h = ctypes.c_void_p()
    rc = vr.lib().vr_build(ctypes.c_void_p(buf.ctypes.data), a["n"], a["d"], a["dtype"], a["maxdim"],
                           a["maxrad"], None, ctypes.byref(h))
    assert rc == status
    assert h.value is None
    assert vr.vr_last_error()


def test_null_arguments():
    h = ctypes.c_void_p()
    assert vr.lib().vr_build(None, 4, 3, vr.VR_I8, 2, 1.0, None, ctypes.byref(h)) == vr.VR_ERR_ARG
    assert vr.lib().vr_complex_dim(None, 0, None) == vr.VR_ERR_ARG
    assert vr.vr_status_string(vr.VR_ERR_RANGE) == "VR_ERR_RANGE"


@pytest.mark.parametrize("fn", ["vr_sort_keys", "vr_sort_keys_noalloc"])
@pytest.mark.parametrize("n,lo,nb,status", [(-1, 0, 8, vr.VR_ERR_ARG), (4, -1, 8, vr.VR_ERR_ARG),
                                            (4, 60, 5, vr.VR_ERR_ARG), (4, 0, -2, vr.VR_ERR_ARG),
                                            # bit_lo + nbits wraps in 32 bits: must still be refused
                                            (4, 8, 2**31 - 8, vr.VR_ERR_ARG), (4, 2**31 - 1, 1, vr.VR_ERR_ARG),
                                            (4, 65, 0, vr.VR_ERR_ARG), (4, 0, 65, vr.VR_ERR_ARG)])
def test_sort_argument_checks(fn, n, lo, nb, status):
    """Bad sort arguments are rejected before any CUDA call."""
    f = getattr(vr.lib(), fn)
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    buf = np.zeros(8, np.uint64)
    assert f(ctypes.c_void_p(buf.ctypes.data), n, lo, nb, None) == status
    assert f(None, 4, 0, 8, None) == vr.VR_ERR_ARG


@pytest.mark.parametrize("fn,good,bad", [
    ("vr_set_tri_claim", [0, 1, 2], [-1, 3, 8]),
    ("vr_set_tri_key_width", [0, 8], [4, -1, 2]),
])
def test_process_wide_mode_setters(fn, good, bad):
    """The triangle-path setters accept their documented modes and reject
    any other value with VR_ERR_ARG, on the host (no device work); the
    automatic mode is left in place."""
    f = getattr(vr.lib(), fn)
    f.argtypes = [ctypes.c_int32]
    f.restype = ctypes.c_int
    try:
        for v in good:
            assert f(v) == vr.VR_OK, (fn, v)
        for v in bad:
            assert f(v) == vr.VR_ERR_ARG, (fn, v)
    finally:
        assert f(0) == vr.VR_OK


def test_build_stats_layout_matches_header():
    """The binding's vr_build_stats mirror has the header's fields in order
    (five 8-byte fields and the triangle path), so the C struct and the
    ctypes one agree."""
    hdr = open(os.path.join(ROOT, "include", "vr.h")).read()
    body = re.search(r"typedef struct vr_build_stats \{(.*?)\} vr_build_stats;", hdr, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int64_t|double)\s+(\w+);", body)
    assert fields == [f for f, _ in vr.BuildStats._fields_]
    assert ctypes.sizeof(vr.BuildStats) == 8 * len(fields)
