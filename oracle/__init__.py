"""Plain CPU oracle of the Vietoris-Rips filtered-complex build.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
module; the product path (``paper_1809_04424_b300``) never does, and the two
share no code.  The arithmetic lives in ``vr_oracle.c`` (plain C, compiled
without fused multiply-add); this file only marshals arguments.

Passages followed (arXiv 1809.04424): Sec. 2.1 (the Vietoris-Rips
construction and the threshold as time), Sec. 2.2 (the filtered boundary
matrix), Sec. 3 (the integer rank matrix and filtration grades Eirene returns),
Sec. 4.4 (ranking = sort permutation), Algorithm 1 and the caption of Fig. 4
(reduction and pivot -> bar, used for self-checks).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import weakref
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vr_oracle.c")
_HDR = os.path.join(_HERE, "vr_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libvr_oracle.so")
_CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]

I8, I32, F32 = 1, 2, 3
MAXDIM = 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction) if it is stale."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Complex(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("d", ctypes.c_int32), ("maxdim", ctypes.c_int32),
        ("count", ctypes.c_int64 * (MAXDIM + 1)),
        ("verts", ctypes.POINTER(ctypes.c_int32) * (MAXDIM + 1)),
        ("grade", ctypes.POINTER(ctypes.c_int32) * (MAXDIM + 1)),
        ("colptr", ctypes.POINTER(ctypes.c_int64) * (MAXDIM + 1)),
        ("rowidx", ctypes.POINTER(ctypes.c_int32) * (MAXDIM + 1)),
        ("ngrades", ctypes.c_int64),
        ("grade_value", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def _open(path):
    lib = ctypes.CDLL(path)
    lib.vro_build.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                              ctypes.POINTER(_Complex)]
    lib.vro_build.restype = ctypes.c_int
    lib.vro_build_dmat.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_void_p]
    lib.vro_build_dmat.restype = ctypes.c_int
    lib.vro_free.argtypes = [ctypes.POINTER(_Complex)]
    lib.vro_pair_d2.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32]
    lib.vro_pair_d2.restype = ctypes.c_double
    lib.vro_dense_rank.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.vro_dense_rank.restype = ctypes.c_int
    lib.vro_barcode.argtypes = [ctypes.POINTER(_Complex), ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))]
    lib.vro_barcode.restype = ctypes.c_int
    lib.vro_free_buf.argtypes = [ctypes.c_void_p]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _open(build())
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle returned {code}")
        self.code = code


def _dtype_code(points: np.ndarray) -> int:
    if points.dtype == np.int8:
        return I8
    if points.dtype == np.int32:
        return I32
    if points.dtype == np.float32:
        return F32
    raise TypeError(f"unsupported point dtype {points.dtype}")


def _copy(ptr, count, dtype):
    if count == 0 or not ptr:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(count,)).copy()


@dataclass
class Dim:
    """One dimension of the filtered complex, in filtration order."""
    count: int
    verts: np.ndarray          # (count, k+1) int32
    grade: np.ndarray          # (count,) int32
    colptr: np.ndarray | None  # (count+1,) int64, k >= 1
    rowidx: np.ndarray | None  # ((k+1)*count,) int32, k >= 1


@dataclass
class Complex:
    n: int
    maxdim: int
    dims: list = field(default_factory=list)
    grade_value: np.ndarray = None
    _bars: dict = field(default_factory=dict, repr=False)
    _c: object = field(default=None, repr=False)
    _lib: object = field(default=None, repr=False)

    def barcode(self, dim: int) -> np.ndarray:
        """Bars of dimension `dim` as an (m, 2) int64 array of [birth, death)
        grades, death = -1 for an infinite bar (Algorithm 1 over F2)."""
        if dim not in self._bars:
            self._bars[dim] = _barcode(self._lib, self._c, dim)
        return self._bars[dim]


def _barcode(lib, c, dim):
    nb = ctypes.c_int64()
    pb = ctypes.POINTER(ctypes.c_int64)()
    pe = ctypes.POINTER(ctypes.c_int64)()
    rc = lib.vro_barcode(ctypes.byref(c), dim, ctypes.byref(nb), ctypes.byref(pb), ctypes.byref(pe))
    if rc:
        raise OracleError(rc)
    out = np.stack([_copy(pb, nb.value, np.int64), _copy(pe, nb.value, np.int64)], axis=1) \
        if nb.value else np.zeros((0, 2), np.int64)
    lib.vro_free_buf(pb)
    lib.vro_free_buf(pe)
    return out


def vr_build(points: np.ndarray, maxdim: int, maxrad: float = float("inf"),
             keep_handle: bool = False) -> Complex:
    """Build the filtered complex of an (n, d) point array (int8, int32 or
    float32) up to simplex dimension `maxdim` with inclusive radius cap
    `maxrad`.  With keep_handle=True the C result is kept for barcodes."""
    lib = _load()
    pts = np.ascontiguousarray(points)
    if pts.ndim != 2:
        raise ValueError("points must be (n, d)")
    n, d = pts.shape
    c = _Complex()
    rc = lib.vro_build(pts.ctypes.data, n, d, _dtype_code(pts), maxdim, float(maxrad), ctypes.byref(c))
    if rc:
        raise OracleError(rc)
    return _wrap(lib, c, n, maxdim, keep_handle)


def vr_build_dmat(D: np.ndarray, maxdim: int, maxrad: float = float("inf"),
                  keep_handle: bool = False) -> Complex:
    """Build the filtered complex of a square symmetric (n, n) matrix of edge
    values (int32 or float32): edges from the strict upper triangle, kept iff
    value <= maxrad, grades ranking the values."""
    lib = _load()
    m = np.ascontiguousarray(D)
    if m.ndim != 2 or m.shape[0] != m.shape[1]:
        raise ValueError("D must be (n, n)")
    if m.dtype == np.int32:
        code = 2
    elif m.dtype == np.float32:
        code = 3
    else:
        raise ValueError("D must be int32 or float32")
    n = m.shape[0]
    c = _Complex()
    rc = lib.vro_build_dmat(m.ctypes.data, n, code, maxdim, float(maxrad), ctypes.byref(c))
    if rc:
        raise OracleError(rc)
    return _wrap(lib, c, n, maxdim, keep_handle)


def _wrap(lib, c, n, maxdim, keep_handle):
    cx = Complex(n=n, maxdim=maxdim)
    for k in range(maxdim + 1):
        cnt = c.count[k]
        verts = _copy(c.verts[k], cnt * (k + 1), np.int32).reshape(cnt, k + 1)
        grade = _copy(c.grade[k], cnt, np.int32)
        colptr = _copy(c.colptr[k], cnt + 1, np.int64) if k >= 1 else None
        rowidx = _copy(c.rowidx[k], cnt * (k + 1), np.int32) if k >= 1 else None
        cx.dims.append(Dim(cnt, verts, grade, colptr, rowidx))
    cx.grade_value = _copy(c.grade_value, c.ngrades, np.float64)
    if keep_handle:
        cx._c, cx._lib = c, lib
        weakref.finalize(cx, lib.vro_free, ctypes.byref(c))
    else:
        lib.vro_free(ctypes.byref(c))
    return cx


def pair_d2(points: np.ndarray, i: int, j: int) -> float:
    """Squared distance of one pair by the oracle's step 1."""
    lib = _load()
    pts = np.ascontiguousarray(points)
    return lib.vro_pair_d2(pts.ctypes.data, pts.shape[1], _dtype_code(pts), i, j)


def dense_rank(values) -> np.ndarray:
    """Rank of each value inside the sorted distinct set {0} U values."""
    lib = _load()
    v = np.ascontiguousarray(values, dtype=np.float64)
    r = np.zeros(v.shape[0], dtype=np.int64)
    rc = lib.vro_dense_rank(v.ctypes.data, v.shape[0], r.ctypes.data)
    if rc:
        raise OracleError(rc)
    return r


def betti(cx: Complex, grade: int) -> list:
    """Betti numbers at a grade: bars with birth <= grade < death."""
    out = []
    for k in range(cx.maxdim + 1):
        bars = cx.barcode(k)
        alive = (bars[:, 0] <= grade) & ((bars[:, 1] < 0) | (bars[:, 1] > grade))
        out.append(int(alive.sum()))
    return out


# ---------------------------------------------------- planted-mistake support

class using:
    """Context manager that swaps in another build of the oracle library
    (used by the tests that plant a mistake in a copy of the oracle)."""

    def __init__(self, libpath: str):
        self.libpath = libpath

    def __enter__(self):
        global _lib
        self._saved = _load()
        _lib = _open(self.libpath)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source to `out_path`."""
    d = os.path.dirname(out_path)
    src = os.path.join(d, "vr_oracle_variant.c")
    with open(src, "w") as f:
        f.write(src_text)
    shutil.copy(_HDR, os.path.join(d, "vr_oracle.h"))
    subprocess.check_call(["gcc", *_CFLAGS, "-w", "-o", out_path, src, "-lm"])
    return out_path
