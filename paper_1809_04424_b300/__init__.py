"""Python binding of the B300 Vietoris-Rips builder (libvr_b300.so).

Argument marshalling only: every step of the build runs in the library's
CUDA kernels.  The functions carry the C-ABI names of ``include/vr.h``;
``Complex`` wraps a ``vr_complex*`` handle.  PyTorch, when used, only provides
device memory and the current stream.  There is no CPU fallback: if the
library cannot be loaded the import of any entry point raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VR_OK, VR_ERR_ARG, VR_ERR_RANGE, VR_ERR_UNSUPPORTED, VR_ERR_OOM = 0, 1, 2, 3, 4
VR_ERR_CUDA, VR_ERR_TIMEOUT, VR_ERR_BUSY, VR_ERR_INTERNAL = 5, 6, 7, 8
VR_I8, VR_I32, VR_F32 = 1, 2, 3
VR_MAX_POINTS = 8192

LIB_PATH = _build.LIB


class VRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "VR_OK", 1: "VR_ERR_ARG", 2: "VR_ERR_RANGE", 3: "VR_ERR_UNSUPPORTED", 4: "VR_ERR_OOM",
           5: "VR_ERR_CUDA", 6: "VR_ERR_TIMEOUT", 7: "VR_ERR_BUSY", 8: "VR_ERR_INTERNAL"}


class DimView(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("count", ctypes.c_int64), ("verts", ctypes.c_void_p),
                ("grade", ctypes.c_void_p), ("colptr", ctypes.c_void_p), ("rowidx", ctypes.c_void_p)]


class BuildStats(ctypes.Structure):
    _fields_ = [("kept_edges", ctypes.c_int64), ("triangles", ctypes.c_int64), ("ngrades", ctypes.c_int64),
                ("near_tie_edges", ctypes.c_int64), ("max_rel_dist_err", ctypes.c_double),
                ("tri_order", ctypes.c_int64)]


_lib = None


def lib():
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is None:
        path = LIB_PATH
        if _build.stale():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run paper_1809_04424_b300/build.py")
        L = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.vr_build.argtypes = [vp, i32, i32, ctypes.c_int, i32, dbl, vp, ctypes.POINTER(vp)]
        L.vr_complex_dim.argtypes = [vp, i32, ctypes.POINTER(DimView)]
        L.vr_complex_grade_values.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i64)]
        L.vr_complex_counts.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
        L.vr_complex_stats.argtypes = [vp, ctypes.POINTER(BuildStats)]
        L.vr_complex_to_host.argtypes = [vp, i32, vp, vp, vp, vp]
        L.vr_complex_grade_values_to_host.argtypes = [vp, vp]
        L.vr_complex_free.argtypes = [vp]
        L.vr_complex_free.restype = None
        L.vr_last_error.restype = ctypes.c_char_p
        L.vr_status_string.restype = ctypes.c_char_p
        L.vr_status_string.argtypes = [ctypes.c_int]
        L.vr_complex_status.argtypes = [vp]
        L.vr_inject_alloc_failure.argtypes = [i64]
        L.vr_inject_lookback_stall.argtypes = [i64, i64]
        L.vr_inject_gram_stall.argtypes = [i32, i64]
        L.vr_inject_admission_refusals.argtypes = [i64]
        L.vr_inject_clear.argtypes = []
        L.vr_pool_used_bytes.argtypes = [ctypes.POINTER(i64)]
        for name in ("vr_build", "vr_complex_dim", "vr_complex_grade_values", "vr_complex_counts",
                     "vr_complex_stats", "vr_complex_to_host", "vr_complex_grade_values_to_host",
                     "vr_complex_status", "vr_inject_alloc_failure", "vr_inject_lookback_stall",
                     "vr_inject_gram_stall", "vr_inject_admission_refusals", "vr_inject_clear",
                     "vr_pool_used_bytes"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != VR_OK:
        raise VRError(status, lib().vr_last_error().decode())


def vr_last_error() -> str:
    return lib().vr_last_error().decode()


def vr_status_string(s: int) -> str:
    return lib().vr_status_string(s).decode()


def _dtype_code(dt) -> int:
    name = str(dt).replace("torch.", "")
    return {"int8": VR_I8, "int32": VR_I32, "float32": VR_F32}[name]


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class _DevArray:
    """Zero-copy device view (``__cuda_array_interface__``) of library memory."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {"data": (int(ptr or 0), True), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3}
        self._owner = owner


class Complex:
    """Owner of one ``vr_complex*`` result."""

    def __init__(self, handle: int, owned: bool = True, keepalive=None):
        self.handle = handle
        self._owned = owned
        self._keepalive = keepalive

    def __del__(self):
        if getattr(self, "_owned", False) and self.handle:
            try:
                vr_complex_free(self.handle)
            except Exception:
                pass
            self.handle = None

    def counts(self):
        return vr_complex_counts(self.handle)

    def stats(self) -> dict:
        return vr_complex_stats(self.handle)

    def status(self) -> int:
        """vr_complex_status: waits for the build and returns what the device
        reported after the build's last size read (VR_OK or an error code)."""
        return vr_complex_status(self.handle)

    def dim(self, k: int) -> dict:
        """Zero-copy torch views of dimension k's device arrays."""
        import torch
        v = vr_complex_dim(self.handle, k)
        out = {"count": v.count,
               "verts": torch.as_tensor(_DevArray(v.verts, (v.count, k + 1), "<i4", self), device="cuda"),
               "grade": torch.as_tensor(_DevArray(v.grade, (v.count,), "<i4", self), device="cuda")}
        if k >= 1:
            out["colptr"] = torch.as_tensor(_DevArray(v.colptr, (v.count + 1,), "<i8", self), device="cuda")
            out["rowidx"] = torch.as_tensor(_DevArray(v.rowidx, ((k + 1) * v.count,), "<i4", self), device="cuda")
        return out

    def to_host(self, k: int) -> dict:
        return vr_complex_to_host(self.handle, k)

    def barcode(self, dim: int, stream=None) -> np.ndarray:
        """Bars of dimension `dim` as an (m, 2) int64 array of [birth, death)
        grades (death -1: infinite), computed on the device."""
        L = lib()
        L.vr_complex_barcode.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_int64)]
        L.vr_complex_barcode.restype = ctypes.c_int
        L.vr_complex_bars_to_host.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        L.vr_complex_bars_to_host.restype = ctypes.c_int
        nb = ctypes.c_int64()
        _check(L.vr_complex_barcode(ctypes.c_void_p(self.handle), int(dim), ctypes.c_void_p(stream or 0),
                                    ctypes.byref(nb)))
        b = np.zeros(nb.value, np.int32)
        d = np.zeros(nb.value, np.int32)
        _check(L.vr_complex_bars_to_host(ctypes.c_void_p(self.handle), int(dim), ctypes.c_void_p(b.ctypes.data),
                                         ctypes.c_void_p(d.ctypes.data)))
        return np.stack([b, d], axis=1).astype(np.int64) if nb.value else np.zeros((0, 2), np.int64)

    def grade_values(self) -> np.ndarray:
        return vr_complex_grade_values_to_host(self.handle)


# ---------------------------------------------------------------- C-ABI names

def vr_build(points, maxdim: int, maxrad: float = float("inf"), stream=None, n=None, d=None, dtype=None) -> Complex:
    """Build the filtered VR complex of `points` ((n, d) int8/int32/float32).
    `points` may be a CUDA torch tensor (device pointer) or a numpy array
    (host pointer, copied in by the library)."""
    if hasattr(points, "data_ptr"):
        ptr = points.data_ptr()
        n0, d0 = points.shape
        code = _dtype_code(points.dtype)
        keep = points
    elif isinstance(points, np.ndarray):
        keep = np.ascontiguousarray(points)
        ptr = keep.ctypes.data
        n0, d0 = keep.shape
        code = _dtype_code(keep.dtype)
    else:  # raw pointer with explicit sizes
        ptr, n0, d0, code, keep = int(points), n, d, dtype, None
    if hasattr(points, "is_contiguous") and not points.is_contiguous():
        raise ValueError("points must be contiguous")
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else stream
    _check(lib().vr_build(ctypes.c_void_p(ptr), int(n0), int(d0), code, int(maxdim), float(maxrad),
                          ctypes.c_void_p(s), ctypes.byref(h)))
    return Complex(h.value)


def vr_build_dmat(D, maxdim: int, maxrad: float = float("inf"), stream=None, n=None, dtype=None) -> Complex:
    """Build the filtered complex of a square symmetric (n, n) matrix of edge
    values (int32 or float32; CUDA tensor, numpy array, or raw pointer with
    n and dtype).  The cap applies to the values themselves."""
    if hasattr(D, "data_ptr"):
        if not D.is_contiguous():
            raise ValueError("D must be contiguous")
        ptr, n0, code = D.data_ptr(), D.shape[0], _dtype_code(D.dtype)
        if D.dim() != 2 or D.shape[1] != n0:
            raise ValueError("D must be (n, n)")
    elif isinstance(D, np.ndarray):
        keep = np.ascontiguousarray(D)
        if keep.ndim != 2 or keep.shape[0] != keep.shape[1]:
            raise ValueError("D must be (n, n)")
        ptr, n0, code = keep.ctypes.data, keep.shape[0], _dtype_code(keep.dtype)
    else:
        ptr, n0, code = int(D), n, dtype
    L = lib()
    L.vr_build_dmat.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.vr_build_dmat.restype = ctypes.c_int
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else stream
    _check(L.vr_build_dmat(ctypes.c_void_p(ptr), int(n0), code, int(maxdim), float(maxrad), ctypes.c_void_p(s),
                           ctypes.byref(h)))
    return Complex(h.value)


def vr_complex_status(handle) -> int:
    return lib().vr_complex_status(ctypes.c_void_p(handle))


# ------------------------------------------------------ fault injection
# (include/vr_inject.h: host-side and bounded-wait faults for tests)

def vr_inject_alloc_failure(nth: int) -> None:
    _check(lib().vr_inject_alloc_failure(int(nth)))


def vr_inject_lookback_stall(tile: int, wait_limit: int) -> None:
    _check(lib().vr_inject_lookback_stall(int(tile), int(wait_limit)))


def vr_inject_gram_stall(tile: int, wait_limit: int) -> None:
    _check(lib().vr_inject_gram_stall(int(tile), int(wait_limit)))


def vr_inject_admission_refusals(k: int) -> None:
    _check(lib().vr_inject_admission_refusals(int(k)))


def vr_inject_clear() -> None:
    _check(lib().vr_inject_clear())


def vr_pool_used_bytes() -> int:
    v = ctypes.c_int64()
    _check(lib().vr_pool_used_bytes(ctypes.byref(v)))
    return v.value


class GramAccuracy(ctypes.Structure):
    _fields_ = [("max_rel_d_err", ctypes.c_double), ("max_norm_err", ctypes.c_double), ("beta", ctypes.c_double),
                ("kept_pairs", ctypes.c_int64), ("band_pairs", ctypes.c_int64)]


def vr_gram_accuracy_check(points, maxrad: float, split: int = 0, stream=None) -> dict:
    """Tensor-core distance tiles against the canonical FP64 values on device
    float32 points (a CUDA tensor): max relative error in d over the kept
    pairs, the normalised error, beta, kept and band pair counts."""
    L = lib()
    L.vr_gram_accuracy_check.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(GramAccuracy)]
    L.vr_gram_accuracy_check.restype = ctypes.c_int
    a = GramAccuracy()
    s = _current_stream() if stream is None else stream
    _check(L.vr_gram_accuracy_check(ctypes.c_void_p(points.data_ptr()), points.shape[0], points.shape[1],
                                    float(maxrad), int(split), ctypes.c_void_p(s), ctypes.byref(a)))
    return {f: getattr(a, f) for f, _ in GramAccuracy._fields_}


def vr_set_gram_split(split: int) -> None:
    L = lib()
    L.vr_set_gram_split.argtypes = [ctypes.c_int32]
    L.vr_set_gram_split.restype = ctypes.c_int
    _check(L.vr_set_gram_split(int(split)))


def vr_set_tri_key_width(nbytes: int) -> None:
    """0: automatic max-edge triangle keys (32-bit when the edge indices
    fit), 8: always 64-bit."""
    L = lib()
    L.vr_set_tri_key_width.argtypes = [ctypes.c_int32]
    L.vr_set_tri_key_width.restype = ctypes.c_int
    _check(L.vr_set_tri_key_width(int(nbytes)))


def vr_set_tri_claim(mode: int) -> None:
    """Max-edge key space: 0 automatic (claimed by the generator, no count
    first), 1 counted, 2 claimed with tiny sub-buffers (the counted generator
    takes over; tests)."""
    L = lib()
    L.vr_set_tri_claim.argtypes = [ctypes.c_int32]
    L.vr_set_tri_claim.restype = ctypes.c_int
    _check(L.vr_set_tri_claim(int(mode)))


def vr_complex_dim(handle, k: int) -> DimView:
    v = DimView()
    _check(lib().vr_complex_dim(ctypes.c_void_p(handle), k, ctypes.byref(v)))
    return v


def vr_complex_grade_values(handle):
    p, n = ctypes.c_void_p(), ctypes.c_int64()
    _check(lib().vr_complex_grade_values(ctypes.c_void_p(handle), ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def vr_complex_counts(handle):
    c = (ctypes.c_int64 * 4)()
    m = ctypes.c_int32()
    _check(lib().vr_complex_counts(ctypes.c_void_p(handle), c, ctypes.byref(m)))
    return [c[k] for k in range(max(3, m.value + 1))], m.value


def vr_complex_stats(handle) -> dict:
    s = BuildStats()
    _check(lib().vr_complex_stats(ctypes.c_void_p(handle), ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in BuildStats._fields_}


def vr_complex_to_host(handle, k: int) -> dict:
    counts, _ = vr_complex_counts(handle)
    m = counts[k]
    verts = np.zeros((m, k + 1), np.int32)
    grade = np.zeros(m, np.int32)
    colptr = np.zeros(m + 1, np.int64) if k >= 1 else None
    rowidx = np.zeros((k + 1) * m, np.int32) if k >= 1 else None
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None
    _check(lib().vr_complex_to_host(ctypes.c_void_p(handle), k, ptr(verts), ptr(grade), ptr(colptr), ptr(rowidx)))
    return {"count": m, "verts": verts, "grade": grade, "colptr": colptr, "rowidx": rowidx}


def vr_complex_grade_values_to_host(handle) -> np.ndarray:
    _, n = vr_complex_grade_values(handle)
    out = np.zeros(n, np.float64)
    _check(lib().vr_complex_grade_values_to_host(ctypes.c_void_p(handle), ctypes.c_void_p(out.ctypes.data)))
    return out


def vr_complex_free(handle) -> None:
    lib().vr_complex_free(ctypes.c_void_p(handle))


# ---------------------------------------------------------------- batches

def _sort_call(fn, keys, bit_lo, nbits, stream):
    """keys: a CUDA uint64/int64 tensor (contiguous), sorted in place."""
    if not (hasattr(keys, "is_cuda") and keys.is_cuda and keys.is_contiguous() and keys.element_size() == 8):
        raise TypeError("keys must be a contiguous 8-byte CUDA tensor")
    L = lib()
    f = getattr(L, fn)
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    s = stream if stream is not None else _current_stream()
    _check(f(ctypes.c_void_p(keys.data_ptr()), keys.numel(), bit_lo, nbits, ctypes.c_void_p(s)))
    return keys


def vr_sort_keys(keys, bit_lo: int, nbits: int, stream=None):
    """Stable radix sort of 64-bit keys in place on bits [bit_lo, bit_lo + nbits)."""
    return _sort_call("vr_sort_keys", keys, bit_lo, nbits, stream)


def vr_sort_keys_noalloc(keys, bit_lo: int, nbits: int, stream=None):
    """The same sort, one CTA, no allocation (at most 131072 keys)."""
    return _sort_call("vr_sort_keys_noalloc", keys, bit_lo, nbits, stream)


class Batch:
    """Owner of one ``vr_batch*``: per-cloud results as non-owning views."""

    def __init__(self, handle: int, keepalive=None):
        self.handle = handle
        self._keep = keepalive

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                vr_batch_free(self.handle)
            except Exception:
                pass
            self.handle = None

    def info(self) -> dict:
        return vr_batch_info(self.handle)

    def get(self, cloud: int):
        """(status, Complex view or None) of one cloud; the view lives as long
        as this batch."""
        view, st = vr_batch_get(self.handle, cloud)
        return st, (Complex(view, owned=False, keepalive=self) if view else None)


def _set_batch_types(L):
    if getattr(L, "_batch_types", False):
        return
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.vr_build_batch.argtypes = [vp, vp, i32, i32, ctypes.c_int, vp, vp, vp, ctypes.POINTER(vp)]
    L.vr_build_batch.restype = ctypes.c_int
    L.vr_batch_get.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int)]
    L.vr_batch_get.restype = ctypes.c_int
    L.vr_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]
    L.vr_batch_info.restype = ctypes.c_int
    L.vr_batch_free.argtypes = [vp]
    L.vr_batch_free.restype = None
    L.vr_batch_set_shape.argtypes = [ctypes.POINTER(BatchShape)]
    L.vr_batch_set_shape.restype = ctypes.c_int
    L.vr_batch_get_shape.argtypes = [ctypes.POINTER(BatchShape), ctypes.POINTER(i32), ctypes.POINTER(BatchShape),
                                     ctypes.POINTER(ctypes.c_double), i32]
    L.vr_batch_get_shape.restype = ctypes.c_int
    L.vr_batch_tune_reset.argtypes = []
    L.vr_batch_tune_reset.restype = ctypes.c_int
    L._batch_types = True


class BatchShape(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("order", ctypes.c_int32)]


def vr_batch_set_shape(ctas_per_sm: int = 0, order: int = 0) -> None:
    """Pin the one-launch batch shape on this thread (ctas_per_sm 0: tuned)."""
    L = lib()
    _set_batch_types(L)
    sh = BatchShape(int(ctas_per_sm), int(order))
    _check(L.vr_batch_set_shape(ctypes.byref(sh)))


def vr_batch_get_shape(max_cand: int = 64) -> dict:
    """The shape of the last batch on this thread and the tuner's candidates
    (shape, device ms) when its class was tuned."""
    L = lib()
    _set_batch_types(L)
    used = BatchShape()
    n = ctypes.c_int32()
    cand = (BatchShape * max_cand)()
    ms = (ctypes.c_double * max_cand)()
    _check(L.vr_batch_get_shape(ctypes.byref(used), ctypes.byref(n), cand, ms, max_cand))
    return {"used": (used.ctas_per_sm, used.order),
            "candidates": [((cand[k].ctas_per_sm, cand[k].order), ms[k]) for k in range(min(n.value, max_cand))]}


def vr_batch_tune_reset() -> None:
    L = lib()
    _set_batch_types(L)
    _check(L.vr_batch_tune_reset())


def vr_build_batch(points, offsets, maxdim=None, maxrad=None, stream=None) -> Batch:
    """Build every cloud of a row-concatenated point array (CUDA tensor or
    numpy array) with host row `offsets` (n_clouds + 1)."""
    L = lib()
    _set_batch_types(L)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nc = off.shape[0] - 1
    md = None if maxdim is None else np.ascontiguousarray(np.broadcast_to(maxdim, (nc,)), dtype=np.int32)
    mr = None if maxrad is None else np.ascontiguousarray(np.broadcast_to(maxrad, (nc,)), dtype=np.float64)
    if hasattr(points, "data_ptr"):
        ptr, d, code, keep = points.data_ptr(), points.shape[1], _dtype_code(points.dtype), points
    else:
        keep = np.ascontiguousarray(points)
        ptr, d, code = keep.ctypes.data, keep.shape[1], _dtype_code(keep.dtype)
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else stream
    cp = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None
    _check(L.vr_build_batch(ctypes.c_void_p(ptr), cp(off), nc, d, code, cp(md), cp(mr), ctypes.c_void_p(s),
                            ctypes.byref(h)))
    return Batch(h.value, keepalive=(keep, off, md, mr))


def vr_batch_get(handle, cloud: int):
    v, st = ctypes.c_void_p(), ctypes.c_int()
    _check(lib().vr_batch_get(ctypes.c_void_p(handle), cloud, ctypes.byref(v), ctypes.byref(st)))
    return v.value, st.value


def vr_batch_info(handle) -> dict:
    nc, tot, nf = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().vr_batch_info(ctypes.c_void_p(handle), ctypes.byref(nc), ctypes.byref(tot), ctypes.byref(nf)))
    return {"n_clouds": nc.value, "total_simplices": tot.value, "n_failed": nf.value}


def vr_batch_free(handle) -> None:
    L = lib()
    _set_batch_types(L)
    L.vr_batch_free(ctypes.c_void_p(handle))


# ---------------------------------------------------------------- serving

class ServerStats(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_int64) for nm in ("submitted", "completed", "failed", "deferred", "batches",
                                                "large_builds", "queued")]


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_queue", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("max_batch_clouds", ctypes.c_int32), ("device", ctypes.c_int32),
                ("n_large_workers", ctypes.c_int32)]


def _set_server_types(L):
    if getattr(L, "_server_types", False):
        return
    vp = ctypes.c_void_p
    L.vr_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    L.vr_server_create.restype = ctypes.c_int
    L.vr_serve_submit.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, ctypes.c_int32,
                                  ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]
    L.vr_serve_submit.restype = ctypes.c_int
    L.vr_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(vp)]
    L.vr_serve_poll.restype = ctypes.c_int
    L.vr_server_destroy.argtypes = [vp]
    L.vr_server_destroy.restype = ctypes.c_int
    L.vr_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.vr_server_get_stats.restype = ctypes.c_int
    L._server_types = True


class Server:
    """A continuous-batching request server (vr_server_*)."""

    def __init__(self, mem_budget_bytes=0, max_queue=0, n_streams=0, max_batch_clouds=0, device=-1,
                 n_large_workers=0):
        L = lib()
        _set_server_types(L)
        o = ServerOpts(mem_budget_bytes, max_queue, n_streams, max_batch_clouds, device, n_large_workers)
        h = ctypes.c_void_p()
        _check(L.vr_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value

    def submit(self, points: np.ndarray, maxdim: int, maxrad: float) -> int:
        """Queue one cloud (numpy array, copied before return); returns its
        ticket.  Raises VRError (VR_ERR_BUSY when the queue is full)."""
        return vr_serve_submit(self.handle, points, maxdim, maxrad)

    def poll(self, ticket: int, timeout_us: int = 10_000_000) -> Complex:
        return vr_serve_poll(self.handle, ticket, timeout_us)

    def stats(self) -> dict:
        """vr_server_get_stats as a dict of counters."""
        st = ServerStats()
        _check(lib().vr_server_get_stats(ctypes.c_void_p(self.handle), ctypes.byref(st)))
        return {nm: getattr(st, nm) for nm, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            vr_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vr_server_create(**kw) -> Server:
    return Server(**kw)


def vr_serve_submit(handle, points, maxdim, maxrad) -> int:
    L = lib()
    _set_server_types(L)
    p = np.ascontiguousarray(points)
    t = ctypes.c_uint64()
    _check(L.vr_serve_submit(ctypes.c_void_p(handle), ctypes.c_void_p(p.ctypes.data), p.shape[0], p.shape[1],
                             _dtype_code(p.dtype), int(maxdim), float(maxrad), ctypes.byref(t)))
    return t.value


def vr_serve_poll(handle, ticket, timeout_us=10_000_000) -> Complex:
    L = lib()
    _set_server_types(L)
    h = ctypes.c_void_p()
    _check(L.vr_serve_poll(ctypes.c_void_p(handle), ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(h)))
    return Complex(h.value)


def vr_server_destroy(handle) -> None:
    L = lib()
    _set_server_types(L)
    L.vr_server_destroy(ctypes.c_void_p(handle))
