"""The allocation-free sort entry point, checked against numpy's stable
argsort and against vr_build.

vr_sort_keys_noalloc is for callers that cannot allocate device memory when
they rank edges (their framework's allocator owns the GPU memory, or their
memory budget is fixed at start-up).  Fed the edge keys of a cloud in (i, j)
order, it must reproduce exactly the (distance, i, j) edge order and the
squared distances that vr_build returns for that cloud.  Two different calls
run back to back on the shared scratch array, then the first one again.
This file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

import paper_1809_04424_b300 as vr
import synth

pytestmark = pytest.mark.gpu


def lex_keys(points, maxrad):
    """Edge keys (d2 << 26) | (i << 13) | j of the kept pairs, in (i, j)
    order, with exact integer squared distances."""
    p = points.astype(np.int64)
    n = p.shape[0]
    iu, ju = np.triu_indices(n, 1)
    d2 = ((p[iu] - p[ju]) ** 2).sum(axis=1)
    if not math.isinf(maxrad):
        keep = d2 <= math.floor(maxrad * maxrad)
        iu, ju, d2 = iu[keep], ju[keep], d2[keep]
    keys = (d2.astype(np.uint64) << np.uint64(26)) | (iu.astype(np.uint64) << np.uint64(13)) | ju.astype(np.uint64)
    return keys, int(d2.max()).bit_length() if d2.size else 1


def sort_noalloc(torch, keys, nbits):
    dev = torch.from_numpy(keys.view(np.int64)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    L = vr.lib()
    L.vr_sort_keys_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p]
    L.vr_sort_keys_noalloc.restype = ctypes.c_int
    rc = L.vr_sort_keys_noalloc(ctypes.c_void_p(dev.data_ptr()), keys.size, 26, nbits, ctypes.c_void_p(s))
    assert rc == vr.VR_OK, vr.vr_last_error()
    torch.cuda.synchronize()
    return dev.cpu().numpy().view(np.uint64)


def check_cloud(torch, cloud):
    keys, nbits = lex_keys(cloud.points, cloud.maxrad)
    out = sort_noalloc(torch, keys, nbits)
    # A sort defined without this library: numpy's stable argsort on the
    # distance field alone (the (i, j) input order breaks its ties).
    np.testing.assert_array_equal(out, keys[np.argsort(keys >> np.uint64(26), kind="stable")])
    ref = vr.vr_build(torch.from_numpy(cloud.points).cuda(), 1, cloud.maxrad)
    e = ref.to_host(1)
    gv = ref.grade_values()
    ij = np.stack([(out >> np.uint64(13)) & np.uint64(8191), out & np.uint64(8191)], axis=1).astype(np.int32)
    np.testing.assert_array_equal(ij, e["verts"])
    np.testing.assert_array_equal((out >> np.uint64(26)).astype(np.float64), gv[e["grade"]])


def test_noalloc_sort_matches_vr_build_twice():
    import torch
    assert torch.cuda.is_available()
    check_cloud(torch, synth.config1())      # 2016 keys
    check_cloud(torch, synth.config2())      # 74934 keys, same scratch array
    check_cloud(torch, synth.config1())      # leftovers of the larger call do not matter


def test_noalloc_sort_rejects_oversize():
    import torch
    L = vr.lib()
    L.vr_sort_keys_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p]
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    rc = L.vr_sort_keys_noalloc(ctypes.c_void_p(buf.data_ptr()), 131073, 0, 8, None)
    assert rc == vr.VR_ERR_RANGE
    assert "exceeds" in vr.vr_last_error()
