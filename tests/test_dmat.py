"""Distance-matrix input (Sec. 3: Eirene takes a square symmetric matrix,
e.g. the Hamming distances of the HIV benchmark) against the oracle's matrix
build, bit for bit."""
import math

import numpy as np
import pytest

import oracle
import paper_1809_04424_b300 as vr
import synth
from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def gpu_build_dmat(torch, D, maxdim, maxrad, on_device=True):
    src = torch.from_numpy(np.ascontiguousarray(D)).cuda() if on_device else D
    c = vr.vr_build_dmat(src, maxdim, maxrad)
    out = {"counts": c.counts()[0], "gv": c.grade_values(), "stats": c.stats()}
    for k in range(maxdim + 1):
        out[k] = c.to_host(k)
    return out


def check(torch, D, maxdim, maxrad, on_device=True):
    g = gpu_build_dmat(torch, D, maxdim, maxrad, on_device)
    assert_same(g, oracle.vr_build_dmat(D, maxdim, maxrad), maxdim)
    return g


def test_hiv_shaped_hamming_matrix(torch):
    """1088 sequences, cap at the 10th percentile: 59,846 edges, 2,106,840
    triangles, 51 grades (ties everywhere), in full."""
    D = synth.hamming_matrix()
    cap = synth.hamming_cap(D, 0.1)
    g = check(torch, D, 2, cap)
    assert g["counts"] == [1088, 59846, 2106840]


@pytest.mark.parametrize("maxdim", [1, 2])
def test_float_euclidean_matrix(torch, maxdim):
    g = synth.rng(31)
    p = g.normal(size=(600, 5))
    D = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)).astype(np.float32)
    D = np.minimum(D, D.T)                      # exactly symmetric after rounding
    iu = np.triu_indices(600, 1)
    cap = float(np.quantile(D[iu], 0.06))
    check(torch, D, maxdim, cap)


def random_symmetric(n, dtype, g, hi):
    a = g.integers(0, hi, size=(n, n))
    m = np.triu(a, 1)
    m = m + m.T
    if dtype == np.float32:
        return (m * 0.5).astype(np.float32)
    return m.astype(dtype)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 100, 257])
@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_ragged_sizes_and_caps(torch, n, dtype):
    g = synth.rng(70 + n)
    D = random_symmetric(n, dtype, g, 40)
    for cap in (math.inf, 6.0, 0.0):
        check(torch, D, 2, cap)


def test_beyond_dense_table(torch):
    """n = 4097: triangles through the neighbour CSR instead of the dense
    edge-index table."""
    g = synth.rng(4097)
    D = random_symmetric(4097, np.int32, g, 200)
    g2 = check(torch, D, 2, 3.0)
    assert g2["counts"][2] > 1000


def test_matches_point_build(torch):
    """A float32 matrix of a cloud's integer squared distances, capped at
    r^2, gives the same complex as the point build capped at r."""
    p = synth.random_cloud(300, 3, np.int32, seed=8, lo=-40, hi=40)
    D = ((p[:, None, :].astype(np.int64) - p[None, :, :]) ** 2).sum(-1).astype(np.float32)
    a = gpu_build_dmat(torch, D, 2, 400.0)
    c = vr.vr_build(torch.from_numpy(p).cuda(), 2, 20.0)
    for k in range(3):
        b = c.to_host(k)
        for f in ("verts", "grade", "colptr", "rowidx"):
            if b.get(f) is not None:
                np.testing.assert_array_equal(a[k][f], b[f])
    np.testing.assert_array_equal(a["gv"], c.grade_values())


def test_host_matrix(torch):
    D = synth.hamming_matrix(n=200, seed=5)
    check(torch, D, 2, synth.hamming_cap(D, 0.2), on_device=False)


@pytest.mark.parametrize("kind", ["asymmetric", "negative", "nan"])
def test_invalid_matrices(torch, kind):
    D = random_symmetric(40, np.float32, synth.rng(3), 10)
    if kind == "asymmetric":
        D[3, 17] += 0.5
    elif kind == "negative":
        D[5, 6] = D[6, 5] = -1.0
    else:
        D[7, 8] = D[8, 7] = np.nan
    with pytest.raises(vr.VRError) as e:
        vr.vr_build_dmat(torch.from_numpy(D).cuda(), 2)
    assert e.value.status == vr.VR_ERR_ARG
