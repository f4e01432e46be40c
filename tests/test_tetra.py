"""Tetrahedra (maxdim 3) and their barcodes against the oracle, bit for bit:
simplices, grades, (grade, lex) order, the triangle-face boundary columns,
and bars of dimensions 0..3."""
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


def build(torch, pts, maxrad, dmat=False):
    src = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    c = vr.vr_build_dmat(src, 3, maxrad) if dmat else vr.vr_build(src, 3, maxrad)
    g = {"counts": c.counts()[0], "gv": c.grade_values(), "stats": c.stats()}
    for k in range(4):
        g[k] = c.to_host(k)
    return c, g


def check(torch, pts, maxrad, dmat=False, bars=True):
    c, g = build(torch, pts, maxrad, dmat)
    o = (oracle.vr_build_dmat if dmat else oracle.vr_build)(pts, 3, maxrad, keep_handle=bars)
    assert_same(g, o, 3)
    if bars:
        for k in range(4):
            np.testing.assert_array_equal(c.barcode(k), o.barcode(k), err_msg=f"bars of dimension {k}")
    return g


def test_boundary_of_4_simplex(torch):
    g = check(torch, np.eye(5, dtype=np.int32), math.inf)
    assert g["counts"] == [5, 10, 10, 5]


@pytest.mark.parametrize("n,dtype,cap", [(1, np.int8, math.inf), (4, np.int32, math.inf), (9, np.int32, math.inf),
                                         (40, np.int8, 60.0), (70, np.float32, 55.0), (130, np.int32, 40.0)])
def test_random_clouds(torch, n, dtype, cap):
    check(torch, synth.random_cloud(n, 3, dtype, seed=3000 + n), cap)


def test_torus_300(torch):
    c = synth.config2(n=300)
    g = check(torch, c.points, c.maxrad, bars=False)
    assert g["counts"][3] > 100000


def test_torus_200_bars(torch):
    c = synth.config2(n=200)
    check(torch, c.points, c.maxrad)


def test_float_ngon_and_lattice(torch):
    check(torch, synth.ngon(24, 2.0), 2.6)
    ax = np.arange(-2, 3)
    pts = np.stack(np.meshgrid(ax, ax, ax), -1).reshape(-1, 3).astype(np.int8)
    check(torch, pts, 1.5)


def test_many_grades_unpacked_keys(torch):
    """A float cloud with more than 2^12 distinct edge lengths: the
    tetrahedron keys carry a lexicographic position instead of the vertices."""
    g0 = synth.rng(77)
    pts = g0.normal(size=(400, 3)).astype(np.float32)
    g = check(torch, pts, 0.9, bars=False)
    assert len(g["gv"]) > 4097 and g["counts"][3] > 1000


def test_beyond_dense_table(torch):
    """n = 4500 (> 4096): edge indices through the neighbour CSR."""
    g0 = synth.rng(45)
    pts = g0.integers(-12, 13, size=(4500, 3)).astype(np.int8)
    g = check(torch, pts, 1.8, bars=False)
    assert g["counts"][3] > 100


def test_distance_matrix(torch):
    D = synth.hamming_matrix(n=150, seed=11)
    check(torch, D, synth.hamming_cap(D, 0.1), dmat=True)


def test_batch_rejects_maxdim_3(torch):
    pts = torch.from_numpy(synth.random_cloud(20, 3, np.int8, seed=1)).cuda()
    with pytest.raises(vr.VRError) as e:
        vr.vr_build_batch(pts, [0, 20], maxdim=[3], maxrad=[math.inf])
    assert e.value.status == vr.VR_ERR_UNSUPPORTED
