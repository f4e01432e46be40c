"""Persistence barcodes computed on the device (Algorithm 1 over F2, the
pivot/bar rule of Fig. 4) against the oracle's column reduction: the same
bars in the same order (the pairing of a filtered complex is unique)."""
import math

import numpy as np
import pytest

import oracle
import paper_1809_04424_b300 as vr
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def check_bars(torch, pts, maxdim, maxrad, dims=None):
    c = vr.vr_build(torch.from_numpy(np.ascontiguousarray(pts)).cuda(), maxdim, maxrad)
    o = oracle.vr_build(pts, maxdim, maxrad, keep_handle=True)
    for k in (dims if dims is not None else range(maxdim + 1)):
        g = c.barcode(k)
        want = o.barcode(k)
        assert g.shape == want.shape, (k, g.shape, want.shape)
        np.testing.assert_array_equal(g, want, err_msg=f"bars of dimension {k}")
    return c


def test_config1(torch):
    c = synth.config1()
    check_bars(torch, c.points, 2, 60.0)


@pytest.mark.parametrize("n,dtype,cap", [(1, np.int32, math.inf), (2, np.int8, math.inf), (33, np.int32, 40.0),
                                         (65, np.float32, 60.0), (120, np.int8, 25.0), (257, np.int32, 30.0)])
def test_random_clouds(torch, n, dtype, cap):
    pts = synth.random_cloud(n, 3, dtype, seed=n)
    for maxdim in (0, 1, 2):
        check_bars(torch, pts, maxdim, cap)


def set_dense_min(m):
    import ctypes
    L = vr.lib()
    L.vr_set_barcode_dense_min.argtypes = [ctypes.c_int64]
    L.vr_set_barcode_dense_min.restype = ctypes.c_int
    assert L.vr_set_barcode_dense_min(m) == 0


@pytest.mark.parametrize("dense_min", [0, 1, 64, -1])
def test_dense_column_continuation(torch, dense_min):
    """Working columns continued as bitsets (from the first entry, from
    short lengths, never) give the oracle's bars: the addition order and the
    pairs do not depend on the column's representation."""
    try:
        set_dense_min(dense_min)
        c = synth.config2(n=300)
        check_bars(torch, c.points, 2, c.maxrad)
        pts = synth.random_cloud(120, 3, np.int8, seed=120)
        check_bars(torch, pts, 2, 25.0)
        check_bars(torch, synth.circle_samples(150, 3), 2, 0.6)
    finally:
        set_dense_min(4096)


def test_torus_small(torch):
    """A torus: one H0 class, two long H1 classes, many ties."""
    c = synth.config2(n=300)
    cx = check_bars(torch, c.points, 2, c.maxrad)
    assert (cx.barcode(0)[:, 1] == -1).sum() >= 1


def test_lattice_ties(torch):
    ax = np.arange(-3, 4)
    pts = np.stack(np.meshgrid(ax, ax, ax[:3]), -1).reshape(-1, 3).astype(np.int32)
    check_bars(torch, pts, 2, 1.5)
    check_bars(torch, pts, 2, math.inf)


@pytest.mark.parametrize("n", [12, 40])
def test_float_ngon(torch, n):
    check_bars(torch, synth.ngon(n, 3.0), 2, 7.0)


def test_circle_samples(torch):
    check_bars(torch, synth.circle_samples(150, 3), 2, 0.6)


def test_torus_600(torch):
    c = synth.config2(n=600)
    check_bars(torch, c.points, 2, c.maxrad, dims=(0, 1))


def test_headline_torus_euler_every_grade(torch):
    """The full headline torus (2.4M triangles; the oracle's reduction takes
    about a minute): at every grade g the alternating count of simplices of
    grade <= g equals the alternating count of bars alive at g."""
    c = synth.config2()
    cx = vr.vr_build(torch.from_numpy(c.points).cuda(), 2, c.maxrad)
    ng = len(cx.grade_values())
    chi = np.zeros(ng, np.int64)
    for k in range(3):
        gk = cx.to_host(k)["grade"]
        chi += (-1) ** k * np.cumsum(np.bincount(gk, minlength=ng))
    alive = np.zeros(ng + 1, np.int64)
    for k in range(3):
        bars = cx.barcode(k)
        d = np.where(bars[:, 1] < 0, ng, bars[:, 1])
        delta = np.zeros(ng + 1, np.int64)
        np.add.at(delta, bars[:, 0], (-1) ** k)
        np.add.at(delta, d, -((-1) ** k))
        alive += delta
    np.testing.assert_array_equal(np.cumsum(alive)[:ng], chi)
    assert (cx.barcode(0)[:, 1] == -1).sum() >= 1


def test_dmat_bars(torch):
    D = synth.hamming_matrix(n=300, seed=9)
    cap = synth.hamming_cap(D, 0.15)
    c = vr.vr_build_dmat(torch.from_numpy(D).cuda(), 2, cap)
    o = oracle.vr_build_dmat(D, 2, cap, keep_handle=True)
    for k in (0, 1):
        np.testing.assert_array_equal(c.barcode(k), o.barcode(k))
