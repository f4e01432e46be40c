"""Distance tiles on the tensor cores (tcgen05 Gram) against the CUDA-core
kernel and the oracle, and the float Gram error bound measured on
adversarial inputs."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import paper_1809_04424_b300 as vr
import synth
from test_gpu_parity import assert_same, gpu_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def set_path(mode):
    L = vr.lib()
    L.vr_set_gram_path.argtypes = [ctypes.c_int32]
    L.vr_set_gram_path.restype = ctypes.c_int
    assert L.vr_set_gram_path(mode) == 0


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("case", ["torus", "gauss", "ragged_f", "ragged_i8"])
def test_both_distance_paths_match_oracle(torch, mode, case):
    """Tensor-core (1) and CUDA-core (2) distance tiles give the oracle's
    complex, including ragged tile tails (n not a multiple of 128)."""
    if case == "torus":
        c = synth.config2(n=700)
        pts, md, r = c.points, 2, c.maxrad
    elif case == "gauss":
        c = synth.config3(n=500)
        pts, md, r = c.points, 2, c.maxrad
    elif case == "ragged_f":
        pts, md, r = synth.random_cloud(200, 7, np.float32, seed=5, lo=-3, hi=3), 2, 2.5
    else:
        pts, md, r = synth.random_cloud(333, 5, np.int8, seed=6), 2, 60.0
    try:
        set_path(mode)
        g = gpu_build(torch, pts, md, r)
    finally:
        set_path(0)
    assert_same(g, oracle.vr_build(pts, md, r), md)


@pytest.mark.parametrize("seed,scale,d", [(1, 1.0, 32), (2, 1000.0, 64), (3, 1e-3, 16), (4, 50.0, 3)])
def test_float_gram_error_within_quarter_beta(torch, seed, scale, d):
    """Every pair's tensor-core d^2 is within beta/4 of the canonical FP64
    value, relative to |y_i|^2 + |y_j|^2: clustered points far from the
    origin (large norms against small distances) and mixed magnitudes."""
    g = synth.rng(900 + seed)
    base = g.normal(size=(1, d)) * 10 * scale
    pts = (base + g.normal(size=(600, d)) * scale * g.uniform(0.01, 1.0, size=(600, 1))).astype(np.float32)
    dev = torch.from_numpy(pts).cuda()
    L = vr.lib()
    L.vr_gram_error_check.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.vr_gram_error_check.restype = ctypes.c_int
    worst, beta = ctypes.c_double(), ctypes.c_double()
    assert L.vr_gram_error_check(ctypes.c_void_p(dev.data_ptr()), 600, d, None, ctypes.byref(worst),
                                 ctypes.byref(beta)) == 0, vr.vr_last_error()
    assert 0 <= worst.value <= beta.value / 4, (worst.value, beta.value)


def test_band_list_overflow_falls_back_exactly(torch):
    """Two tight clusters 100 apart with the cap at exactly 100: every one of
    the 1050^2 cross pairs lies within beta of the cap, more than the near-cap
    list holds, so the build redoes the bitmap on the CUDA cores and still
    gives the oracle's complex."""
    g = synth.rng(77)
    a = g.normal(size=(1050, 4)) * 1e-3
    b = g.normal(size=(1050, 4)) * 1e-3
    b[:, 0] += 100.0
    pts = np.concatenate([a, b]).astype(np.float32)
    try:
        set_path(1)
        gc = gpu_build(torch, pts, 1, 100.0)
    finally:
        set_path(0)
    assert_same(gc, oracle.vr_build(pts, 1, 100.0), 1)


def set_split(split):
    vr.vr_set_gram_split(split)


@pytest.mark.parametrize("case", ["gauss", "ragged_f", "clustered_far"])
def test_three_way_split_matches_oracle(torch, case):
    """The three-way float split (hi, mid, lo: six products per k-step) on the
    forced tensor-core path gives the oracle's complex."""
    if case == "gauss":
        c = synth.config3(n=900)
        pts, md, r = c.points, 2, c.maxrad
    elif case == "ragged_f":
        pts, md, r = synth.random_cloud(333, 29, np.float32, seed=8, lo=-3, hi=3), 2, 9.0
    else:
        g = synth.rng(12)
        pts = (g.normal(size=(1, 20)) * 500 + g.normal(size=(400, 20))).astype(np.float32)
        md, r = 2, 4.5
    try:
        set_path(1)
        set_split(3)
        gsplit = gpu_build(torch, pts, md, r)
    finally:
        set_split(2)
        set_path(0)
    assert_same(gsplit, oracle.vr_build(pts, md, r), md)


@pytest.mark.parametrize("seed,scale,d", [(1, 1.0, 32), (2, 1000.0, 64), (4, 50.0, 3)])
def test_both_splits_within_quarter_beta_and_three_way_tighter(torch, seed, scale, d):
    """Both splits stay within beta/4 of the canonical FP64 value (normalised
    by |y_i|^2 + |y_j|^2); the three-way split's relative error in d over
    the kept pairs is below the two-way split's."""
    g = synth.rng(900 + seed)
    base = g.normal(size=(1, d)) * 10 * scale
    pts = (base + g.normal(size=(600, d)) * scale * g.uniform(0.01, 1.0, size=(600, 1))).astype(np.float32)
    dev = torch.from_numpy(pts).cuda()
    q = pts.astype(np.float64)
    d2 = ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1)[np.triu_indices(600, 1)]
    r = math.sqrt(float(np.quantile(d2, 0.2)))
    a2 = vr.vr_gram_accuracy_check(dev, r, split=2)
    a3 = vr.vr_gram_accuracy_check(dev, r, split=3)
    for a in (a2, a3):
        assert 0 <= a["max_norm_err"] <= a["beta"] / 4, a
        assert a["kept_pairs"] > 0 and 0 <= a["band_pairs"] <= 600 * 599 // 2
    assert a3["max_rel_d_err"] <= a2["max_rel_d_err"], (a2, a3)
    # kept pairs are the pairs with canonical d^2 <= r^2: same count for both splits
    assert a2["kept_pairs"] == a3["kept_pairs"]
