"""Batched builds: every cloud of a batch must equal the oracle's complex bit
for bit (and so vr_build's), whatever the mix of sizes, dtypes, caps and
maxdims; clouds too large for the fused path, tiny clouds and bad clouds
included."""
import math
import os
from concurrent.futures import ThreadPoolExecutor

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


def concat(clouds):
    pts = np.concatenate([c.points for c in clouds], axis=0)
    off = np.concatenate([[0], np.cumsum([c.n for c in clouds])]).astype(np.int64)
    return pts, off


def check_batch(torch, clouds, on_device=True):
    pts, off = concat(clouds)
    src = torch.from_numpy(pts).cuda() if on_device else pts
    b = vr.vr_build_batch(src, off, [c.maxdim for c in clouds], [c.maxrad for c in clouds])
    for i, c in enumerate(clouds):
        st, view = b.get(i)
        assert st == vr.VR_OK, (i, st)
        g = {"gv": view.grade_values()}
        for k in range(c.maxdim + 1):
            g[k] = view.to_host(k)
        assert_same(g, oracle.vr_build(c.points, c.maxdim, c.maxrad), c.maxdim)
    return b


def oracle_many(clouds):
    """Oracle complexes of many clouds, built by host threads (the oracle's C
    call releases the interpreter lock, so they run in parallel)."""
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        return list(ex.map(lambda c: oracle.vr_build(c.points, c.maxdim, c.maxrad), clouds))


@pytest.mark.timeout(900)
def test_full_sphere_batch_4096_clouds(torch):
    """The whole uneven sphere workload (4096 clouds, n ~ U[32, 512], int8,
    cap 40, maxdim 2) in one vr_build_batch; every cloud equals the oracle."""
    clouds = synth.config4(4096)
    refs = oracle_many(clouds)
    pts, off = concat(clouds)
    b = vr.vr_build_batch(torch.from_numpy(pts).cuda(), off, 2, 40.0)
    info = b.info()
    assert info["n_failed"] == 0
    total = 0
    for i, c in enumerate(clouds):
        st, view = b.get(i)
        assert st == vr.VR_OK, (i, st)
        g = {"gv": view.grade_values()}
        for k in range(3):
            g[k] = view.to_host(k)
        assert_same(g, refs[i], 2)
        total += sum(d.count for d in refs[i].dims)
    assert info["total_simplices"] == total


def test_sphere_batch_int8(torch):
    """64 clouds of the uneven sphere workload (n in [32, 512], cap 40)."""
    b = check_batch(torch, synth.config4(64))
    assert b.info()["n_failed"] == 0


def test_mixed_float_batch(torch):
    g = synth.rng(55)
    clouds = []
    for k in range(40):
        n = int(g.integers(2, 300))
        pts = synth.gaussian_mixture(n, 16, g)
        clouds.append(synth.Cloud(pts, int(g.integers(0, 3)), float(g.uniform(4, 9))))
    check_batch(torch, clouds)


def test_batch_with_fallback_and_tiny_clouds(torch):
    g = synth.rng(66)
    clouds = [synth.Cloud(np.zeros((1, 3), np.int8), 2, math.inf),
              synth.Cloud(g.integers(-127, 128, size=(1300, 3)).astype(np.int8), 2, 12.0),  # single-cloud path
              synth.Cloud(g.integers(-5, 6, size=(40, 3)).astype(np.int8), 1, math.inf),
              synth.Cloud(np.full((30, 3), 4, np.int8), 2, math.inf)]                      # all ties
    check_batch(torch, clouds)


def test_batch_int32_and_host_input(torch):
    g = synth.rng(77)
    clouds = [synth.Cloud(g.integers(-1000, 1000, size=(int(n), 4)).astype(np.int32), 2, 700.0)
              for n in g.integers(10, 200, size=20)]
    check_batch(torch, clouds, on_device=False)


def test_bad_cloud_fails_alone(torch):
    good = synth.gaussian_mixture(50, 3, synth.rng(1))
    bad = good.copy()
    bad[3, 1] = np.nan
    clouds = [synth.Cloud(good, 2, 5.0), synth.Cloud(bad, 2, 5.0), synth.Cloud(good, 1, 5.0)]
    pts, off = concat(clouds)
    b = vr.vr_build_batch(torch.from_numpy(pts).cuda(), off, 2, 5.0)
    assert b.get(0)[0] == vr.VR_OK and b.get(2)[0] == vr.VR_OK
    assert b.get(1)[0] == vr.VR_ERR_ARG and b.get(1)[1] is None
    assert b.info()["n_failed"] == 1


@pytest.mark.parametrize("cps,order", [(1, 0), (1, 1), (2, 0), (3, 1)])
def test_pinned_shapes_give_the_same_complexes(torch, cps, order):
    """The one-launch batch under each pinned launch shape (CTAs per SM,
    work-list order): every cloud still equals the oracle."""
    clouds = synth.config4(96)
    vr.vr_batch_set_shape(cps, order)
    try:
        check_batch(torch, clouds)
        used = vr.vr_batch_get_shape()["used"]
        assert used[1] == order and 1 <= used[0] <= cps
    finally:
        vr.vr_batch_set_shape(0)


def test_tuner_records_candidates(torch):
    vr.vr_batch_tune_reset()
    clouds = synth.config4(128)
    check_batch(torch, clouds)
    info = vr.vr_batch_get_shape()
    assert len(info["candidates"]) >= 2
    assert info["used"] in [c for c, _ in info["candidates"]]
    assert all(ms > 0 for _, ms in info["candidates"])
    best = min(info["candidates"], key=lambda c: c[1])[0]
    assert info["used"] == best


def test_batch_outgrowing_the_arenas_is_rebuilt_exactly(torch):
    """A class first seen with sparse clouds, then with much denser ones of
    the same sizes: the second batch overflows the arenas sized from the
    first and is rebuilt into exact ones."""
    vr.vr_batch_set_shape(2, 0)
    try:
        g = synth.rng(88)
        sizes = g.integers(200, 257, size=40)
        sparse = [synth.Cloud(synth.quantize(synth.sphere(int(m), g), 100.0), 2, 20.0) for m in sizes]
        dense = [synth.Cloud(c.points, 2, 60.0) for c in sparse]
        check_batch(torch, sparse)
        check_batch(torch, dense)
        check_batch(torch, sparse)
    finally:
        vr.vr_batch_set_shape(0)
