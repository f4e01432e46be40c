"""Serving: requests submitted while others run are batched, admitted by
memory and overlapped; every result must be bit-for-bit the one vr_build
gives for the same request alone (and the oracle's), in any mix."""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import paper_1809_04424_b300 as vr
import synth
from test_gpu_parity import assert_same

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def alone(torch, c):
    cx = vr.vr_build(torch.from_numpy(c.points).cuda(), c.maxdim, c.maxrad)
    return result_dict(cx, c.maxdim)


def result_dict(cx, maxdim):
    g = {"gv": cx.grade_values()}
    for k in range(maxdim + 1):
        g[k] = cx.to_host(k)
    return g


def same(a, b, maxdim):
    assert a["gv"].tobytes() == b["gv"].tobytes()
    for k in range(maxdim + 1):
        for f in ("count", "verts", "grade", "colptr", "rowidx"):
            x, y = a[k][f], b[k][f]
            if isinstance(x, np.ndarray):
                np.testing.assert_array_equal(x, y)
            else:
                assert x == y


def requests(seed, count, nmax=1400):
    g = synth.rng(seed)
    out = []
    while len(out) < count:
        c = synth.config5_request(g)
        if c.n <= nmax:
            out.append(c)
    return out


def test_mixed_stream_equals_alone(torch):
    reqs = requests(11, 150)
    srv = vr.Server(n_streams=3, max_batch_clouds=64)
    tickets = [srv.submit(c.points, c.maxdim, c.maxrad) for c in reqs]
    for c, t in zip(reqs, tickets):
        got = result_dict(srv.poll(t, 20_000_000), c.maxdim)
        same(got, alone(torch, c), c.maxdim)
    for c in reqs[:12]:  # and the oracle, for a sample
        got = alone(torch, c)
        assert_same(got, oracle.vr_build(c.points, c.maxdim, c.maxrad), c.maxdim)
    srv.close()


def test_config5_stream_sample_equals_oracle(torch):
    """The first 300 requests of the 20000-request serving stream, as drawn
    (n log-uniform in [50, 5000], int8 d=3 and float32 d=16, maxdim 1 or 2,
    per-request caps), all submitted at once: requests above 1400 points take
    the server's single-cloud workers, the rest its batches.  Every result
    equals the oracle's complex."""
    reqs = synth.config5(300)[1]
    big = [c for c in reqs if c.n > 1400]
    assert any(c.points.dtype == np.int8 for c in big) and any(c.points.dtype == np.float32 for c in big)
    assert max(c.n for c in reqs) > 4000
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        refs = list(ex.map(lambda c: oracle.vr_build(c.points, c.maxdim, c.maxrad), reqs))
    srv = vr.Server(n_streams=3, max_batch_clouds=256, n_large_workers=4)
    tickets = [srv.submit(c.points, c.maxdim, c.maxrad) for c in reqs]
    for c, t, ref in zip(reqs, tickets, refs):
        assert_same(result_dict(srv.poll(t, 120_000_000), c.maxdim), ref, c.maxdim)
    srv.close()


def test_small_memory_budget_defers_but_completes(torch):
    reqs = requests(12, 60, nmax=600)
    srv = vr.Server(mem_budget_bytes=2 << 20, n_streams=2, max_batch_clouds=32)
    tickets = [srv.submit(c.points, c.maxdim, c.maxrad) for c in reqs]
    for c, t in zip(reqs, tickets):
        same(result_dict(srv.poll(t, 20_000_000), c.maxdim), alone(torch, c), c.maxdim)
    srv.close()


def test_bad_request_fails_alone_and_unknown_ticket():
    srv = vr.Server()
    good = synth.gaussian_mixture(40, 3, synth.rng(3))
    bad = good.copy()
    bad[0, 0] = np.inf
    t1 = srv.submit(good, 2, 5.0)
    t2 = srv.submit(bad, 2, 5.0)
    t3 = srv.submit(good, 1, 5.0)
    assert srv.poll(t1).counts()[0][0] == 40
    with pytest.raises(vr.VRError) as e:
        srv.poll(t2)
    assert e.value.status == vr.VR_ERR_ARG
    assert srv.poll(t3).counts()[1] == 1
    with pytest.raises(vr.VRError) as e:
        srv.poll(10**9, 1000)
    assert e.value.status == vr.VR_ERR_ARG
    with pytest.raises(vr.VRError) as e:
        srv.submit(good, 3, 5.0)
    assert e.value.status == vr.VR_ERR_UNSUPPORTED
    srv.close()


def test_queue_full_is_busy_and_accepted_complete():
    srv = vr.Server(max_queue=4, n_streams=1, max_batch_clouds=2)
    pts = synth.random_cloud(300, 3, np.int8, seed=9)
    tickets, busy = [], 0
    for _ in range(400):
        try:
            tickets.append(srv.submit(pts, 2, 30.0))
        except vr.VRError as e:
            assert e.status == vr.VR_ERR_BUSY
            busy += 1
    assert busy > 0
    ref = None
    for t in tickets:
        r = srv.poll(t, 20_000_000).counts()[0]
        ref = ref or r
        assert r == ref
    srv.close()
