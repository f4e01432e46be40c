"""Failure handling, exercised without faulting, trapping or hanging a GPU.

Every fault here is made on the host or by a kernel that withholds a signal
under a short bounded wait (include/vr_inject.h):
  * the n-th device allocation fails: the call returns VR_ERR_OOM and gives
    back everything it had allocated (the stream-ordered pool's used bytes
    return to where they were), for vr_build, vr_build_batch and the server;
  * one tile of a radix digit pass never publishes its count: later tiles'
    look-back waits give up and the build reports VR_ERR_TIMEOUT (at the next
    size read, or through vr_complex_status when it happens after the last);
  * one tensor-core distance tile never signals MMA completion: its wait
    gives up, the build reports VR_ERR_TIMEOUT;
  * the server's memory admission refuses batches: the clouds go back to the
    queue and complete later;
  * vr_serve_poll with a 1 us timeout on a pending ticket: VR_ERR_TIMEOUT,
    then the ticket completes.
After each fault the next call on the same stream is bit-exact against the
oracle."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1809_04424_b300 as vr
import synth
from test_gpu_parity import assert_same

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(autouse=True)
def disarm():
    yield
    vr.vr_inject_clear()
    vr.lib().vr_set_gram_path(0)


def result_dict(cx, maxdim):
    g = {"gv": cx.grade_values()}
    for k in range(maxdim + 1):
        g[k] = cx.to_host(k)
    return g


def check_against_oracle(torch, cloud):
    cx = vr.vr_build(torch.from_numpy(cloud.points).cuda(), cloud.maxdim, cloud.maxrad)
    assert cx.status() == vr.VR_OK
    assert_same(result_dict(cx, cloud.maxdim), oracle.vr_build(cloud.points, cloud.maxdim, cloud.maxrad),
                cloud.maxdim)


def pool_used(torch):
    torch.cuda.synchronize()
    return vr.vr_pool_used_bytes()


def fail_each_allocation(torch, call, max_allocs=64):
    """Make the 1st, 2nd, ... allocation of `call` fail until a run makes
    fewer allocations than that (it then succeeds).  Each failing run must
    return VR_ERR_OOM and leave the pool's used bytes as they were.
    Returns how many allocations the call makes."""
    call()  # warm: persistent per-thread buffers are made once
    base = pool_used(torch)
    for k in range(1, max_allocs + 1):
        vr.vr_inject_alloc_failure(k)
        try:
            r = call()
        except vr.VRError as e:
            assert e.status == vr.VR_ERR_OOM, (k, e)
            del e
            assert pool_used(torch) == base, f"allocation {k} failed and {pool_used(torch) - base} bytes stayed"
            continue
        vr.vr_inject_alloc_failure(0)
        del r
        assert pool_used(torch) == base
        return k - 1
    raise AssertionError(f"more than {max_allocs} allocations")


def test_vr_build_out_of_memory_at_every_allocation(torch):
    c = synth.config2()
    src = torch.from_numpy(c.points).cuda()
    n = fail_each_allocation(torch, lambda: vr.vr_build(src, c.maxdim, c.maxrad))
    assert n >= 3
    check_against_oracle(torch, c)


def test_float_tensor_core_build_out_of_memory(torch):
    """The tensor-core distance path's own allocations (operands, norms,
    near-cap list) included."""
    vr.lib().vr_set_gram_path(1)
    c = synth.config3(n=700)
    src = torch.from_numpy(c.points).cuda()
    n = fail_each_allocation(torch, lambda: vr.vr_build(src, c.maxdim, c.maxrad))
    assert n >= 6
    check_against_oracle(torch, c)


def test_batch_out_of_memory_at_every_allocation(torch):
    clouds = synth.config4(48)
    pts = np.concatenate([c.points for c in clouds], axis=0)
    off = np.concatenate([[0], np.cumsum([c.n for c in clouds])]).astype(np.int64)
    dev = torch.from_numpy(pts).cuda()
    n = fail_each_allocation(torch, lambda: vr.vr_build_batch(dev, off, 2, 40.0))
    assert n >= 3
    b = vr.vr_build_batch(dev, off, 2, 40.0)
    for i, c in enumerate(clouds[:12]):
        st, view = b.get(i)
        assert st == vr.VR_OK
        assert_same(result_dict(view, 2), oracle.vr_build(c.points, 2, 40.0), 2)


def test_server_out_of_memory_fails_requests_then_recovers(torch):
    reqs = [synth.Cloud(synth.quantize(synth.sphere(int(m), synth.rng(int(m))), 100.0), 2, 40.0)
            for m in (60, 90, 120, 150, 180, 210)]
    srv = vr.Server(n_streams=1, max_batch_clouds=2, n_large_workers=1)
    for c in reqs[:2]:  # warm: the slot's buffers exist
        srv.poll(srv.submit(c.points, c.maxdim, c.maxrad), 60_000_000)
    base = pool_used(torch)
    vr.vr_inject_alloc_failure(1)
    tickets = [srv.submit(c.points, c.maxdim, c.maxrad) for c in reqs]
    failed = 0
    for c, t in zip(reqs, tickets):
        try:
            got = result_dict(srv.poll(t, 60_000_000), c.maxdim)
            assert_same(got, oracle.vr_build(c.points, c.maxdim, c.maxrad), c.maxdim)
        except vr.VRError as e:
            assert e.status == vr.VR_ERR_OOM
            failed += 1
    assert failed >= 1
    st = srv.stats()
    assert st["failed"] == failed and st["completed"] == 2 + len(reqs) - failed
    for c in reqs:  # and it keeps serving
        got = result_dict(srv.poll(srv.submit(c.points, c.maxdim, c.maxrad), 60_000_000), c.maxdim)
        assert_same(got, oracle.vr_build(c.points, c.maxdim, c.maxrad), c.maxdim)
    srv.close()
    assert pool_used(torch) <= base


def test_edge_sort_lookback_timeout_then_exact(torch):
    """Torus workload: 74,934 edge keys (74 tiles of 1024) -- tile 1 of the
    first digit pass withholds its count."""
    c = synth.config2()
    src = torch.from_numpy(c.points).cuda()
    vr.vr_inject_lookback_stall(1, 2000)
    with pytest.raises(vr.VRError) as e:
        vr.vr_build(src, c.maxdim, c.maxrad)
    assert e.value.status == vr.VR_ERR_TIMEOUT
    del e
    check_against_oracle(torch, c)


def test_triangle_sort_timeout_reported_late_then_exact(torch):
    """The triangle grade sort runs after the build's last size read: the
    timeout comes back through vr_complex_status and vr_complex_to_host.
    Tile 100 exists only in the triangle sort (590 tiles; the edge sort has
    74)."""
    c = synth.config2()
    src = torch.from_numpy(c.points).cuda()
    vr.vr_inject_lookback_stall(100, 2000)
    cx = vr.vr_build(src, c.maxdim, c.maxrad)
    assert cx.status() == vr.VR_ERR_TIMEOUT
    with pytest.raises(vr.VRError) as e:
        cx.to_host(2)
    assert e.value.status == vr.VR_ERR_TIMEOUT
    del cx, e
    check_against_oracle(torch, c)


def test_sort_primitive_timeout_then_exact(torch):
    g = synth.rng(4)
    keys = g.integers(0, 2**63, size=1_000_000, dtype=np.uint64)
    dev = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    vr.vr_inject_lookback_stall(5, 2000)
    with pytest.raises(vr.VRError) as e:
        vr.vr_sort_keys(dev, 0, 24)
    assert e.value.status == vr.VR_ERR_TIMEOUT
    dev = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    vr.vr_sort_keys(dev, 0, 24)
    torch.cuda.synchronize()
    field = keys & np.uint64((1 << 24) - 1)
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), keys[np.argsort(field, kind="stable")])


@pytest.mark.parametrize("dtype", ["float32", "int8"])
def test_gram_tile_timeout_then_exact(torch, dtype):
    """Tensor-core distance tiles forced on (700 points: 21 tiles); tile 7
    issues no MMA, its completion wait gives up."""
    vr.lib().vr_set_gram_path(1)
    if dtype == "float32":
        c = synth.config3(n=700)
    else:
        g = synth.rng(21)
        c = synth.Cloud(g.integers(-60, 61, size=(700, 24)).astype(np.int8), 2, 140.0)
    src = torch.from_numpy(c.points).cuda()
    vr.vr_inject_gram_stall(7, 4000)
    with pytest.raises(vr.VRError) as e:
        vr.vr_build(src, c.maxdim, c.maxrad)
    assert e.value.status == vr.VR_ERR_TIMEOUT
    del e
    check_against_oracle(torch, c)


def test_admission_refusals_defer_then_complete(torch):
    g = synth.rng(31)
    reqs = []
    while len(reqs) < 40:
        c = synth.config5_request(g)
        if c.n <= 600:
            reqs.append(c)
    srv = vr.Server(n_streams=2, max_batch_clouds=8)
    vr.vr_inject_admission_refusals(3)
    tickets = [srv.submit(c.points, c.maxdim, c.maxrad) for c in reqs]
    for c, t in zip(reqs, tickets):
        got = result_dict(srv.poll(t, 60_000_000), c.maxdim)
        assert_same(got, oracle.vr_build(c.points, c.maxdim, c.maxrad), c.maxdim)
    st = srv.stats()
    assert st["deferred"] >= 3 and st["completed"] == len(reqs) and st["failed"] == 0
    srv.close()


def test_poll_timeout_on_pending_ticket(torch):
    """A ticket held pending: every admission refused until the hook is
    cleared.  Polls with 1 us and 20 ms time out; after the hook is cleared
    the same ticket completes with the result vr_build gives alone."""
    c = synth.config5_request(synth.rng(43))
    while c.n > 600:
        c = synth.config5_request(synth.rng(c.n))
    srv = vr.Server(n_streams=1)
    vr.vr_inject_admission_refusals(10**9)
    t = srv.submit(c.points, c.maxdim, c.maxrad)
    for wait_us in (1, 20_000):
        with pytest.raises(vr.VRError) as e:
            srv.poll(t, wait_us)
        assert e.value.status == vr.VR_ERR_TIMEOUT
    vr.vr_inject_clear()
    got = result_dict(srv.poll(t, 60_000_000), c.maxdim)
    assert_same(got, oracle.vr_build(c.points, c.maxdim, c.maxrad), c.maxdim)
    assert srv.stats()["deferred"] >= 1
    srv.close()
