"""The bench's multi-rank host logic on CPU: two gloo ranks (one process per
rank, as torchrun launches them on GPUs) shard the units with no overlap and
no gap, meet at the barrier, and agree on the slowest rank's time and the
whole-job rate.  No GPU and no data-path collective is involved."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_units, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(backend="gloo")
    lo, hi = r.shard(n_units)
    r.barrier()
    my_time = 1.0 + rank          # rank 1 is the slowest
    slowest = r.max(my_time)
    units = r.sum(hi - lo)
    out[rank] = (lo, hi, slowest, units, bench.whole_job_rate(units, slowest))
    r.close()


@pytest.mark.parametrize("n_units", [1, 7, 4096])
def test_two_ranks_shard_and_aggregate(n_units):
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, n_units, out), nprocs=world, join=True)
        res = [out[r] for r in range(world)]
    spans = sorted((lo, hi) for lo, hi, *_ in res)
    assert spans[0][0] == 0 and spans[-1][1] == n_units
    assert spans[0][1] == spans[1][0]                   # contiguous, disjoint
    assert abs((spans[0][1] - spans[0][0]) - (spans[1][1] - spans[1][0])) <= 1
    for lo, hi, slowest, units, rate in res:
        assert slowest == 2.0                           # max over ranks
        assert units == n_units
        assert rate == n_units / 2.0


def test_single_rank_is_identity(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(backend="gloo")
    assert r.shard(10) == (0, 10)
    assert r.max(3.5) == 3.5 and r.sum(4) == 4
    r.close()
