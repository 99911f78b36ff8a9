"""The N > 1 bench path on CPU: two gloo ranks, replicas with max-over-ranks timing.

bench.py runs one independent replica per GPU (the protocol's party axis is
local, so there is no data-path collective); the only cross-rank step is the
timing reduction.  Here two CPU processes check that the whole-job value uses
the slowest rank's time and counts every rank's units, and that a rank that
never joins makes the others fail with an error instead of hanging.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [0.50, 0.80][rank]            # rank 1 is the slow replica
    slowest = bench.job_time(local, world)
    q.put((rank, slowest, bench.whole_job_rate(10, world, slowest)))
    dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in out:
        assert slowest == pytest.approx(0.80)
        assert rate == pytest.approx(2 * 10 / 0.80)


def _lonely(port, q):
    sys.path.insert(0, ROOT)
    from datetime import timedelta
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        dist.init_process_group("gloo", rank=0, world_size=2, timeout=timedelta(seconds=3))
        q.put("joined")
    except Exception as e:     # the peer never arrives: an error, not a hang
        q.put(type(e).__name__)


def test_missing_rank_fails_fast():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_lonely, args=(_free_port(), q))
    p.start()
    p.join(60)
    assert p.exitcode == 0
    assert q.get(timeout=5) != "joined"
