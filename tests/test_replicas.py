"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks, each timing
its own replica, agree on the slowest rank's time, and the whole-job value
is that time per body.  The solve itself has no data-parallel split (one
body per GPU), so no other collective exists to test."""

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


def _rank(rank, world, port, times, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, w, local, dist = bench._dist(backend="gloo")
    try:
        m = bench.max_over_ranks(times[r], dist, "cpu")
        dist.barrier()
        q.put((r, w, local, m, bench.replica_value_s(m, w)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [40.5, 43.25]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, local, m, v in out:
        assert w == 2 and local == r and m == 43.25
        assert v == pytest.approx(43.25 / 1000.0 / 2)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.replica_value_s(40.0, 1) == 0.04
