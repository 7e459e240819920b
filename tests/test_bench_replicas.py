"""The bench's multi-rank path on the CPU: independent replicas on two `gloo`
ranks, whole-job time = the slowest rank's, value = units of all ranks / that
time.  No GPU and no data-path collective are involved."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [2.0, 3.0, 2.5][rank]           # seconds this replica took
        secs, value = bench.job_time_and_value(local, 600.0, world, device="cpu")
        q.put((rank, secs, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_aggregation_takes_slowest_rank(world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(world))
    slowest = max([2.0, 3.0, 2.5][:world])
    for rank, secs, value in got:
        assert secs == slowest
        assert value == pytest.approx(600.0 * world / slowest)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_time_and_value(4.0, 100.0, 1) == (4.0, 25.0)
