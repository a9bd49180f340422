"""The N > 1 host logic of bench.py (one process per GPU, independent
replicas, max-over-ranks timing) with world_size 2 on CPU over gloo."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [1.5, 2.5][rank]  # rank 1 is the slow one
        got = bench.max_over_ranks(secs, world, "cpu")
        rate = bench.aggregate_rate(world, 3, 1000, got)
        out.put((rank, got, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    # every rank sees the slowest rank's time; the rate counts both ranks' work
    assert [r[1] for r in res] == [2.5, 2.5]
    assert all(abs(r[2] - 2 * 3 * 1000 / 2.5) < 1e-9 for r in res)


def test_one_rank_is_local():
    import bench
    assert bench.max_over_ranks(1.25, 1, None) == 1.25
    assert bench.aggregate_rate(1, 4, 10, 2.0) == 20.0
