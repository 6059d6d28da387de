"""Host logic of the N > 1 bench path on CPU: two ranks over gloo (127.0.0.1).  Every rank runs
its own problem (its own shift seed); the job's step time is the slowest rank's, and the job's
throughput counts every rank's units over that time.  No GPU and no data-path collective."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms_local = [10.0, 25.0][rank]
        ms, value = bench.job_time_and_value(ms_local, 1000.0, world)
        out.put((rank, ms, value, bench.rank_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_all_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.spawn(_rank_main, args=(world, port, q), nprocs=world, join=True)
    res = sorted(q.get() for _ in range(world))
    for rank, ms, value, seed in res:
        assert ms == 25.0                           # max over ranks
        assert value == pytest.approx(world * 1000.0 / 0.025)
    assert res[0][3] != res[1][3]                   # independent problems per rank


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    ms, value = bench.job_time_and_value(20.0, 500.0, 1)
    assert ms == 20.0 and value == pytest.approx(500.0 / 0.02)
