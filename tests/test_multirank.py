"""Host logic of the N > 1 path on CPU, ranks over gloo (127.0.0.1): the job's step time is the
slowest rank's and its throughput counts every rank's units over that time; one SOV problem
split by path ranges over the ranks (per-rank pairs, an all-gather, the combine) gives the
estimate of the whole problem.  No GPU."""
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
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_all_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.spawn(_rank_main, args=(world, port, q), nprocs=world, join=True)
    res = sorted(q.get() for _ in range(world))
    for rank, ms, value in res:
        assert ms == 25.0                           # max over ranks
        assert value == pytest.approx(world * 1000.0 / 0.025)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    ms, value = bench.job_time_and_value(20.0, 500.0, 1)
    assert ms == 20.0 and value == pytest.approx(500.0 / 0.02)


# ----------------------------------------------------------------- one problem split over ranks

def _shard_main(rank, world, port, out):
    """Rank `rank` of an SOV problem split by path ranges: the oracle's log-weights of this
    rank's paths, their per-shift pairs, an all-gather over gloo, and the combined estimate."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle
    from paper_2405_14892_gb300 import inputs, shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        n = 30
        c = inputs.grid_coords(6)[:n]
        L, _ = oracle.cholesky(oracle.matern(c, 1.0, 0.2, 1.5, nugget=1e-4))
        a = np.full(n, -np.inf)
        b = inputs.uniform_limits(n, -0.5, 1.5, 3)
        q = oracle.QMC(101, 6, 17)

        def partial_fn(p0, p1):
            lw = oracle.sov_logw(a, b, L, q, paths=(p0, p1))
            return torch.tensor(oracle.shift_partials(lw, p0, q.Ns, q.M).ravel())

        def gather_fn(pairs):
            bufs = [torch.empty_like(pairs) for _ in range(world)]
            dist.all_gather(bufs, pairs)
            return bufs

        def combine_fn(bufs):
            return oracle.combine_partials([x.numpy().reshape(q.M, 2) for x in bufs], q.Ns, q.M)

        est = shard.sharded_estimate(partial_fn, gather_fn, combine_fn, q.Ntot, world, rank)
        out.put((rank, est, shard.shard_range(q.Ntot, world, rank)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_problem_over_ranks_matches_the_whole_estimate(world):
    """World-size 2 and 3 gloo runs of one problem split by path ranges (606 paths: the cuts fall
    inside shifts) give, on every rank, the oracle's estimate of all paths."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle
    from paper_2405_14892_gb300 import inputs
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.spawn(_shard_main, args=(world, port, q), nprocs=world, join=True)
    res = sorted(q.get() for _ in range(world))
    n = 30
    c = inputs.grid_coords(6)[:n]
    L, _ = oracle.cholesky(oracle.matern(c, 1.0, 0.2, 1.5, nugget=1e-4))
    a = np.full(n, -np.inf)
    b = inputs.uniform_limits(n, -0.5, 1.5, 3)
    qm = oracle.QMC(101, 6, 17)
    ref = oracle.estimate(oracle.sov_logw(a, b, L, qm), qm.M)
    ranges = [r[2] for r in res]
    assert ranges[0][0] == 0 and ranges[-1][1] == qm.Ntot
    assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
    for rank, est, _ in res:
        assert abs(est[0] - ref[0]) <= 1e-13 * abs(ref[0])
        assert abs(est[1] - ref[1]) <= 1e-13 * ref[1]
        assert abs(est[2] - ref[2]) <= 1e-10 * ref[2]


def test_shard_ranges_cover_the_rule_in_balance():
    sys.path.insert(0, ROOT)
    from paper_2405_14892_gb300 import shard
    for total in (0, 1, 7, 20000, 20001):
        for world in (1, 2, 3, 8):
            rs = [shard.shard_range(total, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == total
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [p1 - p0 for p0, p1 in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)
