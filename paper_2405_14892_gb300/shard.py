"""One SOV problem split over several GPUs (one process per GPU, torch.distributed).

The lattice paths are independent QMC samples (Sec. IV-C: the samples of Alg. 2 are processed
in parallel), so every rank sweeps a contiguous range of them with the same factor and limits
(mvn_sov_partial), the ranks exchange their per-shift pairs (2 * n_shifts doubles each, one
all-gather), and every rank combines them into the estimate (mvn_sov_combine).  The factor is
not split: each rank holds its own copy (the Cholesky does not divide into independent units).

Argument marshalling and the exchange only; every step of the computation runs in the library.
"""
from __future__ import annotations

from typing import Callable


def shard_range(n_paths: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced path range [p0, p1) of rank `rank` among `world` ranks (the first
    n_paths % world ranks take one path more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    base, extra = divmod(int(n_paths), world)
    p0 = rank * base + min(rank, extra)
    return p0, p0 + base + (1 if rank < extra else 0)


def sharded_estimate(partial_fn: Callable, gather_fn: Callable, combine_fn: Callable,
                     n_paths: int, world: int, rank: int):
    """The shard protocol: this rank's pairs for its range, all ranks' pairs gathered in rank
    order, and the combined estimate.  partial_fn(p0, p1) -> pairs; gather_fn(pairs) -> the
    world's pairs stacked in rank order; combine_fn(stacked) -> (log P, P, err)."""
    p0, p1 = shard_range(n_paths, world, rank)
    return combine_fn(gather_fn(partial_fn(p0, p1)))


def sov_sharded(a, b, L, n_points: int, n_shifts: int, seed: int, prec: str = "fp64",
                err_k: float = 3.0, group=None, out3=None):
    """mvn_sov over all ranks of `group` (default: the world): the same estimate as one GPU's
    mvn_sov on the whole rule (to rounding where a rank's range cuts a shift).  Every rank must
    call it with the same arguments; returns out3 on every rank."""
    import torch
    import torch.distributed as dist

    from . import mvn

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    n_paths = int(n_points) * int(n_shifts)

    def partial_fn(p0, p1):
        return mvn.mvn_sov_partial(a, b, L, n_points, n_shifts, seed, p0, p1, prec=prec,
                                   err_k=err_k)

    def gather_fn(pairs):
        if world == 1:
            return pairs
        allp = torch.empty(world * pairs.numel(), dtype=pairs.dtype, device=pairs.device)
        dist.all_gather_into_tensor(allp, pairs, group=group)
        return allp

    def combine_fn(stacked):
        return mvn.mvn_sov_combine(stacked, n_points, n_shifts, err_k=err_k, out3=out3)

    return sharded_estimate(partial_fn, gather_fn, combine_fn, n_paths, world, rank)
