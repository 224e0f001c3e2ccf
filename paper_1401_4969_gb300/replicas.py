"""Host-side logic of multi-process runs: one process per GPU, no data-path collective.

A single eigenproblem does not shard (Algorithm 4.2 is one solve); N processes run N
independent replicas of it. A batch of independent eigenproblems shards by problem: each
rank solves a contiguous share of the batch and no data moves between ranks. Timing is
the maximum over ranks of each rank's device time, and the whole-job rate counts the
units every rank processed.
"""
from __future__ import annotations


def env_ranks(environ=None) -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process if unset)."""
    import os

    e = os.environ if environ is None else environ
    return int(e.get("RANK", 0)), int(e.get("LOCAL_RANK", 0)), int(e.get("WORLD_SIZE", 1))


def batch_share(batch: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of the problems of a batch that `rank` solves: contiguous, sizes differ by
    at most one, every problem on exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(batch, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank number over the process group (the slowest rank sets the time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_this_rank: float, ms_this_rank: float, dist=None, device=None) -> tuple[float, float]:
    """(units per second of the whole job, slowest rank's ms): all ranks' units over the
    maximum time."""
    ms = max_over_ranks(ms_this_rank, dist, device)
    units = sum_over_ranks(units_this_rank, dist, device)
    return units / (ms / 1e3), ms
