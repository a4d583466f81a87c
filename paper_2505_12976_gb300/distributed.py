"""Multi-process pieces of the path (torch.distributed, one process per GPU).

The work partitions two ways (Sect. 2.1):

* independent elections: each rank runs its own, no collective;
* one election's tally: d[i][j] counts the voters ranking i above j, a sum
  over voters, so each rank tallies a contiguous shard of the ballots and one
  int32 sum all-reduce gives every rank the whole d exactly. The closure of
  d is not sharded: each rank closes the summed d (replicas).

Host orchestration only: the tally itself is the library's (schulze_tally).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def voter_shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of the ballots rank `rank` of `world` tallies: contiguous,
    sizes differing by at most one, covering 0..n-1 once."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def tally_voter_sharded(ranks_local: torch.Tensor, m: int, flags: int = 0, ctx=None, group=None,
                        tally=None) -> torch.Tensor:
    """d of the whole election from this rank's shard of the ballots: the
    local tally (schulze_tally, or `tally(ranks, m, flags=..., ctx=...)`)
    summed over the ranks of `group` by one all-reduce. Every rank gets d."""
    if tally is None:
        from . import schulze_tally as tally
    d = tally(ranks_local, m, flags=flags, ctx=ctx)
    if d.dtype != torch.int32:
        raise TypeError("the tally must be int32")
    dist.all_reduce(d, op=dist.ReduceOp.SUM, group=group)
    return d


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest of the ranks' values (step times: the job is as slow as
    its slowest rank)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
