"""Frequency-parallel sharding of the X-stage across ranks.

The paper parallelises the X-stage by frequency: each GPU processes its own
sub-band of channels and no data moves between GPUs (Sec. 2.1).  A rank
therefore owns a contiguous band of channels and runs the whole X-stage on it;
the only inter-rank traffic is host-side coordination (a barrier and the
maximum of the ranks' step times), never visibility data.
"""

from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local_rank: int


def rank_info() -> RankInfo:
    return RankInfo(int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
                    int(os.environ.get("LOCAL_RANK", 0)))


def channel_band(rank: int, world: int, n_channels_total: int) -> tuple[int, int]:
    """Contiguous channel range [c0, c1) of one rank; bands differ by at most one channel."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(n_channels_total, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def init(backend: str) -> RankInfo:
    """Join the process group when launched with several ranks (env:// rendezvous)."""
    info = rank_info()
    if info.world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
    return info


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the step time of the slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
