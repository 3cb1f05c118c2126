"""Host-side rank logic for running independent replicas of the solve, one
process per GPU.

The method's solve has no exchange step between independent problems (each
field, or each snapshot of a batch, is its own linear system), so N ranks run
N replicas with no data-path collective.  The only collectives are the
timing ones: a barrier on both sides of the timed region, the maximum of the
ranks' times and the sum of the ranks' work.  The backend is whatever the
process group was initialised with (NCCL on GPUs, gloo on CPU in tests).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class RankInfo:
    rank: int
    world: int
    local: int

    @classmethod
    def from_env(cls) -> "RankInfo":
        return cls(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                   int(os.environ.get("LOCAL_RANK", "0")))


class RankGroup:
    """Barrier / max / sum over the ranks of the default process group.

    With one rank every call is the identity and no process group is needed.
    ``device`` is where the reduction buffers live ("cuda" under NCCL, "cpu"
    under gloo)."""

    def __init__(self, info: RankInfo, device: str = "cpu"):
        self.info = info
        self.device = device

    def barrier(self) -> None:
        if self.info.world > 1:
            import torch.distributed as dist

            dist.barrier()

    def _reduce(self, x: float, op_name: str) -> float:
        if self.info.world == 1:
            return float(x)
        import torch
        import torch.distributed as dist

        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, "MAX")

    def sum(self, x: float) -> float:
        return self._reduce(x, "SUM")


def shard(count: int, rank: int, world: int) -> range:
    """Contiguous share of ``count`` independent instances for ``rank``: the
    first ``count % world`` ranks take one extra.  The shares are disjoint and
    cover 0..count-1."""
    if world < 1 or not 0 <= rank < world or count < 0:
        raise ValueError(f"bad shard request count={count} rank={rank} world={world}")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def aggregate_throughput(units_this_rank: float, ms_this_rank: float, group: RankGroup) -> tuple[float, float]:
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time.  Returns (units per second, max milliseconds)."""
    ms_max = group.max(ms_this_rank)
    units = group.sum(units_this_rank)
    return units / (ms_max / 1e3), ms_max
