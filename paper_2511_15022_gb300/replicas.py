"""Multi-GPU replicas (one process per GPU, launched by torchrun): every rank optimises its
own independent hologram; the only collectives are a barrier around the timed region and
a max over ranks of the measured times.  One hologram is far too small to shard and the
method has no exchange step, so no data-path collective exists.

These helpers hold the rank bookkeeping of the benchmark so that it can be exercised on
CPU (gloo) as well as on GPUs (NCCL).
"""
from __future__ import annotations

import os
from dataclasses import dataclass
from typing import Sequence

import torch


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local_rank: int

    @property
    def is_root(self) -> bool:
        return self.rank == 0


def rank_info() -> RankInfo:
    """RANK / WORLD_SIZE / LOCAL_RANK from the environment torchrun sets (1 process if
    absent)."""
    return RankInfo(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                    int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base: int, rank: int) -> int:
    """Seed of a rank's hologram: every rank optimises a different one."""
    return base + rank


def max_over_ranks(values: Sequence[float], device=None) -> list:
    """Element-wise maximum of per-rank values (times) across the process group; the
    values themselves when there is no group."""
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def aggregate_throughput(steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput (steps per second summed over the replicas) from the slowest
    rank's time for `steps` steps: every rank finishes its `steps` within ms_max."""
    return world * steps / (ms_max / 1000.0)
