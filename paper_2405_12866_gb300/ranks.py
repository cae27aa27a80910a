"""Host-side logic of multi-GPU runs (one process per GPU).

QFactor-Sample instantiations of different targets are independent, so the
work shards across ranks with no collective on the data path: every rank
instantiates its own targets (weak scaling).  Collectives are used only to
combine the measurement: the slowest rank's time and the sum of converged
instantiations.
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def target_seeds(rank: int, n: int, stride: int = 100000) -> list[int]:
    """Seeds of the n targets a rank instantiates; disjoint across ranks."""
    if n > stride // 2:
        raise ValueError("more targets per rank than half the seed stride")
    return [rank * stride + i for i in range(n)]


def warmup_seeds(rank: int, n: int, stride: int = 100000) -> list[int]:
    """Seeds of the n untimed warm-up targets of a rank: the upper half of
    its seed range, disjoint from target_seeds and from other ranks."""
    if n > stride // 2:
        raise ValueError("more warm-up targets per rank than half the seed stride")
    return [rank * stride + stride // 2 + i for i in range(n)]


def combine(values_max, values_sum, device=None):
    """All-reduce across ranks: the maximum of values_max (times) and the
    sum of values_sum (counts).  Returns two lists of floats; a single
    process returns its inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values_max], [float(v) for v in values_sum]
    tm = torch.tensor([float(v) for v in values_max], dtype=torch.float64, device=device)
    ts = torch.tensor([float(v) for v in values_sum], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return tm.tolist(), ts.tolist()
