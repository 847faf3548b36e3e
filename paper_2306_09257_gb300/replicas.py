"""Replica bookkeeping for running independent designs on several GPUs.

One evaluation does not shard (the slab elimination is sequential in the
slab rows and every row's inverse would be needed on every GPU), so several
GPUs run independent designs: each rank owns a disjoint set of seeds and no
collective touches the data path.  The only collective is the max over ranks
of the timed region, used to report whole-job throughput.
"""
from __future__ import annotations

from typing import List


def replica_seeds(rank: int, designs: int, per_design: int, base: int = 0) -> List[List[int]]:
    """Seeds of rank `rank`: designs x per_design integers, disjoint across
    ranks and designs."""
    return [[base + 1000 * rank + 100 * b + i for i in range(per_design)] for b in range(designs)]


def max_over_ranks(value: float) -> float:
    """Max of a host float over all ranks of the default process group (the
    value itself if torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(world_size: int, designs: int, steps: int, max_ms: float) -> float:
    """Evaluations per second of the whole job: every rank evaluates
    designs x steps designs within the slowest rank's time."""
    return world_size * designs * steps / (max_ms / 1000.0)
