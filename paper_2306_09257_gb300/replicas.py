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


# ---------------------------------------------------------------------------
# Multi-start optimisation (paper Sec. 3: the beam splitter is optimised from
# 1000 random initial guesses and the best final design is kept).  The starts
# are independent, so each rank runs its own share on its own GPU; the only
# communication is one host gather of the per-rank results at the end.
# ---------------------------------------------------------------------------

def partition_starts(n_starts: int, world_size: int, rank: int) -> List[int]:
    """Start indices of `rank`: a round-robin share, disjoint across ranks and
    covering 0 .. n_starts - 1."""
    return list(range(rank, n_starts, world_size))


def multistart(run_one, n_starts: int, rank: int = None, world_size: int = None):
    """Run `run_one(start)` for this rank's starts and gather to rank 0.

    run_one(start) -> (f_final, design, history) with a float objective (lower
    is better), the final design (any picklable object, e.g. the permittivity
    slab as a NumPy array) and a per-start history (e.g. the list of f per
    iteration).  Returns on rank 0 a dict with the global best
    (f, design, start, rank) and every start's (start, rank, f, history) in
    start order; on the other ranks None.  Without an initialised process
    group the calling process is the only rank."""
    import torch.distributed as dist
    dist_on = dist.is_available() and dist.is_initialized()
    if world_size is None:
        world_size = dist.get_world_size() if dist_on else 1
    if rank is None:
        rank = dist.get_rank() if dist_on else 0
    local = []
    best = None
    for st in partition_starts(n_starts, world_size, rank):
        f, design, hist = run_one(st)
        local.append((st, rank, float(f), hist))
        if best is None or f < best[0]:
            best = (float(f), design, st, rank)
    mine = {"best": best, "runs": local}
    if dist_on and world_size > 1:
        allr = [None] * world_size
        dist.all_gather_object(allr, mine)  # host objects; works on gloo and nccl groups
    else:
        allr = [mine]
    if rank != 0:
        return None
    runs = sorted((r for part in allr for r in part["runs"]), key=lambda r: r[0])
    bests = [part["best"] for part in allr if part["best"] is not None]
    gbest = min(bests, key=lambda b: (b[0], b[2])) if bests else None
    return {"best_f": gbest[0] if gbest else None, "best_design": gbest[1] if gbest else None,
            "best_start": gbest[2] if gbest else None, "best_rank": gbest[3] if gbest else None,
            "runs": runs}


def optimize_start(solver, w, start: int, kind: str, orders, target: float, iters: int, seed_base: int = 10 ** 6):
    """One start of the multi-start beam-splitter optimisation on this rank's
    GPU: the seeded filtered-threshold design `seed_base + start` of workload
    `w`, optimised by the Armijo line search (optim.optimize) with every
    evaluation on the solver.  Returns (f_final, eps_final, f history)."""
    from . import optim
    eps0 = w.eps_slab(seed_base + start)
    eps, hist = optim.optimize(solver, eps0, w.eps_sub, w.eps_clad, w.j0, kind, orders, target, iters)
    return hist.f[-1], eps, hist.f
