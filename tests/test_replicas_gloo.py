"""Multi-process (gloo, world size 2, CPU) check of the replica logic used
by bench.py for N > 1: disjoint seeds per rank and the max-over-ranks time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2306_09257_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = replicas.replica_seeds(rank, designs=3, per_design=4)
    local_ms = 100.0 + 50.0 * rank
    m = replicas.max_over_ranks(local_ms)
    out[rank] = (seeds, m, replicas.whole_job_throughput(world, 3, 5, m))
    dist.destroy_process_group()


def test_two_rank_replicas():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    s0, m0, v0 = out[0]
    s1, m1, v1 = out[1]
    flat0 = {x for row in s0 for x in row}
    flat1 = {x for row in s1 for x in row}
    assert len(flat0) == 12 and len(flat1) == 12 and not (flat0 & flat1)
    assert m0 == m1 == 150.0
    assert v0 == v1 == pytest.approx(2 * 3 * 5 / 0.150)


def _quadratic_start(start):
    """CPU stand-in for one optimisation start: gradient descent on a seeded
    quadratic, f = |x - c|^2 + start * 0.01 (so the best start is known)."""
    import numpy as np
    rng = np.random.default_rng(start)
    x = rng.normal(size=4)
    c = np.arange(4.0)
    hist = []
    for _ in range(20):
        hist.append(float(np.sum((x - c) ** 2) + 0.01 * start))
        x = x - 0.25 * 2 * (x - c)
    f = float(np.sum((x - c) ** 2) + 0.01 * start)
    hist.append(f)
    return f, x, hist


def _ms_worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2306_09257_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = replicas.multistart(_quadratic_start, 7)
    out[rank] = res
    dist.destroy_process_group()


def test_two_rank_multistart_gathers_the_best():
    from paper_2306_09257_gb300 import replicas
    assert replicas.partition_starts(7, 2, 0) == [0, 2, 4, 6]
    assert replicas.partition_starts(7, 2, 1) == [1, 3, 5]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_ms_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[1] is None
    r = out[0]
    assert [x[0] for x in r["runs"]] == list(range(7))
    assert [x[1] for x in r["runs"]] == [0, 1, 0, 1, 0, 1, 0]
    # the same starts run in one process give the same results (no data-path collective)
    single = replicas.multistart(_quadratic_start, 7, rank=0, world_size=1)
    assert [x[2] for x in r["runs"]] == [x[2] for x in single["runs"]]
    assert r["best_start"] == 0 and r["best_rank"] == 0
    assert r["best_f"] == min(x[2] for x in r["runs"])
    assert all(h[-1] <= h[0] for _, _, _, h in r["runs"])
