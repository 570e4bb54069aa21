"""Replica plumbing across two processes (gloo, CPU): max-over-ranks timing,
whole-job weak-scaling rate, and the tensor-to-rank assignment of the
batched workload."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2012_03550_gb300 import dist as D
    D.init("gloo")
    try:
        assert D.world() == (world, rank, rank)
        D.barrier()
        secs = 1.0 + rank          # rank 1 is the slow one
        rate, tmax = D.weak_scaling_rate(100.0 * (rank + 1), secs)
        mine = D.shard([5, 1, 4, 4, 3, 9, 2], world, rank)
        out[rank] = (rate, tmax, tuple(mine))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    r0, r1 = out[0], out[1]
    # total units 100 + 200 over the slowest rank's 2 s
    assert r0[0] == pytest.approx(150.0) and r1[0] == pytest.approx(150.0)
    assert r0[1] == 2.0 and r1[1] == 2.0
    # the two shards partition the items and balance the weights
    assert sorted(r0[2] + r1[2]) == list(range(7))
    w = [5, 1, 4, 4, 3, 9, 2]
    loads = [sum(w[i] for i in r0[2]), sum(w[i] for i in r1[2])]
    assert abs(loads[0] - loads[1]) <= max(w)


def test_single_process_defaults():
    from paper_2012_03550_gb300 import dist as D
    assert D.max_over_ranks(3.5) == 3.5
    assert D.shard([1, 2, 3], 1, 0) == [0, 1, 2]
