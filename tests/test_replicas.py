"""The N>1 (replicas) path of the benchmark on CPU: world_size-2 gloo ranks
shard ligands without overlap and reduce time (max) and work (sum)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2007_03678_gb300.replicas import reduce_run, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(10, rank, world)
    ms, units = reduce_run(100.0 + 50.0 * rank, float(len(mine) * 1000), dist)
    q.put((rank, mine, ms, units))
    dist.destroy_process_group()


def test_shard_partitions():
    from paper_2007_03678_gb300.replicas import shard
    parts = [shard(11, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == list(range(11))
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def test_reduce_single_process():
    from paper_2007_03678_gb300.replicas import reduce_run
    assert reduce_run(12.5, 7.0) == (12.5, 7.0)


def test_two_rank_gloo_reduction():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, ms0, u0), (r1, m1, ms1, u1) = out
    assert set(m0).isdisjoint(m1) and sorted(m0 + m1) == list(range(10))
    assert ms0 == ms1 == 150.0
    assert u0 == u1 == 10 * 1000.0
