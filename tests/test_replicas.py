"""The multi-GPU split as world-size-2 ``gloo`` process groups on the CPU:
disjoint realisations per rank, round-robin shards that partition a batch,
and the max / sum / gather reductions the benchmark and batch runs use."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_math_0508111_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = replicas.realisation_seeds(3, rank)
        problems = list(range(10))
        mine = replicas.shard(problems, rank, world)
        t = replicas.max_over_ranks(1.5 + rank)          # rank 1 is the slower one
        tot = replicas.sum_over_ranks(len(mine))
        gathered = replicas.gather_to_root({"rank": rank, "seeds": seeds, "mine": mine})
        q.put((rank, seeds, mine, t, tot, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_split_and_reductions():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s0, s1 = set(res[0][1]), set(res[1][1])
    assert not (s0 & s1)                                  # different lattices per rank
    assert sorted(res[0][2] + res[1][2]) == list(range(10))  # shards partition the batch
    assert res[0][3] == res[1][3] == 2.5                   # max over ranks
    assert res[0][4] == res[1][4] == 10                    # sum over ranks
    g = res[0][5]
    assert [x["rank"] for x in g] == [0, 1] and res[1][5] is None


def test_single_process_fallbacks():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.sum_over_ranks(4) == 4.0
    assert replicas.gather_to_root("x") == ["x"]
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
