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


def _batch_main(rank, world, port, q):
    """Each rank takes its balanced share of a mixed-L batch; the root
    gathers every rank's (problem, result) list."""
    import torch.distributed as dist
    import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        recipe = workloads.batch_recipe(24, seed=42)
        work = [replicas.problem_work(r["L"], r["k"]) for r in recipe]
        mem = [r["L"] ** 3 * 400 for r in recipe]
        mine = replicas.balanced_shard(work, mem, world, mem_budget=50 ** 3 * 400)[rank]
        # a stand-in result per problem (the real run solves it on this rank's GPU)
        results = [(i, recipe[i]["seed"], sum(work[j] for j in [i])) for i in mine]
        load = replicas.sum_over_ranks(0.0)  # a collective between the ranks
        gathered = replicas.gather_to_root(results)
        q.put((rank, mine, load, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_balanced_batch():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_batch_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import workloads
    recipe = workloads.batch_recipe(24, seed=42)
    work = [replicas.problem_work(r["L"], r["k"]) for r in recipe]
    m0, m1 = res[0][1], res[1][1]
    assert sorted(m0 + m1) == list(range(24)) and not set(m0) & set(m1)
    w0, w1 = sum(work[i] for i in m0), sum(work[i] for i in m1)
    # greedy LPT: the imbalance is at most the largest single problem
    assert abs(w0 - w1) <= max(work)
    g = res[0][3]
    assert res[1][3] is None and [x[0] for x in g[0]] == m0 and [x[0] for x in g[1]] == m1
    assert [x[1] for x in g[0] + g[1]] == [recipe[i]["seed"] for i in m0 + m1]


def test_balanced_shard_rules():
    # decreasing work, each to the least-loaded rank: 9 | 7, 2 | 5, 4 -> loads 9, 9, 9
    work = [5.0, 9.0, 2.0, 7.0, 4.0]
    parts = replicas.balanced_shard(work, [1] * 5, 3)
    assert sorted(sum(parts, [])) == [0, 1, 2, 3, 4]
    loads = [sum(work[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(work)
    assert parts == [[1], [2, 3], [0, 4]]
    # one rank takes everything; the budget rejects a too-large problem
    assert replicas.balanced_shard(work, [1] * 5, 1) == [[0, 1, 2, 3, 4]]
    with pytest.raises(ValueError):
        replicas.balanced_shard(work, [1, 1, 10, 1, 1], 2, mem_budget=5)
    assert replicas.balanced_shard([], [], 4) == [[], [], [], []]
    # more ranks than problems: the extra ranks get nothing
    assert replicas.balanced_shard([1.0, 2.0], [1, 1], 4) == [[1], [0], [], []]


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
