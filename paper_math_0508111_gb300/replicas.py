"""Replica-parallel runs over several GPUs (one process per GPU).

The method has no data-parallel split of one lattice (the triangular solves
of the preconditioner are sequential across levels), so several GPUs solve
independent problems: disorder realisations, or the requests of a batch.
These helpers hold the host logic of that split -- which rank takes which
problem, and the reductions of timings and results -- and run unchanged over
the ``gloo`` (CPU) or ``nccl`` backends of ``torch.distributed``.  No
collective touches the data path: each rank's solves are self-contained.
"""
import torch
import torch.distributed as dist


def realisation_seeds(count, rank, base=1, stride=100000):
    """Disorder seeds of this rank's `count` realisations: disjoint blocks
    base + stride * rank + i, so every rank solves different lattices."""
    return [base + stride * rank + i for i in range(count)]


def shard(items, rank, world):
    """Round-robin share of a problem list for this rank (rank r takes items
    r, r + world, ...); the shares partition the list."""
    return list(items[rank::world])


def balanced_shard(work, mem, world, mem_budget=None):
    """Greedy partition of independent problems over `world` ranks by
    estimated work, under a per-rank device-memory budget.

    work[i], mem[i]: estimated work and device bytes of problem i (for the
    Anderson eigensolves work grows with the lattice size n = L^3 and mem is
    the library's jd_server_estimate).  Problems are taken in decreasing
    work (ties: lower index first) and each goes to the rank with the least
    work so far (ties: lower rank) among the ranks whose largest problem
    would still fit mem_budget -- every rank solves its problems one or a
    few at a time, so the budget bounds the largest problem, not the sum.
    A problem larger than the budget everywhere raises ValueError.  Returns
    one ascending index list per rank; together they partition range(len)."""
    n = len(work)
    if len(mem) != n:
        raise ValueError("work and mem must have the same length")
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(n), key=lambda j: (-work[j], j)):
        if mem_budget is not None and mem[i] > mem_budget:
            raise ValueError("problem %d needs %d bytes, more than the budget %d" % (i, mem[i], mem_budget))
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += work[i]
        out[r].append(i)
    return [sorted(o) for o in out]


def problem_work(L, k):
    """Work estimate of one eigensolve on an L^3 lattice with k pairs: the
    setup and every sweep of the solve are linear in n = L^3, and the
    number of outer steps grows with k (one locked pair every few steps)."""
    return float(L) ** 3 * (1.0 + 0.2 * k)


def _device(backend):
    return torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")


def max_over_ranks(x):
    """Largest value of x over all ranks (the job's wall time is that of its
    slowest rank); x itself when not distributed."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device(dist.get_backend()))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x):
    """Sum of x over all ranks (e.g. eigenpairs solved by the whole job)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device(dist.get_backend()))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_to_root(obj, root=0):
    """Per-rank Python objects (e.g. result lists) collected on `root` in
    rank order; other ranks get None."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == root else None
    dist.gather_object(obj, out, dst=root)
    return out
