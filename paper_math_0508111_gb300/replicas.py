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
