"""Sharding one product across devices by leaves.

The 7^d leaf products of one recursion tree are independent (the paper runs
them as parallel tasks, Sec. III-C and Alg. 4); each rank computes the leaves
of its share with ``stark_mul_leaves`` (its partial C is the sum of those
leaves' signed combine contributions), and one sum all-reduce over the ranks
gives every rank C = A.B.  This is the only exchange the path has.

Argument marshalling only: the products run in libstark.so; the reduction
is torch.distributed's (NCCL on GPUs).
"""
from __future__ import annotations


def leaf_range(leaves: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced share [begin, end) of ``leaves`` for ``rank``:
    the first ``leaves % world`` ranks take one extra leaf."""
    if world <= 0 or not 0 <= rank < world or leaves < 0:
        raise ValueError("bad world/rank/leaves")
    base, extra = divmod(leaves, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def mul_sharded(plan, A, B, C, group=None, stream=None):
    """C = A @ B on every rank of ``group``: local leaves, then one sum all-reduce.

    ``plan`` is a :class:`paper_1811_07325_gb300.stark.Plan` (or any object with
    ``leaves`` and ``mul_leaves(A, B, begin, end, C, stream)``)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    begin, end = leaf_range(plan.leaves, world, rank)
    plan.mul_leaves(A, B, begin, end, C=C, stream=stream)
    dist.all_reduce(C, op=dist.ReduceOp.SUM, group=group)
    return C
