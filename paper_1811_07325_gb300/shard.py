"""Sharding one product across devices by leaves.

The 7^d leaf products of one recursion tree are independent (the paper runs
them as parallel tasks, Sec. III-C and Alg. 4, and measures strong scaling
over executors, Sec. V-F).  Each rank takes a balanced contiguous range of
leaves (``leaf_range``) and a plan restricted to it (``shard_plan``: the
workspace and the divide cover only the subtrees holding those leaves), and
computes its partial C (the sum of its leaves' signed combine
contributions) with ``stark_mul_leaves``.  One sum reduce-scatter gives each
rank its block of rows of C = A.B (``mul_sharded_rows``, the default), or
one sum all-reduce gives every rank all of C (``mul_sharded``).  That
reduction is the only exchange the path has.

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


def shard_plan(n: int, depth: int, dtype, world: int, rank: int):
    """A plan for this rank's leaves of an n x n product at ``depth``
    (``stark_plan_set_shard`` on ``leaf_range``), or a whole plan when the
    rank's range is everything (one rank) or empty."""
    from . import stark
    p = stark.Plan(n, depth, dtype)
    begin, end = leaf_range(p.leaves, world, rank)
    if begin < end and (begin, end) != (0, p.leaves):
        p.set_shard(begin, end)
    return p


def _rank_leaves(plan, world, rank):
    shard = getattr(plan, "shard", None)
    return shard if shard is not None else leaf_range(plan.leaves, world, rank)


def mul_sharded(plan, A, B, C, group=None, stream=None):
    """C = A @ B on every rank of ``group``: local leaves, then one sum all-reduce.

    ``plan`` is a :class:`paper_1811_07325_gb300.stark.Plan` (or any object with
    ``leaves`` and ``mul_leaves(A, B, begin, end, C, stream)``)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    begin, end = _rank_leaves(plan, world, rank)
    plan.mul_leaves(A, B, begin, end, C=C, stream=stream)
    dist.all_reduce(C, op=dist.ReduceOp.SUM, group=group)
    return C


def row_block(n: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [begin, end) of C held by ``rank`` after ``mul_sharded_rows``:
    blocks of ceil(n / world) rows, the last ones shorter or empty."""
    if world <= 0 or not 0 <= rank < world or n < 0:
        raise ValueError("bad world/rank/n")
    rb = -(-n // world)
    return min(rank * rb, n), min((rank + 1) * rb, n)


def mul_sharded_rows(plan, A, B, group=None, stream=None):
    """Rows of C = A @ B, one block per rank of ``group``: local leaves into a
    partial C, then one sum reduce-scatter over row blocks.

    Returns ``(begin, end, rows)``: ``rows`` holds C[begin:end] (a view of a
    ceil(n / world) x n buffer; rows past ``end - begin`` are padding)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = plan.n
    rb = -(-n // world)
    partial = torch.empty((world * rb, n), dtype=A.dtype, device=A.device)
    partial[n:].zero_()  # padding rows of the last block (the product overwrites the first n)
    begin, end = _rank_leaves(plan, world, rank)
    plan.mul_leaves(A, B, begin, end, C=partial[:n], stream=stream)
    out = torch.empty((rb, n), dtype=A.dtype, device=A.device)
    dist.reduce_scatter_tensor(out, partial, op=dist.ReduceOp.SUM, group=group)
    r0, r1 = row_block(n, world, rank)
    return r0, r1, out
