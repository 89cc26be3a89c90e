"""Restart points sharded across ranks (one process per GPU).

Points are independent, so each rank runs its own slice of the B points on its
own replica of the instance; restart draws are keyed by the global point index
(``b_offset``), so a sharded run draws exactly what a single process would.
Between rounds the ranks exchange only what the restart heuristics need: an OR
of the "some point is a model" flags and, for the ERWA weighting (Sec. 5,
"Weighting Heuristics"), the per-constraint violation counts U_c summed over
all ranks' points, after which every rank applies the same weight update.
"""
from __future__ import annotations


def shard(B_total: int, rank: int, world: int):
    """(b_offset, B_local): this rank's contiguous slice of the global points."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(B_total, world)
    B_local = base + (1 if rank < extra else 0)
    b_offset = rank * base + min(rank, extra)
    return b_offset, B_local


def combine_round(solved, unsat_counts=None, group=None) -> bool:
    """All-reduce of one round's results: returns whether any rank's point is a
    model, and sums ``unsat_counts`` (int32 [m], in place) over the ranks.
    Tensors live on the device the process group's backend uses (CUDA for NCCL,
    CPU for gloo)."""
    import torch
    import torch.distributed as dist

    flag = solved.any().to(torch.int32).reshape(1)
    dist.all_reduce(flag, op=dist.ReduceOp.MAX, group=group)
    if unsat_counts is not None:
        dist.all_reduce(unsat_counts, op=dist.ReduceOp.SUM, group=group)
    return bool(flag.item())
