"""Data-parallel split of a window grid across ranks, one GPU per rank.

Match windows are independent, so the forward needs no collective: each rank
matches a contiguous band of grid rows, and the 32-byte result records are
concatenated in rank order.  The backward keeps every window's six affine
gradients with its window; the only quantity the ranks share is the
whitening-exponent gradient, one float per level summed over the whole batch,
which is an all-reduce (sum) of n_levels floats.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def row_bands(n_rows: int, world: int):
    """Contiguous, near-equal [start, stop) row ranges, one per rank (the first
    n_rows % world ranks take one row more)."""
    if n_rows < 0 or world < 1:
        raise ValueError("need n_rows >= 0 and world >= 1")
    base, extra = divmod(n_rows, world)
    bands, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        bands.append((start, stop))
        start = stop
    return bands


def shard_rows(items, n_rows: int, n_cols: int, rank: int, world: int):
    """This rank's windows of a row-major n_rows x n_cols grid (origins,
    levels or any per-window array whose first axis is the window): the grid
    rows of its band, contiguous."""
    if len(items) != n_rows * n_cols:
        raise ValueError("items must hold one entry per grid window, row-major")
    start, stop = row_bands(n_rows, world)[rank]
    return items[start * n_cols: stop * n_cols]


def gather_results(local: torch.Tensor, group=None) -> torch.Tensor:
    """Concatenate every rank's [b_r, 8] int32 result records in rank order
    (each rank gets the whole batch's results)."""
    world = dist.get_world_size(group)
    count = torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device)
    counts = [torch.zeros_like(count) for _ in range(world)]
    dist.all_gather(counts, count, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts)
    pad = torch.zeros((m, local.shape[1]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])


def allreduce_grad_w(grad_w: torch.Tensor, group=None) -> torch.Tensor:
    """Sum the per-level whitening-exponent gradients over the ranks, in place."""
    dist.all_reduce(grad_w, op=dist.ReduceOp.SUM, group=group)
    return grad_w
