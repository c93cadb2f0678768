"""Row-sharded fitness of one population over several GPUs (one process each).

The grid's rows are split into contiguous bands, one per rank (`band_rows`).
Each rank loads its band as a domain (`Context.load_domain` with `rows`: the points
and coordinates are those of the full grid's rows) and computes, for every
tree, the binary64 sum of squared residuals over its band
(`Context.fitness_sse_dev`).  The ranks then exchange these [T] sums -- T
doubles per rank, the only data that crosses between GPUs -- and every rank
adds them in rank order and forms sqrt(sum / (W*H)), the RMSE of Sec. 4.1 over
the whole grid.  The exchange is an all-gather followed by a fixed-order sum
on each rank rather than an all-reduce, so every rank holds the same bits
whatever order the collective library would have added in.

Argument marshalling and the exchange only: the sums come from the library's
kernels.
"""
from __future__ import annotations

import math

import torch
import torch.distributed as dist


def band_rows(H: int, rank: int, world: int) -> tuple[int, int]:
    """(first row, number of rows) of rank `rank`'s band of an H-row grid:
    contiguous bands whose sizes differ by at most one row, in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    lo = H * rank // world
    hi = H * (rank + 1) // world
    return lo, hi - lo


def reduce_band_sse(sse: torch.Tensor, n_points: int, group=None) -> torch.Tensor:
    """RMSE of every tree over the whole grid from this rank's band sums.

    sse: float64 [T] (this rank's binary64 sums of squared residuals; on the
    device the process group's backend works on).  n_points: W*H of the full
    grid.  Returns float64 [T] on sse's device: sqrt(sum over ranks, added in
    rank order, / n_points), +inf where that is not finite.  Without an
    initialised process group the rank is alone."""
    if sse.dtype != torch.float64 or sse.dim() != 1:
        raise ValueError("sse must be a float64 vector")
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    sse = sse.contiguous()
    if world == 1:
        parts = [sse]
    else:
        parts = [torch.empty_like(sse) for _ in range(world)]
        dist.all_gather(parts, sse, group=group)
    total = parts[0].clone()
    for p in parts[1:]:
        total += p
    r = torch.sqrt(total / float(n_points))
    return torch.where(torch.isfinite(r), r, torch.full_like(r, math.inf))


def sharded_fitness(ctx, pop, n_trees: int, band_dom, n_points: int, group=None, stream=None) -> torch.Tensor:
    """Fitness of the n_trees trees of `pop` over the full grid of n_points
    points, this rank holding the band `band_dom` (a domain loaded with
    Context.load_domain(..., rows=band_rows(H, rank, world)) on this rank's
    GPU).  Every rank passes its own band; all receive the same float64 [T]
    RMSE."""
    sse = torch.empty(n_trees, dtype=torch.float64, device="cuda")
    ctx.fitness_sse_dev(pop, band_dom, sse, stream=stream)
    if stream is not None:
        torch.cuda.current_stream().wait_stream(stream)
    return reduce_band_sse(sse, n_points, group=group)
