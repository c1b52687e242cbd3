"""Multi-GPU host logic for the FMM-IPM map (one process per GPU).

The deflection of a ray depends only on the stars, so the targets shard
freely (Sec. 2.1: targets are independent of the deflectors; Sec. 2.4 already
splits the image plane into chunks).  Two modes:

* independent maps -- every rank builds its own plan and computes its own
  map (e.g. a different star-field realisation); no collective on the data
  path, weak scaling;
* one map in strips -- every rank holds the same plan (the tree is cheap to
  replicate), computes the cells of a contiguous strip of grid rows into a
  full-size local map, and one sum all-reduce of the map completes it (IPM is
  additive over cells).

Only host logic lives here; the compute runs in liblens on each rank's GPU.
"""
from __future__ import annotations

from typing import List, Tuple

import torch
import torch.distributed as dist


def row_strips(ny: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous, balanced strips of cell rows [r0, r0+n) covering [0, ny)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(ny, world)
    out, r0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((r0, n))
        r0 += n
    return out


def strip_grid(grid, r0: int, nrows: int):
    """The sub-grid of cell rows [r0, r0+nrows) of a grid (same x0, h, nx)."""
    from .synth import Grid
    return Grid(x0=grid.x0, y0=grid.y0 + r0 * grid.h, h=grid.h, nx=grid.nx, ny=nrows)


def allreduce_map(mp: torch.Tensor) -> torch.Tensor:
    """Sum the ranks' partial maps in place (the only collective of the path)."""
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(mp, op=dist.ReduceOp.SUM)
    return mp


def allreduce_ledger(stats: dict, keys, device) -> dict:
    """Sum the ranks' flux ledgers."""
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return dict(stats)
    t = torch.tensor([float(stats[k]) for k in keys], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = dict(stats)
    for k, v in zip(keys, t.tolist()):
        out[k] = v
    return out


def max_over_ranks(value: float, device) -> float:
    """Maximum of a per-rank timing (the job's time is its slowest rank)."""
    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
