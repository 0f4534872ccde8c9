"""Work split across ranks (one process per GPU).

A program's fitness needs nothing from any other program, and the paper
splits the population between the GPUs of a machine (Sec. 2.1.2).  Two
ways to use several ranks follow from that:

* independent populations (islands): every rank evolves its own population
  of the same problem with its own seed; no data crosses ranks.  This is
  what ``bench.py --gpus N`` times (weak scaling).
* one population split into contiguous slices (``Evolver(split=True)``):
  every rank holds the whole population, evaluates rows
  ``shard_range(P, r, world)`` (the C-ABI takes the slice as pointers at
  that row offset) and optimises their constants; the fitness slices (P
  doubles, :func:`gather_fitness`) and the optimised constants
  (:func:`gather_rows`) are all-gathered once per generation, and every
  rank then runs the same selection and variation from the same seed, so
  the populations stay identical without sending programs.

Timing over ranks is the maximum (:func:`max_over_ranks`), work the sum.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(P: int, rank: int, world: int) -> tuple[int, int]:
    """(offset, count) of rank's contiguous slice of P items; the first
    P % world ranks take one extra item."""
    if world < 1 or not 0 <= rank < world or P < 0:
        raise ValueError(f"bad shard: P={P} rank={rank} world={world}")
    base, extra = divmod(P, world)
    return rank * base + min(rank, extra), base + (1 if rank < extra else 0)


def gather_fitness(local: torch.Tensor, P: int, group=None) -> torch.Tensor:
    """All-gather per-rank fitness slices (last axis = this rank's programs)
    into the whole population's fitness, in program order."""
    world = dist.get_world_size(group)
    counts = [shard_range(P, r, world)[1] for r in range(world)]
    rank = dist.get_rank(group)
    if local.shape[-1] != counts[rank]:
        raise ValueError(f"rank {rank} holds {local.shape[-1]} programs, its slice has {counts[rank]}")
    width = max(counts)
    buf = torch.full(local.shape[:-1] + (width,), float("nan"), dtype=local.dtype, device=local.device)
    buf[..., : local.shape[-1]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[..., :c] for p, c in zip(parts, counts)], dim=-1)


def gather_rows(local: torch.Tensor, P: int, group=None) -> torch.Tensor:
    """All-gather per-rank row slices (first axis = this rank's programs)
    into the whole population's rows, in program order."""
    world = dist.get_world_size(group)
    counts = [shard_range(P, r, world)[1] for r in range(world)]
    rank = dist.get_rank(group)
    if local.shape[0] != counts[rank]:
        raise ValueError(f"rank {rank} holds {local.shape[0]} rows, its slice has {counts[rank]}")
    width = max(counts)
    buf = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    buf[: local.shape[0]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def _reduce(value: float, op, device=None, group=None) -> float:
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op, group=group)
    return float(t.item())


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Largest value over ranks (the timing of a step that every rank runs)."""
    return _reduce(value, dist.ReduceOp.MAX, device, group)


def sum_over_ranks(value: float, device=None, group=None) -> float:
    """Sum over ranks (work units)."""
    return _reduce(value, dist.ReduceOp.SUM, device, group)
