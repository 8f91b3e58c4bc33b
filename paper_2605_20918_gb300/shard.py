"""Sharding over ranks (one process per GPU).

The geometries of an MD-like sequence are independent problems: rank r of W takes the steps
r, r + W, r + 2W, ...  No data moves between ranks; the only collective is the maximum of the
timed region over ranks.  Within one system the colours are independent block-Lanczos
problems on a replicated H; `colour_partition` deals them to ranks for the decomposition whose
one exchange is an all-gather of the Ritz pairs before mu.
"""
from __future__ import annotations


def rank_steps(rank: int, world: int, n_steps: int) -> list[int]:
    """Global step indices handled by `rank` (n_steps per rank, interleaved over ranks)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return [rank + world * i for i in range(n_steps)]


def colour_partition(sizes, world: int) -> list[list[int]]:
    """Colours of one system dealt to `world` ranks for the colour-partitioned decomposition
    (independent block-Lanczos problems on a replicated H): largest colours first, each to the
    rank with the fewest molecules so far (ties to the lower rank); every rank's list ascending."""
    if world < 1:
        raise ValueError("world < 1")
    load = [0] * world
    out = [[] for _ in range(world)]
    for c in sorted(range(len(sizes)), key=lambda c: (-int(sizes[c]), c)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(c)
        load[r] += int(sizes[c])
    return [sorted(x) for x in out]


def geometry_of(step: int, n_geometries: int) -> int:
    """Geometry of the sequence used by a global step (the sequence is reused cyclically)."""
    return step % n_geometries


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_build(t_max: float, steps_per_rank: int, world: int) -> float:
    """Whole-job time per P build: the slowest rank's time over all ranks' builds."""
    return t_max / (steps_per_rank * world)
