"""Host logic of runs on several GPUs.  The streams are independent (the
paper parametrises every thread's generator: Sec. "Parallelizing RNGs"), so
the path shards with no collective on the data path: each rank owns its own
streams, and the ranks only agree on timing.

- rank_seed: rank r's generator of n streams is seeded with seed + r * n, so
  its stream s starts splitmix64 at seed + r * n + s — the same point as
  stream r * n + s of one generator of world * n streams seeded with seed.
  Streams of different ranks therefore never share a seeding point, and for
  the kinds without per-stream multipliers (xor128, XORSHIFT8) rank r
  produces exactly that generator's streams r * n .. (r + 1) * n - 1.
- max_over_ranks: the slowest rank's time, which the whole job's rate uses.
- job_rate: samples of all ranks over that time (weak scaling).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_seed(seed: int, rank: int, n_streams: int) -> int:
    return (seed + rank * n_streams) % (1 << 64)


def max_over_ranks(value: float, device: torch.device | str = "cpu") -> float:
    """The maximum of `value` over the ranks of the default process group
    (the value itself when no group is initialised)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(samples_per_rank: int, world: int, seconds_max: float) -> float:
    """Samples per second of the whole job: every rank's samples over the
    slowest rank's time."""
    return world * samples_per_rank / seconds_max
