"""Host logic of runs on several GPUs.  The streams are independent (the
paper parametrises every thread's generator: Sec. "Parallelizing RNGs"), so
the path shards with no collective on the data path: each rank owns a
contiguous range of one global generator's streams, and the ranks only agree
on timing.

- shard_spec: rank r of `world` ranks with n streams each holds global
  streams r * n .. (r + 1) * n - 1 of the generator (kind, seed): a handle
  made by rng_create_range(kind, r * n, n, seed), with those streams'
  multipliers and seeds.  When world * n streams exceed the kind's
  multiplier table (MWC32 and KISS at 2^22 streams per rank), the rank
  keeps the table's first n multipliers and shifts its seed by r * n
  instead (rank_seed): its streams then start splitmix64 at the same points
  as the global streams, on the same multipliers as rank 0.
- max_over_ranks: the slowest rank's time, which the whole job's rate uses.
- job_rate: samples of all ranks over that time (weak scaling).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import capi

# largest stream count of each kind (include/rng.h)
MAX_STREAMS = {0: capi.RNG_MAX_STREAMS_MWC, 1: capi.RNG_MAX_STREAMS_XOR,
               2: capi.RNG_MAX_STREAMS_MWC, 3: capi.RNG_MAX_STREAMS_MWC16,
               4: capi.RNG_MAX_STREAMS_XS8, 5: capi.RNG_MAX_STREAMS_MWC16}


def rank_seed(seed: int, rank: int, n_streams: int) -> int:
    return (seed + rank * n_streams) % (1 << 64)


def shard_spec(kind: int, rank: int, world: int, n_streams: int, seed: int) -> tuple[int, int]:
    """(s_begin, seed) to create rank `rank`'s handle with: rng_create_range
    (kind, s_begin, n_streams, seed) holds global streams s_begin ..
    s_begin + n_streams - 1.  s_begin is 0, with the seed shifted, when the
    global generator would have more streams than the kind allows."""
    if world * n_streams <= MAX_STREAMS[kind]:
        return rank * n_streams, seed % (1 << 64)
    return 0, rank_seed(seed, rank, n_streams)


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
