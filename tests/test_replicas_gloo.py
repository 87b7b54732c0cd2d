"""The multi-GPU host logic with two gloo ranks on the CPU (no GPU): each
rank's stream range is its slice of one generator's streams, multipliers
included, and the job's time is the slowest rank's."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

from paper_1101_1846_gb300 import replicas  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = replicas.max_over_ranks(1.0 + rank)       # rank 1 is the slow one
        seed = replicas.rank_seed(42, rank, 1000)
        results[rank] = (t, seed, replicas.job_rate(5000, world, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert res[0][0] == res[1][0] == 2.0
    assert res[0][1] == 42 and res[1][1] == 1042
    assert res[0][2] == res[1][2] == 2 * 5000 / 2.0


def _rank_outputs(kind, rank, world, n, seed, steps):
    """What rng_create_range(kind, s_begin, n, seed') computes, for the
    (s_begin, seed') of shard_spec: the handle's stream s takes multiplier
    s_begin + s of the table and starts splitmix64 at seed' + s_begin + s
    (oracle, CPU)."""
    import oracle
    s_begin, seed_r = replicas.shard_spec(kind, rank, world, n, seed)
    table = oracle.multipliers_for(kind, s_begin + n)
    a = None if table is None else table[s_begin:s_begin + n]
    st = oracle.seed_streams(kind, a, (seed_r + s_begin) % (1 << 64), np.arange(n))
    return oracle.generate(kind, a, st, steps, oracle.U32)[0]


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 5])
def test_rank_streams_are_the_global_generators_streams(kind):
    """Rank r's n streams are streams r*n .. (r+1)*n - 1 of one generator of
    world*n streams, multipliers included (oracle, CPU)."""
    import oracle
    n, world, seed = 64, 3, 7
    table = oracle.multipliers_for(kind, world * n)
    whole = oracle.seed_streams(kind, table, seed, np.arange(world * n))
    ref, _ = oracle.generate(kind, table, whole, 16, oracle.U32)
    for r in range(world):
        out = _rank_outputs(kind, r, world, n, seed, 16)
        assert np.array_equal(out, ref[:, r * n:(r + 1) * n]), (kind, r)


def test_shard_spec_falls_back_to_shifted_seeds_beyond_the_table():
    n = replicas.MAX_STREAMS[0]
    assert replicas.shard_spec(0, 0, 1, n, 5) == (0, 5)
    assert replicas.shard_spec(0, 1, 2, n, 5) == (0, 5 + n)   # 2n > 2^22 multipliers
    assert replicas.shard_spec(1, 1, 2, n, 5) == (n, 5)       # xor128 has no table


def test_no_group_means_own_value():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.rank_seed(2**64 - 1, 1, 1) == 0
