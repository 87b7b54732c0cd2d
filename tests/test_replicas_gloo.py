"""The multi-GPU host logic with two gloo ranks on the CPU (no GPU): rank
seeding covers a single generator's streams without overlap, and the job's
time is the slowest rank's."""
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


def test_rank_streams_are_the_global_generators_streams():
    """For xor128 (no per-stream multipliers) rank r's n streams are streams
    r*n .. (r+1)*n - 1 of one generator of world*n streams (oracle, CPU)."""
    import oracle
    n, world, seed = 64, 3, 7
    whole = oracle.seed_streams(oracle.XOR128, None, seed, np.arange(world * n))
    ref, _ = oracle.generate(oracle.XOR128, None, whole, 16, oracle.U32)
    for r in range(world):
        st = oracle.seed_streams(oracle.XOR128, None, replicas.rank_seed(seed, r, n),
                                 np.arange(n))
        out, _ = oracle.generate(oracle.XOR128, None, st, 16, oracle.U32)
        assert np.array_equal(out, ref[:, r * n:(r + 1) * n])


def test_no_group_means_own_value():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.rank_seed(2**64 - 1, 1, 1) == 0
