"""Host-side wave scheduling (no GPU): pieces cover every instance's rows in
order, a wave holds at most one piece per instance and fits the budget."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1101_1846_gb300 import scheduler, workloads


def check(streams, rows, budget, chunk):
    waves = scheduler.chunked_waves(streams, rows, budget, chunk)
    covered = [0] * len(streams)
    for w in waves:
        assert w, "empty wave"
        ids = [p.inst for p in w]
        assert len(ids) == len(set(ids))
        used = sum(4 * streams[p.inst] * p.rows for p in w)
        assert used <= budget or len(w) == 1
        for p in w:
            assert p.rows >= 1
            assert p.row0 == covered[p.inst]  # rows in order, no gap
            if chunk > 0:
                assert p.rows <= chunk
            covered[p.inst] += p.rows
    assert covered == list(rows)
    return waves


@pytest.mark.parametrize("chunk", [0, 1, 7, 2048])
def test_random_instances(chunk):
    rng = np.random.Generator(np.random.PCG64(3))
    streams = rng.integers(1, 5000, 300).tolist()
    rows = rng.integers(0, 9000, 300).tolist()
    check(streams, rows, 64 << 20, chunk)


def test_batched_workload_waves_fit():
    inst = workloads.batched_instances(2000, 1234)
    waves = check([i.n_streams for i in inst], [i.n_per_stream for i in inst],
                  8 << 30, 2048)
    assert max(p.rows for w in waves for p in w) <= 2048


def test_oversized_piece_alone():
    waves = check([1000, 10], [100, 5], 4 * 1000 * 10, 0)
    assert len(waves[0]) == 1 and waves[0][0].inst == 0


def test_laned_waves_keep_each_instance_in_one_lane_and_in_order():
    rng = np.random.Generator(np.random.PCG64(8))
    streams = rng.integers(1, 3000, 200).tolist()
    rows = rng.integers(1, 5000, 200).tolist()
    waves = scheduler.laned_waves(streams, rows, 32 << 20, 300, lanes=2)
    covered = [0] * len(streams)
    lane_of = {}
    for lane, w in waves:
        assert sum(4 * streams[p.inst] * p.rows for p in w) <= 32 << 20 or len(w) == 1
        for p in w:
            assert lane_of.setdefault(p.inst, lane) == lane == p.inst % 2
            assert p.row0 == covered[p.inst]
            covered[p.inst] += p.rows
    assert covered == rows
    lanes = [lane for lane, _ in waves]
    assert lanes[:4] == [0, 1, 0, 1]
