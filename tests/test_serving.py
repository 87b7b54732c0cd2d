"""The serving engine (rng_server_*): every request's output equals the
oracle's replay of the client's sequence, the same whether the request is
served alone or batched with others, under an HBM budget that makes
requests wait for admission."""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1101_1846_gb300 import build, capi, workloads  # noqa: E402
from paper_1101_1846_gb300.serving import Server, replay  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


def client_sequences(kind, n, seed, total):
    """The first `total` samples of a client's sequence (uint32 and float32
    bits): the generator's stream-interleaved output read row by row."""
    a = oracle.multipliers(n, 32) if kind != oracle.XOR128 else None
    st = oracle.seed_streams(kind, a, seed, np.arange(n))
    rows = max(1, math.ceil(total / n))
    u, _ = oracle.generate(kind, a, st, rows, oracle.U32)
    f, _ = oracle.generate(kind, a, st, rows, oracle.F32)
    return u.reshape(-1)[:total], f.reshape(-1)[:total].view(np.uint32)


def make_log(count, n_clients, hi, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.floor(np.exp(rng.random(count) * np.log(hi))).astype(int) + 1
    return [workloads.Request(0.0, int(rng.integers(0, n_clients)), int(sizes[i]),
                              int(rng.integers(0, 2))) for i in range(count)]


def run_all(server, log, one_at_a_time=False):
    """Submit the log (all at once, or one request at a time), collect every
    output by request index."""
    outs = {}
    if one_at_a_time:
        for i, r in enumerate(log):
            rid = server.submit(r.client, r.n_samples, r.fmt)
            server.drain()
            done = dict(server.take())
            assert rid in done
            outs[i] = (server.result(rid), server.copy(rid).cpu().numpy().view(np.uint32))
            server.release(rid)
        return outs
    rids = [server.submit(r.client, r.n_samples, r.fmt) for r in log]
    server.drain()
    done = dict(server.take())
    assert set(done) == set(rids)
    for i, rid in enumerate(rids):
        outs[i] = (server.result(rid), server.copy(rid).cpu().numpy().view(np.uint32))
        server.release(rid)
    return outs


def check_against_oracle(server, log, outs, kind, n):
    totals = {}
    for r in log:
        totals[r.client] = totals.get(r.client, 0) + r.n_samples
    seqs = {c: client_sequences(kind, n, server.client_seed(c), t) for c, t in totals.items()}
    cursor = {c: 0 for c in totals}
    for i, r in enumerate(log):
        info, got = outs[i]
        assert info["client"] == r.client and info["n"] == r.n_samples
        assert info["start"] == cursor[r.client]  # ranges in submission order
        u, f = seqs[r.client]
        exp = (u if r.fmt == oracle.U32 else f)[cursor[r.client]:cursor[r.client] + r.n_samples]
        assert np.array_equal(got, exp), i
        cursor[r.client] += r.n_samples


def test_mixed_requests_equal_oracle_and_alone():
    n, clients = 1003, 3  # odd stream count: realigned rows, wrapped windows
    log = make_log(60, clients, 20000, seed=12)
    mixed = Server(capi.RNG_KISS, clients, n, seed_base=77, budget_bytes=64 << 20,
                   chunk_rows=2)
    outs = run_all(mixed, log)
    check_against_oracle(mixed, log, outs, oracle.KISS, n)
    st = mixed.stats()
    # a tick advances each client by at most chunk_rows * n samples
    per_client = [sum(r.n_samples for r in log if r.client == c) for c in range(clients)]
    assert st["completed"] == len(log)
    assert st["ticks"] >= max(-(-t // (2 * n)) for t in per_client)
    mixed.close()
    alone = Server(capi.RNG_KISS, clients, n, seed_base=77, budget_bytes=64 << 20,
                   chunk_rows=2)
    outs2 = run_all(alone, log, one_at_a_time=True)
    for i in outs:
        assert np.array_equal(outs[i][1], outs2[i][1]), i
    alone.close()


SIZES = [5, 1, 2000, 3, 1003, 1004, 7, 4096, 9, 1, 1, 2, 333, 1, 64]


@pytest.mark.parametrize("kind,n", [(oracle.KISS, 1003), (oracle.KISS, 1024), (oracle.KISS, 3),
                                    (oracle.MWC, 1001), (oracle.XOR128, 1000)])
def test_one_piece_spans_requests_of_mixed_formats(kind, n):
    """Many small requests of one client, formats alternating request by
    request (requests of one sample put two format changes inside one
    16-byte store), all admitted at once: their outputs sit back to back in
    the arena, so one piece of the client's sequence runs through all of them
    in a single tick, its format map flipping at every request boundary; and
    every output equals the oracle's."""
    log = [workloads.Request(0.0, 0, size, i % 2) for i, size in enumerate(SIZES * 3)]
    total = sum(r.n_samples for r in log)
    rows = -(-total // n)
    s = Server(kind, 1, n, seed_base=5, budget_bytes=64 << 20, chunk_rows=rows)
    outs = run_all(s, log)
    check_against_oracle(s, log, outs, kind, n)
    assert s.stats()["ticks"] == 1
    s.close()


@pytest.mark.parametrize("kind", [oracle.MWC, oracle.XOR128])
def test_other_kinds_equal_oracle(kind):
    n, clients = 640, 2
    log = make_log(20, clients, 5000, seed=3 + kind)
    s = Server(kind, clients, n, seed_base=5, budget_bytes=32 << 20, chunk_rows=3)
    outs = run_all(s, log)
    check_against_oracle(s, log, outs, kind, n)
    s.close()


def test_plan_shape_keeps_outputs():
    """Another kernel shape, set before the first tick and changed between
    two halves of the log (the lanes' plans are rebuilt), gives the oracle's
    outputs; invalid shapes are refused."""
    n, clients = 1024, 4
    log = make_log(40, clients, 30000, seed=21)
    s = Server(capi.RNG_KISS, clients, n, seed_base=9, budget_bytes=64 << 20, chunk_rows=4,
               plan_shape=(128, 2))
    outs = run_all(s, log[:20])
    capi.check(capi.lib().rng_server_set_plan_shape(s.h, 256, 0))
    outs2 = run_all(s, log[20:])
    outs.update({20 + i: v for i, v in outs2.items()})
    check_against_oracle(s, log, outs, oracle.KISS, n)
    for bad in ((0, 0), (96, 0), (1024, 0), (256, -1), (256, 33)):
        assert capi.lib().rng_server_set_plan_shape(s.h, *bad) == capi.RNG_ERR_ARG
    s.close()


def test_admission_waits_for_budget():
    n, clients = 512, 2
    state = clients * n * 20
    s = Server(capi.RNG_KISS, clients, n, seed_base=1, budget_bytes=state + (1 << 20) + 4096,
               chunk_rows=4)
    arena = s.stats()["arena_size"]
    log = [workloads.Request(0.0, i % clients, 100_000, i % 2) for i in range(12)]
    rids = [s.submit(r.client, r.n_samples, r.fmt) for r in log]
    s.progress()
    assert s.stats()["waiting"] > 0  # only a few outputs fit at once
    max_used, outs = 0, {}
    while len(outs) < len(rids):
        s.progress()
        for rid, _ in s.take():
            outs[rid] = s.copy(rid).cpu().numpy().view(np.uint32)
            s.release(rid)
        max_used = max(max_used, s.stats()["arena_used"])
    assert max_used <= arena
    check_against_oracle(s, log, {i: ({"client": r.client, "n": r.n_samples,
                                        "start": 100_000 * (i // clients)}, outs[rids[i]])
                                   for i, r in enumerate(log)}, oracle.KISS, n)
    with pytest.raises(capi.RngError):
        s.submit(0, arena // 4 + 1, 0)  # larger than the whole arena
    s.close()


def test_admission_looks_past_a_waiting_head():
    """Client 0's second large request waits for space; client 1's small
    requests behind it are admitted at once (each client's requests still in
    order), and every output equals the oracle's."""
    n, clients = 512, 2
    s = Server(capi.RNG_KISS, clients, n, seed_base=4,
               budget_bytes=clients * n * 20 + (1 << 20) + 8192, chunk_rows=4)
    arena = s.stats()["arena_size"]
    big, small = int(0.6 * arena) // 4, int(0.1 * arena) // 4
    log = [workloads.Request(0.0, 0, big, 0), workloads.Request(0.0, 0, big, 1),
           workloads.Request(0.0, 1, small, 1), workloads.Request(0.0, 1, small, 0)]
    rids = [s.submit(r.client, r.n_samples, r.fmt) for r in log]
    s.progress()
    st = s.stats()
    assert st["admitted"] == 3 and st["waiting"] == 1  # only the second large one waits
    outs = {}
    while len(outs) < len(rids):
        s.progress()
        for rid, _ in s.take():
            outs[rid] = s.copy(rid).cpu().numpy().view(np.uint32)
            s.release(rid)
    starts = [0, big, 0, small]
    check_against_oracle(s, log, {i: ({"client": r.client, "n": r.n_samples,
                                        "start": starts[i]}, outs[rids[i]])
                                   for i, r in enumerate(log)}, oracle.KISS, n)
    s.close()


def test_drain_reports_blocked_admission():
    n = 256
    s = Server(capi.RNG_XOR128, 1, n, seed_base=2, budget_bytes=n * 16 + (1 << 20) + 8192,
               chunk_rows=8)
    arena = s.stats()["arena_size"]
    a = s.submit(0, (arena - 28) // 4, 0)  # fills the arena (28 bytes of placement room)
    b = s.submit(0, 1024, 0)
    with pytest.raises(capi.RngError):
        s.drain()  # b cannot be admitted until a is released
    s.release(a)
    s.drain()
    assert {rid for rid, _ in s.take()} >= {b}
    s.close()


def test_realtime_replay_small():
    log = workloads.request_log(rate_hz=400.0, duration_s=0.5, n_clients=4, lo_bytes=1024,
                                hi_bytes=4 << 20, seed=9)
    s = Server(capi.RNG_KISS, 4, 4096, seed_base=3, budget_bytes=256 << 20, chunk_rows=16)
    res = replay(s, log, realtime=True)
    summ = res.summary()
    assert summ["requests"] == len(log) and summ["samples"] == sum(r.n_samples for r in log)
    assert res.latencies_s.min() >= 0 and np.isfinite(summ["p99_ms"])
    s.close()


def test_submit_many_and_release_many():
    n, clients = 777, 4
    log = make_log(40, clients, 9000, seed=21)
    s = Server(capi.RNG_KISS, clients, n, seed_base=11, budget_bytes=32 << 20, chunk_rows=5)
    ids = s.submit_many(np.array([r.client for r in log]), np.array([r.n_samples for r in log]),
                        np.array([r.fmt for r in log]))
    assert ids.tolist() == list(range(len(log)))
    s.drain()
    got, _ = s.take_arrays()
    assert sorted(got.tolist()) == ids.tolist()
    outs = {i: (s.result(int(rid)), s.copy(int(rid)).cpu().numpy().view(np.uint32))
            for i, rid in enumerate(ids)}
    check_against_oracle(s, log, outs, oracle.KISS, n)
    s.release_many(ids)
    assert s.stats()["arena_used"] == 0
    with pytest.raises(capi.RngError):  # nothing is queued if one request is invalid
        s.submit_many(np.array([0, clients]), np.array([5, 5]), np.array([0, 0]))
    assert s.stats()["submitted"] == len(log)
    s.close()


def test_copy_on_user_stream_and_to_host():
    """rng_server_copy enqueues on the stream it is given: torch's current
    stream (a side stream here), or pinned host memory as the target."""
    n, clients = 300, 2
    log = make_log(8, clients, 4000, seed=5)
    s = Server(capi.RNG_KISS, clients, n, seed_base=9, budget_bytes=16 << 20, chunk_rows=3)
    rids = [s.submit(r.client, r.n_samples, r.fmt) for r in log]
    s.drain()
    s.take()
    side = torch.cuda.Stream()
    outs = {}
    for i, rid in enumerate(rids):
        with torch.cuda.stream(side):
            dev = s.copy(rid)
        host = s.copy(rid, out=torch.empty(log[i].n_samples, dtype=torch.int32,
                                           pin_memory=True))
        assert torch.equal(dev.cpu(), host)
        outs[i] = (s.result(rid), host.numpy().view(np.uint32))
    check_against_oracle(s, log, outs, oracle.KISS, n)
    s.release_many(np.array(rids))
    s.close()
