"""Parity of the inline consumers (rng_generate_reduce), the jump-ahead
(rng_jump) and split generation (few streams, long sequences cut into
jumped segments) with the oracle, through the C-ABI.  Integer results:
bit-exact."""
from __future__ import annotations

import ctypes
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1101_1846_gb300 import build, capi  # noqa: E402
from paper_1101_1846_gb300.generator import Generator  # noqa: E402

KINDS = [oracle.MWC, oracle.XOR128, oracle.KISS]
OPS = [oracle.SUM_U32, oracle.SUM_U24, oracle.DISC]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


@functools.lru_cache(maxsize=1)
def _table(k=8192):
    return oracle.multipliers(k, 32)


def oracle_a(kind, n):
    return None if kind == oracle.XOR128 else _table()[:n]


def seeded(kind, n, seed):
    return oracle.seed_streams(kind, oracle_a(kind, n), seed, np.arange(n))


def gpu_state(g: Generator) -> np.ndarray:
    """Device state as the oracle's (n, 4) uint32 array."""
    w = g.get_state().numpy().view(np.uint32)  # (words, n)
    st = np.zeros((g.n_streams, 4), np.uint32)
    st[:, :w.shape[0]] = w.T
    return st


def u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def bits(t: torch.Tensor) -> np.ndarray:
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


class split_set:
    """Sets the split threshold of `kind` (0: off) for a block."""

    def __init__(self, kind, log2_rows):
        self.kind, self.log2_rows, self.saved = kind, log2_rows, ctypes.c_int()

    def __enter__(self):
        capi.check(capi.lib().gbrng_get_split(self.kind, ctypes.byref(self.saved)))
        capi.check(capi.lib().gbrng_set_split(self.kind, self.log2_rows))

    def __exit__(self, *exc):
        capi.check(capi.lib().gbrng_set_split(self.kind, self.saved.value))


# ----------------------------------------------------------- consumers
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("split", [True, False], ids=["split", "whole"])
def test_reduce_equals_oracle_and_carries_state(kind, op, split):
    n, seed = 1003, 21
    with split_set(kind, 0 if not split else {0: 6, 1: 8, 2: 7}[kind]):
        _reduce_twice_then_generate(kind, op, n, seed)


def _reduce_twice_then_generate(kind, op, n, seed):
    g = Generator(kind, n, seed)
    st = seeded(kind, n, seed)
    for steps in (777, 1024):  # an odd count leaves an unpaired output
        got = u64(g.generate_reduce(steps, op))
        exp, st = oracle.reduce(kind, oracle_a(kind, n), st, steps, op)
        assert np.array_equal(got, exp), steps
        assert np.array_equal(gpu_state(g), st)
    # the outputs that follow are those of the continued sequence
    out = bits(g.generate(5))
    exp, _ = oracle.generate(kind, oracle_a(kind, n), st, 5, oracle.U32)
    assert np.array_equal(out, exp)
    g.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("op", OPS)
def test_reduce_split_equals_oracle(kind, op):
    # 8 streams x 5001 outputs: split into segments of 64 (MWC), 128 (KISS)
    # or 1024 (xor128) rows that start from jumped states
    n, seed, steps = 8, 5, 5001
    g = Generator(kind, n, seed)
    got = u64(g.generate_reduce(steps, op))
    exp, st = oracle.reduce(kind, oracle_a(kind, n), seeded(kind, n, seed), steps, op)
    assert np.array_equal(got, exp)
    assert np.array_equal(gpu_state(g), st)
    g.close()


def test_reduce_zero_steps_and_bad_args():
    g = Generator(oracle.KISS, 64, 1)
    before = gpu_state(g)
    out = torch.full((64,), 7, dtype=torch.int64, device="cuda")
    g.generate_reduce(0, capi.RNG_DISC, out=out)
    assert np.array_equal(u64(out), np.zeros(64, np.uint64))
    assert np.array_equal(gpu_state(g), before)
    with pytest.raises(capi.RngError):
        g.generate_reduce(10, 3, out=out)
    with pytest.raises(capi.RngError):  # misaligned output
        capi.check(capi.lib().rng_generate_reduce(g.h, 10, 0, out.data_ptr() + 4))
    assert np.array_equal(gpu_state(g), before)
    g.close()


def test_disc_estimates_pi_at_scale():
    n, steps = 1 << 16, 2048
    g = Generator(oracle.KISS, n, 99)
    cnt = int(u64(g.generate_reduce(steps, capi.RNG_DISC)).sum())
    pairs = n * steps // 2
    p = cnt / pairs
    sd = np.sqrt(np.pi / 4 * (1 - np.pi / 4) / pairs)
    assert abs(p - np.pi / 4) < 6 * sd
    g.close()


# --------------------------------------------------------------- jumps
@pytest.mark.parametrize("kind", KINDS)
def test_jump_equals_oracle(kind):
    n, seed = 1000, 8
    g = Generator(kind, n, seed)
    st = seeded(kind, n, seed)
    for k in (0, 1, 63, (1 << 20) + 3, (1 << 63) + 12345, (1 << 64) - 1):
        g.jump(k)
        st = oracle.jump_streams(kind, oracle_a(kind, n), st, k)
        assert np.array_equal(gpu_state(g), st), k
    out = bits(g.generate(16))
    exp, _ = oracle.generate(kind, oracle_a(kind, n), st, 16, oracle.U32)
    assert np.array_equal(out, exp)
    g.close()


@pytest.mark.parametrize("kind", KINDS)
def test_jump_then_generate_equals_stepping(kind):
    n, seed, k = 96, 4, 12345
    g = Generator(kind, n, seed)
    g.jump(k)
    got = bits(g.generate(10))
    full, _ = oracle.generate(kind, oracle_a(kind, n), seeded(kind, n, seed), k + 10, oracle.U32)
    assert np.array_equal(got, full[k:])
    g.close()


# ------------------------------------------------------ split generation
@pytest.mark.parametrize("kind,n,steps", [(oracle.MWC, 64, 5000), (oracle.KISS, 64, 5000),
                                          (oracle.XOR128, 8, 20000), (oracle.KISS, 8, 300),
                                          (oracle.MWC, 4, 100_000),
                                          # rows 16- but not 32-byte aligned: barrier-synced
                                          (oracle.MWC, 12, 5000), (oracle.KISS, 20, 3000),
                                          (oracle.XOR128, 12, 5000)])
@pytest.mark.parametrize("fmt", [oracle.U32, oracle.F32])
def test_split_generate_equals_oracle(kind, n, steps, fmt):
    seed = 17
    g = Generator(kind, n, seed)
    got = bits(g.generate(steps, fmt))
    st = seeded(kind, n, seed)
    exp, st = oracle.generate(kind, oracle_a(kind, n), st, steps, fmt)
    assert np.array_equal(got, np.ascontiguousarray(exp).view(np.uint32))
    assert np.array_equal(gpu_state(g), st)
    got2 = bits(g.generate(3, fmt))
    exp2, _ = oracle.generate(kind, oracle_a(kind, n), st, 3, fmt)
    assert np.array_equal(got2, np.ascontiguousarray(exp2).view(np.uint32))
    g.close()


@pytest.mark.parametrize("kind", [oracle.MWC, oracle.KISS])
def test_split_jump_table_grows_and_rebuilds(kind):
    """One handle through split calls whose segment counts and lengths
    change: the per-handle MWC jump table is allocated by the first, grown
    when a call needs more segments, and rebuilt when the segment length
    changes; consumer calls share it.  Every output and state equals the
    oracle's."""
    n, seed = 64, 29
    g = Generator(kind, n, seed)
    a = oracle_a(kind, n)
    st = seeded(kind, n, seed)
    # a few segments (allocates), many (grows), then longer segments
    # (rebuilds); the consumer calls go back to the default length (rebuild)
    # and then need more segments again (grow)
    for steps, log2_rows in ((300, None), (6000, None), (700, 8)):
        if log2_rows is None:
            got = bits(g.generate(steps))
        else:
            with split_set(kind, log2_rows):
                got = bits(g.generate(steps))
        exp, st = oracle.generate(kind, a, st, steps, oracle.U32)
        assert np.array_equal(got, exp), steps
        assert np.array_equal(gpu_state(g), st), steps
    for steps in (2500, 12000):
        got = u64(g.generate_reduce(steps, oracle.SUM_U32))
        exp, st = oracle.reduce(kind, a, st, steps, oracle.SUM_U32)
        assert np.array_equal(got, exp), steps
        assert np.array_equal(gpu_state(g), st), steps
    got = bits(g.generate(4000))
    exp, st = oracle.generate(kind, a, st, 4000, oracle.U32)
    assert np.array_equal(got, exp)
    g.close()


def test_split_mwc_4096_by_4096_equals_oracle():
    """The few-streams configuration: MWC, 4096 streams x 4096 outputs."""
    n, steps, seed = 4096, 4096, 42
    g = Generator(oracle.MWC, n, seed)
    got = bits(g.generate(steps))
    exp, st = oracle.generate(oracle.MWC, oracle_a(oracle.MWC, n), seeded(oracle.MWC, n, seed),
                              steps, oracle.U32)
    assert np.array_equal(got, exp)
    assert np.array_equal(gpu_state(g), st)
    g.close()


@pytest.mark.parametrize("kind", KINDS)
def test_split_range_leaves_other_streams(kind):
    n, seed, steps = 4096, 3, 3000
    g = Generator(kind, n, seed)
    out = torch.zeros((steps, n), dtype=torch.int32, device="cuda")
    g.generate_range(512, 1024, steps, out, ld=n, offset=512)
    st = seeded(kind, n, seed)
    exp, st_new = oracle.generate(kind, oracle_a(kind, n)[512:1024] if kind != oracle.XOR128
                                  else None, st[512:1024], steps, oracle.U32)
    got = bits(out)
    assert np.array_equal(got[:, 512:1024], exp)
    assert not got[:, :512].any() and not got[:, 1024:].any()
    full = gpu_state(g)
    assert np.array_equal(full[512:1024], st_new)
    assert np.array_equal(full[:512], st[:512]) and np.array_equal(full[1024:], st[1024:])
    g.close()


@pytest.mark.parametrize("kind", KINDS)
def test_split_off_gives_the_same_outputs(kind):
    n, steps = 64, 4000
    a, b = Generator(kind, n, 1), Generator(kind, n, 1)
    split = bits(a.generate(steps))
    with split_set(kind, 0):
        plain = bits(b.generate(steps))
    assert np.array_equal(split, plain)
    assert np.array_equal(gpu_state(a), gpu_state(b))
    a.close()
    b.close()


def test_device_view_describes_the_handle():
    g = Generator(oracle.KISS, 300, 2)
    v = g.device_view()
    assert (v.kind, v.state_words, v.n_streams) == (oracle.KISS, 4, 300)
    assert v.state and v.mult and v.device == torch.cuda.current_device()
    x = Generator(oracle.XOR128, 40, 2).device_view()
    assert x.mult is None and x.state_words == 4
    g.close()


@pytest.mark.parametrize("kind", [oracle.MWC, oracle.KISS])
def test_split_calls_captured_in_a_cuda_graph(kind):
    """A split call captured in a CUDA graph powers its jumps itself (the
    handle's multiplier table is not built during a capture), so a direct
    call made before the first replay, with another segment length, and the
    replays all continue the one sequence."""
    n, seed = 64, 23
    g = Generator(kind, n, seed)
    out = torch.empty((4096, n), dtype=torch.int32, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=side):
        g.generate(4096, oracle.U32, out=out)
    first = bits(g.generate(2048))          # not captured; another segment length
    graph.replay()
    second = bits(out)
    graph.replay()
    third = bits(out)
    exp, st = oracle.generate(kind, oracle_a(kind, n), seeded(kind, n, seed), 2048 + 2 * 4096,
                              oracle.U32)
    assert np.array_equal(first, exp[:2048])
    assert np.array_equal(second, exp[2048:6144])
    assert np.array_equal(third, exp[6144:])
    assert np.array_equal(gpu_state(g), st)
    g.close()
