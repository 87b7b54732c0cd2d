"""Parity of the paper's own generators on the CUDA path (through the C-ABI)
with the oracle: the two-part base-2^16 MWC, the r = 8 XorShift of Eq. 5
and KISS in the xor form.  Bit-exact for uint32 and FP32."""
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
from paper_1101_1846_gb300.generator import BatchItem, Generator, generate_batch  # noqa: E402

PAPER = [oracle.MWC16X2, oracle.XORSHIFT8, oracle.KISS_XOR]
FMTS = [oracle.U32, oracle.F32]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


@functools.lru_cache(maxsize=1)
def _pairs():
    return oracle.mwc16_pairs(capi.RNG_MAX_STREAMS_MWC16)


def oracle_a(kind, n):
    return _pairs()[:n] if kind in (oracle.MWC16X2, oracle.KISS_XOR) else None


def seeded(kind, n, seed):
    return oracle.seed_streams(kind, oracle_a(kind, n), seed, np.arange(n))


def gpu_state(g: Generator) -> np.ndarray:
    w = g.get_state().numpy().view(np.uint32)  # (words, n)
    st = np.zeros((g.n_streams, oracle.words(g.kind)), np.uint32)
    st[:, :w.shape[0]] = w.T
    return st


def bits(t: torch.Tensor) -> np.ndarray:
    return t.cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def obits(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a).view(np.uint32)


def test_pair_table_equals_oracle():
    k = capi.RNG_MAX_STREAMS_MWC16
    out = torch.empty(k, dtype=torch.int32, device="cuda")
    capi.check(capi.lib().rng_mwc16_pairs(k, ctypes.c_void_p(out.data_ptr())))
    assert np.array_equal(bits(out), _pairs())
    with pytest.raises(capi.RngError):
        capi.check(capi.lib().rng_mwc16_pairs(k + 1, ctypes.c_void_p(out.data_ptr())))


@pytest.mark.parametrize("kind", PAPER)
@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("n", [1, 3, 4, 5, 8, 33, 64, 1003, 4096])
def test_generate_equals_oracle_with_state_carry(kind, fmt, n):
    seed = 1000 + n
    g = Generator(kind, n, seed)
    st = seeded(kind, n, seed)
    for steps in (7, 64):
        got = bits(g.generate(steps, fmt))
        exp, st = oracle.generate(kind, oracle_a(kind, n), st, steps, fmt)
        assert np.array_equal(got, obits(exp)), steps
        assert np.array_equal(gpu_state(g), st)
    g.close()


@pytest.mark.parametrize("kind", PAPER)
def test_unaligned_rows_and_ranges(kind):
    n, steps, seed = 1000, 40, 3
    g = Generator(kind, n, seed)
    st = seeded(kind, n, seed)
    out = torch.zeros(steps * 1003 + 8, dtype=torch.int32, device="cuda")
    # streams [101, 702) with a row stride of 1003 at an odd word offset
    g.generate_range(101, 702, steps, out, ld=1003, offset=5)
    a = oracle_a(kind, n)
    exp, st_new = oracle.generate(kind, a[101:702] if a is not None else None, st[101:702],
                                  steps, oracle.U32)
    got = bits(out)[5:5 + steps * 1003].reshape(steps, 1003)[:, :601]
    assert np.array_equal(got, exp)
    full = gpu_state(g)
    assert np.array_equal(full[101:702], st_new)
    assert np.array_equal(full[:101], st[:101]) and np.array_equal(full[702:], st[702:])
    g.close()


@pytest.mark.parametrize("kind,n,steps", [(oracle.MWC16X2, 8, 5000), (oracle.KISS_XOR, 64, 4096),
                                          (oracle.XORSHIFT8, 8, 3000),
                                          (oracle.MWC16X2, 4096, 1000),
                                          # every pair; rows 16- but not 32-byte aligned
                                          (oracle.MWC16X2, 76636, 600),
                                          (oracle.KISS_XOR, 76636, 600)])
def test_few_streams_long_sequences(kind, n, steps):
    # MWC16X2 and KISS_XOR split into jumped segments; XORSHIFT8 does not
    seed = 9
    g = Generator(kind, n, seed)
    got = bits(g.generate(steps))
    exp, st = oracle.generate(kind, oracle_a(kind, n), seeded(kind, n, seed), steps, oracle.U32)
    assert np.array_equal(got, exp)
    assert np.array_equal(gpu_state(g), st)
    g.close()


@pytest.mark.parametrize("kind", PAPER)
@pytest.mark.parametrize("op", [oracle.SUM_U32, oracle.SUM_U24, oracle.DISC])
@pytest.mark.parametrize("n,steps", [(8, 3001), (5000, 300)])
def test_reduce_equals_oracle(kind, op, n, steps):
    seed = 12
    g = Generator(kind, n, seed)
    got = g.generate_reduce(steps, op).cpu().numpy().view(np.uint64)
    exp, st = oracle.reduce(kind, oracle_a(kind, n), seeded(kind, n, seed), steps, op)
    assert np.array_equal(got, exp)
    assert np.array_equal(gpu_state(g), st)
    g.close()


@pytest.mark.parametrize("kind", PAPER)
def test_jump_equals_oracle(kind):
    n, seed = 300, 8
    g = Generator(kind, n, seed)
    st = seeded(kind, n, seed)
    a = oracle_a(kind, n)
    for k in (0, 1, 77, (1 << 33) + 5, (1 << 64) - 1):
        g.jump(k)
        st = oracle.jump_streams(kind, a, st, k)
        assert np.array_equal(gpu_state(g), st), k
    g.close()


@pytest.mark.parametrize("kind", PAPER)
def test_host_delivery_and_checkpoint(kind):
    n, steps, seed = 500, 33, 4
    g = Generator(kind, n, seed)
    saved = g.get_state()
    host = g.generate_host(steps)
    exp, _ = oracle.generate(kind, oracle_a(kind, n), seeded(kind, n, seed), steps, oracle.U32)
    assert np.array_equal(host.numpy().view(np.uint32), exp)
    g.set_state(saved)
    assert np.array_equal(bits(g.generate(steps)), exp)
    bad = saved.clone()
    bad[:, 7] = 0  # all words of stream 7 zero (MWC parts: a fixed point)
    with pytest.raises(capi.RngError):
        g.set_state(bad)
    g.close()


def test_limits_and_batched_kinds():
    g = Generator(oracle.MWC16X2, capi.RNG_MAX_STREAMS_MWC16, 1)
    assert g.n_streams == capi.RNG_MAX_STREAMS_MWC16 and g.words == 2
    out = torch.empty((2, g.n_streams), dtype=torch.int32, device="cuda")
    with pytest.raises(capi.RngError):
        generate_batch([BatchItem(g, 2, out, oracle.U32)])
    g.close()
    assert not capi.lib().rng_create(oracle.KISS_XOR, capi.RNG_MAX_STREAMS_MWC16 + 1, 1)
    assert capi.lib().rng_last_error() == capi.RNG_ERR_ARG
    x = Generator(oracle.XORSHIFT8, 64, 1)
    assert x.words == 8
    x.close()
