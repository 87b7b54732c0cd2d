"""Device seeding (rng_create) against the oracle on seeds that force every
redraw and reduction branch of the state mapping, for all six kinds.

The seeds are found by inverting splitmix64's finaliser
(test_oracle_seeding.seed_giving), so that a chosen stream's draw is a
chosen word: an MWC fixed point, a carry that needs reducing, y = 0 for
KISS, a bad part of the two-part base-2^16 MWC.  The expected states come
from the oracle only."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import test_oracle_seeding as sd  # noqa: E402
from paper_1101_1846_gb300 import build, capi  # noqa: E402
from paper_1101_1846_gb300.generator import Generator  # noqa: E402

N = 64


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


def _cases(kind: int, a_tab) -> list[tuple[int, int, int]]:
    """(stream, draw index, word) triples that reach the mapping's branches."""
    out = []
    for s in (0, 5, 37, N - 1):
        if kind in (oracle.MWC, oracle.KISS):
            a = int(a_tab[s])
            out += [(s, 0, 0), (s, 0, (a - 1) << 32 | 0xFFFFFFFF), (s, 0, a << 32),
                    (s, 0, (0xFFFFFFFF << 32) | 77)]
        if kind in (oracle.KISS, oracle.KISS_XOR):
            out += [(s, 1, 0x13579BDF00000000), (s, 1, 0)]
        if kind in (oracle.MWC16X2, oracle.KISS_XOR):
            ap = int(a_tab[s])
            a1, a2 = ap & 0xFFFF, ap >> 16
            out += [(s, 0, 0), (s, 0, 0x2345_6789 << 32), (s, 0, 0x0000_0001_0003),
                    (s, 0, ((a1 - 1) << 16) | 0xFFFF | (0x0777_0001 << 32)),
                    (s, 0, (((a2 - 1) << 16 | 0xFFFF) << 32) | 0x0005_0009),
                    (s, 0, 0xFFFF_FFFF_FFFF_FFFF)]
        if kind in (oracle.XOR128, oracle.XORSHIFT8):
            out += [(s, 0, 0), (s, 1, 0)]
    return out


@pytest.mark.parametrize("kind", range(6))
def test_device_seeding_takes_every_redraw_branch(kind):
    a_tab = oracle.multipliers_for(kind, N)
    for s, idx, word in _cases(kind, a_tab):
        seed = sd.seed_giving(word, s, idx)
        with Generator(kind, N, seed) as g:
            got = g.get_state().numpy().view(np.uint32).T
        exp = oracle.seed_streams(kind, a_tab, seed, np.arange(N))
        assert np.array_equal(got, exp[:, :got.shape[1]]), (kind, s, idx, hex(word))
        # the same seed also fixes the outputs that follow
        if s == 5:
            with Generator(kind, N, seed) as g:
                out = g.generate(9).cpu().view(torch.int32).numpy().view(np.uint32)
            ref, _ = oracle.generate(kind, a_tab, exp, 9, oracle.U32)
            assert np.array_equal(out, ref), (kind, s, idx)


@pytest.mark.parametrize("kind", range(6))
def test_range_handle_is_the_slice_of_the_whole_generator(kind):
    """rng_create_range(kind, s_begin, n, seed) gives the streams s_begin ..
    s_begin + n - 1 of rng_create(kind, s_begin + n, seed): the same
    multipliers, states and outputs, over two carried calls; and the oracle
    agrees."""
    n, s_begin, seed, steps = 300, 1000, 4242, 17
    with Generator(kind, s_begin + n, seed) as whole, \
            Generator(kind, n, seed, s_begin=s_begin) as part:
        for _ in range(2):
            w = whole.generate(steps).cpu().view(torch.int32).numpy().view(np.uint32)
            p = part.generate(steps).cpu().view(torch.int32).numpy().view(np.uint32)
            assert np.array_equal(p, w[:, s_begin:])
        ws = whole.get_state().numpy()
        assert np.array_equal(part.get_state().numpy(), ws[:, s_begin:])
    table = oracle.multipliers_for(kind, s_begin + n)
    a = None if table is None else table[s_begin:]
    st = oracle.seed_streams(kind, a, seed + s_begin, np.arange(n))
    exp, _ = oracle.generate(kind, a, st, 2 * steps, oracle.U32)
    assert np.array_equal(p, exp[steps:])


def test_range_handle_rejects_ranges_beyond_the_table():
    L = capi.lib()
    assert L.rng_create_range(0, capi.RNG_MAX_STREAMS_MWC - 10, 11, 1) is None
    assert L.rng_last_error() == capi.RNG_ERR_ARG
    h = L.rng_create_range(0, capi.RNG_MAX_STREAMS_MWC - 10, 10, 1)
    assert h
    L.rng_destroy(h)
