"""Pins for the oracle's consumers (numbers used inline, only the final state
stored: Sec. "Performance evaluation") and its jump-ahead (sequence
splitting: Sec. "Parallelizing RNGs").  Each check_* raises AssertionError
when the oracle gets the fact wrong; test_oracle_mutants.py plants mistakes
in copies of oracle.c and expects one of these checks to fail."""
from __future__ import annotations

import math

import numpy as np

import oracle

M32 = 1 << 32
M64 = 1 << 64


# ------------------------------------------------------------ consumers
def check_sum_closed_forms():
    n = 100_003
    ramp = np.arange(n, dtype=np.uint64)
    assert oracle.sum_u32(ramp.astype(np.uint32)) == n * (n - 1) // 2
    # the low byte is not part of the 24-bit integer
    noisy = ((ramp << np.uint64(8)) | np.uint64(0xAB)).astype(np.uint32)
    assert oracle.sum_u24(noisy) == n * (n - 1) // 2
    top = np.full(3 * 65_536, M32 - 1, dtype=np.uint32)
    assert oracle.sum_u32(top) == (M32 - 1) * len(top)
    assert oracle.sum_u24(top) == ((M32 - 1) >> 8) * len(top)
    assert oracle.sum_u32(top[:0]) == 0 and oracle.sum_u24(top[:0]) == 0


def _lattice_sequence(g: int, noise: int = 0) -> np.ndarray:
    """Points (i h, j h) of a g x g grid (h = 2^24 / g) as consecutive pairs
    of outputs, row by row; `noise` fills the low byte."""
    h = (1 << 24) // g
    i, j = np.meshgrid(np.arange(g, dtype=np.uint64), np.arange(g, dtype=np.uint64),
                       indexing="ij")
    pts = np.stack([i.ravel() * h, j.ravel() * h], axis=1)
    return ((pts << np.uint64(8)) | np.uint64(noise)).astype(np.uint32).ravel()


def check_disc_lattice_count():
    """Grid points inside the quarter disc, counted row by row with integer
    square roots: for x = i h, the j with (j h)^2 < 2^48 - x^2 are those with
    j h <= isqrt(2^48 - 1 - x^2)."""
    for g, noise in ((512, 0), (300, 0x5C), (1000, 0xFF)):
        h = (1 << 24) // g
        expect = sum(min(math.isqrt((1 << 48) - 1 - (i * h) ** 2) // h + 1, g)
                     for i in range(g))
        seq = _lattice_sequence(g, noise)
        assert oracle.disc_count(seq) == expect, (g, noise)
        # an odd trailing output is unpaired and ignored
        assert oracle.disc_count(np.append(seq, np.uint32(0))) == expect
    # with g = 512 the grid is exact: i^2 + j^2 < 512^2
    assert oracle.disc_count(_lattice_sequence(512)) == sum(
        math.isqrt(512 * 512 - 1 - i * i) + 1 for i in range(512))


def check_disc_estimates_pi():
    """Over 2^21 KISS points the fraction inside is pi/4 within 5 standard
    deviations of a binomial proportion."""
    n, steps = 64, 1 << 16
    a = oracle.multipliers(n, 32)
    st = oracle.seed_streams(oracle.KISS, a, 2024, np.arange(n))
    out, _ = oracle.reduce(oracle.KISS, a, st, steps, oracle.DISC)
    pairs = n * (steps // 2)
    p = int(out.sum()) / pairs
    sd = math.sqrt((math.pi / 4) * (1 - math.pi / 4) / pairs)
    assert abs(p - math.pi / 4) < 5 * sd, p


def check_sum_means():
    """The mean output of each kind is within 6 standard deviations of the
    uniform mean (2^32 - 1)/2; the 24-bit mean of (2^24 - 1)/2."""
    n, steps = 32, 1 << 15
    for kind in (oracle.MWC, oracle.XOR128, oracle.KISS):
        a = oracle.multipliers(n, 32) if kind != oracle.XOR128 else None
        st = oracle.seed_streams(kind, a, 77, np.arange(n))
        for op, top in ((oracle.SUM_U32, M32), (oracle.SUM_U24, 1 << 24)):
            out, _ = oracle.reduce(kind, a, st, steps, op)
            mean = sum(int(v) for v in out) / (n * steps)
            sd = top / math.sqrt(12 * n * steps)
            assert abs(mean - (top - 1) / 2) < 6 * sd, (kind, op, mean)


def check_reduce_advances_like_generate():
    n, steps = 5, 777
    for kind in (oracle.MWC, oracle.XOR128, oracle.KISS, oracle.MWC16X2, oracle.XORSHIFT8,
                 oracle.KISS_XOR):
        a = oracle.multipliers_for(kind, n)
        st = oracle.seed_streams(kind, a, 3, np.arange(n))
        u, st_gen = oracle.generate(kind, a, st, steps, oracle.U32)
        for op, fn in ((oracle.SUM_U32, oracle.sum_u32), (oracle.SUM_U24, oracle.sum_u24),
                       (oracle.DISC, oracle.disc_count)):
            out, st_red = oracle.reduce(kind, a, st, steps, op)
            assert np.array_equal(st_red, st_gen)
            assert [int(v) for v in out] == [fn(u[:, s].copy()) for s in range(n)]


def test_sum_closed_forms():
    check_sum_closed_forms()


def test_disc_lattice_count():
    check_disc_lattice_count()


def test_disc_estimates_pi():
    check_disc_estimates_pi()


def test_sum_means():
    check_sum_means()


def test_reduce_advances_like_generate():
    check_reduce_advances_like_generate()


# ---------------------------------------------------------------- jumps
JUMPS = (0, 1, 2, 3, 31, 32, 33, 1000, (1 << 17) + 5)


ALL_KINDS = (oracle.MWC, oracle.XOR128, oracle.KISS, oracle.MWC16X2, oracle.XORSHIFT8,
             oracle.KISS_XOR)


def check_jump_equals_stepping():
    """The state after jump(k) equals the state after k single steps."""
    n = 3
    for kind in ALL_KINDS:
        a = oracle.multipliers_for(kind, n)
        st = oracle.seed_streams(kind, a, 11, np.arange(n))
        for s in range(n):
            for k in JUMPS:
                ai = int(a[s]) if a is not None else 0
                _, stepped = oracle.stream(kind, ai, st[s], k, oracle.U32)
                jumped = oracle.jump(kind, ai, st[s], k)
                assert np.array_equal(stepped, jumped), (kind, s, k)


def check_jump_composes():
    rng = np.random.Generator(np.random.PCG64(8))
    for kind in ALL_KINDS:
        a = oracle.multipliers_for(kind, 2)
        a0 = int(a[0]) if a is not None else 0
        st = oracle.seed_streams(kind, a, 5, np.arange(2))
        for _ in range(4):
            j = int(rng.integers(0, 1 << 62)) * 3
            k = int(rng.integers(0, 1 << 62))
            two = oracle.jump(kind, a0, oracle.jump(kind, a0, st[0], j), k)
            one = oracle.jump(kind, a0, st[0], (j + k) % M64)
            assert np.array_equal(two, one), (kind, j, k)


def check_mwc_jump_lehmer():
    """jump(k) multiplies t = a x + c by b^-k mod p (Python integers)."""
    b = M32
    a_tab = oracle.multipliers(3, 32)
    st = oracle.seed_streams(oracle.MWC, a_tab, 9, np.arange(3))
    for s, a in enumerate(int(v) for v in a_tab):
        p = a * b - 1
        t = a * int(st[s][0]) + int(st[s][1])
        for k in (1, 10 ** 9, (1 << 63) + 12345):
            tk = (pow(b, -k, p) * t) % p
            x, c = oracle.mwc_jump(a, int(st[s][0]), int(st[s][1]), k)
            assert (x, c) == (tk // a, tk % a), (a, k)


def check_jump_periods():
    """One jump by a part's period returns to the start; a jump by a proper
    divisor of it does not.  MWC: the order of a modulo the safe prime
    p = a b - 1 is q = (p - 1)/2 (b is a square, a = b^-1); xorshift32:
    2^32 - 1; LCG: 2^32 (Hull-Dobell)."""
    for a in (int(v) for v in oracle.multipliers(3, 32)):
        q = (a * M32 - 2) // 2
        for x, c in ((123456789, 4321), (M32 - 2, a - 1)):
            assert oracle.mwc_jump(a, x, c, q) == (x, c)
            assert oracle.mwc_jump(a, x, c, q - 1) != (x, c)
    for a in (int(v) for v in oracle.multipliers(2000, 16)[-3:]):
        q = (a * (1 << 16) - 2) // 2
        assert oracle.mwc_jump(a, 12345, 7, q, 16) == (12345, 7)
        assert oracle.mwc_jump(a, 12345, 7, q - 1, 16) != (12345, 7)
    for y in (1, 0xDEADBEEF):
        assert oracle.xorshift32_jump(y, M32 - 1) == y
        for f in (3, 5, 17, 257, 65537):
            assert oracle.xorshift32_jump(y, (M32 - 1) // f) != y
    for z in (0, 987654321):
        assert oracle.lcg_jump(z, M32) == z
        assert oracle.lcg_jump(z, M32 // 2) != z


def test_jump_equals_stepping():
    check_jump_equals_stepping()


def test_jump_composes():
    check_jump_composes()


def test_mwc_jump_lehmer():
    check_mwc_jump_lehmer()


def test_jump_periods():
    check_jump_periods()
