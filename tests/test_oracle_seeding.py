"""Pins for the oracle's seeding, for every generator kind (no GPU).

The paper gives every thread its own seeds (Sec. "Parallelizing RNGs",
parametrisation) but not how they are made.  Here they come from
splitmix64 (Steele, Lea and Flood, OOPSLA 2014) started at seed + s for
stream s, and the draws r0, r1, ... map to each kind's state as follows:

* MWC32: x = lo32(r), c = hi32(r) mod a; the two fixed points (0, 0) and
  (2^32 - 1, a - 1) are drawn again (the Lehmer form needs 0 < a x + c < p).
* xor128: (s0, s1, s2, s3) = (lo32 r0, hi32 r0, lo32 r1, hi32 r1), drawn
  again while all four are zero.
* KISS: (x, c) as MWC32, then y = lo32 and z = hi32 of the next draw; while
  y = 0, y is the lo32 of the draw after.
* MWC16X2 (the paper's two-part base-2^16 MWC): from one draw, part one
  x = bits 0-15, c = bits 16-31 mod a1; part two x = bits 32-47,
  c = bits 48-63 mod a2 (a1, a2 the low and high halves of the packed pair);
  each part packed as x | c << 16; drawn again while either part is a fixed
  point (0, 0) or (2^16 - 1, a - 1).
* XORSHIFT8 (Eq. 5): words 2i, 2i + 1 = lo32, hi32 of draw i (i < 4),
  drawn again while all eight are zero.
* KISS_XOR: the pair as MWC16X2, then y and the LCG word as KISS.

This file restates that mapping with Python integers, with its own
splitmix64 (pinned to published outputs), and compares the oracle with it.
The redraw branches are reached on purpose: splitmix64's finaliser is a
bijection of 64-bit words, so inverting it gives the seed whose draw for a
stream is any chosen word (all zero, a fixed point, y = 0).
"""
from __future__ import annotations

import json
from pathlib import Path

import numpy as np
import pytest

import oracle

GOLD = json.loads((Path(__file__).resolve().parent / "golden" /
                   "splitmix64_vectors.json").read_text())
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
C1, C2 = 0xBF58476D1CE4E5B9, 0x94D049BB133111EB


# ------------------------------------------------ splitmix64, Python ints
def mix(z: int) -> int:
    """splitmix64's output function of the advanced state."""
    z = ((z ^ (z >> 30)) * C1) & M64
    z = ((z ^ (z >> 27)) * C2) & M64
    return z ^ (z >> 31)


def draws(z: int, k: int) -> list[int]:
    """k successive splitmix64 outputs from state z."""
    out = []
    for _ in range(k):
        z = (z + GAMMA) & M64
        out.append(mix(z))
    return out


def _unxorshift_right(v: int, k: int) -> int:
    """Inverse of v -> v ^ (v >> k) on 64-bit words (k >= 1)."""
    r = v
    for _ in range(64 // k + 1):
        r = v ^ (r >> k)
    return r


def unmix(r: int) -> int:
    """The advanced state z with mix(z) = r."""
    z = _unxorshift_right(r, 31)
    z = (z * pow(C2, -1, 1 << 64)) & M64
    z = _unxorshift_right(z, 27)
    z = (z * pow(C1, -1, 1 << 64)) & M64
    return _unxorshift_right(z, 30)


def seed_giving(first_draw: int, s: int, draw_index: int = 0) -> int:
    """The seed for which stream s's draw number draw_index is first_draw."""
    z_before = (unmix(first_draw) - GAMMA * (draw_index + 1)) & M64
    return (z_before - s) & M64


# ---------------------------------------- the documented state mapping
def lo32(v: int) -> int:
    return v & 0xFFFFFFFF


def hi32(v: int) -> int:
    return v >> 32


class Draws:
    def __init__(self, seed: int, s: int):
        self.z = (seed + s) & M64

    def next(self) -> int:
        self.z = (self.z + GAMMA) & M64
        return mix(self.z)


def _mwc_pair(d: Draws, a: int) -> tuple[int, int]:
    while True:
        r = d.next()
        x, c = lo32(r), hi32(r) % a
        if (x, c) != (0, 0) and (x, c) != (0xFFFFFFFF, a - 1):
            return x, c


def _mwc16_pair(d: Draws, a_pair: int) -> tuple[int, int]:
    a1, a2 = a_pair & 0xFFFF, a_pair >> 16
    while True:
        r = d.next()
        x1, c1 = r & 0xFFFF, ((r >> 16) & 0xFFFF) % a1
        x2, c2 = (r >> 32) & 0xFFFF, (r >> 48) % a2
        bad1 = (x1, c1) in ((0, 0), (0xFFFF, a1 - 1))
        bad2 = (x2, c2) in ((0, 0), (0xFFFF, a2 - 1))
        if not bad1 and not bad2:
            return x1 | (c1 << 16), x2 | (c2 << 16)


def _y_and_lcg(d: Draws) -> tuple[int, int]:
    r = d.next()
    y, z = lo32(r), hi32(r)
    while y == 0:
        y = lo32(d.next())
    return y, z


def expected_state(kind: int, a: int | None, seed: int, s: int) -> list[int]:
    d = Draws(seed, s)
    if kind == oracle.MWC:
        return list(_mwc_pair(d, a))
    if kind == oracle.XOR128:
        while True:
            r0, r1 = d.next(), d.next()
            w = [lo32(r0), hi32(r0), lo32(r1), hi32(r1)]
            if any(w):
                return w
    if kind == oracle.KISS:
        x, c = _mwc_pair(d, a)
        return [x, c, *_y_and_lcg(d)]
    if kind == oracle.MWC16X2:
        return list(_mwc16_pair(d, a))
    if kind == oracle.XORSHIFT8:
        while True:
            w = []
            for _ in range(4):
                r = d.next()
                w += [lo32(r), hi32(r)]
            if any(w):
                return w
    if kind == oracle.KISS_XOR:
        p1, p2 = _mwc16_pair(d, a)
        return [p1, p2, *_y_and_lcg(d)]
    raise ValueError(kind)


# ---------------------------------------------------------------- checks
def check_splitmix64_published_vectors():
    """The oracle's splitmix64 (C) and this file's (Python ints) both give
    the published outputs."""
    v = GOLD["first_outputs_from_1234567"]
    assert draws(v["seed"], 5) == v["values"]
    z, got = v["seed"], []
    for _ in range(5):
        z, r = oracle.splitmix64(z)
        got.append(r)
    assert got == v["values"], got
    f = GOLD["fifths_from_987654321"]
    counts, z = [0] * 5, f["seed"]
    for _ in range(f["draws"]):
        z, r = oracle.splitmix64(z)
        counts[(r * 5) >> 64] += 1
    assert counts == f["counts"], counts
    assert oracle.splitmix64(0)[1] == GOLD["first_output_from_0"]["value"]


def _compare(kind: int, a_tab, seed: int, ids) -> None:
    ids = np.asarray(ids, dtype=np.uint64)
    a = None if a_tab is None else np.asarray([a_tab[int(s)] for s in ids], np.uint32)
    got = oracle.seed_streams(kind, a, seed, ids)
    for i, s in enumerate(ids):
        exp = expected_state(kind, None if a is None else int(a[i]), seed, int(s))
        row = [int(w) for w in got[i]]
        # rows are padded to the kind's state width; padding stays zero
        assert row == exp + [0] * (len(row) - len(exp)), (kind, seed, int(s), row, exp)


N_TAB = 2048


def _tables():
    return {k: oracle.multipliers_for(k, N_TAB) for k in range(6)}


def check_seeding_mapping(kind: int, tables=None):
    """The oracle's seeding equals the documented mapping on thousands of
    streams and several seeds, including seeds near 2^64 (seed + s wraps)."""
    tables = tables or _tables()
    a = tables[kind]
    for seed in (0, 7, 42, 1234, M64 - 100):
        _compare(kind, a, seed, range(0, N_TAB, 3 if seed else 1))


def check_seeding_redraws(kind: int, tables=None):
    """Seeds chosen by inverting the finaliser so that the first draws of a
    stream hit each redraw and reduction branch of the mapping."""
    tables = tables or _tables()
    a_tab = tables[kind]
    cases = []  # (stream, draw index, word)
    s = 5
    if kind in (oracle.MWC, oracle.KISS):
        a = int(a_tab[s])
        cases += [
            (s, 0, 0),                                     # (x, c) = (0, 0)
            (s, 0, (a - 1) << 32 | 0xFFFFFFFF),            # the top fixed point
            (s, 0, a << 32),                               # c = a mod a = 0, x = 0
            (s, 0, (0xFFFFFFFF << 32) | 12345),            # c needs the reduction
        ]
    if kind in (oracle.KISS, oracle.KISS_XOR):
        cases += [(s, 1, 0xABCDEF0100000000), (s, 1, 0)]  # y = 0 after the MWC draw
    if kind in (oracle.MWC16X2, oracle.KISS_XOR):
        ap = int(a_tab[s])
        a1, a2 = ap & 0xFFFF, ap >> 16
        cases += [
            (s, 0, 0),                                     # both parts (0, 0)
            (s, 0, 0x1234_5678 << 32),                     # part one (0, 0)
            (s, 0, 0x0000_0001_0003),                      # part two (0, 0)
            (s, 0, ((a1 - 1) << 16) | 0xFFFF | (0x0777_0001 << 32)),  # part one's top point
            (s, 0, (((a2 - 1) << 16 | 0xFFFF) << 32) | 0x0005_0009),  # part two's top point
            (s, 0, 0xFFFF_FFFF_FFFF_FFFF),                 # both carries reduced
        ]
    if kind in (oracle.XOR128, oracle.XORSHIFT8):
        # An all-zero draw set is out of reach: it needs two successive
        # outputs equal to 0, and mix() is a bijection. A zero first word
        # still has to be kept as it is.
        cases += [(s, 0, 0), (s, 1, 0)]
    assert cases
    for stream, idx, word in cases:
        seed = seed_giving(word, stream, idx)
        assert draws((seed + stream) & M64, idx + 1)[idx] == word
        _compare(kind, a_tab, seed, [stream])


KINDS = [oracle.MWC, oracle.XOR128, oracle.KISS, oracle.MWC16X2, oracle.XORSHIFT8,
         oracle.KISS_XOR]


# ----------------------------------------------------------------- tests
def test_unmix_inverts_mix():
    rng = np.random.default_rng(3)
    for w in [0, 1, M64, GAMMA] + [int(v) for v in rng.integers(0, 2**63, 200)]:
        assert mix(unmix(w)) == w


def test_splitmix64_published_vectors():
    check_splitmix64_published_vectors()


@pytest.fixture(scope="module")
def tables():
    return _tables()


@pytest.mark.parametrize("kind", KINDS)
def test_seeding_mapping(kind, tables):
    check_seeding_mapping(kind, tables)


@pytest.mark.parametrize("kind", KINDS)
def test_seeding_redraws(kind, tables):
    check_seeding_redraws(kind, tables)
