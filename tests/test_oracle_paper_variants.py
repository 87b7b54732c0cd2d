"""Pins for the oracle's versions of the paper's own generators: the
two-part base-2^16 MWC (Methods / MWC), Panneton's r = 8 XorShift (Eq. 5)
and KISS in the paper's xor form (Background / KISS).  Each check_* raises
AssertionError when the oracle gets the fact wrong; test_oracle_mutants.py
plants mistakes in copies of oracle.c and expects one of them to fail."""
from __future__ import annotations

import itertools
import math

import numpy as np

import oracle

M32 = 1 << 32
B16 = 1 << 16

# 2^256 - 1 = F0 F1 ... F7 (Fermat numbers F_k = 2^(2^k) + 1), with the
# published factorisations of F5, F6 and F7.
F256 = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721, 59649589127497217,
        5704689200685129054721]


def _probable_prime(n: int) -> bool:
    """Miller-Rabin with the first twelve prime bases (deterministic below
    3.3e24), written here with Python integers."""
    if n < 2:
        return False
    bases = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37]
    for p in bases:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in bases:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _gf2_matrix(step_words, nwords: int) -> np.ndarray:
    """Columns: images of the unit vectors under a GF(2)-linear step on
    nwords 32-bit words (bit b of word k is row 32k + b)."""
    n = 32 * nwords
    m = np.zeros((n, n), np.float32)
    for j in range(n):
        st = [0] * nwords
        st[j // 32] = 1 << (j % 32)
        img = step_words(st)
        for k, w in enumerate(img):
            for b in range(32):
                if (int(w) >> b) & 1:
                    m[32 * k + b, j] = 1.0
    return m


def _gf2_pow(m: np.ndarray, e: int) -> np.ndarray:
    # float32 products are exact here: every entry of a product is a count
    # of at most 256 ones
    r = np.eye(m.shape[0], dtype=np.float32)
    b = m.copy()
    while e:
        if e & 1:
            r = np.mod(r @ b, 2.0)
        b = np.mod(b @ b, 2.0)
        e >>= 1
    return r


# ---------------------------------------------------------- multipliers
def check_mwc16_pairs_lexicographic():
    table = [int(v) for v in oracle.multipliers(2000, 16)]
    assert len(table) == 392
    expect = [a | (b << 16) for a, b in itertools.combinations(table, 2)]
    got = oracle.mwc16_pairs(len(expect) + 10)
    assert len(got) == 392 * 391 // 2
    assert [int(v) for v in got] == expect


def test_mwc16_pairs_lexicographic():
    check_mwc16_pairs_lexicographic()


# ------------------------------------------------------- two-part MWC
def check_mwc16x2_closed_form():
    """With b = 2^16, a part's packed word z = x + c b after a step is the
    previous Lehmer value t = a x + c, and t_n = b^-n t_0 mod (a b - 1).
    Output n is ((z << 16) + w) mod 2^32 of the words after step n+1."""
    pairs = oracle.mwc16_pairs(400)
    for s in (0, 1, 391, 399):
        ap = int(pairs[s])
        a1, a2 = ap & 0xFFFF, ap >> 16
        p1, p2 = a1 * B16 - 1, a2 * B16 - 1
        st = oracle.seed_streams(oracle.MWC16X2, pairs[s:s + 1], 42, np.array([s]))[0]
        z0, w0 = int(st[0]), int(st[1])
        t1 = a1 * (z0 & 0xFFFF) + (z0 >> 16)
        t2 = a2 * (w0 & 0xFFFF) + (w0 >> 16)
        out, _ = oracle.stream(oracle.MWC16X2, ap, st, 3000, oracle.U32)
        for n in (0, 1, 2, 17, 1000, 2999):
            z = pow(B16, -n, p1) * t1 % p1
            w = pow(B16, -n, p2) * t2 % p2
            assert int(out[n]) == ((z << 16) + w) % M32, (s, n)


def check_mwc16x2_parts_are_base16_mwcs():
    """Each packed word follows Eq. 2-3 with b = 2^16 (the pinned MWC step)."""
    rng = np.random.Generator(np.random.PCG64(4))
    pairs = oracle.mwc16_pairs(1000)
    for _ in range(100):
        ap = int(pairs[rng.integers(0, 1000)])
        a1, a2 = ap & 0xFFFF, ap >> 16
        z = int(rng.integers(0, B16)) | (int(rng.integers(0, a1)) << 16)
        w = int(rng.integers(0, B16)) | (int(rng.integers(0, a2)) << 16)
        _, new = oracle.mwc16x2_step(ap, [z, w])
        x1, c1 = oracle.mwc_step(a1, z & 0xFFFF, z >> 16, 16)
        x2, c2 = oracle.mwc_step(a2, w & 0xFFFF, w >> 16, 16)
        assert new == [x1 | (c1 << 16), x2 | (c2 << 16)]


def test_mwc16x2_closed_form():
    check_mwc16x2_closed_form()


def test_mwc16x2_parts_are_base16_mwcs():
    check_mwc16x2_parts_are_base16_mwcs()


# ------------------------------------------------------ r = 8 XorShift
def _xs8_words(st):
    return oracle.xorshift8_step(st)[1]


def check_xorshift8_full_period():
    """Eq. 5's 256 x 256 matrix M over GF(2) has M^(2^256-1) = I and
    M^((2^256-1)/q) != I for every prime q dividing 2^256 - 1: period
    2^256 - 1 from any nonzero state (Panneton's full-period claim)."""
    order = (1 << 256) - 1
    assert math.prod(F256) == order and all(_probable_prime(q) for q in F256)
    m = _gf2_matrix(_xs8_words, 8)
    eye = np.eye(256, dtype=np.float32)
    assert np.array_equal(_gf2_pow(m, order), eye)
    for q in F256:
        assert not np.array_equal(_gf2_pow(m, order // q), eye), q


def check_xorshift8_shift_register():
    rng = np.random.Generator(np.random.PCG64(9))
    for _ in range(50):
        st = [int(v) for v in rng.integers(0, M32, 8)]
        out, new = oracle.xorshift8_step(st)
        assert out == new[7] and new[:7] == st[1:]


def check_xorshift8_lags():
    """The new word depends on exactly v_{n-1}, v_{n-4}, v_{n-5}, v_{n-7} and
    v_{n-8} (Eq. 5 has s = 7 xorshifts spread over five lags)."""
    for k in range(8):
        st = [0] * 8
        st[k] = 0x80000001
        out, _ = oracle.xorshift8_step(st)
        lag = 8 - k
        assert (out != 0) == (lag in (1, 4, 5, 7, 8)), lag


def test_xorshift8_full_period():
    check_xorshift8_full_period()


def test_xorshift8_shift_register_and_lags():
    check_xorshift8_shift_register()
    check_xorshift8_lags()


# ------------------------------------------------------------ KISS xor
def check_kiss_xor_is_parts():
    """(MWC xor LCG) + XorShift mod 2^32, each part stepped on its own."""
    pairs = oracle.mwc16_pairs(64)
    st = oracle.seed_streams(oracle.KISS_XOR, pairs, 5, np.arange(64))
    for s in range(0, 64, 7):
        ap = int(pairs[s])
        zw, y, z = [int(st[s][0]), int(st[s][1])], int(st[s][2]), int(st[s][3])
        cur = [int(v) for v in st[s]]
        for _ in range(200):
            out, cur = oracle.kiss_xor_step(ap, cur)
            m, zw = oracle.mwc16x2_step(ap, zw)
            y = oracle.xorshift32_step(y)
            z = oracle.lcg_step(z)
            assert out == ((m ^ z) + y) % M32


def test_kiss_xor_is_parts():
    check_kiss_xor_is_parts()


# ------------------------------------------------------------- seeding
def test_seeding_valid_states():
    n = 3000
    pairs = oracle.mwc16_pairs(n)
    for kind in (oracle.MWC16X2, oracle.KISS_XOR):
        st = oracle.seed_streams(kind, pairs, 77, np.arange(n))
        for part, shift in ((0, 0), (1, 16)):
            a = (pairs.astype(np.int64) >> shift) & 0xFFFF
            x, c = st[:, part].astype(np.int64) & 0xFFFF, st[:, part].astype(np.int64) >> 16
            assert np.all(c < a)
            assert not np.any((x == 0) & (c == 0))
            assert not np.any((x == 0xFFFF) & (c == a - 1))
        if kind == oracle.KISS_XOR:
            assert np.all(st[:, 2] != 0)
    st = oracle.seed_streams(oracle.XORSHIFT8, None, 77, np.arange(n))
    assert st.shape == (n, 8) and np.all(st.any(axis=1))
    # draws come from splitmix64 started at seed + s: stream s of seed 77
    # equals stream 0 of seed 77 + s
    one = oracle.seed_streams(oracle.XORSHIFT8, None, 77 + 5, np.array([0]))
    assert np.array_equal(one[0], st[5])
