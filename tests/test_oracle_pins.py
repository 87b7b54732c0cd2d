"""Pins for the oracle: facts the paper or mathematics fixes, checked against
oracle/ on the CPU (no GPU).  Each check_* function raises AssertionError
when the oracle gets the fact wrong; tests/test_oracle_mutants.py runs the
same checks against copies of the oracle with a planted mistake and expects
them to fail."""
from __future__ import annotations

import hashlib
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle

GOLD = Path(__file__).resolve().parent / "golden"
PAPER = json.loads((GOLD / "paper_values.json").read_text())
M32 = 1 << 32


# --------------------------------------------------------------- helpers
def sieve(n: int) -> np.ndarray:
    """Boolean primality of 0..n-1 by the sieve of Eratosthenes."""
    is_p = np.ones(n, bool)
    is_p[:2] = False
    for i in range(2, int(n ** 0.5) + 1):
        if is_p[i]:
            is_p[i * i::i] = False
    return is_p


SMALL = np.nonzero(sieve(1 << 16))[0].astype(np.uint64)


def trial_division_prime(values: np.ndarray) -> np.ndarray:
    """Primality of values < 2^32 by trial division with every prime < 2^16."""
    v = np.asarray(values, dtype=np.uint64)
    res = v >= 2
    for p in SMALL:
        div = (v % p == 0) & (v != p)
        res &= ~div
    return res


def gf2_matrix_from_step(step, nbits: int) -> np.ndarray:
    """Columns are the images of the unit vectors under a GF(2)-linear step
    (state given and returned as an integer of nbits bits)."""
    m = np.zeros((nbits, nbits), np.int64)
    for i in range(nbits):
        img = step(1 << i)
        for r in range(nbits):
            m[r, i] = (img >> r) & 1
    return m


def gf2_pow(m: np.ndarray, e: int) -> np.ndarray:
    n = m.shape[0]
    r = np.eye(n, dtype=np.int64)
    b = m.copy()
    while e:
        if e & 1:
            r = (r @ b) & 1
        b = (b @ b) & 1
        e >>= 1
    return r


def full_period_gf2(m: np.ndarray, prime_factors) -> bool:
    """The map has period 2^n - 1 on nonzero states iff M^(2^n-1) = I and
    M^((2^n-1)/q) != I for every prime q dividing 2^n - 1."""
    n = m.shape[0]
    order = (1 << n) - 1
    assert math.prod(prime_factors) == order
    eye = np.eye(n, dtype=np.int64)
    if not np.array_equal(gf2_pow(m, order), eye):
        return False
    return all(not np.array_equal(gf2_pow(m, order // q), eye)
               for q in prime_factors)


# ---------------------------------------------------------- primality
def check_primality_exhaustive(limit=1 << 18):
    ref = sieve(limit)
    got = np.array([oracle.is_prime(n) for n in range(limit)])
    bad = np.nonzero(ref != got)[0]
    assert bad.size == 0, f"primality wrong at {bad[:10]}"


def check_primality_near_2_32_and_semiprimes():
    lo = M32 - (1 << 16)
    vals = np.arange(lo, M32, dtype=np.uint64)
    ref = trial_division_prime(vals)
    got = np.array([oracle.is_prime(int(v)) for v in vals])
    assert np.array_equal(ref, got)
    primes = vals[ref][-40:]
    for i in range(0, 40, 2):
        p, q = int(primes[i]), int(primes[i + 1])
        assert not oracle.is_prime(p * q), (p, q)


def check_strong_pseudoprime():
    # Composite by its factorisation (checked here), yet a strong probable
    # prime to every prime base up to 23: a Miller-Rabin with too few bases
    # accepts it.
    n = 3825123056546413051
    assert 149491 * 747451 * 34233211 == n
    assert not oracle.is_prime(n)


def check_mwc16_multiplier_count():
    m = oracle.multipliers(2000, 16)
    assert len(m) == PAPER["mwc16_multiplier_count"]["value"]


def check_mwc16_multipliers_brute_force():
    a = np.arange(1, 1 << 16, dtype=np.uint64)
    p = a * (1 << 16) - 1
    q = (p - 1) // 2
    ok = trial_division_prime(q) & trial_division_prime(p)
    expect = a[ok][::-1].astype(np.uint32)
    got = oracle.multipliers(2000, 16)
    assert np.array_equal(expect, got)


def test_primality_exhaustive():
    check_primality_exhaustive()


def test_primality_near_2_32_and_semiprimes():
    check_primality_near_2_32_and_semiprimes()


def test_strong_pseudoprime_rejected():
    check_strong_pseudoprime()


def test_mwc16_multiplier_count_is_papers_392():
    check_mwc16_multiplier_count()


def test_mwc16_multipliers_equal_brute_force():
    check_mwc16_multipliers_brute_force()


def test_multiplier_ranges_concatenate():
    full = oracle.multipliers(300, 32)
    hi = M32 - 1
    parts = []
    while sum(len(p) for p in parts) < 300:
        parts.append(oracle.multipliers_range(hi, hi - 50000 + 1, 32))
        hi -= 50000
    assert np.array_equal(np.concatenate(parts)[:300], full)


def test_multiplier_table_32_largest_first_and_valid():
    m = oracle.multipliers(64, 32).astype(np.int64)
    assert np.all(np.diff(m) < 0) and m[0] < M32
    # the gap above the first entry holds no valid multiplier
    for a in range(int(m[0]) + 1, M32):
        assert not oracle.is_safe_multiplier(a, 32)


def test_golden_multiplier_file_matches_oracle():
    path = GOLD / "multipliers_b32.json"
    if not path.exists():
        pytest.skip("golden multiplier file not generated")
    doc = json.loads(path.read_text())
    table = oracle.multipliers(4096, 32)
    h = hashlib.sha256(table.astype("<u4").tobytes()).hexdigest()
    assert h == doc["prefix"]["4096"]["sha256"]
    idx = np.array(doc["sample_index"])
    a = np.array(doc["sample_a"], dtype=np.int64)
    sel = idx < 4096
    assert np.array_equal(table[idx[sel]].astype(np.int64), a[sel])
    # the sampled entries beyond 4096 satisfy the condition and descend
    assert np.all(np.diff(a) < 0)
    for v in a[~sel][::97]:
        assert oracle.is_safe_multiplier(int(v), 32)


# ---------------------------------------------------------------- MWC
def check_mwc_lehmer_closed_form():
    """With p = a b - 1 and t_n = a x_n + c_n, t_{n+1} = b^-1 t_n mod p and
    the output x_{n+1} = t_n mod b (the MWC/Lehmer correspondence).  The
    closed form is computed with Python integers and pow(); the oracle steps
    Eq. 2-3 one at a time."""
    b = M32
    a_tab = oracle.multipliers(3, 32)
    for s, a in enumerate(a_tab):
        a = int(a)
        p = a * b - 1
        st = oracle.seed_streams(oracle.MWC, a_tab[s:s + 1], 42, np.array([s]))[0]
        t0 = a * int(st[0]) + int(st[1])
        assert 0 < t0 < p
        out, _ = oracle.stream(oracle.MWC, a, st, 2000, oracle.U32)
        for n in (0, 1, 2, 3, 10, 999, 1999):
            t_n = (pow(b, -n, p) * t0) % p
            assert int(out[n]) == t_n % b, (a, n)
        # a long jump: output 10^6 (computed by stepping the oracle)
        far, _ = oracle.stream(oracle.MWC, a, st, 10 ** 6, oracle.U32)
        n = 10 ** 6 - 1
        assert int(far[n]) == ((pow(b, -n, p) * t0) % p) % b


def check_mwc_period_base_2_16():
    """Brute-force period of the base-2^16 MWC equals (a b - 2)/2 for the
    smallest valid multipliers (order of b modulo the safe prime a b - 1)."""
    m16 = oracle.multipliers(2000, 16)
    for a in [int(v) for v in m16[-3:]]:
        expect = (a * (1 << 16) - 2) // 2
        assert oracle.mwc_period(a, 12345, 7, 16, 4 * expect) == expect, a


def check_mwc_fixed_points():
    a = int(oracle.multipliers(1, 32)[0])
    assert oracle.mwc_step(a, 0, 0) == (0, 0)
    assert oracle.mwc_step(a, M32 - 1, a - 1) == (M32 - 1, a - 1)


def test_mwc_lehmer_closed_form():
    check_mwc_lehmer_closed_form()


def test_mwc_period_base_2_16():
    check_mwc_period_base_2_16()


def test_mwc_fixed_points():
    check_mwc_fixed_points()


# ------------------------------------------------------------ xorshift32
def _xs32_matrix():
    return gf2_matrix_from_step(oracle.xorshift32_step, 32)


def check_xorshift32_full_period_gf2():
    assert full_period_gf2(_xs32_matrix(), [3, 5, 17, 257, 65537])


def check_xorshift32_brute_force_period():
    assert oracle.xorshift32_period(1) == PAPER["xorshift32_period"]["value"]


def test_xorshift32_full_period_gf2():
    check_xorshift32_full_period_gf2()


@pytest.mark.slow
def test_xorshift32_brute_force_period():
    check_xorshift32_brute_force_period()


# ---------------------------------------------------------------- LCG
def check_lcg_constants():
    g = PAPER["lcg_constants"]
    assert oracle.lcg_step(0) == g["c"]
    assert (oracle.lcg_step(1) - oracle.lcg_step(0)) % g["m"] == g["a"]
    rng = np.random.Generator(np.random.PCG64(3))
    for z in rng.integers(0, M32, 200):
        assert oracle.lcg_step(int(z)) == (g["a"] * int(z) + g["c"]) % g["m"]


def check_lcg_period():
    assert oracle.lcg_period(0) == M32


def test_lcg_constants_are_papers():
    check_lcg_constants()


@pytest.mark.slow
def test_lcg_full_period():
    check_lcg_period()


# -------------------------------------------------------------- xor128
def _xor128_as_int(v: int) -> int:
    st = [(v >> (32 * i)) & 0xFFFFFFFF for i in range(4)]
    _, new = oracle.xor128_step(st)
    return sum(int(w) << (32 * i) for i, w in enumerate(new))


F128 = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721]


def check_xor128_full_period_gf2():
    assert full_period_gf2(gf2_matrix_from_step(_xor128_as_int, 128), F128)


def check_xor128_output_is_new_last_word():
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(50):
        st = [int(v) for v in rng.integers(0, M32, 4)]
        out, new = oracle.xor128_step(st)
        assert out == new[3] and new[:3] == st[1:]


def test_xor128_full_period_gf2():
    check_xor128_full_period_gf2()


def test_xor128_output_and_shift_register():
    check_xor128_output_is_new_last_word()


def test_xor128_linear():
    rng = np.random.Generator(np.random.PCG64(6))
    for _ in range(50):
        u = int(rng.integers(0, 2**63)) | (int(rng.integers(0, 2**63)) << 64)
        v = int(rng.integers(0, 2**63)) | (int(rng.integers(0, 2**63)) << 64)
        assert _xor128_as_int(u ^ v) == _xor128_as_int(u) ^ _xor128_as_int(v)


# ---------------------------------------------------------------- KISS
def check_kiss_is_sum_of_parts():
    a = int(oracle.multipliers(1, 32)[0])
    st = [123456789, 1000, 362436069, 521288629]
    x, c, y, z = st
    cur = list(st)
    for _ in range(500):
        out, cur = oracle.kiss_step(a, cur)
        x, c = oracle.mwc_step(a, x, c)
        y = oracle.xorshift32_step(y)
        z = oracle.lcg_step(z)
        assert out == (x + y + z) % M32
        assert cur == [x, c, y, z]


def test_kiss_is_sum_of_parts():
    check_kiss_is_sum_of_parts()


# ---------------------------------------------------------------- FP32
def check_uniform_exact():
    rng = np.random.Generator(np.random.PCG64(8))
    us = list(rng.integers(0, M32, 2000)) + [0, 1, 255, 256, M32 - 1]
    for u in us:
        f = oracle.to_unit_f32(int(u))
        assert 0.0 <= f < 1.0
        assert f * 2 ** 24 == int(u) >> 8
    assert oracle.to_unit_f32(M32 - 1) == 1.0 - 2.0 ** -24


def test_uniform_exact_and_in_range():
    check_uniform_exact()


# ------------------------------------------------------------ splitmix64
def test_splitmix64_increment_is_golden_ratio():
    """The increment is the odd integer nearest 2^64 / phi."""
    z1, _ = oracle.splitmix64(0)
    x = (math.isqrt(5 << 128) - (1 << 64)) // 2  # floor(2^64 (sqrt5-1)/2)
    odd = x if x & 1 else x + 1
    assert z1 == odd


def test_splitmix64_published_first_output():
    _, r = oracle.splitmix64(0)
    assert r == 0xE220A8397B1DCDAF


# ------------------------------------------------------------- seeding
def test_seeding_invariants():
    n = 4096
    a = oracle.multipliers(n, 32)
    ids = np.arange(n)
    mwc = oracle.seed_streams(oracle.MWC, a, 42, ids)
    assert np.all(mwc[:, 1] < a)
    assert not np.any((mwc[:, 0] == 0) & (mwc[:, 1] == 0))
    assert not np.any((mwc[:, 0] == M32 - 1) & (mwc[:, 1] == a - 1))
    xs = oracle.seed_streams(oracle.XOR128, None, 7, ids)
    assert np.all(xs.any(axis=1))
    ks = oracle.seed_streams(oracle.KISS, a, 7, ids)
    assert np.all(ks[:, 2] != 0) and np.all(ks[:, 1] < a)


def test_seeding_draws_splitmix_from_seed_plus_stream():
    a = oracle.multipliers(16, 32)
    for s in range(16):
        _, r0 = oracle.splitmix64(42 + s)
        st = oracle.seed_streams(oracle.MWC, a[s:s + 1], 42, np.array([s]))[0]
        assert int(st[0]) == r0 & 0xFFFFFFFF
        assert int(st[1]) == (r0 >> 32) % int(a[s])


def test_generate_layout_is_stream_interleaved():
    n, k = 37, 19
    a = oracle.multipliers(n, 32)
    for kind in (oracle.MWC, oracle.XOR128, oracle.KISS):
        st = oracle.seed_streams(kind, a, 9, np.arange(n))
        out, st2 = oracle.generate(kind, a, st, k, oracle.U32)
        for s in range(n):
            col, fin = oracle.stream(kind, int(a[s]), st[s], k, oracle.U32)
            assert np.array_equal(out[:, s], col)
            assert np.array_equal(st2[s], fin)
        f, _ = oracle.generate(kind, a, st, k, oracle.F32)
        assert np.array_equal(f * np.float32(2 ** 24),
                              (out >> 8).astype(np.float32))
