"""Pins for the oracle's battery counts (monobit, top-byte frequency,
serial pairs, birthday spacings) on synthetic outputs whose counts follow
from their construction, and sanity of the statistics on generator output.
Each check_* raises AssertionError when the oracle gets a count wrong;
test_oracle_mutants.py plants mistakes and expects one of them to fail."""
from __future__ import annotations

import math

import numpy as np

import oracle

M32 = 1 << 32


def _interleave(streams: list[np.ndarray]) -> np.ndarray:
    """Stream-interleaved block: column s is stream s's outputs."""
    return np.ascontiguousarray(np.stack(streams, axis=1).astype(np.uint32))


def check_ones_and_bytes():
    u = np.arange(1 << 16, dtype=np.uint32).reshape(-1, 4)
    c = oracle.battery_counts(u)
    assert c["ones"] == 16 * (1 << 15)  # each of 16 bits is one in half of 0..2^16-1
    assert c["bytes"][0] == 1 << 16 and c["bytes"][1:].sum() == 0  # all below 2^24
    top = (np.arange(256, dtype=np.uint64) << np.uint64(24)) | np.uint64(0xABCDE)
    u = np.tile(top.astype(np.uint32), 12).reshape(-1, 8)
    c = oracle.battery_counts(u)
    assert np.array_equal(c["bytes"], np.full(256, 12, np.uint64))
    assert c["ones"] == 12 * sum(bin(int(v)).count("1") for v in top)


def check_serial_pairs_within_streams():
    # stream 0 repeats the pair (1, 2), stream 1 the pair (3, 4), stream 2
    # walks every cell (a, b) once; an odd trailing output is unpaired
    k = 256
    s0 = np.tile(np.array([1, 2], np.uint64), k) << np.uint64(28)
    s1 = np.tile(np.array([3, 4], np.uint64), k) << np.uint64(28)
    cells = np.arange(256, dtype=np.uint64)
    s2 = np.stack([cells >> np.uint64(4), cells & np.uint64(15)], axis=1).ravel() << np.uint64(28)
    u = _interleave([s0 | 7, s1 | 99, s2 | 12345])
    u = np.vstack([u, np.full((1, 3), 0xF0000000, np.uint32)])
    hist = oracle.battery_counts(u)["serial"]
    expect = np.ones(256, np.uint64)
    expect[1 * 16 + 2] += k
    expect[3 * 16 + 4] += k
    assert np.array_equal(hist, expect)


def _birthday_sample(spacings: np.ndarray, rng) -> np.ndarray:
    """512 outputs whose top 24 bits are the birthdays with these spacings
    (first birthday = first spacing), in shuffled order, low byte noise."""
    b = np.cumsum(spacings.astype(np.uint64))
    assert b[-1] < (1 << 24)
    rng.shuffle(b)
    return ((b << np.uint64(8)) | rng.integers(0, 256, 512).astype(np.uint64)).astype(np.uint32)


def check_birthday_repeats():
    """Samples built from spacing lists with a known number of repeats: a
    list of 512 distinct spacings has none; replacing r of them by copies of
    other values (each copy a new repeat) gives r."""
    rng = np.random.Generator(np.random.PCG64(17))
    want = [0, 1, 2, 3, 5, 8, 14, 15, 40, 0, 2, 2]
    streams = []
    for r in want:
        sp = rng.permutation(np.arange(1, 513, dtype=np.int64))
        for i in range(r):
            sp[i] = sp[-1 - (i % 5)]  # copies of five values never replaced
        assert 512 - len(np.unique(sp)) == r
        streams.append(sp)
    # the 12 samples laid out as 4 streams x 3 blocks
    cols = []
    for s in range(4):
        cols.append(np.concatenate([_birthday_sample(streams[3 * s + b], rng) for b in range(3)]))
    u = _interleave(cols)
    u = np.vstack([u, np.zeros((100, 4), np.uint32)])  # a partial block is not a sample
    c = oracle.battery_counts(u)
    expect = np.zeros(16, np.uint64)
    for s in range(4):
        for b in range(3):
            expect[min(want[3 * s + b], 15)] += 1
    assert c["birthday_samples"] == 12
    assert np.array_equal(c["birthday"], expect)


def check_birthday_cap_and_order():
    """At most 4096 samples, taken block by block across the streams: with
    3000 streams of two blocks, the samples are block 0 of every stream and
    block 1 of streams 0..1095.  Each sample's repeat count encodes where it
    came from."""
    rng = np.random.Generator(np.random.PCG64(23))
    n = 3000
    base = rng.permutation(np.arange(1, 513, dtype=np.int64))

    def sample(r):
        sp = base.copy()
        for i in range(r):
            sp[i] = sp[-1 - (i % 5)]
        b = np.cumsum(sp.astype(np.uint64))
        return ((b << np.uint64(8)) | np.uint64(3)).astype(np.uint32)

    r_of = {(0, "lo"): 1, (1, "lo"): 2, (1, "hi"): 9}
    blk0 = sample(1)
    b1_lo, b1_hi = sample(2), sample(9)
    cols = [np.concatenate([blk0, b1_lo if s < 1096 else b1_hi]) for s in range(n)]
    c = oracle.battery_counts(_interleave(cols), birthday_max=4096)
    assert c["birthday_samples"] == 4096
    expect = np.zeros(16, np.uint64)
    expect[r_of[(0, "lo")]] = n
    expect[r_of[(1, "lo")]] = 4096 - n
    assert np.array_equal(c["birthday"], expect)


def _poisson_chi2_p(hist: np.ndarray, lam: float) -> float:
    n = int(hist.sum())
    probs = [math.exp(-lam) * lam ** k / math.factorial(k) for k in range(7)]
    probs.append(1 - sum(probs))
    obs = list(hist[:7].astype(float)) + [float(hist[7:].sum())]
    chi2 = sum((o - n * p) ** 2 / (n * p) for o, p in zip(obs, probs))
    # upper tail of chi-square with 7 degrees of freedom (odd dof series)
    x = chi2 / 2
    return math.erfc(math.sqrt(x)) + math.exp(-x) * sum(
        x ** (k + 0.5) / math.gamma(k + 1.5) for k in range(3))


def check_statistics_on_kiss_and_a_weyl_sequence():
    """KISS looks uniform to all four counts; the Weyl sequence j * 0x9E3779B9
    has perfect byte frequencies but fails the birthday spacings."""
    n, rows = 64, 512 * 32
    a = oracle.multipliers(n, 32)
    u, _ = oracle.generate(oracle.KISS, a, oracle.seed_streams(oracle.KISS, a, 5, np.arange(n)),
                           rows, oracle.U32)
    c = oracle.battery_counts(u)
    N = c["n_outputs"]
    assert abs(c["ones"] - 16 * N) < 6 * math.sqrt(8 * N)
    exp = N / 256
    chi_b = float((((c["bytes"].astype(float) - exp) ** 2) / exp).sum())
    assert 150 < chi_b < 380  # 255 degrees of freedom
    assert c["birthday_samples"] == n * 32
    assert _poisson_chi2_p(c["birthday"], 2.0) > 1e-4
    weyl = (np.arange(512 * 64, dtype=np.uint64) * np.uint64(0x9E3779B9)) % np.uint64(M32)
    w = oracle.battery_counts(weyl.astype(np.uint32).reshape(-1, 1))
    assert w["birthday"][15] == w["birthday_samples"]  # every sample: 15 or more repeats


def test_ones_and_bytes():
    check_ones_and_bytes()


def test_serial_pairs_within_streams():
    check_serial_pairs_within_streams()


def test_birthday_repeats():
    check_birthday_repeats()


def test_birthday_cap_and_order():
    check_birthday_cap_and_order()


def test_statistics_on_kiss_and_a_weyl_sequence():
    check_statistics_on_kiss_and_a_weyl_sequence()
