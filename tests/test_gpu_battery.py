"""The battery's counts on the device (rng_battery) against the oracle's on
the same outputs, and the statistics of every generator kind."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import test_oracle_battery as tob  # noqa: E402
from paper_1101_1846_gb300 import battery, build, capi  # noqa: E402
from paper_1101_1846_gb300.generator import Generator  # noqa: E402

ALL = [oracle.MWC, oracle.XOR128, oracle.KISS, oracle.MWC16X2, oracle.XORSHIFT8,
       oracle.KISS_XOR]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


def device_counts(u: np.ndarray) -> dict:
    rows, n = u.shape
    t = torch.from_numpy(np.ascontiguousarray(u).view(np.int32)).cuda()
    return battery.counts(t, n, rows)


def same(a: dict, b: dict):
    assert a["n_outputs"] == b["n_outputs"] and a["ones"] == b["ones"]
    assert a["birthday_samples"] == b["birthday_samples"]
    for k in ("bytes", "serial", "birthday"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("kind", ALL)
@pytest.mark.parametrize("n,rows", [(300, 1537), (1024, 1024), (7, 2049), (3000, 1024)])
def test_counts_equal_oracle_on_oracle_outputs(kind, n, rows):
    a = oracle.multipliers_for(kind, n)
    st = oracle.seed_streams(kind, a, 77 + n, np.arange(n))
    u, _ = oracle.generate(kind, a, st, rows, oracle.U32)
    c = device_counts(u)
    same(c, oracle.battery_counts(u))
    assert c["birthday_samples"] == min((rows // 512) * n, capi.RNG_BATTERY_BIRTHDAY_MAX)


def test_counts_of_designed_samples():
    rng = np.random.Generator(np.random.PCG64(3))
    cols = []
    want = []
    for s in range(6):
        blocks = []
        for b in range(2):
            r = int(rng.integers(0, 20))
            sp = rng.permutation(np.arange(1, 513, dtype=np.int64))
            for i in range(r):
                sp[i] = sp[-1 - (i % 5)]
            want.append(min(r, 15))
            blocks.append(tob._birthday_sample(sp, rng))
        cols.append(np.concatenate(blocks))
    u = tob._interleave(cols)
    c = device_counts(u)
    expect = np.zeros(16, np.uint64)
    for r in want:
        expect[r] += 1
    assert np.array_equal(c["birthday"], expect)
    same(c, oracle.battery_counts(u))


def test_counts_many_rows_one_stream():
    # more than 65535 x 64 row pairs: the count kernel widens its row tiles
    rows = 2 * 65535 * 64 + 1001
    rng = np.random.Generator(np.random.PCG64(5))
    u = rng.integers(0, 1 << 32, size=(rows, 1), dtype=np.uint64).astype(np.uint32)
    same(device_counts(u), oracle.battery_counts(u))


def test_rejects_bad_arguments():
    c = capi.rng_battery_counts()
    with pytest.raises(capi.RngError):
        capi.check(capi.lib().rng_battery(None, 4, 4, c, None))
    t = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.RngError):
        capi.check(capi.lib().rng_battery(t.data_ptr(), 0, 4, c, None))


@pytest.mark.parametrize("kind", ALL)
def test_every_kind_passes_the_battery(kind):
    """2^21 birthday samples per kind (2^20 streams x 1024 outputs; the pair
    kinds 76,636 x 16,384), compared with the repeat count's law at 512 days
    in 2^24, not its Poisson limit."""
    n, rows = ((1 << 20, 1024) if kind not in (oracle.MWC16X2, oracle.KISS_XOR)
               else (capi.RNG_MAX_STREAMS_MWC16, 16384))
    stats = battery.run(kind, n, rows, 2024)
    assert stats["birthday"]["samples"] == capi.RNG_BATTERY_BIRTHDAY_MAX
    assert battery.passed(stats), stats
    mu, var = battery.birthday_moments()
    se = (var / stats["birthday"]["samples"]) ** 0.5
    assert abs(stats["birthday"]["mean_repeats"] - mu) < 6 * se


def test_birthday_samples_stop_at_the_cap():
    n, rows = (1 << 20) + 8, 1024  # 2^21 + 16 samples available
    with Generator(oracle.XOR128, n, 5) as g:
        u = g.generate(rows)
        c = battery.counts(u, n, rows)
    assert c["birthday_samples"] == capi.RNG_BATTERY_BIRTHDAY_MAX
    assert int(c["birthday"].sum()) == capi.RNG_BATTERY_BIRTHDAY_MAX


def test_a_bad_sequence_fails():
    # a Weyl sequence: perfect byte frequencies, hopeless birthday spacings
    j = np.arange(512 * 256, dtype=np.uint64)
    u = ((j * np.uint64(0x9E3779B9)) % np.uint64(1 << 32)).astype(np.uint32).reshape(-1, 1)
    stats = battery.statistics(device_counts(u))
    assert stats["birthday"]["p"] < 1e-12 and not battery.passed(stats)
