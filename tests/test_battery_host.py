"""Host-side statistics of the battery (no GPU): chi-square and normal
p-values formed from counts, checked against scipy's distributions and
against counts whose statistic is known."""
from __future__ import annotations

import math

import numpy as np
import pytest

pytest.importorskip("torch")
stats_mod = pytest.importorskip("scipy.stats")

from paper_1101_1846_gb300 import battery  # noqa: E402


def counts(ones, n, bytes_, serial, bday):
    return {"n_outputs": n, "ones": ones, "bytes": np.array(bytes_, np.uint64),
            "serial": np.array(serial, np.uint64), "birthday_samples": int(np.sum(bday)),
            "birthday": np.array(bday, np.uint64)}


def test_statistics_match_scipy():
    rng = np.random.Generator(np.random.PCG64(1))
    b = rng.multinomial(1 << 20, [1 / 256] * 256)
    s = rng.multinomial(1 << 19, [1 / 256] * 256)
    pois = rng.poisson(2.0, 4096)
    bday = np.bincount(np.minimum(pois, 15), minlength=16)
    n = 1 << 20
    ones = 16 * n + 1234
    st = battery.statistics(counts(ones, n, b, s, bday))
    chi_b, p_b = stats_mod.chisquare(b)
    assert st["frequency"]["chi2"] == pytest.approx(chi_b) and st["frequency"]["p"] == pytest.approx(p_b)
    chi_s, p_s = stats_mod.chisquare(s)
    assert st["serial"]["p"] == pytest.approx(p_s)
    z = 1234 / math.sqrt(8 * n)
    assert st["monobit"]["p"] == pytest.approx(2 * stats_mod.norm.sf(z))
    probs = list(battery.birthday_pmf()[:7])
    probs.append(1 - sum(probs))
    obs = list(bday[:7]) + [bday[7:].sum()]
    chi, p = stats_mod.chisquare(obs, np.array(probs) * sum(obs))
    assert st["birthday"]["p"] == pytest.approx(p)
    assert battery.passed(st)


def _repeat_counts(samples: int, seed: int) -> np.ndarray:
    """Marsaglia's statistic on days drawn by numpy's PCG64 (a generator of
    another family than any in this library): 512 days in 2^24, spacings =
    first day and neighbour differences, repeats among the sorted spacings."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = np.zeros(64, np.int64)
    for _ in range(samples // 4096):
        d = np.sort(rng.integers(0, 1 << 24, (4096, 512), dtype=np.int64), axis=1)
        sp = np.empty_like(d)
        sp[:, 0] = d[:, 0]
        sp[:, 1:] = np.diff(d, axis=1)
        sp.sort(axis=1)
        hist += np.bincount((sp[:, 1:] == sp[:, :-1]).sum(axis=1), minlength=64)[:64]
    return hist


def test_birthday_distribution_fits_an_independent_simulation():
    """The derived law of the repeat count (birthday_pmf) against 2^19 samples
    of another generator family: it fits, while Poisson(2), the asymptotic
    law, is rejected at this sample size; the simulated mean and variance
    agree with birthday_moments within four standard errors."""
    h = _repeat_counts(1 << 19, 2026)
    n = h.sum()
    mu, var = battery.birthday_moments()
    k = np.arange(64)
    m_sim = (k * h).sum() / n
    v_sim = (k * k * h).sum() / n - m_sim ** 2
    assert abs(m_sim - mu) < 4 * math.sqrt(var / n)
    assert abs(v_sim - var) < 4 * math.sqrt(2 * var * var / n)
    obs = list(h[:7]) + [h[7:].sum()]
    for probs, ok in ((battery.birthday_pmf(), True),
                      (np.array([stats_mod.poisson.pmf(k, 2.0) for k in range(64)]), False)):
        e = np.array(list(probs[:7]) + [1 - probs[:7].sum()]) * n
        _, p = stats_mod.chisquare(obs, e)
        assert (p > 1e-3) if ok else (p < 1e-6), (ok, p)


def test_too_perfect_and_too_skewed_fail():
    n = 256 * 1000
    flat = counts(16 * n, n, [1000] * 256, [500] * 256, [0] * 16)
    assert not battery.passed(battery.statistics(flat))  # p = 1: too good to be random
    skew = [1000] * 256
    skew[0] = 2000
    bad = counts(16 * n, n, skew, [500] * 256, [0] * 16)
    assert battery.statistics(bad)["frequency"]["p"] < 1e-6
