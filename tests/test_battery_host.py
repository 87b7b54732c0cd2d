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
    lam = 2.0
    probs = [stats_mod.poisson.pmf(k, lam) for k in range(7)]
    probs.append(1 - sum(probs))
    obs = list(bday[:7]) + [bday[7:].sum()]
    chi, p = stats_mod.chisquare(obs, np.array(probs) * sum(obs))
    assert st["birthday"]["p"] == pytest.approx(p)
    assert battery.passed(st)


def test_too_perfect_and_too_skewed_fail():
    n = 256 * 1000
    flat = counts(16 * n, n, [1000] * 256, [500] * 256, [0] * 16)
    assert not battery.passed(battery.statistics(flat))  # p = 1: too good to be random
    skew = [1000] * 256
    skew[0] = 2000
    bad = counts(16 * n, n, skew, [500] * 256, [0] * 16)
    assert battery.statistics(bad)["frequency"]["p"] < 1e-6
