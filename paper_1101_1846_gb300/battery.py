"""A small statistical battery over generator outputs: the device counts four
tests of the DIEHARD / TestU01 families (rng_battery), and this module forms
the statistics and p-values from the counts.  The paper assesses its
generators with DIEHARD and TestU01 (Sec. "Performance evaluation"); those
suites are not part of this library, so this is a smoke test of the same
kind, not a replacement.

  monobit    z = (ones - 16 N) / sqrt(8 N), two-sided normal p-value
  frequency  chi-square of the 256 top-byte bins, 255 degrees of freedom
  serial     chi-square of the 256 pair cells, 255 degrees of freedom
  birthday   chi-square of the samples' repeat counts against their
             distribution at m = 512 days in a year of n = 2^24 (birthday_pmf),
             bins 0..6 and >= 7, 7 degrees of freedom
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import capi
from .generator import Generator

BIRTHDAY_DAYS, BIRTHDAY_YEAR = 512, 1 << 24


def birthday_moments(m: int = BIRTHDAY_DAYS, n: int = BIRTHDAY_YEAR) -> tuple[float, float]:
    """Mean and variance of the repeat count R of m birthdays in a year of n
    days (m spacings: the first day and the neighbour differences).

    The m spacings behave as m of the m + 1 exchangeable gaps of m uniform
    points in [0, n) (Dirichlet(1, ..., 1) scaled by n): two given gaps are
    equal with probability p = m / (2n) (the density of their difference at
    0), three with q3 = m (m - 1) / (3 n^2), and two disjoint pairs both
    equal with m (m - 1) / (4 n^2), slightly less than p^2.  With P2 and P3
    the numbers of equal pairs and triples, R = P2 - P3 + ... (a value
    shared by k spacings adds k - 1 = C(k,2) - C(k,3) + ... to R), so
        E[R]   = C(m,2) p - C(m,3) q3,
        Var[R] = Var[P2] - 2 Cov[P2, P3] + Var[P3],  Cov[P2, P3] = 3 E[P3],
    with Var[P2] summed over pairs of pairs: equal, sharing one spacing, or
    disjoint.  At m = 512, n = 2^24: E[R] = 1.98920, Var[R] = 1.96417, where
    the Poisson limit m^3 / (4n) = 2 has both equal to 2."""
    p = m / (2 * n)
    q3 = m * (m - 1) / (3 * n * n)
    pairs = math.comb(m, 2)
    e2 = pairs * p
    e3 = math.comb(m, 3) * q3
    var2 = (pairs * p * (1 - p) + m * (m - 1) * (m - 2) * (q3 - p * p)
            + pairs * math.comb(m - 2, 2) * (m * (m - 1) / (4 * n * n) - p * p))
    return e2 - e3, var2 - 2 * 3 * e3 + e3


def birthday_pmf(kmax: int = 64, m: int = BIRTHDAY_DAYS, n: int = BIRTHDAY_YEAR) -> np.ndarray:
    """P(R = k), k < kmax: the Poisson law of R's mean with the second-order
    Charlier term that carries R's variance (the factorial cumulant
    d = Var[R] - E[R], here -0.025):
        P(k) = pi(k) + (d / 2) (pi(k) - 2 pi(k - 1) + pi(k - 2)),
    pi the Poisson(E[R]) probabilities.  (An independent simulation of 2^26
    samples with numpy's PCG64 fits it: chi-square 7.5 on 7 degrees of
    freedom; Poisson(2) scores 8825.)"""
    mu, var = birthday_moments(m, n)
    d = var - mu
    pi = np.array([math.exp(-mu) * mu ** k / math.factorial(k) for k in range(kmax)])
    pi1 = np.concatenate([[0.0], pi[:-1]])
    pi2 = np.concatenate([[0.0, 0.0], pi[:-2]])
    return pi + d / 2 * (pi - 2 * pi1 + pi2)


def counts(u: torch.Tensor, n_streams: int, n_per_stream: int,
           stream: torch.cuda.Stream | None = None) -> dict:
    """Battery counts of a device tensor of n_per_stream x n_streams outputs
    (rng_generate's layout).  Synchronises `stream`."""
    assert u.is_cuda and u.is_contiguous() and u.element_size() == 4
    assert u.numel() >= n_streams * n_per_stream
    s = stream if stream is not None else torch.cuda.current_stream()
    c = capi.rng_battery_counts()
    capi.check(capi.lib().rng_battery(ctypes.c_void_p(u.data_ptr()), n_streams, n_per_stream,
                                      ctypes.byref(c), ctypes.c_void_p(s.cuda_stream)),
               "rng_battery")
    return {"n_outputs": int(c.n_outputs), "ones": int(c.ones),
            "bytes": np.array(c.bytes[:], dtype=np.uint64),
            "serial": np.array(c.serial[:], dtype=np.uint64),
            "birthday_samples": int(c.birthday_samples),
            "birthday": np.array(c.birthday[:], dtype=np.uint64)}


def _chi2_sf(x: float, dof: int) -> float:
    from scipy.special import gammaincc
    return float(gammaincc(dof / 2.0, x / 2.0))


def _uniform_chi2(hist: np.ndarray) -> tuple[float, float]:
    h = hist.astype(np.float64)
    n = h.sum()
    if n == 0:
        return float("nan"), float("nan")
    e = n / len(h)
    chi2 = float(((h - e) ** 2 / e).sum())
    return chi2, _chi2_sf(chi2, len(h) - 1)


def statistics(c: dict) -> dict:
    """Statistics and p-values from battery counts."""
    out = {}
    N = c["n_outputs"]
    if N:
        z = (c["ones"] - 16.0 * N) / math.sqrt(8.0 * N)
        out["monobit"] = {"z": z, "p": math.erfc(abs(z) / math.sqrt(2.0))}
    chi2, p = _uniform_chi2(c["bytes"])
    out["frequency"] = {"chi2": chi2, "dof": 255, "p": p}
    chi2, p = _uniform_chi2(c["serial"])
    out["serial"] = {"chi2": chi2, "dof": 255, "p": p}
    m = c["birthday_samples"]
    if m:
        pmf = birthday_pmf()
        probs = list(pmf[:7])
        probs.append(1.0 - sum(probs))
        h = c["birthday"].astype(np.float64)
        obs = np.concatenate([h[:7], [h[7:].sum()]])
        exp = m * np.array(probs)
        chi2 = float(((obs - exp) ** 2 / exp).sum())
        mean = float((np.arange(16) * h).sum() / m)
        out["birthday"] = {"chi2": chi2, "dof": 7, "p": _chi2_sf(chi2, 7), "samples": m,
                           "mean_repeats": mean}
    return out


def run(kind: int, n_streams: int, n_per_stream: int, seed: int,
        generator: Generator | None = None) -> dict:
    """Generates n_per_stream uint32 outputs of n_streams streams on the
    device and returns the battery's statistics (the tests read the raw 32
    bits, so the FP32 format is not a meaningful input)."""
    g = generator if generator is not None else Generator(kind, n_streams, seed)
    u = g.generate(n_per_stream, capi.RNG_U32)
    res = statistics(counts(u, g.n_streams, n_per_stream))
    if generator is None:
        g.close()
    return res


def passed(stats: dict, alpha: float = 1e-6) -> bool:
    """No p-value below alpha or above 1 - alpha."""
    ps = [v["p"] for v in stats.values() if "p" in v and not math.isnan(v["p"])]
    return all(alpha < p < 1 - alpha for p in ps)
