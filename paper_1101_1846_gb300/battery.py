"""A small statistical battery over generator outputs: the device counts four
tests of the DIEHARD / TestU01 families (rng_battery), and this module forms
the statistics and p-values from the counts.  The paper assesses its
generators with DIEHARD and TestU01 (Sec. "Performance evaluation"); those
suites are not part of this library, so this is a smoke test of the same
kind, not a replacement.

  monobit    z = (ones - 16 N) / sqrt(8 N), two-sided normal p-value
  frequency  chi-square of the 256 top-byte bins, 255 degrees of freedom
  serial     chi-square of the 256 pair cells, 255 degrees of freedom
  birthday   chi-square of the samples' repeat counts against Poisson(2),
             bins 0..6 and >= 7, 7 degrees of freedom
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import capi
from .generator import Generator

BIRTHDAY_MEAN = 512 ** 3 / (4 * 2 ** 24)  # = 2


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
        lam = BIRTHDAY_MEAN
        probs = [math.exp(-lam) * lam ** k / math.factorial(k) for k in range(7)]
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
