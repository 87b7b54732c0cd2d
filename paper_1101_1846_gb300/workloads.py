"""Seeded synthetic workloads.  This module holds none of the generators'
arithmetic: it only fixes sizes, seeds and the random draws that shape the
batched and serving workloads (numpy's PCG64), so that the CUDA path and the
oracle are driven by the same inputs.

The paper measures each generator on one large call (about 4e7 numbers per
call on its card, Sec. "Performance evaluation" and Tables I-III); the
workloads below scale that to a GB300 and add the batched and serving
shapes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MWC, XOR128, KISS = 0, 1, 2
U32, F32 = 0, 1
KIND_NAMES = {MWC: "mwc", XOR128: "xor128", KISS: "kiss"}
FMT_NAMES = {U32: "u32", F32: "f32"}


@dataclass(frozen=True)
class Plain:
    """One generator, one or more calls of n_per_stream outputs per stream."""
    name: str
    kinds: tuple
    n_streams: int
    n_per_stream: int
    seed: int
    fmts: tuple = (U32, F32)
    calls: int = 1


# MWC, 4096 streams x 4096 outputs, seeds 42 + s.
MWC_4K = Plain("mwc_4096x4096", (MWC,), 4096, 4096, 42, (U32,))
# xor128 and KISS, 2^20 streams x 1024 outputs, seeds 7 + s.
XOR_KISS_1M = Plain("xor128_kiss_2^20x1024", (XOR128, KISS), 1 << 20, 1024, 7)
# Full device: each kind at 2^22 streams x 1024 outputs per call (2^32 samples,
# 16 GiB per call), 10 calls with the state carried on the device.
FULL_4M = Plain("full_2^22x1024x10", (MWC, XOR128, KISS), 1 << 22, 1024, 42,
                (U32, F32), calls=10)


def sample_streams(n_streams: int, k: int, seed: int = 11) -> np.ndarray:
    """Sorted stream indices for sampled comparisons: both ends, the
    boundaries of 4-stream groups and 512-stream tiles, and random picks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    picks = {0, 1, 2, 3, n_streams - 1, n_streams - 2, n_streams - 3, n_streams - 4}
    for b in (4, 512, 4096):
        if n_streams > b:
            picks.update({b - 1, b, b + 1})
    picks.update(rng.choice(n_streams, size=min(k, n_streams), replace=False).tolist())
    return np.array(sorted(p for p in picks if 0 <= p < n_streams), dtype=np.int64)


# ------------------------------------------------------------- batched
@dataclass(frozen=True)
class Instance:
    kind: int
    n_streams: int
    n_per_stream: int
    fmt: int
    seed: int


def loguniform_int(rng: np.random.Generator, lo: int, hi: int, size: int) -> np.ndarray:
    """floor(lo * (hi/lo)^U), U uniform on [0, 1); values in [lo, hi)."""
    u = rng.random(size)
    return np.floor(lo * np.exp(u * np.log(hi / lo))).astype(np.int64)


def batched_instances(count: int = 10_000, seed: int = 1234, streams_range=(32, 65536),
                      steps_range=(16, 65536)) -> list[Instance]:
    """Uneven batched workload: kinds uniform over the three generators,
    stream counts log-uniform in [32, 65536], outputs per stream log-uniform
    in [16, 65536], uint32/FP32 drawn per instance, one seed per instance.
    Stream counts are not rounded, so about three quarters of the instances
    take the scalar-store path.  Smaller ranges give the same recipe scaled
    down (for tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = rng.integers(0, 3, count)
    streams = loguniform_int(rng, streams_range[0], streams_range[1], count)
    steps = loguniform_int(rng, steps_range[0], steps_range[1], count)
    fmts = rng.integers(0, 2, count)
    seeds = rng.integers(0, 2**63, count, dtype=np.int64)
    return [Instance(int(kinds[i]), int(streams[i]), int(steps[i]), int(fmts[i]),
                     int(seeds[i])) for i in range(count)]


def waves(instances: list[Instance], budget_bytes: int) -> list[list[int]]:
    """Splits instance indices, in order, into waves whose outputs fit in
    budget_bytes (an instance larger than the budget gets a wave alone)."""
    out, cur, used = [], [], 0
    for i, ins in enumerate(instances):
        b = 4 * ins.n_streams * ins.n_per_stream
        if cur and used + b > budget_bytes:
            out.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += b
    if cur:
        out.append(cur)
    return out


# ------------------------------------------------------------- serving
@dataclass(frozen=True)
class Request:
    t: float        # arrival time, seconds from the start
    client: int     # client id
    n_samples: int  # samples requested (bytes / 4)
    fmt: int


def request_log(rate_hz: float = 20_000.0, duration_s: float = 10.0,
                n_clients: int = 256, lo_bytes: int = 1024,
                hi_bytes: int = 256 << 20, seed: int = 5) -> list[Request]:
    """Poisson arrivals at rate_hz, clients uniform, sizes log-uniform on
    [lo_bytes, hi_bytes] rounded down to whole 4-byte samples, formats
    uniform over uint32/FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rate_hz * duration_s * 1.2) + 64
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    t = t[t < duration_s]
    m = len(t)
    clients = rng.integers(0, n_clients, m)
    sizes = loguniform_int(rng, lo_bytes, hi_bytes + 1, m) // 4
    fmts = rng.integers(0, 2, m)
    return [Request(float(t[i]), int(clients[i]), int(sizes[i]), int(fmts[i]))
            for i in range(m)]
