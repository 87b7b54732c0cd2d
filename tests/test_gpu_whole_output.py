"""Every output element of the two large workloads against the oracle.

* xor128 and KISS at 2^20 streams x 1024 outputs, seeds 7 + s, uint32 and
  FP32: each call compared element by element.
* MWC, xor128 and KISS at 2^22 streams x 1024 outputs (16 GiB per call),
  seeds 42 + s: the 1st and the 10th call of a handle, state carried on the
  device through calls 2-9, compared element by element in both formats,
  and the state after the 10th call.

The oracle runs in host threads over blocks of 2^16 streams (its C calls
release the GIL), each thread carrying its block's state from call to call;
its multiplier table is its own search, checked against the stored digest
of the oracle's table before use."""
from __future__ import annotations

import hashlib
import json
import os
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1101_1846_gb300 import build, capi  # noqa: E402
from paper_1101_1846_gb300.generator import Generator  # noqa: E402

GOLD = json.loads((Path(__file__).resolve().parent / "golden" /
                   "multipliers_b32.json").read_text())
BLOCK = 1 << 16
STEPS = 1024
THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


@pytest.fixture(scope="module")
def table():
    """The oracle's first 2^22 multipliers (its own search, in spawned
    processes), checked against the stored digest."""
    a = oracle.multipliers(1 << 22, 32)
    assert hashlib.sha256(a.astype("<u4").tobytes()).hexdigest() == \
        GOLD["prefix"][str(1 << 22)]["sha256"]
    return a


def _host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().view(torch.int32).numpy().view(np.uint32)


class Blocks:
    """The oracle's state of every block of streams, advanced call by call."""

    def __init__(self, kind, a, n, seed):
        self.kind, self.n = kind, n
        self.a = None if kind == oracle.XOR128 else a
        self.ranges = [(s, min(s + BLOCK, n)) for s in range(0, n, BLOCK)]
        self.pool = ThreadPoolExecutor(THREADS)
        self.state = list(self.pool.map(
            lambda r: oracle.seed_streams(kind, self._a(r), seed, np.arange(*r)), self.ranges))

    def _a(self, r):
        return None if self.a is None else self.a[r[0]:r[1]]

    def compare(self, got: np.ndarray, fmt: int) -> list:
        """Blocks whose next call (from the current state, not advanced)
        differs from `got` in format fmt."""
        def one(i):
            r = self.ranges[i]
            exp, _ = oracle.generate(self.kind, self._a(r), self.state[i], STEPS, fmt)
            return None if np.array_equal(got[:, r[0]:r[1]], exp.view(np.uint32)) else r
        return [r for r in self.pool.map(one, range(len(self.ranges))) if r is not None]

    def advance(self, calls: int) -> None:
        def one(i):
            st = self.state[i]
            for _ in range(calls):
                _, st = oracle.generate(self.kind, self._a(self.ranges[i]), st, STEPS, oracle.U32)
            return st
        self.state = list(self.pool.map(one, range(len(self.ranges))))

    def words(self) -> np.ndarray:
        return np.concatenate(self.state)

    def close(self):
        self.pool.shutdown()


@pytest.mark.parametrize("kind", [oracle.XOR128, oracle.KISS])
def test_2p20x1024_every_element(kind, table):
    n = 1 << 20
    ref = Blocks(kind, table[:n], n, 7)
    try:
        for fmt in (oracle.U32, oracle.F32):
            with Generator(kind, n, 7) as g:
                got = _host(g.generate(STEPS, fmt))
            assert ref.compare(got, fmt) == [], (kind, fmt)
    finally:
        ref.close()


@pytest.mark.parametrize("kind", [oracle.MWC, oracle.XOR128, oracle.KISS])
def test_full_device_1st_and_10th_call_every_element(kind, table):
    """Handle A makes calls 1-10 as u32 x 9 then f32; handle B (same seed)
    f32 then u32 x 9.  Calls 1 and 10 of both are compared in full, and
    both handles' states after call 10."""
    n = 1 << 22
    ref = Blocks(kind, table, n, 42)
    out = torch.empty((STEPS, n), dtype=torch.int32, device="cuda")
    try:
        with Generator(kind, n, 42) as ga, Generator(kind, n, 42) as gb:
            ga.generate(STEPS, oracle.U32, out=out)
            assert ref.compare(_host(out), oracle.U32) == [], "call 1 u32"
            gb.generate(STEPS, oracle.F32, out=out)
            assert ref.compare(_host(out), oracle.F32) == [], "call 1 f32"
            for _ in range(8):
                ga.generate(STEPS, oracle.U32, out=out)
                gb.generate(STEPS, oracle.U32, out=out)
            ref.advance(9)
            ga.generate(STEPS, oracle.F32, out=out)
            assert ref.compare(_host(out), oracle.F32) == [], "call 10 f32"
            gb.generate(STEPS, oracle.U32, out=out)
            assert ref.compare(_host(out), oracle.U32) == [], "call 10 u32"
            ref.advance(1)
            exp = ref.words()
            for g in (ga, gb):
                st = g.get_state().numpy().view(np.uint32).T
                assert np.array_equal(st, exp[:, :st.shape[1]])
    finally:
        del out
        ref.close()
        torch.cuda.empty_cache()
