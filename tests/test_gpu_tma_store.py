"""The TMA bulk-store path of the aligned generate kernel (launch hint 2):
outputs and state equal the oracle's, including a last CTA with few
streams, and nothing past the output is written."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1101_1846_gb300 import build, capi  # noqa: E402
from paper_1101_1846_gb300.generator import Generator  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


class tma_hint:
    """The shape (1, 256, hint) for calls of fewer than 2^21 streams (size
    class 0, which every call of this file is)."""

    def __init__(self, kind, fmt, hint):
        self.kind, self.fmt, self.hint = kind, fmt, hint
        self.saved = [ctypes.c_int() for _ in range(3)]

    def __enter__(self):
        capi.check(capi.lib().gbrng_get_launch_class(self.kind, self.fmt, 0,
                                                     *[ctypes.byref(v) for v in self.saved]))
        capi.check(capi.lib().gbrng_set_launch_class(self.kind, self.fmt, 0, 1, 256, self.hint))

    def __exit__(self, *exc):
        capi.check(capi.lib().gbrng_set_launch_class(self.kind, self.fmt, 0,
                                                     *[v.value for v in self.saved]))


@pytest.mark.parametrize("hint", [2])
@pytest.mark.parametrize("kind", range(6))
@pytest.mark.parametrize("fmt", [oracle.U32, oracle.F32])
@pytest.mark.parametrize("n,steps", [(8, 5), (1032, 64), (4096, 7), (1 << 16, 33)])
def test_tma_store_path_equals_oracle(hint, kind, fmt, n, steps):
    if kind in (oracle.MWC16X2, oracle.KISS_XOR) and n > capi.RNG_MAX_STREAMS_MWC16:
        pytest.skip("beyond the pair count")
    seed = 50 + n
    a = oracle.multipliers_for(kind, n)
    st = oracle.seed_streams(kind, a, seed, np.arange(n))
    g = Generator(kind, n, seed)
    out = torch.full((steps + 1, n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    with tma_hint(kind, fmt, hint):
        for call in range(2):
            g.generate(steps, fmt, out=out)
            got = out.cpu().numpy().view(np.uint32)
            exp, st = oracle.generate(kind, a, st, steps, fmt)
            assert np.array_equal(got[:steps], np.ascontiguousarray(exp).view(np.uint32)), call
            assert np.all(got[steps] == 0x5A5A5A5A)
    w = g.get_state().numpy().view(np.uint32).T
    assert np.array_equal(w, st[:, :w.shape[1]])
    g.close()
