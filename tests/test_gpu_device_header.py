"""The public device header used from outside the library: a user kernel,
compiled here on its own against include/ only, steps a handle's streams
through gbrng::Engine (rng_get_device_view) and counts points of the quarter
disc; its counts and the state it leaves must equal the oracle's."""
from __future__ import annotations

import ctypes
import shutil
import subprocess
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

INCLUDE = Path(__file__).resolve().parents[1] / "include"

USER_CU = r'''
#include <cuda_runtime.h>
#include "gbrng_device.cuh"

template <int KIND>
__global__ void quarter_disc(rng_device_view v, unsigned steps, unsigned long long *hits)
{
    const unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (s >= v.n_streams)
        return;
    gbrng::Engine<KIND> e;
    e.load(v, s);
    unsigned long long inside = 0;
    for (unsigned j = 1; j < steps; j += 2) {
        const float x = e.next_f32(), y = e.next_f32();
        // exact in integers: x = X 2^-24, y = Y 2^-24
        const unsigned long long X = (unsigned long long)(x * 16777216.0f);
        const unsigned long long Y = (unsigned long long)(y * 16777216.0f);
        inside += (X * X + Y * Y) < (1ull << 48);
    }
    if (steps & 1)
        e.next();
    hits[s] = inside;
    e.store(v, s);
}

extern "C" int user_quarter_disc(const rng_device_view *v, unsigned steps, void *hits,
                                 void *stream)
{
    const unsigned threads = 128;
    const unsigned blocks = (unsigned)((v->n_streams + threads - 1) / threads);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long *h = static_cast<unsigned long long *>(hits);
    switch (v->kind) {
    case RNG_MWC32: quarter_disc<RNG_MWC32><<<blocks, threads, 0, st>>>(*v, steps, h); break;
    case RNG_XOR128: quarter_disc<RNG_XOR128><<<blocks, threads, 0, st>>>(*v, steps, h); break;
    case RNG_KISS: quarter_disc<RNG_KISS><<<blocks, threads, 0, st>>>(*v, steps, h); break;
    case RNG_MWC16X2: quarter_disc<RNG_MWC16X2><<<blocks, threads, 0, st>>>(*v, steps, h); break;
    case RNG_XORSHIFT8: quarter_disc<RNG_XORSHIFT8><<<blocks, threads, 0, st>>>(*v, steps, h); break;
    default: quarter_disc<RNG_KISS_XOR><<<blocks, threads, 0, st>>>(*v, steps, h); break;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
'''


@pytest.fixture(scope="module")
def user_lib(tmp_path_factory):
    build.build()
    capi.lib()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tmp_path_factory.mktemp("user_kernel")
    src, so = d / "user.cu", d / "libuser.so"
    src.write_text(USER_CU)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-I", str(INCLUDE), "-o", str(so),
                    str(src)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.user_quarter_disc.restype = ctypes.c_int
    lib.user_quarter_disc.argtypes = [ctypes.POINTER(capi.rng_device_view), ctypes.c_uint,
                                      ctypes.c_void_p, ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("kind", [oracle.MWC, oracle.XOR128, oracle.KISS, oracle.MWC16X2,
                                  oracle.XORSHIFT8, oracle.KISS_XOR])
def test_user_kernel_through_the_device_header(user_lib, kind):
    n, steps, seed = 777, 513, 31
    g = Generator(kind, n, seed)
    v = g.device_view()
    hits = torch.zeros(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    assert user_lib.user_quarter_disc(ctypes.byref(v), steps, ctypes.c_void_p(hits.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream)) == 0
    torch.cuda.synchronize()
    a = oracle.multipliers_for(kind, n)
    st = oracle.seed_streams(kind, a, seed, np.arange(n))
    exp, st = oracle.reduce(kind, a, st, steps, oracle.DISC)
    assert np.array_equal(hits.cpu().numpy().view(np.uint64), exp)
    # the user kernel's state write-back is the library's state: the next
    # library call continues the sequence
    out = g.generate(4).cpu().view(torch.int32).numpy().view(np.uint32)
    nxt, _ = oracle.generate(kind, a, st, 4, oracle.U32)
    assert np.array_equal(out, nxt)
    g.close()
