"""The allocation-free batched launch (rng_generate_batch_noalloc) gives the
same outputs and state as rng_generate_batch, on two calls in a row.

It serves callers that cannot allocate device memory when they need samples
(a pool allocator that owns the device budget, or a loop that must not be
synchronised by cudaMalloc/cudaFree).  This file is named so that pytest
collects it last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1101_1846_gb300 import build, capi  # noqa: E402
from paper_1101_1846_gb300.generator import Generator  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


def _instances(count=48, seed=2024):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        kind = int(rng.integers(0, 3))
        n = int(np.floor(np.exp(rng.random() * np.log(4000.0))))  # 1 .. 3999 streams
        steps = int(rng.integers(1, 200))
        fmt = int(rng.integers(0, 2))
        out.append((kind, n, steps, fmt, 500 + i))
    return out


def _twin(instances):
    gens, outs = [], []
    for i, (kind, n, steps, _fmt, seed) in enumerate(instances):
        gens.append(Generator(kind, n, seed))
        extra = 1 if i % 5 == 2 else 0  # some outputs only 4-byte aligned
        buf = torch.zeros(n * steps + extra, dtype=torch.int32, device="cuda")
        outs.append(buf[extra:])
    return gens, outs


def _items(instances, gens, outs):
    arr = (capi.rng_batch_item * len(instances))()
    for k, ((_, _, steps, fmt, _), g, o) in enumerate(zip(instances, gens, outs)):
        arr[k].h = g.h
        arr[k].n_per_stream = steps
        arr[k].out = o.data_ptr()
        arr[k].fmt = fmt
    return arr


def test_noalloc_batch_equals_batch_on_two_calls():
    ins = _instances()
    ga, oa = _twin(ins)
    gb, ob = _twin(ins)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    L = capi.lib()
    for call in range(2):
        assert L.rng_generate_batch(_items(ins, ga, oa), len(ins), sp) == capi.RNG_OK
        assert L.rng_generate_batch_noalloc(_items(ins, gb, ob), len(ins), sp) == capi.RNG_OK
        torch.cuda.synchronize()
        for k in range(len(ins)):
            assert torch.equal(oa[k], ob[k]), (call, k)
            assert torch.equal(ga[k].get_state(), gb[k].get_state()), (call, k)


def test_noalloc_batch_allocates_no_device_memory():
    """After a first call (which loads the kernel and looks up the scratch
    address), further calls leave the device's free memory and torch's
    allocator exactly as they were."""
    ins = _instances(count=24, seed=99)
    gens, outs = _twin(ins)
    arr = _items(ins, gens, outs)
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = capi.lib()
    assert L.rng_generate_batch_noalloc(arr, len(ins), sp) == capi.RNG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert L.rng_generate_batch_noalloc(arr, len(ins), sp) == capi.RNG_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_batch_rejects_work_beyond_its_capacity():
    g = Generator(capi.RNG_XOR128, 1 << 25, 9)  # 65536 tiles of 512 streams
    out = torch.zeros(1 << 25, dtype=torch.int32, device="cuda")
    before = g.get_state()
    arr = (capi.rng_batch_item * 1)()
    arr[0].h, arr[0].n_per_stream, arr[0].out, arr[0].fmt = g.h, 1, out.data_ptr(), 0
    st = capi.lib().rng_generate_batch_noalloc(
        arr, 1, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == capi.RNG_ERR_ARG
    torch.cuda.synchronize()
    assert torch.equal(g.get_state(), before)
    assert int(out.abs().sum()) == 0
