"""Parity of the CUDA path (through the C-ABI) with the oracle: bit-exact for
uint32 and for the FP32 uniforms, which are exact by construction."""
from __future__ import annotations

import ctypes
import functools
import hashlib
import json
from pathlib import Path

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1101_1846_gb300 import autotune, build, capi, workloads  # noqa: E402
from paper_1101_1846_gb300.generator import (BatchItem, Generator, Plan,  # noqa: E402
                                             generate_batch, multipliers)

GOLD = json.loads((Path(__file__).resolve().parent / "golden" /
                   "multipliers_b32.json").read_text())
KINDS = [oracle.MWC, oracle.XOR128, oracle.KISS]
FMTS = [oracle.U32, oracle.F32]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


@functools.lru_cache(maxsize=1)
def _oracle_table(k=16384):
    return oracle.multipliers(k, 32)


def oracle_a(n: int) -> np.ndarray:
    assert n <= 16384
    return _oracle_table()[:n]


def golden_a(idx: np.ndarray) -> np.ndarray:
    lookup = dict(zip(GOLD["sample_index"], GOLD["sample_a"]))
    return np.array([lookup[int(i)] for i in idx], dtype=np.uint32)


def golden_streams(n: int) -> np.ndarray:
    idx = np.array(GOLD["sample_index"], dtype=np.int64)
    return idx[idx < n]


def bits(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().contiguous().view(torch.int32).numpy().view(np.uint32)


def obits(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a).view(np.uint32)


def expect_full(kind, n, seed, steps, fmt, state=None):
    a = oracle_a(n) if kind != oracle.XOR128 else None
    st = oracle.seed_streams(kind, a, seed, np.arange(n)) if state is None else state
    return oracle.generate(kind, a, st, steps, fmt)


# ------------------------------------------------------------ multipliers
def test_multiplier_table_equals_oracle():
    gpu = bits(multipliers(4096))
    assert np.array_equal(gpu, oracle_a(4096))


@pytest.mark.parametrize("k", [1 << 20, 1 << 22])
def test_multiplier_table_digest_equals_oracle(k):
    gpu = bits(multipliers(k)).astype("<u4")
    assert hashlib.sha256(gpu.tobytes()).hexdigest() == GOLD["prefix"][str(k)]["sha256"]
    idx = np.array(GOLD["sample_index"])
    assert np.array_equal(gpu[idx[idx < k]], golden_a(idx[idx < k]))


# ------------------------------------------------- small sizes, full compare
SIZES = [(1, 9), (3, 33), (4, 7), (5, 1), (31, 16), (32, 5), (100, 33), (1000, 9),
         (4096, 3), (4100, 17), (5003, 8), (16384, 2)]


@pytest.mark.parametrize("n,steps", SIZES)
@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("kind", KINDS)
def test_full_parity_small(kind, fmt, n, steps):
    seed = 99991 + n
    g = Generator(kind, n, seed)
    out = g.generate(steps, fmt)
    torch.cuda.synchronize()
    exp, st = expect_full(kind, n, seed, steps, fmt)
    assert np.array_equal(bits(out), obits(exp))
    got_state = bits(g.get_state())
    assert np.array_equal(got_state, st[:, :g.words].T)


@pytest.mark.parametrize("kind", KINDS)
def test_state_carries_across_calls(kind):
    n, seed = 1028, 5
    g = Generator(kind, n, seed)
    parts = [g.generate(k, oracle.U32) for k in (5, 17, 1, 40)]
    torch.cuda.synchronize()
    got = np.concatenate([bits(p) for p in parts])
    exp, _ = expect_full(kind, n, seed, 63, oracle.U32)
    assert np.array_equal(got, obits(exp))


@pytest.mark.parametrize("kind", KINDS)
def test_unaligned_output_same_result(kind):
    n, steps, seed = 512, 12, 77
    buf = torch.zeros(n * steps + 1, dtype=torch.int32, device="cuda")
    view = buf[1:]  # 4-byte aligned, not 16-byte aligned: scalar-store kernel
    g = Generator(kind, n, seed)
    g.generate(steps, oracle.U32, out=view)
    torch.cuda.synchronize()
    exp, _ = expect_full(kind, n, seed, steps, oracle.U32)
    assert np.array_equal(bits(view).reshape(steps, n), obits(exp))
    assert int(buf[0]) == 0


@pytest.mark.parametrize("offset", [0, 1, 2, 3, 4, 6])
@pytest.mark.parametrize("n,steps", [(5, 13), (130, 7), (517, 9), (4099, 5), (1024, 6),
                                     (2052, 11), (6000, 10)])
@pytest.mark.parametrize("kind", KINDS)
def test_rows_at_every_alignment(kind, n, steps, offset):
    """Rows start at every word offset mod 8 (odd stream counts, outputs
    shifted by 0-6 words): the sector-aligned, the barrier and the realigned
    kernels, the edge lanes' 4-byte stores and the tail streams all land
    where the layout says."""
    seed = 4242 + n
    fmt = oracle.F32 if (n + offset) % 2 else oracle.U32
    buf = torch.full((n * steps + 8,), -7, dtype=torch.int32, device="cuda")
    view = buf[offset:offset + n * steps]
    g = Generator(kind, n, seed)
    g.generate(steps, fmt, out=view)
    torch.cuda.synchronize()
    exp, st = expect_full(kind, n, seed, steps, fmt)
    assert np.array_equal(bits(view).reshape(steps, n), obits(exp))
    rest = torch.cat([buf[:offset], buf[offset + n * steps:]])
    assert torch.all(rest == -7)  # nothing written outside the output
    assert np.array_equal(bits(g.get_state()), st[:, :g.words].T)


@pytest.mark.parametrize("kind", KINDS)
def test_generate_range_advances_only_its_streams(kind):
    """rng_generate_range on [s0, s1) with a row stride and an offset, then a
    full call: streams in the range are ahead by the range's steps."""
    n, seed = 1003, 91
    g = Generator(kind, n, seed)
    a = oracle_a(n) if kind != oracle.XOR128 else None
    st = oracle.seed_streams(kind, a, seed, np.arange(n))
    for (s0, s1, k, ld, off) in [(5, 262, 7, 300, 1), (0, 1003, 3, 1003, 0),
                                 (512, 1000, 4, 491, 2), (999, 1003, 9, 4, 3)]:
        buf = torch.full((off + (k - 1) * ld + (s1 - s0) + 5,), -9, dtype=torch.int32,
                         device="cuda")
        g.generate_range(s0, s1, k, buf, ld, oracle.U32, offset=off)
        torch.cuda.synchronize()
        exp, st_sub = oracle.generate(kind, a[s0:s1] if a is not None else None,
                                      st[s0:s1], k, oracle.U32)
        st[s0:s1] = st_sub
        got = bits(buf)
        for j in range(k):
            row = got[off + j * ld: off + j * ld + (s1 - s0)]
            assert np.array_equal(row, obits(exp[j])), (s0, s1, j)
        written = np.zeros(len(got), bool)
        for j in range(k):
            written[off + j * ld: off + j * ld + (s1 - s0)] = True
        assert np.all(got[~written] == np.uint32(2**32 - 9))
    out = g.generate(5, oracle.F32)
    torch.cuda.synchronize()
    exp, st = oracle.generate(kind, a, st, 5, oracle.F32)
    assert np.array_equal(bits(out), obits(exp))
    assert np.array_equal(bits(g.get_state()), st[:, :g.words].T)


def test_batch_disjoint_ranges_of_one_handle():
    """Several items of the same generator with disjoint stream ranges in one
    plan equal the same range calls made one after another."""
    n, seed = 2050, 17
    ranges = [(0, 700, 33), (700, 701, 5), (701, 1500, 12), (1503, 2050, 40)]
    gb, gp = Generator(oracle.KISS, n, seed), Generator(oracle.KISS, n, seed)
    ob = [torch.zeros(k * (e - b), dtype=torch.int32, device="cuda") for b, e, k in ranges]
    op = [torch.zeros_like(o) for o in ob]
    plan = Plan([BatchItem(gb, k, o, oracle.F32, s_begin=b, s_end=e, ld=e - b)
                 for (b, e, k), o in zip(ranges, ob)])
    plan.launch()
    for (b, e, k), o in zip(ranges, op):
        gp.generate_range(b, e, k, o, e - b, oracle.F32)
    torch.cuda.synchronize()
    for x, y in zip(ob, op):
        assert torch.equal(x, y)
    assert torch.equal(gb.get_state(), gp.get_state())
    plan.close()
    bad = [BatchItem(gb, 2, ob[0], 0, s_begin=0, s_end=700, ld=700),
           BatchItem(gb, 2, ob[1], 0, s_begin=699, s_end=701, ld=2)]
    with pytest.raises(capi.RngError):
        Plan(bad)


def test_launch_shapes_do_not_change_outputs():
    """Shapes of the small-call class (fewer than 2^21 streams, which n is)."""
    n, steps, seed = 4096, 21, 3
    exp = {k: expect_full(k, n, seed, steps, oracle.F32)[0] for k in KINDS}
    L = capi.lib()
    saved = {}
    for k in KINDS:
        vals = [ctypes.c_int() for _ in range(3)]
        capi.check(L.gbrng_get_launch_class(k, oracle.F32, 0, *[ctypes.byref(x) for x in vals]))
        saved[k] = [x.value for x in vals]
    for v, block, hint in [(1, 64, 0), (2, 128, 1), (2, 512, 0), (1, 512, 1), (2, 32, 0)]:
        for k in KINDS:
            capi.check(L.gbrng_set_launch_class(k, oracle.F32, 0, v, block, hint))
            out = Generator(k, n, seed).generate(steps, oracle.F32)
            torch.cuda.synchronize()
            assert np.array_equal(bits(out), obits(exp[k])), (k, v, block, hint)
    for k in KINDS:
        capi.check(L.gbrng_set_launch_class(k, oracle.F32, 0, *saved[k]))


def test_row_ctas_do_not_change_outputs():
    """The barrier-synced kernels (16-byte rows: n % 8 == 4; realigned rows:
    odd n) with one CTA of 512 threads per SM (a shared-memory reservation)
    and with as many as fit, at sizes that fill the GPU: the two outputs are
    identical, and sampled streams equal the oracle."""
    L = capi.lib()
    steps, seed = 8, 5
    for n, realigned in (((1 << 20) + 4, 0), ((1 << 20) + 3, 1)):
        for k in KINDS:
            idx = np.array(sorted(i for i in golden_streams(n).tolist() if i < (1 << 20)))
            a = golden_a(idx) if k != oracle.XOR128 else None
            st = oracle.seed_streams(k, a, seed, idx)
            for f in FMTS:
                exp, _ = oracle.generate(k, a, st, steps, f)
                v = ctypes.c_int()
                capi.check(L.gbrng_get_row_ctas(k, f, realigned, ctypes.byref(v)))
                outs = []
                for ctas in (0, 1):
                    capi.check(L.gbrng_set_row_ctas(k, f, realigned, ctas))
                    outs.append(Generator(k, n, seed).generate(steps, f))
                    torch.cuda.synchronize()
                capi.check(L.gbrng_set_row_ctas(k, f, realigned, v.value))
                assert torch.equal(outs[0].view(torch.int32), outs[1].view(torch.int32)), (n, k, f)
                got = bits(outs[1].index_select(1, torch.as_tensor(idx, device="cuda")))
                assert np.array_equal(got, obits(exp)), (n, k, f)


def test_launch_ctas_do_not_change_outputs():
    """The aligned vector kernel with one CTA per SM and with as many as fit,
    at 2^21 streams (the size class of the full-device calls): identical
    outputs, and sampled streams equal to the oracle."""
    L = capi.lib()
    n, steps, seed = 1 << 21, 4, 9
    idx = golden_streams(n)
    for k in KINDS:
        a = golden_a(idx) if k != oracle.XOR128 else None
        st = oracle.seed_streams(k, a, seed, idx)
        for f in FMTS:
            exp, _ = oracle.generate(k, a, st, steps, f)
            v, b, h, one = (ctypes.c_int() for _ in range(4))
            capi.check(L.gbrng_get_launch_class(k, f, 1, ctypes.byref(v), ctypes.byref(b),
                                                ctypes.byref(h)))
            capi.check(L.gbrng_get_launch_ctas(k, f, 1, ctypes.byref(one)))
            outs = []
            for shape, ctas in (((1, 512, 1), 0), ((1, 512, 1), 1), ((2, 512, 0), 1)):
                capi.check(L.gbrng_set_launch_class(k, f, 1, *shape))
                capi.check(L.gbrng_set_launch_ctas(k, f, 1, ctas))
                outs.append(Generator(k, n, seed).generate(steps, f))
                torch.cuda.synchronize()
            capi.check(L.gbrng_set_launch_class(k, f, 1, v.value, b.value, h.value))
            capi.check(L.gbrng_set_launch_ctas(k, f, 1, one.value))
            for o in outs[1:]:
                assert torch.equal(outs[0].view(torch.int32), o.view(torch.int32)), (k, f)
            got = bits(outs[1].index_select(1, torch.as_tensor(idx, device="cuda")))
            assert np.array_equal(got, obits(exp)), (k, f)


# --------------------------------------------------------- the workloads
@pytest.mark.parametrize("fmt", FMTS)
def test_mwc_4096x4096_full(fmt):
    w = workloads.MWC_4K
    g = Generator(oracle.MWC, w.n_streams, w.seed)
    out = g.generate(w.n_per_stream, fmt)
    torch.cuda.synchronize()
    exp, _ = expect_full(oracle.MWC, w.n_streams, w.seed, w.n_per_stream, fmt)
    assert np.array_equal(bits(out), obits(exp))


@pytest.mark.parametrize("kind", [oracle.XOR128, oracle.KISS])
def test_xor_kiss_2p20x1024_sampled(kind):
    w = workloads.XOR_KISS_1M
    idx = golden_streams(w.n_streams)
    a = golden_a(idx) if kind != oracle.XOR128 else None
    st = oracle.seed_streams(kind, a, w.seed, idx)
    exp_u, _ = oracle.generate(kind, a, st, w.n_per_stream, oracle.U32)
    exp_f, _ = oracle.generate(kind, a, st, w.n_per_stream, oracle.F32)
    gu = Generator(kind, w.n_streams, w.seed)
    gf = Generator(kind, w.n_streams, w.seed)
    u = gu.generate(w.n_per_stream, oracle.U32)
    f = gf.generate(w.n_per_stream, oracle.F32)
    sel = torch.as_tensor(idx, device="cuda")
    assert np.array_equal(bits(u.index_select(1, sel)), obits(exp_u))
    assert np.array_equal(bits(f.index_select(1, sel)), obits(exp_f))
    # every element: the FP32 output is exactly (u >> 8) * 2^-24 of the uint32 one
    top24 = (u >> 8) & 0xFFFFFF
    assert torch.equal(f, top24.to(torch.float32) * (2.0 ** -24))
    # and both generators end in the same state
    assert torch.equal(gu.get_state(), gf.get_state())


@pytest.mark.parametrize("kind", KINDS)
def test_odd_stream_count_2p20_plus_3_sampled(kind):
    """2^20 + 3 streams: the realigned path at scale, plus a 3-stream tail."""
    n, steps, seed = (1 << 20) + 3, 64, 13
    idx = np.concatenate([golden_streams(n), [n - 3, n - 2, n - 1]])
    idx = np.array(sorted(i for i in set(idx.tolist()) if i < (1 << 20) or
                          kind == oracle.XOR128 or i in set(GOLD["sample_index"])))
    a = golden_a(idx) if kind != oracle.XOR128 else None
    st = oracle.seed_streams(kind, a, seed, idx)
    exp, _ = oracle.generate(kind, a, st, steps, oracle.U32)
    out = Generator(kind, n, seed).generate(steps, oracle.U32)
    got = bits(out.index_select(1, torch.as_tensor(idx, device="cuda")))
    assert np.array_equal(got, obits(exp))


@pytest.mark.parametrize("kind", KINDS)
def test_full_device_10_calls_sampled(kind):
    w = workloads.FULL_4M
    idx = golden_streams(w.n_streams)[::3]
    a = golden_a(idx) if kind != oracle.XOR128 else None
    st = oracle.seed_streams(kind, a, w.seed, idx)
    g = Generator(kind, w.n_streams, w.seed)
    out = torch.empty((w.n_per_stream, w.n_streams), dtype=torch.int32, device="cuda")
    sel = torch.as_tensor(idx, device="cuda")
    for call in range(w.calls):
        fmt = oracle.F32 if call == w.calls - 1 else oracle.U32
        g.generate(w.n_per_stream, fmt, out=out)
        got = bits(out.index_select(1, sel))
        exp, st = oracle.generate(kind, a, st, w.n_per_stream, fmt)
        assert np.array_equal(got, obits(exp)), call
    del out
    torch.cuda.empty_cache()


# --------------------------------------------------------- host delivery
def test_generate_host_matches_device():
    n, steps, seed = 1 << 20, 300, 21  # 1.2 GB: several staging blocks
    d = Generator(oracle.XOR128, n, seed).generate(steps, oracle.U32)
    h = Generator(oracle.XOR128, n, seed).generate_host(steps, oracle.U32)
    assert torch.equal(d.cpu(), h)


@pytest.mark.parametrize("kind", KINDS)
def test_generate_host_small_matches_oracle(kind):
    n, steps, seed = 333, 45, 8
    g = Generator(kind, n, seed)
    h = g.generate_host(steps, oracle.F32)
    exp, _ = expect_full(kind, n, seed, steps, oracle.F32)
    assert np.array_equal(h.view(torch.int32).numpy().view(np.uint32), obits(exp))


# -------------------------------------------------------- checkpoints
@pytest.mark.parametrize("kind", KINDS)
def test_state_checkpoint_roundtrip(kind):
    g = Generator(kind, 2048, 31)
    g.generate(10)
    saved = g.get_state()
    a = g.generate(50).clone()
    g.set_state(saved)
    b = g.generate(50)
    assert torch.equal(a, b)


def test_set_state_rejects_invalid_and_keeps_state():
    g = Generator(oracle.MWC, 64, 1)
    st = g.get_state()
    bad = st.clone()
    bad[1, 5] = -1  # carry 0xFFFFFFFF >= a
    with pytest.raises(capi.RngError):
        g.set_state(bad)
    assert torch.equal(g.get_state(), st)
    x = Generator(oracle.XOR128, 8, 1)
    zero = torch.zeros((4, 8), dtype=torch.int32)
    with pytest.raises(capi.RngError):
        x.set_state(zero)


def test_zero_steps_and_argument_errors():
    g = Generator(oracle.KISS, 16, 2)
    st = g.get_state()
    out = torch.empty(0, dtype=torch.int32, device="cuda")
    assert capi.lib().rng_generate(g.h, 0, None, 0) == 0
    assert torch.equal(g.get_state(), st)
    assert capi.lib().rng_generate(g.h, 4, None, 0) == capi.RNG_ERR_ARG
    buf = torch.empty(64, dtype=torch.int32, device="cuda")
    assert capi.lib().rng_generate(g.h, 4, buf.data_ptr(), 5) == capi.RNG_ERR_ARG
    assert torch.equal(g.get_state(), st)
    del out


# -------------------------------------------------------------- batched
def small_instances(count=60, seed=77):
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = rng.integers(0, 3, count)
    streams = workloads.loguniform_int(rng, 1, 3000, count)
    steps = workloads.loguniform_int(rng, 1, 300, count)
    fmts = rng.integers(0, 2, count)
    return [workloads.Instance(int(kinds[i]), int(streams[i]), int(steps[i]),
                               int(fmts[i]), 1000 + i) for i in range(count)]


def _make(instances, offset_every=7):
    gens, outs = [], []
    for i, ins in enumerate(instances):
        gens.append(Generator(ins.kind, ins.n_streams, ins.seed))
        extra = 1 if i % offset_every == 3 else 0  # some outputs 4-byte aligned only
        buf = torch.zeros(ins.n_streams * ins.n_per_stream + extra, dtype=torch.int32,
                          device="cuda")
        outs.append(buf[extra:])
    return gens, outs


@pytest.mark.parametrize("threads", [0, 32, 256])
def test_batch_equals_plain_and_oracle(threads):
    ins = small_instances()
    gb, ob = _make(ins)
    gp, op = _make(ins)
    plan = Plan([BatchItem(g, i.n_per_stream, o, i.fmt) for g, i, o in zip(gb, ins, ob)],
                threads=threads)
    plan.launch()
    for g, i, o in zip(gp, ins, op):
        g.generate(i.n_per_stream, i.fmt, out=o)
    torch.cuda.synchronize()
    for k in range(len(ins)):
        assert torch.equal(ob[k], op[k]), k
        assert torch.equal(gb[k].get_state(), gp[k].get_state()), k
    for k in range(0, len(ins), 9):
        i = ins[k]
        if i.n_streams <= 16384:
            exp, _ = expect_full(i.kind, i.n_streams, i.seed, i.n_per_stream, i.fmt)
            assert np.array_equal(bits(ob[k]).reshape(i.n_per_stream, i.n_streams),
                                  obits(exp))
    plan.close()


@pytest.mark.parametrize("threads", [32, 128])
def test_batch_many_tails(threads):
    """Many tail tiles (the n % 4 last streams of an item) of mixed lengths,
    tails-only items (fewer than four streams) and the tails of stream
    subranges of one handle, all equal to plain calls."""
    rng = np.random.Generator(np.random.PCG64(31))
    ins = []
    for k in range(150):
        kind, fmt = (oracle.KISS, 0) if k < 100 else (oracle.MWC, 1)
        n = int(rng.choice([1, 2, 3, 5, 6, 7, 9, 13, 30, 61, 203]))
        ins.append(workloads.Instance(kind, n, int(rng.integers(1, 200)), fmt, 500 + k))
    gb, ob = _make(ins, offset_every=5)
    gp, op = _make(ins, offset_every=5)
    plan = Plan([BatchItem(g, i.n_per_stream, o, i.fmt) for g, i, o in zip(gb, ins, ob)],
                threads=threads)
    plan.launch()
    for g, i, o in zip(gp, ins, op):
        g.generate(i.n_per_stream, i.fmt, out=o)
    torch.cuda.synchronize()
    for k in range(len(ins)):
        assert torch.equal(ob[k], op[k]), k
        assert torch.equal(gb[k].get_state(), gp[k].get_state()), k
    plan.close()
    # subranges of one handle, each with a tail
    n, steps = 203, 37
    g1, g2 = Generator(oracle.XOR128, n, 4), Generator(oracle.XOR128, n, 4)
    cuts = [0, 7, 18, 45, 46, 101, 150, 203]
    o1 = torch.zeros(n * steps, dtype=torch.int32, device="cuda")
    o2 = torch.zeros(n * steps, dtype=torch.int32, device="cuda")
    items = [BatchItem(g1, steps, o1[a:], 0, s_begin=a, s_end=b, ld=n)
             for a, b in zip(cuts, cuts[1:])]
    Plan(items, threads=threads).launch()
    g2.generate(steps, 0, out=o2)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    assert torch.equal(g1.get_state(), g2.get_state())


def test_batch_graph_replay_continues_streams():
    ins = small_instances(20, seed=3)
    gb, ob = _make(ins)
    gp, op = _make(ins)
    plan = Plan([BatchItem(g, i.n_per_stream, o, i.fmt) for g, i, o in zip(gb, ins, ob)])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.launch(stream=s)
    for rep in range(2):
        graph.replay()
        for g, i, o in zip(gp, ins, op):
            g.generate(i.n_per_stream, i.fmt, out=o)
        torch.cuda.synchronize()
        for k in range(len(ins)):
            assert torch.equal(ob[k], op[k]), (rep, k)
    plan.close()


def test_generate_batch_rejects_duplicates():
    g = Generator(oracle.MWC, 64, 1)
    o1 = torch.empty(64 * 4, dtype=torch.int32, device="cuda")
    o2 = torch.empty(64 * 4, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.RngError):
        generate_batch([BatchItem(g, 4, o1, 0), BatchItem(g, 4, o2, 0)])
