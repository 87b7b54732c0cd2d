"""The batched configuration as the benchmark runs it: instances cut into
1024-row pieces (and 256-row ones), packed into waves on two lanes
(scheduler.laned_waves), each
wave one persistent launch captured in a CUDA graph, a lane's waves in order
on its own stream and the two lanes overlapping (laned.LanedGraphs).  The
recipe is the 10,000-instance one scaled down (300 instances, streams
log-uniform up to 4096, outputs up to 16 times the piece length) with a wave
budget small enough for many waves, so that many instances carry their state
across waves.

Every piece is checked against the same rows of a plain call of its
instance, every final state against the plain generator's, and every
seventh instance in full against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1101_1846_gb300 import build, capi, laned, scheduler, workloads  # noqa: E402
from paper_1101_1846_gb300.generator import Generator  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    capi.lib()


@pytest.mark.parametrize("chunk,min_carried", [(1024, 60), (256, 100)])
def test_laned_graph_waves_equal_plain_calls_and_oracle(chunk, min_carried):
    inst = workloads.batched_instances(300, 4321, streams_range=(32, 4096),
                                       steps_range=(16, 16 * chunk))
    n_streams = [i.n_streams for i in inst]
    rows = [i.n_per_stream for i in inst]
    pairs = scheduler.laned_waves(n_streams, rows, 16 << 20, chunk, 2)
    assert len(pairs) >= 20 and {lane for lane, _ in pairs} == {0, 1}
    carried = {p.inst for _, w in pairs for p in w if p.row0 > 0}
    assert len(carried) > min_carried  # many instances span several waves

    # one region per wave, so that every piece can be read back afterwards
    sizes = [laned.wave_elems(w, n_streams) for _, w in pairs]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    big = torch.full((int(offs[-1]),), -1, dtype=torch.int32, device="cuda")
    gens = [Generator(i.kind, i.n_streams, i.seed) for i in inst]
    run = laned.LanedGraphs(pairs, gens, [i.fmt for i in inst],
                            lambda k, lane, w: big[int(offs[k]):int(offs[k + 1])])
    run.replay()
    torch.cuda.synchronize()

    plain_gens = [Generator(i.kind, i.n_streams, i.seed) for i in inst]
    # bits as int32, whatever the format
    plain = [g.generate(i.n_per_stream, i.fmt).view(torch.int32)
             for g, i in zip(plain_gens, inst)]
    torch.cuda.synchronize()
    for k, (_, w) in enumerate(pairs):
        for p, o in zip(w, run.outs[k]):
            ref = plain[p.inst][p.row0:p.row0 + p.rows].reshape(-1)
            assert torch.equal(o, ref), (k, p)
    for g, h in zip(gens, plain_gens):
        assert torch.equal(g.get_state(), h.get_state())
    run.close()

    for i in range(0, len(inst), 7):
        ins = inst[i]
        a = oracle.multipliers_for(ins.kind, ins.n_streams)
        st = oracle.seed_streams(ins.kind, a, ins.seed, np.arange(ins.n_streams))
        exp, _ = oracle.generate(ins.kind, a, st, ins.n_per_stream, ins.fmt)
        got = plain[i].cpu().view(torch.int32).numpy().view(np.uint32)
        assert np.array_equal(got, exp.view(np.uint32)), i
    for g in gens + plain_gens:
        g.close()
