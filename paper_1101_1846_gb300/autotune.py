"""Launch-shape autotuner.

Plain kernels: for each (kind, fmt), time the vector kernel under each
candidate shape (groups of four streams per thread V, CTA size, store hint,
one CTA per SM or as many as fit) on a caller-given problem and keep the
fastest through gbrng_set_launch and gbrng_set_launch_ctas (the shapes of
calls of 2^21 streams or more).
Batched plans: time a plan under candidate (CTA size, CTAs per SM) pairs and
return the fastest.  Shapes never change outputs (tests check this), only
speed.  Results can be saved to and loaded from a JSON file keyed by GPU.
"""
from __future__ import annotations

import ctypes
import json
from pathlib import Path

import torch

from . import capi
from .generator import BatchItem, Generator, Plan

PLAIN_CANDIDATES = ([(v, b, h, 0) for v in (1, 2) for b in (128, 256, 512) for h in (0, 1)] +
                    [(v, 512, h, 1) for v in (1, 2) for h in (0, 1)])
PLAN_CANDIDATES = [(512, 1), (64, 0), (128, 0), (256, 0), (512, 0), (128, 4), (256, 2)]


def _time(fn, reps: int, stream) -> float:
    """Median milliseconds of fn() over reps launches (CUDA events)."""
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def get_shape(kind: int, fmt: int) -> tuple[int, int, int, int]:
    """(V, CTA size, store hint, one CTA per SM) of calls of 2^21 streams or more."""
    v, b, h, one = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib = capi.lib()
    capi.check(lib.gbrng_get_launch(kind, fmt, ctypes.byref(v), ctypes.byref(b),
                                    ctypes.byref(h)))
    capi.check(lib.gbrng_get_launch_ctas(kind, fmt, 1, ctypes.byref(one)))
    return v.value, b.value, h.value, one.value


def set_shape(kind: int, fmt: int, shape) -> None:
    """shape: (V, CTA size, store hint[, one CTA per SM])."""
    lib = capi.lib()
    capi.check(lib.gbrng_set_launch(kind, fmt, *shape[:3]), "gbrng_set_launch")
    if len(shape) > 3:
        capi.check(lib.gbrng_set_launch_ctas(kind, fmt, 1, shape[3]), "gbrng_set_launch_ctas")


def tune_plain(n_streams: int = 1 << 22, n_per_stream: int = 256, kinds=(0, 1, 2),
               fmts=(0, 1), candidates=PLAIN_CANDIDATES, reps: int = 5,
               seed: int = 1) -> dict:
    """Picks and installs the fastest shape per (kind, fmt).  Returns
    {(kind, fmt): {"shape": (v, block, hint), "ms": best, "all": {...}}}."""
    stream = torch.cuda.current_stream()
    out = torch.empty((n_per_stream, n_streams), dtype=torch.int32, device="cuda")
    result = {}
    for k in kinds:
        g = Generator(k, n_streams, seed)
        for f in fmts:
            timings = {}
            for shape in candidates:
                set_shape(k, f, shape)
                timings[shape] = _time(lambda: g.generate(n_per_stream, f, out=out,
                                                          stream=stream), reps, stream)
            best = min(timings, key=timings.get)
            set_shape(k, f, best)
            result[(k, f)] = {"shape": best, "ms": timings[best], "all": timings}
        g.close()
    del out
    return result


def tune_plan(items: list[BatchItem], candidates=PLAN_CANDIDATES, reps: int = 3):
    """Times a plan over `items` for each (threads, ctas_per_sm) and returns
    (best_pair, {pair: ms}).  The items' generators advance while timing."""
    stream = torch.cuda.current_stream()
    timings = {}
    for threads, per_sm in candidates:
        plan = Plan(items, threads=threads, ctas_per_sm=per_sm)
        timings[(threads, per_sm)] = _time(lambda: plan.launch(stream), reps, stream)
        plan.close()
    best = min(timings, key=timings.get)
    return best, timings


def save(result: dict, path: Path) -> None:
    name = torch.cuda.get_device_name()
    doc = json.loads(path.read_text()) if path.exists() else {}
    doc[name] = {f"{k}_{f}": list(r["shape"]) for (k, f), r in result.items()}
    path.write_text(json.dumps(doc, indent=1) + "\n")


def load(path: Path) -> bool:
    """Installs the shapes saved for this GPU; False if there are none."""
    if not path.exists():
        return False
    doc = json.loads(path.read_text()).get(torch.cuda.get_device_name())
    if not doc:
        return False
    for key, shape in doc.items():
        k, f = map(int, key.split("_"))
        set_shape(k, f, tuple(shape))
    return True
