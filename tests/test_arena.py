"""The serving engine's output arena (csrc/arena.h, host-only C++), compiled
with the host compiler and driven by random alloc/release scripts, against a
plain model of first-fit allocation over a list of free intervals: same
offsets, same bytes in use, free blocks merged, no two live blocks
overlapping."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
GRANULE = 256


@pytest.fixture(scope="module")
def arena_bin(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = tmp_path_factory.mktemp("arena") / "arena_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-I",
                    str(ROOT / "paper_1101_1846_gb300" / "csrc"), "-o", str(out),
                    str(ROOT / "tests" / "native" / "arena_check.cpp")], check=True)
    return out


class Model:
    """First fit over free intervals kept sorted by offset, merged on release."""

    def __init__(self, size, granule):
        self.g = granule
        self.size = size // granule * granule
        self.free = [[0, self.size]] if self.size else []
        self.used = 0

    def rnd(self, b):
        return (b + self.g - 1) // self.g * self.g

    def alloc(self, b):
        b = self.rnd(b)
        for i, (off, ln) in enumerate(self.free):
            if ln >= b:
                if ln == b:
                    self.free.pop(i)
                else:
                    self.free[i] = [off + b, ln - b]
                self.used += b
                return off
        return None

    def release(self, off, b):
        b = self.rnd(b)
        self.used -= b
        self.free.append([off, b])
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1][1] += ln
            else:
                merged.append([o, ln])
        self.free = merged


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_arena_matches_first_fit_model(arena_bin, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    size = 64 << 20
    model = Model(size, GRANULE)
    live = {}  # offset -> requested bytes
    ops, expect = [], []
    for _ in range(4000):
        if live and (rng.random() < 0.45 or model.used > size * 0.9):
            off = int(rng.choice(sorted(live)))
            b = live.pop(off)
            model.release(off, b)
            ops.append(f"r {off} {b}")
            expect.append(("r", model.used, len(model.free),
                           max((ln for _, ln in model.free), default=0)))
        else:
            b = int(np.exp(rng.random() * np.log(8 << 20))) + 1  # 1 B .. 8 MiB, log-uniform
            off = model.alloc(b)
            ops.append(f"a {b}")
            expect.append(("a", off, model.used))
            if off is not None:
                assert all(off + model.rnd(b) <= o or o + model.rnd(x) <= off
                           for o, x in live.items())
                live[off] = b
    r = subprocess.run([str(arena_bin)], input=f"{size} {GRANULE}\n" + "\n".join(ops) + "\n",
                       capture_output=True, text=True, check=True, timeout=120)
    lines = r.stdout.split("\n")
    assert int(lines[0]) == model.size
    for i, (kind, *vals) in enumerate(expect):
        got = [int(x) for x in lines[1 + i].split()]
        if kind == "a":
            off, used = vals
            assert got == ([1, off, used] if off is not None else [0, 0, used]), i
        else:
            used, blocks, largest = vals
            assert got == [used, blocks, largest], i


def test_arena_release_merges_to_one_block(arena_bin):
    size = 1 << 20
    script = [f"{size} {GRANULE}"] + ["a 1000"] * 4 + ["r 1024 1000", "r 0 1000",
                                                      "r 3072 1000", "r 2048 1000"]
    r = subprocess.run([str(arena_bin)], input="\n".join(script) + "\n", capture_output=True,
                       text=True, check=True, timeout=60)
    lines = r.stdout.split("\n")
    assert [lines[i].split()[1] for i in (1, 2, 3, 4)] == ["0", "1024", "2048", "3072"]
    assert lines[5].split()[:2] == [str(3 * 1024), "2"]   # a hole at 1024, the tail after 4096
    assert lines[6].split()[:2] == [str(2 * 1024), "2"]   # 0 merges with 1024
    assert lines[7].split()[:2] == [str(1024), "2"]       # 3072 merges with the tail
    assert lines[8].split() == ["0", "1", str(size)]  # everything one free block again
