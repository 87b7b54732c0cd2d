"""How one tick's piece of a serving client runs through several of its
requests (csrc/runs.h, host-only C++, compiled with the host compiler):

* placement_pad puts every output at a word index congruent to its first
  sample's index modulo 8, within 28 bytes of its arena block;
* run_piece, on random runs of requests placed that way (outputs anywhere
  in the arena, partly done front request, formats mixed): every window index
  of the piece lands, through its segment's shift, exactly at its sample's
  place in its request's output, in that request's format, with a shift that
  is a multiple of 8 words (the 32-byte phase of the virtual window kept);
  the piece covers the requests in order up to the cap, and segments start
  only where the format or the shift changes."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def runs_bin(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = tmp_path_factory.mktemp("runs") / "runs_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-I",
                    str(ROOT / "paper_1101_1846_gb300" / "csrc"), "-o", str(out),
                    str(ROOT / "tests" / "native" / "runs_check.cpp")], check=True)
    return out


def run(binary, lines):
    r = subprocess.run([str(binary)], input="\n".join(lines) + "\n", capture_output=True,
                       text=True, check=True, timeout=120)
    return r.stdout.strip().split("\n")


def test_placement_pad_keeps_the_word_phase(runs_bin):
    rng = np.random.Generator(np.random.PCG64(3))
    cases = [(4 * int(rng.integers(0, 1 << 40)), int(rng.integers(0, 1 << 50)))
             for _ in range(5000)] + [(0, 0), (4, 0), (28, 1), (256, 7)]
    out = run(runs_bin, [f"a {b} {s}" for b, s in cases])
    for (b, s), line in zip(cases, out):
        pad = int(line)
        assert 0 <= pad <= 28 and pad % 4 == 0
        assert ((b + pad) // 4 - s) % 8 == 0


def random_run(rng):
    """A client's consecutive requests, placed anywhere (phase-aligned)."""
    count = int(rng.integers(1, 9))
    start = int(rng.integers(0, 10**9))
    reqs, info = [], []
    for i in range(count):
        n = int(rng.integers(1, 3000))
        block = 4 * int(rng.integers(0, 1 << 30))
        off = block + 4 * ((start - block // 4) % 8)
        if i and rng.random() < 0.3:  # sometimes right after the previous output
            off = reqs[-1][0] + 4 * reqs[-1][1]
            if (off // 4 - start) % 8:
                off = block + 4 * ((start - block // 4) % 8)
        done = int(rng.integers(0, n)) if i == 0 else 0
        fmt = int(rng.integers(0, 2))
        reqs.append((off, n, done, fmt))
        info.append(start)
        start += n
    return reqs, info


def test_run_piece_stops_at_a_misplaced_request(runs_bin):
    """A request whose output is not at its first sample's phase (mod 8
    words) is never joined to the piece: shifts stay multiples of 8."""
    reqs = [(4 * 8 * 100, 50, 0, 0), (4 * (8 * 900 + 50 + 3), 70, 0, 1), (4 * 8 * 5000, 10, 0, 0)]
    out = run(runs_bin, [f"q 100000 3 " + " ".join(f"{a} {b} {c} {d}" for a, b, c, d in reqs)])
    v = [int(x) for x in out[0].split()]
    assert v[1] == 50 and v[2] == 1 and v[3] == 1


def test_run_piece_places_every_sample(runs_bin):
    rng = np.random.Generator(np.random.PCG64(7))
    cases = []
    for _ in range(1500):
        reqs, starts = random_run(rng)
        cap = int(rng.integers(1, 12000))
        cases.append((reqs, starts, cap))
    lines = [f"q {cap} {len(reqs)} " + " ".join(f"{a} {b} {c} {d}" for a, b, c, d in reqs)
             for reqs, _, cap in cases]
    out = run(runs_bin, lines)
    assert len(out) == len(cases)
    multi = 0
    for (reqs, starts, cap), line in zip(cases, out):
        v = [int(x) for x in line.split()]
        origin, m, touched, nseg = v[:4]
        segs = [tuple(v[4 + 3 * k:7 + 3 * k]) for k in range(nseg)]
        need = [n - d for _, n, d, _ in reqs]
        assert origin == reqs[0][0] // 4 + reqs[0][2]
        assert m == min(cap, sum(need))
        assert touched == next((k + 1 for k in range(len(reqs))
                                if sum(need[:k + 1]) >= m), len(reqs))
        assert segs[0][:3] == (0, reqs[0][3], 0)
        bs = [g[0] for g in segs]
        assert bs == sorted(set(bs)) and all(g[2] % 8 == 0 for g in segs)
        for a, b in zip(segs, segs[1:]):
            assert (a[1], a[2]) != (b[1], b[2])  # a new segment changes something
        # every window index against its request, sample by sample
        i = 0
        for k, (off, n, done, fmt) in enumerate(reqs[:touched]):
            take = min(n - done, m - i)
            idx = np.arange(i, i + take)
            seg = np.searchsorted(bs, idx, side="right") - 1
            shifts = np.array([g[2] for g in segs])[seg]
            fmts = np.array([g[1] for g in segs])[seg]
            phys = origin + idx + shifts
            exp = off // 4 + done + np.arange(take)
            assert np.array_equal(phys, exp) and np.all(fmts == fmt), k
            i += take
        assert i == m
        multi += touched > 1
    assert multi > 500
