"""How the serving engine cuts a client's samples into batch items
(csrc/pieces.h, host-only C++), compiled with the host compiler: for pieces
of every shape (inside one row, across the wrap, whole rows, many rows), the
items write every sample of the piece exactly once, at its place in the
output, from the stream and step the client's sequence assigns it (sample g
is output g // n of stream g % n), with disjoint stream ranges."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def pieces_bin(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = tmp_path_factory.mktemp("pieces") / "pieces_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-I", str(ROOT / "include"), "-I",
                    str(ROOT / "paper_1101_1846_gb300" / "csrc"), "-o", str(out),
                    str(ROOT / "tests" / "native" / "pieces_check.cpp")], check=True)
    return out


def cases():
    rng = np.random.Generator(np.random.PCG64(8))
    out = []
    for n in (1, 3, 4, 7, 64, 1003):
        for c in (0, 1, n - 1, n, 5 * n + n // 2):
            for m in (1, n - 1, n, n + 1, 3 * n, 3 * n + 2):
                if m > 0:
                    out.append((n, c, m))
    for _ in range(300):
        n = int(rng.integers(1, 2000))
        out.append((n, int(rng.integers(0, 50 * n)), int(rng.integers(1, 6 * n))))
    return out


@pytest.mark.parametrize("split", [0, 1])
def test_items_cover_the_piece_exactly_once(pieces_bin, split):
    """With split = 1 the items are also cut at multiples of 8 streams
    (split_aligned), the window placed at word phase c mod 8 as the serving
    engine places outputs: still every sample once, and for n a multiple of
    8 every item of 8 or more streams that starts at a multiple of 8 has
    32-byte aligned rows, and no other item holds a whole aligned block of 8
    streams."""
    cs = cases()
    r = subprocess.run([str(pieces_bin)],
                       input="".join(f"{n} {c} {m} {split}\n" for n, c, m in cs),
                       capture_output=True, text=True, check=True, timeout=120)
    lines = r.stdout.strip().split("\n")
    assert len(lines) == len(cs)
    for (n, c, m), line in zip(cs, lines):
        v = [int(x) for x in line.split()]
        count, items = v[0], [v[1 + 5 * i: 6 + 5 * i] for i in range(v[0])]
        assert 1 <= count <= (12 if split else 4), (n, c, m)
        if split and n % 8 == 0:
            for s_begin, s_end, rows, off, ld in items:
                # stream s's output sits at window offset off + (s - s_begin),
                # word phase (c + off) mod 8 at the item's first stream
                if s_begin % 8 == 0 and s_end - s_begin >= 8:
                    assert (c + off - s_begin) % 8 == 0 and (s_end - s_begin) % 8 == 0
                else:  # nothing aligned left in it to split off
                    assert s_end // 8 * 8 <= (s_begin + 7) // 8 * 8, (n, c, m, s_begin, s_end)
        covered = np.zeros(m, dtype=np.int64)
        ranges = []
        for s_begin, s_end, rows, off, ld in items:
            assert ld == n and 0 <= s_begin < s_end <= n and rows >= 1
            ranges.append((s_begin, s_end))
            for j in range(rows):
                for s in range(s_begin, s_end):
                    k = off + j * n + (s - s_begin)  # window position written
                    assert 0 <= k < m, (n, c, m)
                    covered[k] += 1
                    g = c + k  # the client's sample there
                    assert g % n == s, (n, c, m, s, k)
                    # the item's row j is the stream's (j+1)-th output of this piece
                    first = c + ((s - c) % n)  # the stream's first sample at or after c
                    assert g == first + j * n, (n, c, m, s, j)
        assert (covered == 1).all(), (n, c, m)
        ranges.sort()
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 <= b0, (n, c, m, ranges)
