"""The batched launch's work list (fill_units / order_units in
csrc/batch.cu), built on the CPU by a host-only driver that includes the
library source: for random items of every alignment, every stream of every
item is in exactly one tile (or in the tail that a realigned tile's last warp
runs), each tile points at its first stream's output, the store mode follows
the rows' alignment, tails join a tile only when its last warp holds no group,
and the tiles come longest first."""
from __future__ import annotations

import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
K_TAIL, K_ALIGNED, K_SHIFTED, K_SYNC = 0, 1, 2, 3


@pytest.fixture(scope="module")
def worklist_bin(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(nvcc).exists():
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("worklist") / "worklist_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17",
                    "-I", str(ROOT / "include"), "-I", str(ROOT / "paper_1101_1846_gb300" / "csrc"),
                    "-o", str(out), str(ROOT / "tests" / "native" / "worklist_check.cu")],
                   check=True, capture_output=True, timeout=600)
    return out


def random_items(rng, count):
    items = []
    for _ in range(count):
        kind, fmt = int(rng.integers(0, 3)), int(rng.integers(0, 2))
        n = int(rng.choice([1, 2, 3, 4, 5, 8, 12, 100, 127, 500, 1987, 1988, 1989, 2048, 4099,
                            6000, 9001]))
        if rng.random() < 0.5:
            s_begin, s_end = 0, n
        else:
            s_begin = int(rng.integers(0, n))
            s_end = int(rng.integers(s_begin + 1, n + 1))
        ld = n if rng.random() < 0.7 else n + int(rng.integers(0, 9))
        out_words = int(rng.integers(0, 8)) + 8 * int(rng.integers(0, 1000))
        steps = int(rng.integers(1, 300))
        items.append((kind, fmt, n, s_begin, s_end, ld, out_words, steps))
    return items


def run(worklist_bin, threads, items):
    text = f"{threads} {len(items)}\n" + "".join(" ".join(map(str, it)) + "\n" for it in items)
    r = subprocess.run([str(worklist_bin)], input=text, capture_output=True, text=True,
                       check=True, timeout=120)
    lines = r.stdout.strip().split("\n")
    count = int(lines[0])
    tiles = [tuple(int(x) for x in ln.split()) for ln in lines[1:]]
    assert len(tiles) == count
    return tiles


@pytest.mark.parametrize("threads", [32, 128, 512])
@pytest.mark.parametrize("seed", [1, 2])
def test_tiles_cover_every_stream_once(worklist_bin, threads, seed):
    rng = np.random.Generator(np.random.PCG64(100 * seed + threads))
    items = random_items(rng, 80)
    tiles = run(worklist_bin, threads, items)
    K = threads // 32
    by_item = {i: [] for i in range(len(items))}
    for t in tiles:
        by_item[t[0]].append(t)
    for i, (kind, fmt, n, s_begin, s_end, ld, out_words, steps) in enumerate(items):
        count = s_end - s_begin
        aligned = (count % 4 == 0 and ld % 4 == 0 and out_words % 4 == 0 and n % 4 == 0
                   and s_begin % 4 == 0)
        sectors = aligned and ld % 8 == 0 and out_words % 8 == 0
        main = count & ~3
        covered = np.zeros(count, dtype=np.int64)
        joined = 0
        for (_, mode, s0, cnt, tail, out, st) in by_item[i]:
            assert st == steps
            assert out == out_words + (s0 - s_begin)  # the tile's first stream's element
            assert s_begin <= s0 and s0 + cnt + tail <= s_end
            covered[s0 - s_begin: s0 - s_begin + cnt] += 1
            if mode == K_TAIL:
                assert s0 - s_begin == main and cnt == count - main and tail == 0
            elif aligned:
                assert mode == (K_ALIGNED if sectors else K_SYNC) and tail == 0
                assert cnt <= 4 * threads and cnt % 4 == 0
            else:
                assert mode == K_SHIFTED and cnt % 4 == 0 and cnt <= 4 * (31 * K + 1)
                if tail:
                    # the last realigned tile; its last warp holds no group
                    assert s0 + cnt - s_begin == main and tail == count - main
                    assert cnt // 4 <= 31 * (K - 1)
                    covered[main: count] += 1
                    joined += 1
        assert (covered == 1).all(), (i, items[i])
        if main < count and not aligned and main > 0:
            last = main % (4 * (31 * K + 1)) or 4 * (31 * K + 1)
            assert joined == (1 if last // 4 <= 31 * (K - 1) else 0), (i, items[i])
    # longest first
    assert all(a[6] >= b[6] for a, b in zip(tiles, tiles[1:]))
