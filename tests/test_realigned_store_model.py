"""A CPU model of which lane stores which words in the realigned body
(body_shift / shift_row in csrc/gen_body.cuh), checked exhaustively where
the GPU tests can only sample: for every row alignment R, warp count K and
live group count, every output element of the CTA's range is written exactly
once and nothing outside it.  Also the condition under which the batched
kernel gives a realigned tile's last warp to the item's tail streams: that
warp then holds no live group, and the tail's elements follow the groups'
without overlap."""
from __future__ import annotations

import pytest


def store_roles(K: int, groups: int, R: int) -> dict[int, int]:
    """Element positions (relative to the CTA's first output element) and
    how often each is stored, for K warps of 32 lanes; lane l of warp k holds
    group g = 31k + l (lane 31 of a warp but the last is a halo, holding the
    next warp's first group without owning it)."""
    assert 1 <= groups <= 31 * K + 1
    writes: dict[int, int] = {}

    def put(pos):
        writes[pos] = writes.get(pos, 0) + 1

    for k in range(K):
        for lane in range(32):
            g = 31 * k + lane
            live = g < groups
            owner = live and (lane < 31 or k == K - 1)
            lead = g == 0
            trail = owner and g == groups - 1
            prev = live and lane > 0
            nxt = owner and lane < 31 and g + 1 < groups
            base = 4 * g  # the group's four words sit at base .. base + 3
            if R == 0:
                if owner:  # one aligned chunk
                    for i in range(4):
                        put(base + i)
                continue
            if R in (1, 2):
                if prev:  # chunk C: R words of the lane on the left, then 4 - R own words
                    for i in range(4):
                        put(base - R + i)
            elif nxt:  # R = 3, chunk C + 4: own words 1..3 and word 0 of the next lane
                for i in range(4):
                    put(base + 1 + i)
            if lead:  # the CTA's first lane: its words before the first aligned chunk
                for i in range(4 - R):
                    put(base + i)
            if trail:  # the owner of the last group: its words after the last chunk
                for i in range(4 - R, 4):
                    put(base + i)
    return writes


def check(K, groups, R):
    w = store_roles(K, groups, R)
    assert sorted(w) == list(range(4 * groups)), (K, groups, R)
    assert all(v == 1 for v in w.values()), (K, groups, R)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_every_element_once_small_ctas(K):
    for groups in range(1, 31 * K + 2):
        for R in range(4):
            check(K, groups, R)


def test_every_element_once_16_warps():
    # the batched kernel's 512-thread CTAs: edges of every warp and the ends
    for groups in sorted({1, 2, 3, 30, 31, 32, 33, 61, 62, 63, 64, 250, 464, 465, 466, 467,
                          495, 496, 497}):
        for R in range(4):
            check(16, groups, R)


@pytest.mark.parametrize("K", [2, 4, 16])
def test_tail_warp_holds_no_group(K):
    """The batched kernel joins an item's 1-3 tail streams to its last
    realigned tile when that tile has at most 31 (K - 1) groups; then no lane
    of the last warp, and no halo lane of the warp before it, holds a live
    group, and the tail's elements come right after the groups' ones."""
    for groups in range(1, 31 * (K - 1) + 1):
        live_in_last = [31 * (K - 1) + lane for lane in range(32) if 31 * (K - 1) + lane < groups]
        assert not live_in_last
        assert 31 * (K - 1) >= groups  # warp K - 2's halo lane (group 31 (K - 1)) is idle
        for tail in (1, 2, 3):
            for R in range(4):
                shifted = store_roles(K, groups, R)
                tail_pos = {4 * groups + i for i in range(tail)}
                assert not tail_pos & set(shifted)
                assert sorted(set(shifted) | tail_pos) == list(range(4 * groups + tail))
