"""Host-side scheduling of batched generation.

A generator's state carries from call to call, so an instance that needs R
rows (outputs per stream) can be produced as several consecutive pieces of
at most C rows each: piece k covers rows [k*C, min(R, (k+1)*C)), and the
pieces, run in order, give exactly the rows one call of R would.  Cutting
tall instances this way keeps every tile of a batched launch short, so a
launch does not wait on a few long dependency chains.

chunked_waves() builds the waves: each wave takes the next piece of as many
active instances as fit in a byte budget, in round-robin order, with at most
one piece per instance (two pieces of one generator in the same launch would
advance the same streams twice).  laned_waves() splits the instances into
lanes with waves of their own and interleaves them: waves of one lane must
run in order, waves of different lanes share no instance and may overlap, so
a wave's last tiles run beside the next lane's wave.
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass


@dataclass(frozen=True)
class Piece:
    inst: int   # index of the instance
    row0: int   # first row of this piece in the instance's output
    rows: int   # rows in this piece


def chunked_waves(streams: list[int], rows: list[int], budget_bytes: int,
                  chunk_rows: int, elem_bytes: int = 4) -> list[list[Piece]]:
    """Waves of pieces.  streams[i], rows[i]: instance i's stream count and
    total rows.  chunk_rows <= 0 means whole instances (one piece each).
    Every wave's output fits in budget_bytes, except a single piece that is
    larger than the budget on its own (it gets a wave alone)."""
    n = len(streams)
    done = [0] * n
    queue = deque(i for i in range(n) if rows[i] > 0)
    waves: list[list[Piece]] = []
    while queue:
        wave, used = [], 0
        deferred = []
        for _ in range(len(queue)):
            i = queue.popleft()
            left = rows[i] - done[i]
            take = left if chunk_rows <= 0 else min(left, chunk_rows)
            cost = elem_bytes * streams[i] * take
            if wave and used + cost > budget_bytes:
                # try a shorter piece before deferring the instance
                fit = (budget_bytes - used) // (elem_bytes * streams[i])
                if fit < 1:
                    deferred.append(i)
                    continue
                take, cost = fit, elem_bytes * streams[i] * fit
            wave.append(Piece(i, done[i], take))
            used += cost
            done[i] += take
            if done[i] < rows[i]:
                deferred.append(i)
        queue.extend(deferred)
        waves.append(wave)
    return waves


def laned_waves(streams: list[int], rows: list[int], budget_bytes: int, chunk_rows: int,
                lanes: int = 2, elem_bytes: int = 4) -> list[tuple[int, list[Piece]]]:
    """(lane, wave) pairs, lanes interleaved round-robin.  Instance i belongs
    to lane i % lanes; each lane's waves are chunked_waves() of its own
    instances (with their original indices) under the same budget."""
    per_lane = []
    for ln in range(lanes):
        idx = list(range(ln, len(streams), lanes))
        waves = chunked_waves([streams[i] for i in idx], [rows[i] for i in idx], budget_bytes,
                              chunk_rows, elem_bytes)
        per_lane.append([[Piece(idx[p.inst], p.row0, p.rows) for p in w] for w in waves])
    out = []
    k = 0
    while any(k < len(w) for w in per_lane):
        for ln in range(lanes):
            if k < len(per_lane[ln]):
                out.append((ln, per_lane[ln][k]))
        k += 1
    return out
