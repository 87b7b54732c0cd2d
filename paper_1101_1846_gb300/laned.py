"""Batched waves on lanes, each wave one persistent launch in a CUDA graph.

scheduler.laned_waves() cuts instances into pieces and packs them into
(lane, wave) pairs.  LanedGraphs builds one plan per wave (rng_plan_create)
and captures its launch in a CUDA graph on the lane's stream; replay()
enqueues every wave's graph on its lane's stream after the caller's stream
and makes the caller's stream wait for all lanes.  A lane's waves continue
the same instances, so they run in order on one stream; lanes share no
instance, so their waves overlap on the device.
"""
from __future__ import annotations

from typing import Callable

import torch

from .generator import BatchItem, Generator, Plan
from .scheduler import Piece


def carve(buf: torch.Tensor, wave: list[Piece], n_streams: list[int]) -> list[torch.Tensor]:
    """Consecutive views of `buf` for the pieces of a wave (piece p gets
    n_streams[p.inst] * p.rows elements), each starting 16-byte aligned."""
    outs, off = [], 0
    for p in wave:
        m = n_streams[p.inst] * p.rows
        outs.append(buf[off:off + m])
        off += (m + 3) // 4 * 4
    return outs


def wave_elems(wave: list[Piece], n_streams: list[int]) -> int:
    """Elements carve() needs for a wave."""
    return sum((n_streams[p.inst] * p.rows + 3) // 4 * 4 for p in wave)


class LanedGraphs:
    """Plans and graphs of (lane, wave) pairs.  out_for(k, lane, wave) gives
    the buffer the k-th wave writes into; gens[i] and fmts[i] are instance
    i's generator and format."""

    def __init__(self, laned: list[tuple[int, list[Piece]]], gens: list[Generator],
                 fmts: list[int], out_for: Callable[[int, int, list[Piece]], torch.Tensor],
                 threads: int = 0, ctas_per_sm: int = 0):
        self.lanes = 1 + max(lane for lane, _ in laned)
        self.streams = [torch.cuda.Stream() for _ in range(self.lanes)]
        self.laned = laned
        self.plans, self.graphs, self.outs = [], [], []
        self.tiles = 0
        n_streams = [g.n_streams for g in gens]
        main = torch.cuda.current_stream()
        for k, (lane, wave) in enumerate(laned):
            outs = carve(out_for(k, lane, wave), wave, n_streams)
            items = [BatchItem(gens[p.inst], p.rows, o, fmts[p.inst])
                     for p, o in zip(wave, outs)]
            plan = Plan(items, threads=threads, ctas_per_sm=ctas_per_sm)
            self.tiles += plan.tiles
            s = self.streams[lane]
            s.wait_stream(main)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                plan.launch(s)
            self.plans.append(plan)
            self.graphs.append(graph)
            self.outs.append(outs)
        torch.cuda.synchronize()

    def replay(self) -> None:
        """Every wave once, lanes overlapping, ordered after the current
        stream's work; the current stream then waits for all of them."""
        main = torch.cuda.current_stream()
        for s in self.streams:
            s.wait_stream(main)
        for (lane, _), graph in zip(self.laned, self.graphs):
            with torch.cuda.stream(self.streams[lane]):
                graph.replay()
        for s in self.streams:
            main.wait_stream(s)

    def close(self) -> None:
        torch.cuda.synchronize()
        for plan in self.plans:
            plan.close()
        self.plans, self.graphs = [], []
