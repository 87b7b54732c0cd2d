"""Python face of the serving engine (rng_server_* in include/rng.h): a
wrapper, and a driver that replays a request log with real-time arrivals
and reports latency percentiles and throughput.  All scheduling, admission
and generation happen in the library."""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import capi


class Server:
    def __init__(self, kind: int = capi.RNG_KISS, n_clients: int = 256,
                 streams_per_client: int = 65536, seed_base: int = 0,
                 budget_bytes: int = 40 << 30, chunk_rows: int = 64, tick_bytes: int = 0,
                 plan_shape: tuple[int, int] | None = None):
        h = capi.lib().rng_server_create(kind, n_clients, streams_per_client, seed_base,
                                         budget_bytes, chunk_rows)
        if not h:
            raise capi.RngError(capi.lib().rng_last_error(), "rng_server_create")
        self.h = h
        if tick_bytes:
            capi.check(capi.lib().rng_server_set_tick_bytes(h, tick_bytes))
        if plan_shape is not None:
            capi.check(capi.lib().rng_server_set_plan_shape(h, *plan_shape),
                       "rng_server_set_plan_shape")
        self.kind, self.n_clients, self.streams = kind, n_clients, streams_per_client
        self.seed_base = seed_base
        self._ids = (ctypes.c_uint64 * 4096)()
        self._ms = (ctypes.c_double * 4096)()

    def client_seed(self, client: int) -> int:
        """The seed of a client's generator (seed_base + client * 2^32)."""
        return (self.seed_base + (client << 32)) & (2**64 - 1)

    def submit(self, client: int, n_samples: int, fmt: int) -> int:
        rid = ctypes.c_uint64()
        capi.check(capi.lib().rng_server_submit(self.h, client, n_samples, fmt,
                                                ctypes.byref(rid)), "rng_server_submit")
        return rid.value

    def submit_many(self, clients: np.ndarray, n_samples: np.ndarray,
                    fmts: np.ndarray) -> np.ndarray:
        """Queues len(clients) requests in order; returns their ids."""
        c = np.ascontiguousarray(clients, dtype=np.uint32)
        n = np.ascontiguousarray(n_samples, dtype=np.uint64)
        f = np.ascontiguousarray(fmts, dtype=np.int32)
        ids = np.zeros(len(c), dtype=np.uint64)
        capi.check(capi.lib().rng_server_submit_many(
            self.h, c.ctypes.data, n.ctypes.data, f.ctypes.data, len(c), ids.ctypes.data),
            "rng_server_submit_many")
        return ids

    def take_arrays(self) -> tuple[np.ndarray, np.ndarray]:
        """Completed requests as (ids, device completion times in ms)."""
        ids_all, ms_all = [], []
        ids_view = np.ctypeslib.as_array(self._ids)
        ms_view = np.ctypeslib.as_array(self._ms)
        while True:
            n = capi.lib().rng_server_take(self.h, self._ids, self._ms, len(self._ids))
            ids_all.append(ids_view[:n].copy())
            ms_all.append(ms_view[:n].copy())
            if n < len(self._ids):
                break
        if len(ids_all) == 1:
            return ids_all[0], ms_all[0]
        return np.concatenate(ids_all), np.concatenate(ms_all)

    def release_many(self, ids: np.ndarray) -> None:
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        capi.check(capi.lib().rng_server_release_many(self.h, ids.ctypes.data, len(ids)),
                   "rng_server_release_many")

    def progress(self) -> int:
        return capi.check(capi.lib().rng_server_progress(self.h), "rng_server_progress")

    def drain(self) -> None:
        capi.check(capi.lib().rng_server_drain(self.h), "rng_server_drain")

    def take(self) -> list[tuple[int, float]]:
        out = []
        while True:
            n = capi.lib().rng_server_take(self.h, self._ids, self._ms, 4096)
            out.extend((self._ids[i], self._ms[i]) for i in range(n))
            if n < 4096:
                return out

    def result(self, rid: int) -> dict:
        ptr, n, fmt = ctypes.c_void_p(), ctypes.c_uint64(), ctypes.c_int()
        client, start = ctypes.c_uint32(), ctypes.c_uint64()
        capi.check(capi.lib().rng_server_result(self.h, rid, ctypes.byref(ptr),
                                                ctypes.byref(n), ctypes.byref(fmt),
                                                ctypes.byref(client), ctypes.byref(start)),
                   "rng_server_result")
        return {"n": n.value, "fmt": fmt.value, "client": client.value, "start": start.value}

    def copy(self, rid: int, offset: int = 0, count: int | None = None,
             out: torch.Tensor | None = None) -> torch.Tensor:
        """The request's output (or a slice) as an int32 tensor on the device
        (float requests hold float bits); synchronises torch's current stream."""
        info = self.result(rid)
        count = info["n"] - offset if count is None else count
        if out is None:
            out = torch.empty(count, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        capi.check(capi.lib().rng_server_copy(self.h, rid, ctypes.c_void_p(out.data_ptr()),
                                              offset, count,
                                              ctypes.c_void_p(stream.cuda_stream)),
                   "rng_server_copy")
        stream.synchronize()
        return out

    def release(self, rid: int) -> None:
        capi.check(capi.lib().rng_server_release(self.h, rid), "rng_server_release")

    def stats(self) -> dict:
        v = (ctypes.c_uint64 * 8)()
        capi.check(capi.lib().rng_server_stats(self.h, v))
        keys = ["submitted", "admitted", "completed", "ticks", "samples", "arena_used",
                "arena_size", "waiting"]
        return dict(zip(keys, list(v)))

    def close(self) -> None:
        if getattr(self, "h", None):
            capi.lib().rng_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class RunResult:
    latencies_s: np.ndarray = field(default_factory=lambda: np.zeros(0))
    samples: int = 0
    wall_s: float = 0.0
    requests: int = 0
    max_arena_used: int = 0
    ticks: int = 0
    checked: list = field(default_factory=list)

    def summary(self) -> dict:
        lat = self.latencies_s
        return {
            "requests": self.requests, "samples": self.samples, "wall_s": self.wall_s,
            "gsamples_s": self.samples / self.wall_s / 1e9 if self.wall_s else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "mean_ms": float(lat.mean() * 1e3) if lat.size else None,
            "max_arena_used": self.max_arena_used, "ticks": self.ticks,
        }


def replay(server: Server, log, realtime: bool = True, on_done=None) -> RunResult:
    """Submits log[i] (fields t, client, n_samples, fmt) at its arrival time
    (realtime) or all at once (saturating run), drives the engine until all
    complete, and releases each result (after on_done(rid, request) if
    given).  Request ids are the log indices (a fresh engine numbers
    requests from 0).  Latency = host time the completion is seen minus the
    arrival time."""
    res = RunResult(requests=len(log))
    m = len(log)
    t_arr = np.array([r.t for r in log]) if realtime else np.zeros(m)
    clients = np.array([r.client for r in log], dtype=np.uint32)
    sizes = np.array([r.n_samples for r in log], dtype=np.uint64)
    fmts = np.array([r.fmt for r in log], dtype=np.int32)
    lat = np.zeros(m)
    arrival = np.zeros(m)
    first = server.stats()["submitted"]
    t0 = time.perf_counter()
    i, n_done, loops = 0, 0, 0
    while n_done < m:
        loops += 1
        now = time.perf_counter() - t0
        j = int(np.searchsorted(t_arr, now, side="right")) if realtime else m
        if j > i:
            server.submit_many(clients[i:j], sizes[i:j], fmts[i:j])
            arrival[i:j] = t_arr[i:j] if realtime else now
            i = j
        server.progress()
        ids, _ms = server.take_arrays()
        if ids.size:
            seen = time.perf_counter() - t0
            k = (ids - first).astype(np.int64)
            lat[k] = seen - arrival[k]
            if on_done is not None:
                for rid, kk in zip(ids.tolist(), k.tolist()):
                    on_done(rid, log[kk])
            server.release_many(ids)
            n_done += ids.size
        if loops % 64 == 0:
            res.max_arena_used = max(res.max_arena_used, server.stats()["arena_used"])
        if not ids.size and realtime and i < m and t_arr[i] > now + 2e-4:
            time.sleep(min(1e-4, t_arr[i] - now))
    res.wall_s = time.perf_counter() - t0
    res.latencies_s = lat
    st = server.stats()
    res.samples = st["samples"]
    res.ticks = st["ticks"]
    return res
