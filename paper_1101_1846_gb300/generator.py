"""Python face of the library: PyTorch supplies device memory and streams,
every sample is made by the CUDA kernels behind the C-ABI (capi.py)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import capi


def _stream_ptr(stream: torch.cuda.Stream | None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dtype(fmt: int) -> torch.dtype:
    return torch.int32 if fmt == capi.RNG_U32 else torch.float32


class Generator:
    """n_streams parallel streams of one generator kind on the current
    device.  generate() returns a tensor of shape (n_per_stream, n_streams):
    row j holds output j of every stream (the stream-interleaved layout).
    uint32 outputs are returned in an int32 tensor (same bits)."""

    def __init__(self, kind: int | str, n_streams: int, seed: int, s_begin: int = 0):
        kind = capi.KINDS.get(kind, kind) if isinstance(kind, str) else kind
        if s_begin:  # streams s_begin .. s_begin + n_streams - 1 of one generator
            h = capi.lib().rng_create_range(int(kind), int(s_begin), int(n_streams),
                                            int(seed) & (2**64 - 1))
        else:
            h = capi.lib().rng_create(int(kind), int(n_streams), int(seed) & (2**64 - 1))
        if not h:
            raise capi.RngError(capi.lib().rng_last_error(), "rng_create")
        self.h = h
        self.kind = int(kind)
        self.n_streams = int(n_streams)
        self.seed = int(seed)
        self.s_begin = int(s_begin)
        self.words = capi.lib().rng_state_words(h)
        self.device = torch.cuda.current_device()

    def close(self) -> None:
        if getattr(self, "h", None):
            capi.lib().rng_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _bind(self, stream) -> None:
        capi.check(capi.lib().rng_set_stream(self.h, ctypes.c_void_p(_stream_ptr(stream))),
                   "rng_set_stream")

    def generate(self, n_per_stream: int, fmt: int | str = capi.RNG_U32,
                 out: torch.Tensor | None = None,
                 stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        fmt = capi.FMTS.get(fmt, fmt) if isinstance(fmt, str) else fmt
        if out is None:
            out = torch.empty((n_per_stream, self.n_streams), dtype=_dtype(fmt),
                              device=f"cuda:{self.device}")
        assert out.is_cuda and out.is_contiguous() and out.element_size() == 4
        assert out.numel() >= n_per_stream * self.n_streams
        self._bind(stream)
        capi.check(capi.lib().rng_generate(self.h, n_per_stream,
                                           ctypes.c_void_p(out.data_ptr()), fmt),
                   "rng_generate")
        return out

    def generate_range(self, s_begin: int, s_end: int, n_per_stream: int,
                       out: torch.Tensor, ld: int, fmt: int | str = capi.RNG_U32,
                       offset: int = 0, stream: torch.cuda.Stream | None = None) -> None:
        """Advances streams [s_begin, s_end) only; output j of stream s goes to
        out.view(-1)[offset + j*ld + (s - s_begin)]."""
        fmt = capi.FMTS.get(fmt, fmt) if isinstance(fmt, str) else fmt
        assert out.is_cuda and out.is_contiguous() and out.element_size() == 4
        count = s_end - s_begin
        if n_per_stream:
            assert offset + (n_per_stream - 1) * ld + count <= out.numel()
        self._bind(stream)
        ptr = out.data_ptr() + 4 * offset
        capi.check(capi.lib().rng_generate_range(self.h, s_begin, s_end, n_per_stream,
                                                 ctypes.c_void_p(ptr), ld, fmt),
                   "rng_generate_range")

    def generate_host(self, n_per_stream: int, fmt: int | str = capi.RNG_U32,
                      out: torch.Tensor | None = None,
                      stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        """Same outputs delivered to (pinned) host memory; synchronises."""
        fmt = capi.FMTS.get(fmt, fmt) if isinstance(fmt, str) else fmt
        if out is None:
            out = torch.empty((n_per_stream, self.n_streams), dtype=_dtype(fmt),
                              pin_memory=True)
        assert not out.is_cuda and out.is_contiguous()
        assert out.numel() >= n_per_stream * self.n_streams
        self._bind(stream)
        capi.check(capi.lib().rng_generate_host(self.h, n_per_stream,
                                                ctypes.c_void_p(out.data_ptr()), fmt),
                   "rng_generate_host")
        return out

    def generate_reduce(self, n_per_stream: int, op: int | str = capi.RNG_SUM_U32,
                        out: torch.Tensor | None = None,
                        stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        """Advances every stream n_per_stream times with no output array;
        returns one 64-bit result per stream (an int64 tensor holding the
        uint64 bits): op = RNG_SUM_U32, RNG_SUM_U24 or RNG_DISC
        (rng_generate_reduce)."""
        op = {"sum_u32": capi.RNG_SUM_U32, "sum_u24": capi.RNG_SUM_U24,
              "disc": capi.RNG_DISC}.get(op, op) if isinstance(op, str) else op
        if out is None:
            out = torch.empty(self.n_streams, dtype=torch.int64, device=f"cuda:{self.device}")
        assert out.is_cuda and out.is_contiguous() and out.element_size() == 8
        assert out.numel() >= self.n_streams
        self._bind(stream)
        capi.check(capi.lib().rng_generate_reduce(self.h, n_per_stream, int(op),
                                                  ctypes.c_void_p(out.data_ptr())),
                   "rng_generate_reduce")
        return out

    def jump(self, k: int, stream: torch.cuda.Stream | None = None) -> None:
        """Advances every stream by k steps without producing the outputs
        in between (rng_jump)."""
        self._bind(stream)
        capi.check(capi.lib().rng_jump(self.h, int(k) & (2**64 - 1)), "rng_jump")

    def device_view(self) -> capi.rng_device_view:
        v = capi.rng_device_view()
        capi.check(capi.lib().rng_get_device_view(self.h, ctypes.byref(v)),
                   "rng_get_device_view")
        return v

    def get_state(self) -> torch.Tensor:
        """State words as an int32 tensor (words, n_streams) on the host."""
        buf = torch.empty((self.words, self.n_streams), dtype=torch.int32)
        capi.check(capi.lib().rng_get_state(self.h, ctypes.c_void_p(buf.data_ptr()),
                                            buf.numel() * 4), "rng_get_state")
        return buf

    def set_state(self, state: torch.Tensor) -> None:
        buf = state.to(torch.int32).contiguous().cpu()
        capi.check(capi.lib().rng_set_state(self.h, ctypes.c_void_p(buf.data_ptr()),
                                            buf.numel() * 4), "rng_set_state")


def multipliers(k: int, device: int | None = None) -> torch.Tensor:
    """The first k MWC multipliers from the device table (int32 bits)."""
    dev = torch.cuda.current_device() if device is None else device
    out = torch.empty(k, dtype=torch.int32, device=f"cuda:{dev}")
    with torch.cuda.device(dev):
        capi.check(capi.lib().rng_multipliers(k, ctypes.c_void_p(out.data_ptr())),
                   "rng_multipliers")
    return out


@dataclass
class BatchItem:
    """Generator `gen` advances streams [s_begin, s_end) (s_end = 0: all)
    n_per_stream times; output j of stream s goes to
    out.view(-1)[offset + j*ld + (s - s_begin)] (ld = 0: the stream count)."""
    gen: Generator
    n_per_stream: int
    out: torch.Tensor
    fmt: int
    s_begin: int = 0
    s_end: int = 0
    ld: int = 0
    offset: int = 0


def _items(items: list[BatchItem]):
    arr = (capi.rng_batch_item * len(items))()
    for i, it in enumerate(items):
        assert it.out.is_cuda and it.out.is_contiguous()
        s_end = it.s_end or it.gen.n_streams
        ld = it.ld or it.gen.n_streams
        if it.n_per_stream:
            need = it.offset + (it.n_per_stream - 1) * ld + (s_end - it.s_begin)
            assert it.out.numel() >= need
        arr[i].h = it.gen.h
        arr[i].n_per_stream = it.n_per_stream
        arr[i].out = it.out.data_ptr() + 4 * it.offset
        arr[i].fmt = it.fmt
        arr[i].s_begin = it.s_begin
        arr[i].s_end = it.s_end
        arr[i].ld = it.ld
    return arr


class Plan:
    """A batched launch over many generators (rng_plan_*).  launch() enqueues
    one persistent kernel and can be captured in a CUDA graph."""

    def __init__(self, items: list[BatchItem], threads: int = 0, ctas_per_sm: int = 0):
        self._keep = items  # the plan refers to these tensors and handles
        arr = _items(items)
        p = capi.lib().rng_plan_create(arr, len(items), threads, ctas_per_sm)
        if not p:
            raise capi.RngError(capi.lib().rng_last_error(), "rng_plan_create")
        self.p = p

    @property
    def tiles(self) -> int:
        return int(capi.lib().rng_plan_tiles(self.p))

    @property
    def shape(self) -> tuple[int, int]:
        t, g = ctypes.c_int(), ctypes.c_int()
        capi.check(capi.lib().rng_plan_shape(self.p, ctypes.byref(t), ctypes.byref(g)))
        return t.value, g.value

    def refill(self, items: list[BatchItem], stream: torch.cuda.Stream | None = None) -> None:
        """New work list for the next launch on `stream` (rng_plan_refill)."""
        arr = _items(items)
        capi.check(capi.lib().rng_plan_refill(self.p, arr, len(items),
                                              ctypes.c_void_p(_stream_ptr(stream))),
                   "rng_plan_refill")
        self._keep = items

    def launch(self, stream: torch.cuda.Stream | None = None) -> None:
        capi.check(capi.lib().rng_plan_launch(self.p, ctypes.c_void_p(_stream_ptr(stream))),
                   "rng_plan_launch")

    def close(self) -> None:
        if getattr(self, "p", None):
            capi.lib().rng_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate_batch(items: list[BatchItem], stream: torch.cuda.Stream | None = None) -> None:
    arr = _items(items)
    capi.check(capi.lib().rng_generate_batch(arr, len(items),
                                             ctypes.c_void_p(_stream_ptr(stream))),
               "rng_generate_batch")
