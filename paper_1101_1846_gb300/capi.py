"""ctypes binding of the C-ABI in include/rng.h and include/rng_tune.h.

Argument marshalling only: every step of generation runs in the CUDA library
libgbrng.so.  Functions keep the C names.  Loading fails loudly when the
library has not been built (there is no fallback of any kind).
"""
from __future__ import annotations

import ctypes
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libgbrng.so"

RNG_MWC32, RNG_XOR128, RNG_KISS = 0, 1, 2
RNG_MWC16X2, RNG_XORSHIFT8, RNG_KISS_XOR = 3, 4, 5
RNG_U32, RNG_F32 = 0, 1
RNG_OK, RNG_ERR_ARG, RNG_ERR_OOM, RNG_ERR_CUDA = 0, -1, -2, -3
RNG_ERR_TIMEOUT, RNG_ERR_BUSY, RNG_ERR_NODEV = -4, -5, -6
RNG_MAX_STREAMS_MWC = 1 << 22
RNG_MAX_STREAMS_XOR = 1 << 30
RNG_MAX_STREAMS_MWC16 = 392 * 391 // 2
RNG_MAX_STREAMS_XS8 = 1 << 28
RNG_BATTERY_BIRTHDAY_MAX = 1 << 21

RNG_SUM_U32, RNG_SUM_U24, RNG_DISC = 0, 1, 2

KINDS = {"mwc": RNG_MWC32, "xor128": RNG_XOR128, "kiss": RNG_KISS, "mwc16x2": RNG_MWC16X2,
         "xorshift8": RNG_XORSHIFT8, "kiss_xor": RNG_KISS_XOR}
FMTS = {"u32": RNG_U32, "f32": RNG_F32}


class rng_batch_item(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("n_per_stream", ctypes.c_uint64),
                ("out", ctypes.c_void_p), ("fmt", ctypes.c_int),
                ("s_begin", ctypes.c_uint64), ("s_end", ctypes.c_uint64),
                ("ld", ctypes.c_uint64)]


class rng_device_view(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("device", ctypes.c_int),
                ("state_words", ctypes.c_int), ("n_streams", ctypes.c_uint64),
                ("state", ctypes.c_void_p), ("mult", ctypes.c_void_p)]


class rng_battery_counts(ctypes.Structure):
    _fields_ = [("n_outputs", ctypes.c_uint64), ("ones", ctypes.c_uint64),
                ("bytes", ctypes.c_uint64 * 256), ("serial", ctypes.c_uint64 * 256),
                ("birthday_samples", ctypes.c_uint64), ("birthday", ctypes.c_uint64 * 16)]


# name -> (restype, argtypes); every symbol declared in include/*.h
SIGNATURES = {
    "rng_create": (ctypes.c_void_p, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]),
    "rng_create_range": (ctypes.c_void_p, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_uint64]),
    "rng_destroy": (None, [ctypes.c_void_p]),
    "rng_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "rng_n_streams": (ctypes.c_uint64, [ctypes.c_void_p]),
    "rng_state_words": (ctypes.c_int, [ctypes.c_void_p]),
    "rng_generate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                    ctypes.c_int]),
    "rng_generate_range": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                                          ctypes.c_int]),
    "rng_generate_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_int]),
    "rng_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "rng_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "rng_multipliers": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_void_p]),
    "rng_mwc16_pairs": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_void_p]),
    "rng_generate_reduce": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                           ctypes.c_void_p]),
    "rng_jump": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "rng_battery": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.POINTER(rng_battery_counts), ctypes.c_void_p]),
    "rng_get_device_view": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(rng_device_view)]),
    "rng_plan_create": (ctypes.c_void_p, [ctypes.POINTER(rng_batch_item), ctypes.c_size_t,
                                          ctypes.c_int, ctypes.c_int]),
    "rng_plan_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "rng_plan_refill": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(rng_batch_item),
                                       ctypes.c_size_t, ctypes.c_void_p]),
    "rng_plan_tiles": (ctypes.c_uint64, [ctypes.c_void_p]),
    "rng_plan_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "rng_plan_destroy": (None, [ctypes.c_void_p]),
    "rng_generate_batch": (ctypes.c_int, [ctypes.POINTER(rng_batch_item), ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "rng_generate_batch_noalloc": (ctypes.c_int, [ctypes.POINTER(rng_batch_item),
                                                  ctypes.c_size_t, ctypes.c_void_p]),
    "rng_server_create": (ctypes.c_void_p, [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]),
    "rng_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "rng_server_submit_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_void_p]),
    "rng_server_progress": (ctypes.c_int, [ctypes.c_void_p]),
    "rng_server_release_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_size_t]),
    "rng_server_drain": (ctypes.c_int, [ctypes.c_void_p]),
    "rng_server_take": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "rng_server_result": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "rng_server_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]),
    "rng_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "rng_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "rng_server_set_tick_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "rng_server_set_plan_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "rng_server_destroy": (None, [ctypes.c_void_p]),
    "rng_last_error": (ctypes.c_int, []),
    "rng_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "gbrng_set_launch": (ctypes.c_int, [ctypes.c_int] * 5),
    "gbrng_set_launch_class": (ctypes.c_int, [ctypes.c_int] * 6),
    "gbrng_get_launch_class": (ctypes.c_int, [ctypes.c_int] * 3 +
                               [ctypes.POINTER(ctypes.c_int)] * 3),
    "gbrng_get_launch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int] +
                         [ctypes.POINTER(ctypes.c_int)] * 3),
    "gbrng_set_launch_ctas": (ctypes.c_int, [ctypes.c_int] * 4),
    "gbrng_get_launch_ctas": (ctypes.c_int, [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int)]),
    "gbrng_set_row_ctas": (ctypes.c_int, [ctypes.c_int] * 4),
    "gbrng_get_row_ctas": (ctypes.c_int, [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int)]),
    "gbrng_set_split": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "gbrng_get_split": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gbrng_probe_write": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p]),
    "gbrng_probe_int": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]),
}

_lib = None


class RngError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().rng_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if libgbrng.so has not been built."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -m paper_1101_1846_gb300.build, or __graft_entry__.build())")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str = "") -> int:
    if status < 0:
        raise RngError(status, what)
    return status


def __getattr__(name):
    # capi.rng_generate(...) etc. call straight into the library
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
