"""Oracle for the Marsaglia generators of arXiv:1101.1846 (Hissoiny, Despres
and Ozell, "Using graphics processing units to generate random numbers").

TEST INFRASTRUCTURE ONLY.  A thin ctypes wrapper around ``oracle.c``: plain,
slow, single-threaded C that states each recurrence literally.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package; the product library never does and
shares no code with it.

Kinds: 0 = MWC base 2^32 (Eq. 2-3), 1 = xor128 (Marsaglia 2003), 2 = KISS
(MWC + xorshift32 of Eq. 6 + LCG of Eq. 7, summed mod 2^32), and the paper's
own generators: 3 = two base-2^16 MWCs joined as (z << 16) + w, 4 = Panneton's
r = 8 XorShift (Eq. 5), 5 = KISS as (MWC16X2 xor LCG) + xorshift32.
Formats: 0 = uint32, 1 = float32 uniform (u >> 8) * 2^-24.
State: words(kind) uint32 words per stream (8 for kind 4, else 4; see
``oracle.h``); kinds 0 and 2 take one multiplier per stream, kinds 3 and 5
one packed pair of 16-bit multipliers.
"""
from __future__ import annotations

import contextlib
import ctypes
import multiprocessing as mp
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
BUILD = HERE / "_build"
LIB = BUILD / "liboracle.so"
SOURCES = [HERE / "oracle.c", HERE / "oracle.h"]

MWC, XOR128, KISS, MWC16X2, XORSHIFT8, KISS_XOR = 0, 1, 2, 3, 4, 5
U32, F32 = 0, 1
HAS_MULT = (MWC, KISS, MWC16X2, KISS_XOR)


def words(kind: int) -> int:
    """State words per stream in the oracle's layout."""
    return 8 if kind == XORSHIFT8 else 4

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_lib = None


def build(force: bool = False) -> Path:
    """Compile oracle.c into a shared object (gcc, -O2, no vector flags)."""
    BUILD.mkdir(exist_ok=True)
    stale = not LIB.exists() or any(
        s.stat().st_mtime > LIB.stat().st_mtime for s in SOURCES)
    if force or stale:
        tmp = BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                        "-Wall", "-Wextra", "-o", str(tmp),
                        str(HERE / "oracle.c")], check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


@contextlib.contextmanager
def using(path):
    """Route every call through another build of oracle.c for the duration
    of the block (the tests that plant a mistake in a copy use this)."""
    global _lib
    saved = _lib
    _lib = _load(Path(path))
    try:
        yield
    finally:
        _lib = saved


def compile_variant(src_text: str, out_path) -> Path:
    """Compile a modified copy of oracle.c (tests only)."""
    out_path = Path(out_path)
    c = out_path.with_suffix(".c")
    c.write_text(src_text)
    (out_path.parent / "oracle.h").write_text((HERE / "oracle.h").read_text())
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o",
                    str(out_path), str(c)], check=True)
    return out_path


def _load(path: Path):
    L = ctypes.CDLL(str(path))
    u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "oracle_mulmod_u64": (u64, [u64, u64, u64]),
        "oracle_powmod_u64": (u64, [u64, u64, u64]),
        "oracle_is_prime_u64": (i32, [u64]),
        "oracle_is_safe_multiplier": (i32, [u64, i32]),
        "oracle_multipliers": (u64, [i32, u64, u64, _u32p]),
        "oracle_multipliers_range": (u64, [i32, u64, u64, _u32p, u64]),
        "oracle_mwc16_pairs": (u64, [u64, _u32p]),
        "oracle_mwc16x2_step": (u32, [u32, _u32p]),
        "oracle_xorshift8_step": (u32, [_u32p]),
        "oracle_kiss_xor_step": (u32, [u32, _u32p]),
        "oracle_state_words": (i32, [i32]),
        "oracle_xorshift8_jump": (None, [_u32p, u64]),
        "oracle_splitmix64": (u64, [_u64p]),
        "oracle_seed_stream": (None, [i32, u32, u64, u64, _u32p]),
        "oracle_seed_streams": (None, [i32, _u32p, u64, _u64p, u64, _u32p]),
        "oracle_mwc_step": (u32, [u32, _u32p, _u32p, i32]),
        "oracle_xor128_step": (u32, [_u32p]),
        "oracle_xorshift32_step": (u32, [_u32p]),
        "oracle_lcg_step": (u32, [_u32p]),
        "oracle_kiss_step": (u32, [u32, _u32p]),
        "oracle_step": (u32, [i32, u32, _u32p]),
        "oracle_to_unit_f32": (ctypes.c_float, [u32]),
        "oracle_stream": (None, [i32, u32, _u32p, u64, i32, ctypes.c_void_p]),
        "oracle_generate": (None, [i32, u64, _u32p, _u32p, u64, i32,
                                   ctypes.c_void_p]),
        "oracle_sum_u32": (u64, [_u32p, u64]),
        "oracle_sum_u24": (u64, [_u32p, u64]),
        "oracle_disc_count": (u64, [_u32p, u64]),
        "oracle_reduce": (i32, [i32, u64, _u32p, _u32p, u64, i32, _u64p]),
        "oracle_mwc_jump": (None, [u32, _u32p, _u32p, u64, i32]),
        "oracle_xor128_jump": (None, [_u32p, u64]),
        "oracle_xorshift32_jump": (None, [_u32p, u64]),
        "oracle_lcg_jump": (None, [_u32p, u64]),
        "oracle_jump": (None, [i32, u32, _u32p, u64]),
        "oracle_bat_ones": (u64, [_u32p, u64]),
        "oracle_bat_bytes": (None, [_u32p, u64, _u64p]),
        "oracle_bat_serial": (None, [_u32p, u64, u64, _u64p]),
        "oracle_bat_birthday": (u64, [_u32p, u64, u64, u64, _u64p]),
        "oracle_mwc_period": (u64, [u32, u32, u32, i32, u64]),
        "oracle_xorshift32_period": (u64, [u32]),
        "oracle_lcg_period": (u64, [u32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _p32(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(_u32p)


def _p64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(_u64p)


# ---------------------------------------------------------------- numbers
def is_prime(n: int) -> bool:
    return bool(lib().oracle_is_prime_u64(n))


def is_safe_multiplier(a: int, log2b: int = 32) -> bool:
    return bool(lib().oracle_is_safe_multiplier(a, log2b))


def powmod(b: int, e: int, m: int) -> int:
    return int(lib().oracle_powmod_u64(b, e, m))


def multipliers_range(a_hi: int, a_lo: int, log2b: int = 32) -> np.ndarray:
    """Every valid multiplier in [a_lo, a_hi], descending."""
    cap = max(16, (a_hi - a_lo + 1) // 64 + 64)
    while True:
        out = np.zeros(cap, np.uint32)
        n = int(lib().oracle_multipliers_range(log2b, a_hi, a_lo, _p32(out), cap))
        if n <= cap:
            return out[:n].copy()
        cap = n


def _range_worker(args):
    a_hi, a_lo, log2b = args
    return multipliers_range(a_hi, a_lo, log2b)


def multipliers(k: int, log2b: int = 32, procs: int | None = None,
                chunk: int = 1 << 22) -> np.ndarray:
    """The first k valid multipliers below b, largest first (Sec. on MWC:
    a*b - 1 a safe prime).  Large tables are searched over disjoint ranges
    of a in worker processes (spawned, never forked) and concatenated in
    order; each range is the same single-threaded scan."""
    a_top = (1 << log2b) - 1
    if k <= 16384 or (procs or 0) == 1:
        out = np.zeros(k, np.uint32)
        n = int(lib().oracle_multipliers(log2b, a_top, k, _p32(out)))
        return out[:n]
    procs = procs or os.cpu_count() or 1
    ranges = []
    hi = a_top
    while hi >= 1:
        lo = max(1, hi - chunk + 1)
        ranges.append((hi, lo, log2b))
        hi = lo - 1
    parts, total = [], 0
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for part in pool.imap(_range_worker, ranges):
            parts.append(part)
            total += len(part)
            if total >= k:
                pool.terminate()
                break
    return np.concatenate(parts)[:k]


# ---------------------------------------------------------------- seeding
def splitmix64(z: int) -> tuple[int, int]:
    """One splitmix64 draw: returns (new_state, output)."""
    s = ctypes.c_uint64(z)
    r = lib().oracle_splitmix64(ctypes.byref(s))
    return int(s.value), int(r)


def seed_streams(kind: int, a: np.ndarray | None, seed: int,
                 s_ids: np.ndarray) -> np.ndarray:
    """Initial state (n, words(kind)) uint32 of the streams with indices
    s_ids; a[i] is the multiplier (or packed pair) of stream s_ids[i]."""
    s_ids = np.ascontiguousarray(s_ids, dtype=np.uint64)
    n = len(s_ids)
    st = np.zeros((n, words(kind)), np.uint32)
    ap = None
    if kind in HAS_MULT:
        a = np.ascontiguousarray(a, dtype=np.uint32)
        assert len(a) == n
        ap = _p32(a)
    lib().oracle_seed_streams(kind, ap, seed & (2**64 - 1), _p64(s_ids), n, _p32(st))
    return st


# ---------------------------------------------------------------- steps
def mwc_step(a: int, x: int, c: int, log2b: int = 32) -> tuple[int, int]:
    X, C = ctypes.c_uint32(x), ctypes.c_uint32(c)
    lib().oracle_mwc_step(a, ctypes.byref(X), ctypes.byref(C), log2b)
    return int(X.value), int(C.value)


def _st(st):
    arr = (ctypes.c_uint32 * 4)(*[int(v) for v in st])
    return arr


def xor128_step(st) -> tuple[int, list]:
    arr = _st(st)
    out = lib().oracle_xor128_step(arr)
    return int(out), list(arr)


def xorshift32_step(y: int) -> int:
    Y = ctypes.c_uint32(y)
    return int(lib().oracle_xorshift32_step(ctypes.byref(Y)))


def lcg_step(z: int) -> int:
    Z = ctypes.c_uint32(z)
    return int(lib().oracle_lcg_step(ctypes.byref(Z)))


def kiss_step(a: int, st) -> tuple[int, list]:
    arr = _st(st)
    out = lib().oracle_kiss_step(a, arr)
    return int(out), list(arr)


def mwc16x2_step(a_pair: int, st) -> tuple[int, list]:
    arr = (ctypes.c_uint32 * 2)(*[int(v) for v in st[:2]])
    out = lib().oracle_mwc16x2_step(a_pair, arr)
    return int(out), list(arr)


def xorshift8_step(st) -> tuple[int, list]:
    arr = (ctypes.c_uint32 * 8)(*[int(v) for v in st])
    out = lib().oracle_xorshift8_step(arr)
    return int(out), list(arr)


def kiss_xor_step(a_pair: int, st) -> tuple[int, list]:
    arr = _st(st)
    out = lib().oracle_kiss_xor_step(a_pair, arr)
    return int(out), list(arr)


def mwc16_pairs(k: int) -> np.ndarray:
    """The first k packed multiplier pairs of the paper's two-part MWC."""
    out = np.zeros(k, np.uint32)
    got = lib().oracle_mwc16_pairs(k, _p32(out))
    return out[:got]


def multipliers_for(kind: int, n: int) -> np.ndarray | None:
    """The per-stream multipliers (or packed pairs) of the first n streams."""
    if kind in (MWC, KISS):
        return multipliers(n, 32)
    if kind in (MWC16X2, KISS_XOR):
        return mwc16_pairs(n)
    return None


def to_unit_f32(u: int) -> float:
    return float(np.float32(lib().oracle_to_unit_f32(u)))


# ---------------------------------------------------------------- calls
def generate(kind: int, a: np.ndarray | None, state: np.ndarray,
             n_per_stream: int, fmt: int) -> tuple[np.ndarray, np.ndarray]:
    """One generate call over len(state) streams.  Returns (out, new_state)
    with out of shape (n_per_stream, n_streams): out[j, s] is output j of
    stream s (the stream-interleaved layout)."""
    state = np.array(state, dtype=np.uint32, order="C", copy=True)
    assert state.shape[1] == words(kind)
    n = state.shape[0]
    out = np.zeros((n_per_stream, n), np.uint32 if fmt == U32 else np.float32)
    ap = None
    if kind in HAS_MULT:
        a = np.ascontiguousarray(a, dtype=np.uint32)
        assert len(a) >= n
        ap = _p32(a)
    lib().oracle_generate(kind, n, ap, _p32(state), n_per_stream, fmt,
                          out.ctypes.data_as(ctypes.c_void_p))
    return out, state


def stream(kind: int, a: int, st, n: int, fmt: int) -> tuple[np.ndarray, np.ndarray]:
    """n outputs of one stream, contiguous; returns (out, new_state)."""
    arr = np.array(st, dtype=np.uint32)
    assert len(arr) == words(kind)
    out = np.zeros(n, np.uint32 if fmt == U32 else np.float32)
    lib().oracle_stream(kind, a, _p32(arr), n, fmt,
                        out.ctypes.data_as(ctypes.c_void_p))
    return out, arr


# ------------------------------------------------------------ consumers
SUM_U32, SUM_U24, DISC = 0, 1, 2


def sum_u32(u: np.ndarray) -> int:
    u = np.ascontiguousarray(u, dtype=np.uint32)
    return int(lib().oracle_sum_u32(_p32(u), len(u)))


def sum_u24(u: np.ndarray) -> int:
    u = np.ascontiguousarray(u, dtype=np.uint32)
    return int(lib().oracle_sum_u24(_p32(u), len(u)))


def disc_count(u: np.ndarray) -> int:
    u = np.ascontiguousarray(u, dtype=np.uint32)
    return int(lib().oracle_disc_count(_p32(u), len(u)))


def reduce(kind: int, a: np.ndarray | None, state: np.ndarray, n_per_stream: int,
           op: int) -> tuple[np.ndarray, np.ndarray]:
    """Every stream advances n_per_stream steps; returns (out, new_state)
    with out[s] the consumer `op` over stream s's outputs (uint64)."""
    state = np.array(state, dtype=np.uint32, order="C", copy=True)
    assert state.shape[1] == words(kind)
    n = state.shape[0]
    out = np.zeros(n, np.uint64)
    ap = None
    if kind in HAS_MULT:
        a = np.ascontiguousarray(a, dtype=np.uint32)
        assert len(a) >= n
        ap = _p32(a)
    rc = lib().oracle_reduce(kind, n, ap, _p32(state), n_per_stream, op, _p64(out))
    assert rc == 0, "oracle_reduce: out of memory"
    return out, state


# ----------------------------------------------------------------- jumps
def jump(kind: int, a: int, st, k: int) -> np.ndarray:
    """State of one stream k steps after st (words(kind) uint32 words)."""
    arr = np.array(st, dtype=np.uint32)
    assert len(arr) == words(kind)
    lib().oracle_jump(kind, int(a), _p32(arr), int(k))
    return arr


def jump_streams(kind: int, a: np.ndarray | None, state: np.ndarray, k: int) -> np.ndarray:
    out = np.array(state, dtype=np.uint32, order="C", copy=True)
    for s in range(out.shape[0]):
        lib().oracle_jump(kind, int(a[s]) if a is not None else 0, _p32(out[s]), int(k))
    return out


def mwc_jump(a: int, x: int, c: int, k: int, log2b: int = 32) -> tuple[int, int]:
    X, C = ctypes.c_uint32(x), ctypes.c_uint32(c)
    lib().oracle_mwc_jump(a, ctypes.byref(X), ctypes.byref(C), k, log2b)
    return int(X.value), int(C.value)


def xorshift32_jump(y: int, k: int) -> int:
    Y = ctypes.c_uint32(y)
    lib().oracle_xorshift32_jump(ctypes.byref(Y), k)
    return int(Y.value)


def lcg_jump(z: int, k: int) -> int:
    Z = ctypes.c_uint32(z)
    lib().oracle_lcg_jump(ctypes.byref(Z), k)
    return int(Z.value)


# --------------------------------------------------------------- battery
BIRTHDAY_MAX = 1 << 21  # oracle.h's ORACLE_BAT_BIRTHDAY_MAX


def battery_counts(u: np.ndarray, birthday_max: int = BIRTHDAY_MAX) -> dict:
    """Counts of the four battery tests over u of shape (n_per_stream,
    n_streams), stream-interleaved uint32; at most birthday_max birthday
    samples."""
    u = np.ascontiguousarray(u, dtype=np.uint32)
    rows, n = u.shape
    byte, serial, bday = (np.zeros(256, np.uint64), np.zeros(256, np.uint64),
                          np.zeros(16, np.uint64))
    L = lib()
    ones = int(L.oracle_bat_ones(_p32(u), u.size))
    L.oracle_bat_bytes(_p32(u), u.size, _p64(byte))
    L.oracle_bat_serial(_p32(u), n, rows, _p64(serial))
    samples = int(L.oracle_bat_birthday(_p32(u), n, rows, birthday_max, _p64(bday)))
    return {"n_outputs": int(u.size), "ones": ones, "bytes": byte, "serial": serial,
            "birthday_samples": samples, "birthday": bday}


# ---------------------------------------------------------------- periods
def mwc_period(a: int, x0: int, c0: int, log2b: int, limit: int) -> int:
    return int(lib().oracle_mwc_period(a, x0, c0, log2b, limit))


def xorshift32_period(y0: int) -> int:
    return int(lib().oracle_xorshift32_period(y0))


def lcg_period(z0: int) -> int:
    return int(lib().oracle_lcg_period(z0))
