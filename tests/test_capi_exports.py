"""The C-ABI library builds, loads and exports every function declared in
include/*.h; host-side argument checks work without a GPU."""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

import pytest

from paper_1101_1846_gb300 import build, capi

ROOT = Path(__file__).resolve().parents[1]


def declared_functions() -> set[str]:
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.lib()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for must in ("rng_create", "rng_generate", "rng_destroy", "rng_generate_host",
                 "rng_get_state", "rng_set_state", "rng_plan_create", "rng_plan_launch",
                 "rng_generate_batch", "rng_multipliers", "rng_last_error",
                 "rng_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name
    assert set(capi.SIGNATURES) == declared_functions()


def test_strerror_covers_statuses(lib):
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert lib.rng_strerror(s) not in (None, b"unknown status")
    assert lib.rng_strerror(-99) == b"unknown status"


def test_argument_checks_need_no_gpu(lib):
    # invalid kind / zero or oversized stream counts are rejected first
    assert lib.rng_create(7, 16, 1) is None
    assert lib.rng_last_error() == capi.RNG_ERR_ARG
    assert lib.rng_create(0, 0, 1) is None
    assert lib.rng_last_error() == capi.RNG_ERR_ARG
    assert lib.rng_create(2, capi.RNG_MAX_STREAMS_MWC + 1, 1) is None
    assert lib.rng_last_error() == capi.RNG_ERR_ARG
    assert lib.rng_create_range(2, capi.RNG_MAX_STREAMS_MWC, 1, 1) is None
    assert lib.rng_last_error() == capi.RNG_ERR_ARG
    assert lib.rng_create_range(1, 2**64 - 1, 2, 1) is None  # s_begin + n wraps
    assert lib.rng_last_error() == capi.RNG_ERR_ARG
    assert lib.rng_generate(None, 4, None, 0) == capi.RNG_ERR_ARG
    assert lib.rng_get_state(None, None, 0) == capi.RNG_ERR_ARG
    assert lib.rng_plan_create(None, 0, 0, 0) is None
    assert lib.gbrng_set_launch(0, 0, 3, 256, 0) == capi.RNG_ERR_ARG
    assert lib.gbrng_set_launch(0, 0, 1, 100, 0) == capi.RNG_ERR_ARG
    lib.rng_destroy(None)
    lib.rng_plan_destroy(None)


def test_launch_shape_roundtrip(lib):
    v, b, h = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.gbrng_get_launch(2, 1, ctypes.byref(v), ctypes.byref(b), ctypes.byref(h)) == 0
    old = (v.value, b.value, h.value)
    assert lib.gbrng_set_launch(2, 1, 2, 128, 1) == 0
    lib.gbrng_get_launch(2, 1, ctypes.byref(v), ctypes.byref(b), ctypes.byref(h))
    assert (v.value, b.value, h.value) == (2, 128, 1)
    assert lib.gbrng_set_launch(2, 1, *old) == 0


def test_launch_shape_classes(lib):
    """Class 1 is what gbrng_set_launch / gbrng_get_launch address; class 0
    (calls of fewer than 2^21 streams) is separate."""
    v, b, h = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ref = (ctypes.byref(v), ctypes.byref(b), ctypes.byref(h))
    assert lib.gbrng_get_launch_class(1, 1, 0, *ref) == 0
    small = (v.value, b.value, h.value)
    assert lib.gbrng_get_launch_class(1, 1, 1, *ref) == 0
    large = (v.value, b.value, h.value)
    assert lib.gbrng_set_launch(1, 1, 2, 64, 0) == 0
    lib.gbrng_get_launch_class(1, 1, 1, *ref)
    assert (v.value, b.value, h.value) == (2, 64, 0)
    lib.gbrng_get_launch_class(1, 1, 0, *ref)
    assert (v.value, b.value, h.value) == small
    assert lib.gbrng_set_launch_class(1, 1, 2, 1, 64, 0) == capi.RNG_ERR_ARG
    assert lib.gbrng_set_launch(1, 1, *large) == 0


def test_no_device_reports_nodev(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert lib.rng_create(0, 16, 1) is None
    assert lib.rng_last_error() == capi.RNG_ERR_NODEV


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the Python layer raises; nothing falls back
    to the host (run in a fresh interpreter so the loaded library of this
    process is not involved)."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from pathlib import Path\n"
        "from paper_1101_1846_gb300 import capi\n"
        "capi.LIB_PATH = Path(%r)\n"
        "from paper_1101_1846_gb300.generator import Generator\n"
        "try:\n"
        "    Generator(0, 16, 1)\n"
        "except RuntimeError as e:\n"
        "    print('raised', 'missing' in str(e))\n"
        "else:\n"
        "    print('no error')\n"
    ) % (str(ROOT), str(tmp_path / "absent" / "libgbrng.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.stdout.strip() == "raised True", r.stdout + r.stderr[-2000:]


def test_row_ctas_roundtrip(lib):
    """The CTAs-per-SM choice of the barrier-synced kernels, per (kind, fmt,
    realigned): 0 or 1, anything else rejected; defaults one CTA for the
    memory-bound forms, as many as fit for KISS FP32."""
    v = ctypes.c_int()
    assert lib.gbrng_get_row_ctas(2, 1, 1, ctypes.byref(v)) == 0 and v.value == 0
    assert lib.gbrng_get_row_ctas(0, 0, 1, ctypes.byref(v)) == 0 and v.value == 1
    assert lib.gbrng_set_row_ctas(0, 0, 1, 0) == 0
    lib.gbrng_get_row_ctas(0, 0, 1, ctypes.byref(v))
    assert v.value == 0
    assert lib.gbrng_set_row_ctas(0, 0, 1, 1) == 0
    for bad in [(6, 0, 0, 1), (0, 2, 0, 1), (0, 0, 2, 1), (0, 0, 0, 2), (0, 0, 0, -1)]:
        assert lib.gbrng_set_row_ctas(*bad) == capi.RNG_ERR_ARG
    assert lib.gbrng_get_row_ctas(0, 0, 0, None) == capi.RNG_ERR_ARG


def test_launch_ctas_roundtrip(lib):
    """One CTA per SM for the aligned vector kernel, per (kind, fmt, size
    class): kept when the shape itself is set, 0 or 1 only."""
    v, b, h, one = (ctypes.c_int() for _ in range(4))
    assert lib.gbrng_get_launch_ctas(2, 1, 1, ctypes.byref(one)) == 0 and one.value == 1
    assert lib.gbrng_get_launch_ctas(2, 1, 0, ctypes.byref(one)) == 0 and one.value == 0
    lib.gbrng_get_launch_class(2, 1, 1, ctypes.byref(v), ctypes.byref(b), ctypes.byref(h))
    old = (v.value, b.value, h.value)
    assert lib.gbrng_set_launch_class(2, 1, 1, 2, 256, 1) == 0
    lib.gbrng_get_launch_ctas(2, 1, 1, ctypes.byref(one))
    assert one.value == 1
    assert lib.gbrng_set_launch_ctas(2, 1, 1, 0) == 0
    lib.gbrng_get_launch_ctas(2, 1, 1, ctypes.byref(one))
    assert one.value == 0
    assert lib.gbrng_set_launch_ctas(2, 1, 1, 1) == 0
    assert lib.gbrng_set_launch_class(2, 1, 1, *old) == 0
    for bad in [(6, 0, 0, 1), (0, 2, 0, 1), (0, 0, 2, 1), (0, 0, 0, 2)]:
        assert lib.gbrng_set_launch_ctas(*bad) == capi.RNG_ERR_ARG
    assert lib.gbrng_get_launch_ctas(0, 0, 0, None) == capi.RNG_ERR_ARG
