"""Writes tests/golden/multipliers_b32.json from the oracle alone.

The MWC multiplier table is the list of a < 2^32, largest first, for which
a * 2^32 - 1 is a safe prime (the multiplier condition of the paper's MWC
background section).  Stream s uses entry s.  Tables of 2^20 and 2^22
entries take the single-threaded oracle minutes to rebuild, so this script
stores, for the prefixes the workloads use, the SHA-256 of the table (as
little-endian uint32 bytes) and its last entry, plus the entries at a fixed
set of sampled indices.  Tests compare the device-built table against the
digests and use the sampled entries as oracle inputs.

Run:  python tests/golden/make_multiplier_golden.py   (about two minutes on
eight cores; it calls nothing outside oracle/).
"""
from __future__ import annotations

import hashlib
import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402

PREFIXES = [4096, 1 << 20, 1 << 22]
OUT = Path(__file__).resolve().parent / "multipliers_b32.json"


def sample_indices(k_max: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(20110110))
    idx = set(range(0, 256))
    for k in PREFIXES:
        idx.update(range(max(0, k - 64), k))
    idx.update(rng.choice(k_max, size=2048, replace=False).tolist())
    return np.array(sorted(idx), dtype=np.int64)


def main() -> None:
    t0 = time.time()
    table = oracle.multipliers(PREFIXES[-1], 32)
    assert len(table) == PREFIXES[-1]
    assert np.all(np.diff(table.astype(np.int64)) < 0)
    doc = {
        "what": "MWC base-2^32 multipliers: a < 2^32 with a*2^32-1 a safe "
                "prime, largest first; entry s belongs to stream s",
        "citation": "arXiv:1101.1846, background section on multiply-with-"
                    "carry (safe-prime condition on a*b-1) and the MWC kernel "
                    "section (one multiplier per thread)",
        "generated_by": "tests/golden/make_multiplier_golden.py (oracle only)",
        "prefix": {},
        "sample_index": [],
        "sample_a": [],
    }
    for k in PREFIXES:
        pre = np.ascontiguousarray(table[:k]).astype("<u4")
        doc["prefix"][str(k)] = {
            "sha256": hashlib.sha256(pre.tobytes()).hexdigest(),
            "last": int(pre[-1]),
        }
    idx = sample_indices(PREFIXES[-1])
    doc["sample_index"] = idx.tolist()
    doc["sample_a"] = table[idx].astype(np.int64).tolist()
    OUT.write_text(json.dumps(doc, separators=(",", ":")) + "\n")
    print(f"wrote {OUT} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
