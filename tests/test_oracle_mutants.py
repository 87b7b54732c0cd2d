"""Plants plausible mistakes in copies of oracle.c (on the CPU) and checks
that the pins in test_oracle_pins.py catch each one."""
from __future__ import annotations

from functools import partial

import numpy as np
import pytest

import oracle
import test_oracle_battery as bat
import test_oracle_consumers_jump as cj
import test_oracle_paper_variants as pv
import test_oracle_pins as pins
import test_oracle_seeding as sd

SRC = (oracle.HERE / "oracle.c").read_text()

# (name, text in oracle.c, replacement, pin expected to fail)
MUTANTS = [
    ("xor128 shift 11->10", "uint32_t t = x ^ (x << 11);", "uint32_t t = x ^ (x << 10);",
     pins.check_xor128_full_period_gf2),
    ("xor128 shift 19->18", "st[3] = w ^ (w >> 19)", "st[3] = w ^ (w >> 18)",
     pins.check_xor128_full_period_gf2),
    ("xor128 drops t>>8", "(w >> 19) ^ t ^ (t >> 8);", "(w >> 19) ^ t;",
     pins.check_xor128_full_period_gf2),
    ("xor128 outputs old w", "    return st[3];\n}\n\n/* Eq. 6",
     "    return w;\n}\n\n/* Eq. 6", pins.check_xor128_output_is_new_last_word),
    ("xorshift32 shift 17->15", "v ^= v >> 17;", "v ^= v >> 15;",
     pins.check_xorshift32_full_period_gf2),
    ("xorshift32 right/left swapped", "v ^= v >> 17;", "v ^= v << 17;",
     pins.check_xorshift32_full_period_gf2),
    ("LCG increment off by one", "+ 1234567ull", "+ 1234568ull",
     pins.check_lcg_constants),
    ("LCG multiplier typo", "69069ull *", "69096ull *",
     pins.check_lcg_constants),
    ("MWC x and carry transposed",
     "*x = (uint32_t)(t % b);\n    *c = (uint32_t)(t / b);",
     "*c = (uint32_t)(t % b);\n    *x = (uint32_t)(t / b);",
     pins.check_mwc_lehmer_closed_form),
    ("MWC carry dropped", "(uint64_t)a * (uint64_t)(*x) + (uint64_t)(*c)",
     "(uint64_t)a * (uint64_t)(*x)", pins.check_mwc_period_base_2_16),
    ("KISS in the xor form", "((uint64_t)m + y + z)", "((uint64_t)(m ^ z) + y)",
     pins.check_kiss_is_sum_of_parts),
    ("KISS drops the LCG", "((uint64_t)m + y + z)", "((uint64_t)m + y)",
     pins.check_kiss_is_sum_of_parts),
    ("uniform uses 23 bits", "(float)(u >> 8)", "(float)(u >> 9)",
     pins.check_uniform_exact),
    ("Miller-Rabin with 7 bases", "for (int i = 0; i < 12; ++i) {\n        uint64_t x",
     "for (int i = 0; i < 7; ++i) {\n        uint64_t x",
     pins.check_strong_pseudoprime),
    ("safe-prime test drops q", "return (vq == 1 || miller_rabin(q)) && ",
     "return 1 && ", pins.check_mwc16_multiplier_count),
    ("trial division misses 3", "for (int i = 3; i < 1024; i += 2)",
     "for (int i = 5; i < 1024; i += 2)", pins.check_mwc16_multipliers_brute_force),
    ("sum skips the first output", "for (uint64_t j = 0; j < n; ++j)\n        s += (uint64_t)u[j];",
     "for (uint64_t j = 1; j < n; ++j)\n        s += (uint64_t)u[j];", cj.check_sum_closed_forms),
    ("24-bit sum keeps 25 bits", "s += (uint64_t)(u[j] >> 8);", "s += (uint64_t)(u[j] >> 7);",
     cj.check_sum_closed_forms),
    ("disc count uses 23 bits", "uint64_t X = u[2 * k] >> 8;", "uint64_t X = u[2 * k] >> 9;",
     cj.check_disc_lattice_count),
    ("disc count pairs overlap",
     "uint64_t X = u[2 * k] >> 8;\n        uint64_t Y = u[2 * k + 1] >> 8;",
     "uint64_t X = u[k] >> 8;\n        uint64_t Y = u[k + 1] >> 8;", cj.check_disc_lattice_count),
    ("disc radius squared is 2^47", "X * X + Y * Y < ((uint64_t)1 << 48)",
     "X * X + Y * Y < ((uint64_t)1 << 47)", cj.check_disc_estimates_pi),
    ("MWC jump: x and carry swapped", "*x = (uint32_t)(t / a);\n    *c = (uint32_t)(t % a);",
     "*c = (uint32_t)(t / a);\n    *x = (uint32_t)(t % a);", cj.check_jump_equals_stepping),
    ("MWC jump multiplies by b^k", "oracle_powmod_u64(a, k, p)",
     "oracle_powmod_u64((uint64_t)1 << log2b, k, p)", cj.check_mwc_jump_lehmer),
    ("GF(2) apply drops the top word", "for (int w = 0; w < 8; ++w)\n                r[w] ^= m->col[j][w];",
     "for (int w = 0; w < 3; ++w)\n                r[w] ^= m->col[j][w];", cj.check_jump_equals_stepping),
    ("GF(2) power uses the wrong bit", "if (k & 1)\n            gf2_mul(&result, &base, &result);",
     "if (k & 2)\n            gf2_mul(&result, &base, &result);", cj.check_jump_periods),
    ("LCG jump drops the increment", "RC = (BA * RC + BC) % m;", "RC = (BA * RC) % m;",
     cj.check_jump_equals_stepping),
    ("r=8 XorShift shift 9->8", "t1 ^= t1 << 9;", "t1 ^= t1 << 8;",
     pv.check_xorshift8_full_period),
    ("r=8 XorShift lag 5 read as lag 6", "uint32_t t5 = st[3] ^ (st[3] >> 3);",
     "uint32_t t5 = st[2] ^ (st[2] >> 3);", pv.check_xorshift8_lags),
    ("r=8 XorShift drops R^7", "uint32_t t8 = st[0] ^ (st[0] >> 7);", "uint32_t t8 = st[0];",
     pv.check_xorshift8_full_period),
    ("two-part MWC joined with or", "(((uint64_t)st[0] << 16) + st[1])",
     "(((uint64_t)st[0] << 16) | (st[1] & 0xFFFFu))", pv.check_mwc16x2_closed_form),
    ("two-part MWC parts swapped", "uint32_t a1 = a_pair & 0xFFFFu, a2 = a_pair >> 16;\n    uint32_t x = st[0]",
     "uint32_t a2 = a_pair & 0xFFFFu, a1 = a_pair >> 16;\n    uint32_t x = st[0]",
     pv.check_mwc16x2_closed_form),
    ("paper KISS in the sum form", "((uint64_t)(m ^ z) + y)", "((uint64_t)m + z + y)",
     pv.check_kiss_xor_is_parts),
    ("multiplier pairs reversed", "out[found++] = table[i] | (table[j] << 16);",
     "out[found++] = table[j] | (table[i] << 16);", pv.check_mwc16_pairs_lexicographic),
    ("frequency bins on 7 bits", "hist[u[i] >> 24]++;", "hist[u[i] >> 25]++;",
     bat.check_ones_and_bytes),
    ("serial pairs overlap", "for (uint64_t j = 0; j + 1 < n_per_stream; j += 2) {",
     "for (uint64_t j = 0; j + 1 < n_per_stream; j += 1) {", bat.check_serial_pairs_within_streams),
    ("birthday repeats of days, not spacings", "repeats += d[i] == d[i - 1];",
     "repeats += b[i] == b[i - 1];", bat.check_birthday_repeats),
    ("birthday days of 25 bits", "b[i] = u[(blk * 512 + i) * n_streams + s] >> 8;",
     "b[i] = u[(blk * 512 + i) * n_streams + s] >> 7;", bat.check_birthday_repeats),
    ("birthday without the sample cap", "s < n_streams && samples < max_samples;",
     "s < n_streams;", bat.check_birthday_cap_and_order),
    ("splitmix64 shift 27->26", "r = (r ^ (r >> 27))", "r = (r ^ (r >> 26))",
     sd.check_splitmix64_published_vectors),
    ("stream seed is seed xor s", "uint64_t z = seed + s;", "uint64_t z = seed ^ s;",
     partial(sd.check_seeding_mapping, oracle.XOR128)),
    ("xor128 seed lo/hi swapped", "st[0] = lo32(r0);\n            st[1] = hi32(r0);",
     "st[0] = hi32(r0);\n            st[1] = lo32(r0);", partial(sd.check_seeding_mapping, oracle.XOR128)),
    ("MWC seed carry not reduced", "*c = hi32(r) % a;", "*c = hi32(r);",
     partial(sd.check_seeding_redraws, oracle.MWC)),
    ("MWC seed keeps (0, 0)", "int zero = (*x == 0 && *c == 0);", "int zero = 0;",
     partial(sd.check_seeding_redraws, oracle.MWC)),
    ("MWC seed keeps the top fixed point", "int top = (*x == 0xFFFFFFFFu && *c == a - 1);",
     "int top = 0;", partial(sd.check_seeding_redraws, oracle.MWC)),
    ("KISS seed y and z swapped",
     "st[2] = lo32(r);\n        st[3] = hi32(r);\n        while (st[2] == 0)\n            st[2] = lo32(oracle_splitmix64(&z));\n    }\n}",
     "st[2] = hi32(r);\n        st[3] = lo32(r);\n        while (st[2] == 0)\n            st[2] = lo32(oracle_splitmix64(&z));\n    }\n}",
     partial(sd.check_seeding_mapping, oracle.KISS)),
    ("KISS seed keeps y = 0",
     "        while (st[2] == 0)\n            st[2] = lo32(oracle_splitmix64(&z));\n    }\n}",
     "    }\n}", partial(sd.check_seeding_redraws, oracle.KISS)),
    ("KISS_XOR seed keeps y = 0",
     "        while (st[2] == 0)\n            st[2] = lo32(oracle_splitmix64(&z));\n        return;",
     "        return;", partial(sd.check_seeding_redraws, oracle.KISS_XOR)),
    ("MWC16X2 seed halves swapped",
     "zw[0] = x1 | (c1 << 16);\n            zw[1] = x2 | (c2 << 16);",
     "zw[0] = x2 | (c2 << 16);\n            zw[1] = x1 | (c1 << 16);",
     partial(sd.check_seeding_mapping, oracle.MWC16X2)),
    ("MWC16X2 seed part two from bits 31-46", "(uint32_t)((r >> 32) & 0xFFFFu)",
     "(uint32_t)((r >> 31) & 0xFFFFu)", partial(sd.check_seeding_mapping, oracle.MWC16X2)),
    ("MWC16X2 seed carry one not reduced", "(uint32_t)((r >> 16) & 0xFFFFu) % a1",
     "(uint32_t)((r >> 16) & 0xFFFFu)", partial(sd.check_seeding_mapping, oracle.MWC16X2)),
    ("XORSHIFT8 seed lo/hi swapped", "st[2 * i] = lo32(r);\n                st[2 * i + 1] = hi32(r);",
     "st[2 * i] = hi32(r);\n                st[2 * i + 1] = lo32(r);",
     partial(sd.check_seeding_mapping, oracle.XORSHIFT8)),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, name, old, new, check):
    assert SRC.count(old) == 1, f"mutation anchor not unique: {name}"
    so = oracle.compile_variant(SRC.replace(old, new), tmp_path / "mutant.so")
    with oracle.using(so):
        with pytest.raises(AssertionError):
            check()


def test_unmutated_copy_passes_every_check(tmp_path):
    so = oracle.compile_variant(SRC, tmp_path / "same.so")
    with oracle.using(so):
        for _, _, _, check in MUTANTS:
            check()
    assert np.uint32(1)
