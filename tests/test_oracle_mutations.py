"""Plant one plausible mistake at a time in a copy of the oracle's C source and
check that the pins catch every one of them (CPU only; nothing runs on a GPU)."""
import ctypes
import os
import subprocess

import pytest

import oracle
import oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "ka_oracle.c")

MUTATIONS = {
    "mandelbrot_no_doubling": ("const float ni = (2.0f * zr) * zi + ci;", "const float ni = zr * zi + ci;"),
    "mandelbrot_escape_ge": ("if (rr + ii > 4.0f) break;", "if (rr + ii >= 4.0f) break;"),
    "mandelbrot_sign": ("const float nr = rr - ii + cr;", "const float nr = rr + ii + cr;"),
    "inclusive_scan": ("        o[i] = running;\n        running += v[i];",
                       "        running += v[i];\n        o[i] = running;"),
    "lt_becomes_le": ("return x < param;", "return x <= param;"),
    "topbits_shift": ("return (x >> 28) < param;", "return (x >> 27) < param;"),
    "popcount_31_bits": ("for (int b = 0; b < 32; b++)", "for (int b = 0; b < 31; b++)"),
    "compact_drops_last": ("    for (uint64_t i = 0; i < n; i++) {\n        int keep",
                           "    for (uint64_t i = 0; i + 1 < n; i++) {\n        int keep"),
    "compact_reversed": ("y[k] = x[i];", "y[k] = x[n - 1 - i];"),
    "hash_multiplier": ("2654435761ULL", "2654435769ULL"),
    "splitmix_counter": ("seed + (i + 1) * 0x9E3779B97F4A7C15ULL", "seed + i * 0x9E3779B97F4A7C15ULL"),
    "splitmix_shift": ("(z ^ (z >> 27))", "(z ^ (z >> 28))"),
    "mod_inverted": ("(x % param) != 0u", "(x % param) == 0u"),
    "mask_inverted": ("(x & param) == 0u", "(x & param) != 0u"),
    "interleave_swapped": ("index[2 * i] = chunk_ids[i];\n        index[2 * i + 1] = literals[i];",
                           "index[2 * i] = literals[i];\n        index[2 * i + 1] = chunk_ids[i];"),
    "all_drops_everything": ("case ORA_ALL:          return 1;", "case ORA_ALL:          return 0;"),
    "scatter_off_by_one": ("y[o[i]] = x[i];", "y[o[i] + (o[i] > 0)] = x[i];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, "mutation anchor not found: " + name
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(mutated)])
    bad = oracle.bind(ctypes.CDLL(str(so)))
    oracle.lib()
    prev = oracle.use_library(bad)
    caught = []
    try:
        for check in pins.ALL_PINS:
            try:
                check()
            except (AssertionError, ValueError, IndexError):
                caught.append(check.__name__)
    finally:
        oracle.use_library(prev)
    assert caught, "no pin caught mutation " + name
