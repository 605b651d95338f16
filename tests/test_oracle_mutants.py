"""Planted mistakes in the oracle: each pin must catch its kind of error.

Every case below copies oracle/mhdc_oracle.c, changes one line into a
plausible mistake (a dropped term, a wrong sign, a strict comparison, a
doubled scale, a wrong rounding tie), compiles the copy with gcc into a
temporary library, loads it in place of the oracle's library for the
duration of the case, and checks that the named pin of
tests/test_oracle_pins.py then fails.  The planted mistakes touch only
in-bounds arithmetic and comparisons (no index leaves its array).
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "mhdc_oracle.c")


def _conversion_pin():
    for seed in range(6):
        pins.test_conversion_matches_dense_brute_force(seed)


def _spmv_pin():
    for seed in range(4):
        pins.test_spmv_matches_dense_matvec(seed)


def _example_pin():
    pins.test_example_mhdc_matches_fig12()
    pins.test_example_spmv_all_formats()


# (name, text in the source, replacement, pin that must fail)
MUTANTS = [
    ("absrow_doubled",
     "            a += fabs(val[k]) * fabs(x[col[k]]);",
     "            a += 2.0 * fabs(val[k]) * fabs(x[col[k]]);", pins.check_csr_absrow),
    ("absrow_signed_x",
     "            a += fabs(val[k]) * fabs(x[col[k]]);",
     "            a += fabs(val[k]) * x[col[k]];", pins.check_csr_absrow),
    ("terms_skip_out_of_range",
     "                t++;\n                if (j >= 0 && j < n) a +=",
     "                if (j >= 0 && j < n) t++;\n                if (j >= 0 && j < n) a +=",
     pins.check_mhdc_absrow_terms),
    ("terms_skip_remainder",
     "k < csr_row_ptr[i + 1]; k++, t++)",
     "k < csr_row_ptr[i + 1]; k++)", pins.check_mhdc_absrow_terms),
    ("select_strict_threshold",
     "if (c >= 1 && (double)c >= theta * (double)rows) {",
     "if (c >= 1 && (double)c > theta * (double)rows) {", _conversion_pin),
    ("select_offset_sign",
     "                offs[m++] = (int64_t)col[k] - i;",
     "                offs[m++] = i - (int64_t)col[k];", _conversion_pin),
    ("select_denominator_is_bl",
     "if (c >= 1 && (double)c >= theta * (double)rows) {",
     "if (c >= 1 && (double)c >= theta * (double)bl) {", _conversion_pin),
    ("spmv_drops_remainder",
     "                s += csr_val[k] * x[csr_col[k]];\n            y[i] = s;",
     "                s += csr_val[k] * x[csr_col[k]];\n            y[i] = 0.0 * s;", _spmv_pin),
    ("spmv_remainder_subtracts",
     "                s += csr_val[k] * x[csr_col[k]];\n            y[i] = s;",
     "                s -= csr_val[k] * x[csr_col[k]];\n            y[i] = s;", _example_pin),
    ("bf16_ties_away",
     "if (rem > 0x8000u || (rem == 0x8000u && (q & 1))) q++;",
     "if (rem >= 0x8000u) q++;", pins.test_round_bf16_matches_torch),
    ("f32_ties_away",
     "        if (rem > half || (rem == half && (q & 1))) q++;\n        if (q == (1ull << 24))",
     "        if (rem >= half) q++;\n        if (q == (1ull << 24))", pins.test_round_f32_matches_numpy_cast),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(name, old, new, pin, source, tmp_path, monkeypatch):
    assert source.count(old) == 1, f"mutation site of {name} is not unique"
    if pin is pins.test_round_bf16_matches_torch:
        pytest.importorskip("torch")
    # the unmodified oracle passes the pin
    pin()
    src = tmp_path / "mutant.c"
    src.write_text(source.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
                           "-shared", "-fPIC", "-o", str(so), str(src), "-lm"])
    L = C.CDLL(str(so))
    oracle._declare(L)
    monkeypatch.setattr(oracle, "_lib", L)
    with pytest.raises(AssertionError):
        pin()
