"""Plant plausible mistakes in the oracle and check that the pins catch them.

Each case edits one spot of a copy of ``oracle/rs_oracle.c`` (a dropped term,
a wrong sign, index or bound, a lost tie-break), builds it with gcc into a
temporary library, and runs the pin battery of ``test_oracle_pins.py``
against it.  The original oracle is untouched; the edit happens on the CPU in
a temporary directory.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import test_oracle_pins as pins

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "rs_oracle.c")

MUTATIONS = {
    "no_digit_complement": ("return v < 0 ? 9u - dig : dig;", "return dig;"),
    "sign_order_flipped": ("if (d == 0) return v < 0 ? 0u : 1u;",
                           "if (d == 0) return v < 0 ? 1u : 0u;"),
    "row_walk_exclusive": ("col <= ca->H_Max[row]; col++) {",
                           "col < ca->H_Max[row]; col++) {"),
    "untouched_rows_walked": ("if (ca->H_Min[2 * row] == 0) continue; /* row never touched */",
                              ""),
    "unstable_placement": (
        "for (uint64_t t = 0; t < count; t++) scratch[lo + ca.cursor[cell_of[t]]++] = items[lo + t];",
        "for (uint64_t t = count; t-- > 0;) scratch[lo + ca.cursor[cell_of[t]]++] = items[lo + t];"),
    "pad_symbol_equals_byte0": ("? (uint32_t)ks->chars[beg + (uint64_t)d] + 1u : 0u;",
                                "? (uint32_t)ks->chars[beg + (uint64_t)d] : 0u;"),
    "digit_power_off_by_one": (
        "uint32_t*)ks->keys)[i];\n        return (uint32_t)((v / POW10[ks->D - 1 - d]) % 10u);",
        "uint32_t*)ks->keys)[i];\n        return (uint32_t)((v / POW10[ks->D - d - (d > 0)]) % 10u);"),
    "hmax_wrong_comparison": ("if (ca->H_Max[row] < col) ca->H_Max[row] = col;",
                              "if (ca->H_Max[row] > col) ca->H_Max[row] = col;"),
    "hmin_never_lowered": ("} else if (ca->H_Min[2 * row + 1] > col) {",
                           "} else if (ca->H_Min[2 * row + 1] < col) {"),
    "regen_negative_not_undone": ("mag = (POW10[ks->mag_digits] - 1u) - mag;", ""),
    "float_negatives_not_complemented": ("return negative ? 9u - dig : dig;", "return dig;"),
    "float_nan_before_numbers": ("if (is_nan) return 3u;", "if (is_nan) return 0u;"),
    "emit_u64_wrong_width": ("((uint64_t*)out)[j] = cell;",
                             "((uint32_t*)out)[j] = (uint32_t)cell;"),
    "emit_u32_off_by_one": ("((uint32_t*)out)[j] = (uint32_t)cell;",
                            "((uint32_t*)out)[j] = (uint32_t)cell + (j > 0 && cell > 0);"),
    "bucket_skips_a_dimension": (
        "rc = sort_bucket(ks, items, scratch, bk[i].lo, bk[i].count, next, cell_cap, st);",
        "rc = sort_bucket(ks, items, scratch, bk[i].lo, bk[i].count, next + 1, cell_cap, st);"),
}


def _battery(oracle):
    """Run the pins; return the names of those that failed."""
    failed = []
    checks = [
        ("example1_output", lambda: pins.test_example1_sorted_output(oracle)),
        ("example1_cells_k", lambda: pins.test_example1_cells_and_extraction_cost(oracle)),
        ("maps_definition", lambda: pins.test_traverse_maps_definition(oracle)),
        ("brute_u32", lambda: pins.test_bruteforce_u32(oracle, 4)),
        ("brute_dec", lambda: pins.test_bruteforce_fixed_decimal_signed(oracle, 3)),
        ("brute_str", lambda: pins.test_bruteforce_strings(oracle, 3)),
        ("u32_numpy", lambda: pins.test_u32_vs_numpy_stable(oracle, 1, 2**32, 3000)),
        ("u64_numpy", lambda: pins.test_u64_vs_numpy_stable(oracle, 1)),
        ("u64_regen", lambda: pins.test_u64_small_keys_regenerated(oracle, 1000)),
        ("dec_numpy", lambda: pins.test_fixed_decimal_vs_numpy_stable(oracle, 1)),
        ("dec_regen", lambda: pins.test_fixed_decimal_regenerates_negatives(oracle)),
        ("str_bytes", lambda: pins.test_strings_vs_python_bytes_order(oracle, 1)),
        ("invariants", lambda: pins.test_invariants_random(oracle)),
        ("brute_float", lambda: pins.test_bruteforce_float(oracle, 3)),
        ("float_numpy", lambda: pins.test_float_vs_numpy_stable(oracle, np.float64)),
    ]
    for name, fn in checks:
        try:
            fn()
        except (AssertionError, oracle.OracleError, IndexError, ValueError):
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_battery(oracle):
    assert _battery(oracle) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(oracle, tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutant = tmp_path / "rs_oracle.c"
    mutant.write_text(src.replace(old, new))
    hdr = os.path.join(os.path.dirname(SRC), "rs_oracle.h")
    (tmp_path / "rs_oracle.h").write_text(open(hdr).read())
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", str(mutant), "-o",
                           str(lib)])
    # A mutant may crash (a wrong bound can write out of range), so the
    # battery runs in a child process; any failure or crash counts as caught.
    child = (
        "import sys; sys.path[:0] = [%r, %r]\n"
        "from oracle import oracle as o\n"
        "import test_oracle_mutations as m\n"
        "with o.use_library(%r):\n"
        "    failed = m._battery(o)\n"
        "print('failed:', failed)\n"
        "sys.exit(1 if failed else 0)\n" % (HERE, ROOT, str(lib)))
    r = subprocess.run([sys.executable, "-c", child], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode != 0, f"planted mistake {name} passed every pin: {r.stdout}"
