"""Planted mistakes in the CPU oracle: every one must fail at least one pin.

Each mutant is a copy of ``oracle/swcorr_oracle.c`` with one plausible slip
(a dropped or swapped term, a wrong sign, channel, index or window extent),
built with gcc into a temporary directory and swapped in for the regular
build while the pins of ``test_oracle_pins.py`` run.  A mutant that no pin
rejects would mean the pins do not fix that part of the oracle.  No mutant
reads outside its arrays: they change arithmetic and index maps only.

Not listed, because no input can tell it apart: reporting NaN only when both
channels are constant.  For uint16 and float32 data, n equal values sum
exactly in doubles, so a constant channel's centred sums are exactly 0 and
Eq. 1 gives 0/0 = NaN on its own.
"""
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as P

# (name, original snippet, mutated snippet); each snippet is unique in the source
MUTANTS = [
    ("even window extents swapped",
     "int64_t a = centre - (J->k[d] - 1) / 2;\n    int64_t b = centre + J->k[d] / 2;",
     "int64_t a = centre - J->k[d] / 2;\n    int64_t b = centre + (J->k[d] - 1) / 2;"),
    ("left clip drops the first cell",
     "lo[d] = a < 0 ? 0 : a;",
     "lo[d] = a < 0 ? (J->shape[d] > 1 ? 1 : 0) : a;"),
    ("stride ignored in the window centre",
     "int64_t centre = j[d] * (int64_t)J->stride[d];",
     "int64_t centre = j[d];"),
    ("output index decomposed in the wrong order",
     "for (int d = J->ndim - 1; d >= 0; d--) {\n    j[d] = o % J->oshape[d];",
     "for (int d = 0; d < J->ndim; d++) {\n    j[d] = o % J->oshape[d];"),
    ("cross term uses x twice",
     "    sxy += a * b;\n    sxx += a * a;",
     "    sxy += a * a;\n    sxx += a * a;"),
    ("centring with the wrong sign",
     "double b = value_at(J->dtype, J->y, off) - my;",
     "double b = value_at(J->dtype, J->y, off) + my;"),
    ("mean divided by n + 1",
     "double mx = sum_x / (double)n, my = sum_y / (double)n;",
     "double mx = sum_x / (double)(n + 1), my = sum_y / (double)n;"),
    ("x variance in both factors",
     "c = sxy / sqrt(sxx * syy);",
     "c = sxy / sqrt(sxx * sxx);"),
    ("constant check compares x against y's first value",
     "if (a != x0) x_const = 0;",
     "if (a != y0) x_const = 0;"),
    ("relative variance of x over y's second moment",
     "J->rvx[slot] = (x_const || sum_xx == 0.0) ? 0.0 : sxx / sum_xx;",
     "J->rvx[slot] = (x_const || sum_xx == 0.0) ? 0.0 : sxx / sum_yy;"),
    ("integer cross sum uses x twice",
     "      syy += b * b;\n      sxy += a * b;",
     "      syy += b * b;\n      sxy += a * a;"),
    ("missing-value threshold excludes -999 itself",
     "if (value_at(J->dtype, J->x, off) <= -999.0 || value_at(J->dtype, J->y, off) <= -999.0) missing = 1;",
     "if (value_at(J->dtype, J->x, off) < -999.0 || value_at(J->dtype, J->y, off) <= -999.0) missing = 1;"),
    ("missing values looked for in x only",
     "if (value_at(J->dtype, J->x, off) <= -999.0 || value_at(J->dtype, J->y, off) <= -999.0) missing = 1;",
     "if (value_at(J->dtype, J->x, off) <= -999.0) missing = 1;"),
    ("edge test ignores the far edge",
     "if (a < 0 || b > J->shape[d] - 1) outside = 1;",
     "if (a < 0) outside = 1;"),
    ("integer sum of y squares drops a term",
     "      syy += b * b;\n      sxy += a * b;\n    }",
     "      syy += b * (b - 1);\n      sxy += a * b;\n    }"),
]

# The pins, called with representative parameters; each raises on failure.
PINS = [
    P.test_golden_quadratic_1d,
    P.test_golden_plane_2d,
    P.test_golden_plane_2d_paper_convention,
    P.test_plane_2d_transposed_window_differs,
    P.test_even_window_extent,
    lambda: P.test_exact_rational_tiny_grids(1),
    lambda: P.test_exact_rational_tiny_grids(2),
    lambda: P.test_exact_rational_tiny_grids(3),
    P.test_exact_rational_float_inputs,
    lambda: P.test_whole_grid_windows_equal_corrcoef((9, 11)),
    P.test_windows_equal_scipy_pearsonr,
    P.test_sampled_indices_match_full_grid,
    P.test_invariants,
    P.test_degenerate_cases,
    P.test_constant_window_with_offsets_is_nan,
    P.test_relvar_closed_form,
    lambda: P.test_integer_sums_match_summed_area_table((13, 17), (7, 5), (1, 2)),
    lambda: P.test_integer_sums_match_summed_area_table((5, 6, 7), (3, 5, 3), (2, 1, 1)),
]


def _pins_failing():
    failed = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError) as e:
            failed.append(f"{getattr(pin, '__name__', 'pin')}: {str(e)[:80]}")
    return failed


def test_pins_pass_on_the_regular_build():
    assert _pins_failing() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"snippet for '{name}' not unique in the oracle source"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
                    "-ffp-contract=off", str(mutant), "-o", str(lib), "-lm"], check=True)
    prev = oracle._swap_library(str(lib))
    try:
        failed = _pins_failing()
    finally:
        oracle._swap_library(prev)
    assert failed, f"no pin rejects the planted mistake: {name}"
