"""Pins for the CPU oracle, none of which re-types the oracle's own formula.

* closed forms (golden fixtures derived by hand, tests/golden/);
* the sums form of Pearson (Eq. 2) evaluated in exact rational arithmetic on
  tiny integer grids, against the oracle's two-pass classical form (Eq. 1):
  the identity Eq. 1 == Eq. 2 is the paper's Section 1 premise;
* library special cases: numpy.corrcoef when every clipped window is the
  whole grid, scipy.stats.pearsonr on individual extracted windows;
* invariants of the Pearson coefficient;
* the exact integer window sums (steps 1-3 of Section 1) against an
  independent numpy int64 summed-area table.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    return rows


# ------------------------------------------------------------- closed forms
def test_golden_quadratic_1d():
    rows = _read_golden("quadratic_1d_k3.txt")
    n = len(rows)
    x = np.arange(n, dtype=np.float32)
    y = x * x
    c = oracle.corr(x, y, 3)
    for t, val in rows:
        assert abs(c[int(t)] - float(val)) < 1e-13


def test_golden_plane_2d():
    rows = _read_golden("plane_2d_7x9_k5x3.txt")
    i, j = np.meshgrid(np.arange(7), np.arange(9), indexing="ij")
    x = (i + j).astype(np.uint16) + 100
    y = (i - j + 50).astype(np.uint16)
    c = oracle.corr(x, y, (5, 3))
    for r, col, val in rows:
        if val == "nan":
            assert np.isnan(c[int(r), int(col)])
        else:
            assert abs(c[int(r), int(col)] - float(val)) < 1e-13


def test_golden_plane_2d_paper_convention():
    """The paper's -2 convention (Section 3, result-set paragraph) on a
    hand-derived fixture: edges and windows holding a missing value (x at
    exactly -999, y below it) give -2, the rest the plane closed form; the
    same values at strided centres."""
    rows = _read_golden("plane_2d_paper_6x9_k3x5.txt")
    i, j = np.meshgrid(np.arange(6), np.arange(9), indexing="ij")
    x = (i + j).astype(np.float32)
    y = (i - j + 50).astype(np.float32)
    x[3, 4] = -999.0
    y[1, 7] = -1000.5
    want = np.full((6, 9), np.nan)
    for r, col, val in rows:
        want[int(r), int(col)] = float(val)
    c = oracle.corr(x, y, (3, 5), border="paper")
    assert np.all(np.abs(c - want) < 1e-13)
    cs = oracle.corr(x, y, (3, 5), (2, 3), border="paper")
    assert np.all(np.abs(cs - want[::2, ::3]) < 1e-13)
    # clipped windows are not -2
    assert not np.any(oracle.corr(x, y, (3, 5)) == -2.0)


def test_plane_2d_transposed_window_differs():
    # Swapping the window's row/col extents must flip the sign of the border
    # pattern: catches a transposed k or shape in the index arithmetic.
    i, j = np.meshgrid(np.arange(7), np.arange(9), indexing="ij")
    x = (i + j + 100).astype(np.float32)
    y = (i - j + 50).astype(np.float32)
    a = oracle.corr(x, y, (5, 3))
    b = oracle.corr(x, y, (3, 5))
    assert a[0, 0] > 0.4 and b[0, 0] < 0  # (5,3): rows win; (3,5): cols win


def test_even_window_extent():
    # Even k: window [i - (k-1)//2, i + k//2]; k = 4 at i = 0 covers cells 0..2.
    x = np.array([0, 1, 2, 9, 3, 4], dtype=np.float32)
    y = np.array([0, 1, 2, 0, 0, 0], dtype=np.float32)
    c = oracle.corr(x, y, 4)
    assert abs(c[0] - 1.0) < 1e-15          # cells 0,1,2: identical ramps
    assert abs(c[1] - np.corrcoef(x[0:4], y[0:4])[0, 1]) < 1e-14


# ------------------------------------------- exact rational sums form (Eq. 2)
def _exact_c2_sign(xs, ys):
    n = len(xs)
    sx, sy = sum(xs), sum(ys)
    sxx = sum(v * v for v in xs)
    syy = sum(v * v for v in ys)
    sxy = sum(a * b for a, b in zip(xs, ys))
    num = Fraction(n * sxy - sx * sy)
    vx = Fraction(n * sxx - sx * sx)
    vy = Fraction(n * syy - sy * sy)
    if vx == 0 or vy == 0:
        return None, 0
    return num * num / (vx * vy), (num > 0) - (num < 0)


def _windows(shape, k, stride):
    oshape = [-(-n // s) for n, s in zip(shape, stride)]
    for o in np.ndindex(*oshape):
        sl = []
        for d, jd in enumerate(o):
            lo, hi = oracle.window_bounds(jd * stride[d], k[d], shape[d])
            sl.append(slice(lo, hi + 1))
        yield o, tuple(sl)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_exact_rational_tiny_grids(ndim):
    rng = np.random.default_rng(1234 + ndim)
    for trial in range(30 if ndim < 3 else 12):
        shape = tuple(int(v) for v in rng.integers(1, 10 if ndim < 3 else 6, ndim))
        k = tuple(int(rng.integers(1, 2 * n + 2)) for n in shape)
        stride = tuple(int(v) for v in rng.integers(1, 4, ndim))
        hi = int(rng.choice([3, 50, 65535]))
        x = rng.integers(0, hi + 1, shape).astype(np.uint16)
        y = rng.integers(0, hi + 1, shape).astype(np.uint16)
        c = oracle.corr(x, y, k, stride)
        for o, sl in _windows(shape, k, stride):
            c2, sgn = _exact_c2_sign([int(v) for v in x[sl].ravel()], [int(v) for v in y[sl].ravel()])
            if c2 is None:
                assert np.isnan(c[o])
            else:
                assert abs(c[o] - sgn * math.sqrt(float(c2))) < 1e-13, (shape, k, stride, o)


def test_exact_rational_float_inputs():
    # float32 values are exact binary rationals, so Fraction gives the exact c^2.
    rng = np.random.default_rng(7)
    x = (rng.random((6, 7)) * 10 - 3).astype(np.float32)
    y = (rng.random((6, 7)) * 0.01 + 1e4).astype(np.float32)
    k, stride = (3, 5), (1, 2)
    c = oracle.corr(x, y, k, stride)
    for o, sl in _windows(x.shape, k, stride):
        xs = [Fraction(float(v)) for v in x[sl].ravel()]
        ys = [Fraction(float(v)) for v in y[sl].ravel()]
        c2, sgn = _exact_c2_sign(xs, ys)
        assert abs(c[o] - sgn * math.sqrt(float(c2))) < 1e-10


# ----------------------------------------------------- library special cases
@pytest.mark.parametrize("shape", [(37,), (9, 11), (4, 5, 6)])
def test_whole_grid_windows_equal_corrcoef(shape):
    rng = np.random.default_rng(11)
    x = rng.standard_normal(shape).astype(np.float32)
    y = (0.3 * x + rng.standard_normal(shape)).astype(np.float32)
    k = tuple(2 * n - 1 for n in shape)
    c = oracle.corr(x, y, k)
    ref = np.corrcoef(x.ravel().astype(np.float64), y.ravel().astype(np.float64))[0, 1]
    assert np.allclose(c, ref, rtol=0, atol=1e-13)


def test_windows_equal_scipy_pearsonr():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(5)
    x = rng.random((40, 50)).astype(np.float32)
    y = (-0.8 * x + 0.2 * rng.standard_normal((40, 50))).astype(np.float32)
    k = (7, 5)
    c = oracle.corr(x, y, k)
    for _ in range(200):
        i, j = int(rng.integers(0, 40)), int(rng.integers(0, 50))
        r0, r1 = oracle.window_bounds(i, 7, 40)
        c0, c1 = oracle.window_bounds(j, 5, 50)
        ref = stats.pearsonr(x[r0:r1 + 1, c0:c1 + 1].ravel().astype(np.float64),
                             y[r0:r1 + 1, c0:c1 + 1].ravel().astype(np.float64))[0]
        assert abs(c[i, j] - ref) < 1e-12


def test_sampled_indices_match_full_grid():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 16384, (23, 31)).astype(np.uint16)
    y = rng.integers(0, 16384, (23, 31)).astype(np.uint16)
    full = oracle.corr(x, y, (5, 7), (2, 3))
    idx = rng.integers(0, full.size, 100)
    assert np.array_equal(oracle.corr(x, y, (5, 7), (2, 3), idx=idx), full.ravel()[idx])


# --------------------------------------------------------------- invariants
def test_invariants():
    rng = np.random.default_rng(9)
    x = rng.standard_normal((30, 40)).astype(np.float32)
    y = rng.standard_normal((30, 40)).astype(np.float32)
    c = oracle.corr(x, y, 5)
    assert np.all(np.abs(c) <= 1.0)
    # symmetry
    assert np.array_equal(c, oracle.corr(y, x, 5))
    # c(x, a x + b) = sign(a) on non-constant windows (exact in binary: a, b powers of 2)
    assert np.allclose(oracle.corr(x, (4.0 * x + 2.0).astype(np.float32), 5), 1.0, atol=1e-12)
    assert np.allclose(oracle.corr(x, (-0.5 * x + 8.0).astype(np.float32), 5), -1.0, atol=1e-12)
    # affine invariance c(a x + b, d y + e) = sign(a d) c(x, y)
    c2 = oracle.corr((2.0 * x + 1.0).astype(np.float32), (-8.0 * y + 3.0).astype(np.float32), 5)
    assert np.allclose(c2, -c, atol=1e-9)


def test_degenerate_cases():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 100, (8, 9)).astype(np.uint16)
    y = rng.integers(0, 100, (8, 9)).astype(np.uint16)
    assert np.all(np.isnan(oracle.corr(x, y, 1)))                       # n = 1
    assert np.all(np.isnan(oracle.corr(np.full_like(x, 7), y, 3)))      # constant x
    assert np.all(np.isnan(oracle.corr(x, np.zeros_like(y), 3)))        # constant y
    # a single non-constant cell makes exactly the windows that contain it finite
    z = np.zeros((8, 9), dtype=np.float32)
    z[4, 4] = 1.0
    c = oracle.corr(z, z, 3)
    finite = np.isfinite(c)
    assert finite.sum() == 9 and np.all(c[finite] == 1.0)
    # one-row and one-column grids behave like 1-D series
    row = rng.random(17).astype(np.float32)
    row2 = rng.random(17).astype(np.float32)
    assert np.array_equal(oracle.corr(row[None, :], row2[None, :], (3, 5))[0], oracle.corr(row, row2, 5))
    assert np.array_equal(oracle.corr(row[:, None], row2[:, None], (5, 3))[:, 0], oracle.corr(row, row2, 5))


def test_constant_window_with_offsets_is_nan():
    # The equality check is exact at any offset (Section 3 accuracy note).
    for off in (0.0, 200.0, 1e4, 1e7):
        x = np.full((10, 10), off, dtype=np.float32)
        x[0, 0] = np.float32(off) + np.float32(1.0)
        y = np.random.default_rng(1).random((10, 10)).astype(np.float32)
        c = oracle.corr(x, y, 3)
        assert np.isnan(c[5, 5]) and np.isfinite(c[0, 0])


def test_relvar_closed_form():
    # relvar = sum (v - mean)^2 / sum v^2 over the window (whole grid here):
    # x = 1, 2, 3: 2 / 14; y = 0, 0, 3: 6 / 9
    x = np.array([1, 2, 3], dtype=np.uint16)
    y = np.array([0, 0, 3], dtype=np.uint16)
    c, rx, ry = oracle.corr(x, y, 3, relvar=True)
    assert rx[1] == pytest.approx(1.0 / 7.0, rel=1e-15)
    assert ry[1] == pytest.approx(2.0 / 3.0, rel=1e-15)
    # Pearson of (1, 2, 3) and (0, 0, 3): sxy = 3, sxx = 2, syy = 6
    assert c[1] == pytest.approx(3.0 / np.sqrt(12.0), rel=1e-15)


# ------------------------------------------------------- exact integer sums
def _sat_sums(x, y, k, stride):
    """Window sums via an int64 summed-area table (independent of the oracle)."""
    xs, ys = x.astype(np.int64), y.astype(np.int64)
    planes = [xs, ys, xs * xs, ys * ys, xs * ys]
    nd = x.ndim
    out = []
    for p in planes:
        s = p
        for ax in range(nd):
            s = np.cumsum(s, axis=ax)
        s = np.pad(s, [(1, 0)] * nd)
        oshape = [-(-n // st) for n, st in zip(x.shape, stride)]
        res = np.empty(oshape, dtype=np.int64)
        for o in np.ndindex(*oshape):
            lo, hi = [], []
            for d, jd in enumerate(o):
                a, b = oracle.window_bounds(jd * stride[d], k[d], x.shape[d])
                lo.append(a)
                hi.append(b + 1)
            tot = 0
            for corner in np.ndindex(*([2] * nd)):
                idx = tuple(hi[d] if corner[d] else lo[d] for d in range(nd))
                sign = (-1) ** (nd - sum(corner))
                tot += sign * int(s[idx])
            res[o] = tot
        out.append(res)
    return np.stack(out, axis=-1)


@pytest.mark.parametrize("shape,k,stride", [((50,), (7,), (1,)), ((13, 17), (7, 5), (1, 2)),
                                            ((5, 6, 7), (3, 5, 3), (2, 1, 1))])
def test_integer_sums_match_summed_area_table(shape, k, stride):
    rng = np.random.default_rng(21)
    x = rng.integers(0, 65536, shape).astype(np.uint16)
    y = rng.integers(0, 65536, shape).astype(np.uint16)
    assert np.array_equal(oracle.sums_u16(x, y, k, stride), _sat_sums(x, y, k, stride))
