"""Writes the closed-form golden fixtures in this folder.

The paper prints no worked example with correlation values, so these fixtures
come from inputs whose windowed Pearson coefficient (Eq. 1) has a closed form
derived by hand; this script evaluates those closed forms with exact rational
arithmetic (Python `fractions`/`decimal`), not with the oracle or the CUDA
library.  Run:  python tests/golden/make_golden.py
"""
from decimal import Decimal, getcontext
from fractions import Fraction
import os

getcontext().prec = 40
HERE = os.path.dirname(os.path.abspath(__file__))


def quadratic_1d(n=12):
    # x_i = i, y_i = i^2, window k = 3 centred (Eq. 1 with n = 3 interior).
    # Interior centre t: x = (t-1, t, t+1), y = x^2.  Centred x: (-1, 0, 1);
    # centred y: (-2t + 1/3, -2/3, 2t + 1/3).  sxy = 4t, sxx = 2,
    # syy = 8t^2 + 2/3, so c = 4t / sqrt(2 (8t^2 + 2/3)) = t / sqrt(t^2 + 1/12).
    # Clipped ends (2 cells, both series increasing for i >= 0): c = 1.
    rows = []
    for t in range(n):
        if t == 0 or t == n - 1:
            c = Decimal(1)
        else:
            c2 = Fraction(t * t) / (Fraction(t * t) + Fraction(1, 12))
            c = (Decimal(c2.numerator) / Decimal(c2.denominator)).sqrt()
        rows.append((t, c))
    with open(os.path.join(HERE, "quadratic_1d_k3.txt"), "w") as f:
        f.write("# x_i = i, y_i = i^2 (i = 0..%d), window k = 3, stride 1, clipped borders.\n" % (n - 1))
        f.write("# Closed form of Eq. 1 (classical Pearson): interior c(t) = t / sqrt(t^2 + 1/12),\n")
        f.write("# two-cell border windows c = 1.  Written by make_golden.py (exact rationals).\n")
        f.write("# columns: centre c\n")
        for t, c in rows:
            f.write("%d %s\n" % (t, format(c, ".30f")))


def plane_2d(H=7, W=9, kh=5, kw=3):
    # x = i + j, y = i - j on an H x W grid.  Over a rectangular window the
    # row index i and column index j are uncorrelated, so
    # cov(x, y) = var(i) - var(j) and var(x) = var(y) = var(i) + var(j):
    # c = (vi - vj) / (vi + vj), vi/vj the variances of the clipped index
    # ranges (var of m consecutive integers = (m^2 - 1) / 12).
    def rng(c, k, n):
        lo, hi = max(c - (k - 1) // 2, 0), min(c + k // 2, n - 1)
        return hi - lo + 1
    with open(os.path.join(HERE, "plane_2d_7x9_k5x3.txt"), "w") as f:
        f.write("# x(i,j) = i + j, y(i,j) = i - j on a %dx%d grid (rows x cols), window %dx%d,\n" % (H, W, kh, kw))
        f.write("# stride 1, clipped borders.  Closed form of Eq. 1: c = (vi - vj)/(vi + vj) with\n")
        f.write("# vi = (mi^2 - 1)/12, vj = (mj^2 - 1)/12 for the clipped window extents mi, mj.\n")
        f.write("# Written by make_golden.py (exact rationals).  columns: row col c\n")
        for i in range(H):
            for j in range(W):
                mi, mj = rng(i, kh, H), rng(j, kw, W)
                vi, vj = Fraction(mi * mi - 1, 12), Fraction(mj * mj - 1, 12)
                if vi + vj == 0:
                    s = "nan"
                else:
                    c = (vi - vj) / (vi + vj)
                    s = format(Decimal(c.numerator) / Decimal(c.denominator), ".30f")
                f.write("%d %d %s\n" % (i, j, s))


def plane_2d_paper(H=6, W=9, kh=3, kw=5, miss_x=(3, 4), miss_y=(1, 7)):
    # The paper's result convention (Section 3, result-set paragraph): a
    # window reaching past an edge gives -2, and so does a window holding a
    # missing value (<= -999) in x or y.  Data: x = i + j, y = i - j + 50,
    # with x[miss_x] = -999 (exactly the threshold) and y[miss_y] = -1000.5.
    # Every other window is whole (kh x kw cells, no clipping), so the
    # plane closed form gives c = (vi - vj)/(vi + vj) with vi = (kh^2-1)/12,
    # vj = (kw^2-1)/12 for all of them.
    h1, h2, w1, w2 = (kh - 1) // 2, kh // 2, (kw - 1) // 2, kw // 2
    vi, vj = Fraction(kh * kh - 1, 12), Fraction(kw * kw - 1, 12)
    cw = (vi - vj) / (vi + vj)
    with open(os.path.join(HERE, "plane_2d_paper_6x9_k3x5.txt"), "w") as f:
        f.write("# The paper's -2 convention: x(i,j) = i + j, y(i,j) = i - j + 50 on a %dx%d grid,\n" % (H, W))
        f.write("# x[%d,%d] = -999, y[%d,%d] = -1000.5 (missing values), window %dx%d, stride 1.\n"
                % (miss_x + miss_y + (kh, kw)))
        f.write("# -2 where the window passes an edge or holds a missing cell; else the plane closed\n")
        f.write("# form (vi - vj)/(vi + vj).  Written by make_golden.py (exact rationals).\n")
        f.write("# columns: row col c\n")
        for i in range(H):
            for j in range(W):
                edge = i - h1 < 0 or i + h2 > H - 1 or j - w1 < 0 or j + w2 > W - 1
                holds = any(i - h1 <= r <= i + h2 and j - w1 <= c <= j + w2 for r, c in (miss_x, miss_y))
                s = "-2" if edge or holds else format(Decimal(cw.numerator) / Decimal(cw.denominator), ".30f")
                f.write("%d %d %s\n" % (i, j, s))


if __name__ == "__main__":
    quadratic_1d()
    plane_2d()
    plane_2d_paper()
