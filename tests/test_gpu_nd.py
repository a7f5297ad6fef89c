"""GPU parity of the general n-dimensional path against the CPU oracle.

The general path materialises the five product streams (six with the
paper's missing-value count) and runs one sliding-sum pass per dimension
(Section 1's n-dimensional generalisation); it serves grids of more than
three dimensions, the paper's -2 result convention (Section 3, result-set
paragraph) and the cumulative-sum ablation.  uint16 window sums must equal
the oracle's bit for bit; c within 1e-5 on scored windows; the -2 mask must
equal the oracle's exactly.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import score, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    from paper_1807_06507_gb300 import swcorr
    swcorr.load()
    return swcorr


def run(sw, x, y, k, stride=None, border="clip", flags=0, sums=False):
    dtype = "u16" if x.dtype == np.uint16 else "f32"
    fl = flags | (sw.FLAG_EMIT_SUMS if sums else 0)
    p = sw.Plan(x.shape, k, stride, dtype=dtype, flags=fl, border=border)
    s = torch.zeros((p.outputs(), 5), dtype=torch.int64, device="cuda") if sums else None
    c = p.run(to_dev(x, torch), to_dev(y, torch), sums=s)
    torch.cuda.synchronize()
    p.check_status()
    fb = p.fallbacks()
    out = c.cpu().numpy()
    ss = s.cpu().numpy().reshape(p.oshape + (5,)) if sums else None
    p.close()
    return out, ss, fb


def rand_u16(shape, seed, hi=16384):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, hi, shape).astype(np.uint16)
    y = ((x.astype(np.int64) // 3 + rng.integers(0, hi // 2, shape)) % 65536).astype(np.uint16)
    return x, y


@pytest.mark.parametrize("shape,k,stride", [((6, 7, 9, 20), (3, 5, 3, 7), None),
                                            ((5, 4, 6, 3, 17), (2, 3, 4, 1, 5), (1, 2, 1, 1, 3)),
                                            ((2, 3, 2, 3, 2, 3, 2, 9), (2, 3, 1, 3, 2, 2, 3, 4), None)])
def test_ndim_over_3_u16_bit_exact_sums(sw, shape, k, stride):
    x, y = rand_u16(shape, sum(shape))
    x.reshape(-1)[::97] = 7  # some constant stretches
    c, s, _ = run(sw, x, y, k, stride, sums=True)
    assert np.array_equal(s, oracle.sums_u16(x, y, k, stride))
    score(c, oracle.corr(x, y, k, stride))


@pytest.mark.parametrize("shape,k", [((4, 5, 6, 7, 8), 3), ((3, 9, 4, 30), (3, 5, 1, 7))])
def test_ndim_over_3_f32(sw, shape, k):
    rng = np.random.default_rng(len(shape))
    x = rng.standard_normal(shape).astype(np.float32)
    y = (0.4 * x + rng.standard_normal(shape)).astype(np.float32)
    c, _, _ = run(sw, x, y, k)
    ref, rx, ry = oracle.corr(x, y, k, relvar=True)
    score(c, ref, rx, ry, exact_nan=False)


def test_ndim_4_f32_bright_cell_recomputed(sw):
    rng = np.random.default_rng(9)
    shape = (5, 6, 7, 40)
    x = rng.random(shape).astype(np.float32)
    y = (x + rng.random(shape)).astype(np.float32)
    x[2, 3, 3, 20] = np.float32(1e6)
    c, _, fb = run(sw, x, y, 3)
    ref, rx, ry = oracle.corr(x, y, 3, relvar=True)
    score(c, ref, rx, ry, exact_nan=False)
    assert fb > 0


@pytest.mark.parametrize("shape,k,stride", [((3000,), 31, None), ((120, 333), (5, 7), None),
                                            ((97, 211), (4, 3), (2, 3)), ((9, 30, 41), (3, 5, 7), None),
                                            ((4, 6, 9, 13), (3, 3, 5, 3), (1, 2, 1, 2))])
@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_paper_convention(sw, shape, k, stride, dtype):
    rng = np.random.default_rng(len(shape) * 10 + (dtype == "f32"))
    if dtype == "u16":
        x, y = rand_u16(shape, len(shape))
    else:
        x = (100.0 + rng.standard_normal(shape)).astype(np.float32)
        y = (0.3 * x + rng.standard_normal(shape)).astype(np.float32)
        flat_x, flat_y = x.reshape(-1), y.reshape(-1)
        miss = rng.choice(x.size, max(1, x.size // 500), replace=False)
        flat_x[miss[::2]] = np.float32(-999.0)      # exactly the threshold
        flat_y[miss[1::2]] = np.float32(-5000.25)   # below it
    c, _, _ = run(sw, x, y, k, stride, border="paper")
    ref = oracle.corr(x, y, k, stride, border="paper")
    assert np.array_equal(c == -2.0, ref == -2.0), "the -2 mask differs from the oracle's"
    assert (ref == -2.0).any() and (ref != -2.0).any()
    keep = ref != -2.0
    score(c[keep], ref[keep], exact_nan=(dtype == "u16"))


def test_paper_convention_night_scene(sw):
    from paper_1807_06507_gb300 import workloads as W
    x, y = W.night_scene((600, 800), seed=14)
    c, _, _ = run(sw, x, y, 7, border="paper")
    ref = oracle.corr(x, y, 7, border="paper")
    assert np.array_equal(c == -2.0, ref == -2.0)
    assert np.all(c[:3] == -2.0) and np.all(c[:, -3:] == -2.0)
    score(c[3:-3, 3:-3], oracle.corr(x, y, 7)[3:-3, 3:-3])


@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_cumulative_sum_ablation_equals_sliding(sw, dtype):
    from paper_1807_06507_gb300 import workloads as W
    x, y = W.night_scene((300, 700), seed=15)
    if dtype == "f32":
        x, y = x.astype(np.float32) * np.float32(0.37), y.astype(np.float32)
    k, st = (7, 9), (1, 2)
    c_sat, _, _ = run(sw, x, y, k, st, flags=sw.FLAG_SAT)
    c_nd, _, _ = run(sw, x, y, k, st, border="clip", flags=0)  # fused path
    # the general path's sliding sums on the same grid
    c_gen, _, _ = run(sw, x, y, k, st, flags=sw.FLAG_UNFUSED)
    assert np.array_equal(np.isnan(c_sat), np.isnan(c_gen))
    assert np.allclose(c_sat, c_gen, rtol=0, atol=0, equal_nan=True), "SAT and sliding sums differ"
    if dtype == "u16":  # exact integer sums: the fused kernel's results too, up to its float32 finalize
        score(c_nd, c_gen.astype(np.float64), tol=1e-6)
    ref, rx, ry = oracle.corr(x, y, k, st, relvar=True)
    score(c_sat, ref, rx, ry, exact_nan=(dtype == "u16"))
    score(c_nd, ref, rx, ry, exact_nan=(dtype == "u16"))


@pytest.mark.parametrize("case", ["even_2d_scaled_night", "3d_unequal_spike"])
def test_general_path_float32_high_dynamic_range(sw, case):
    """Window shapes the fused kernels have no instance for run on the general
    path, whose float32 map spans the whole grid; windows it cannot certify
    are recomputed from their own cells (window-local map, then FP64)."""
    from paper_1807_06507_gb300 import workloads as W
    if case == "even_2d_scaled_night":
        vis, ir = W.night_scene((200, 300), seed=16)
        x, y, k = vis.astype(np.float32) * np.float32(0.37), ir.astype(np.float32), (8, 6)
    else:
        rng = np.random.default_rng(17)
        x = rng.standard_normal((12, 30, 40)).astype(np.float32)
        y = (0.5 * x + rng.standard_normal(x.shape)).astype(np.float32)
        x[6, 15, 20] = np.float32(1e6)
        k = (3, 5, 7)
    c, _, fb = run(sw, x, y, k)
    ref, rx, ry = oracle.corr(x, y, k, relvar=True)
    score(c, ref, rx, ry, exact_nan=False)
    assert fb > 0
