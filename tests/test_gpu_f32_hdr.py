"""float32 parity on inputs that stress the fixed-point maps.

Each float32 kernel maps a block of values (2-D: a lane's columns over its
work item; 1-D: a chunk; 3-D: a work item) to integers on a grid of 2^-22 or
so of the block's range.  A single extreme value in a block coarsens that
grid for every window of the block, including windows that do not contain it;
the per-window certificate must catch those windows and recompute them.
These tests plant 1e6 and 1e30 cells among unit-scale data, compare every
window with the FP64 oracle at |dc| <= 1e-5 on scored windows (both relative
variances above 1e-6), and check that the recomputation path ran.  They also
cover windows of more than 1023 cells on the offset random walk (the regime
where the chunk map keeps only 20 bits), and check that data which converts
exactly (integers, offset walks) never takes the recomputation path.
"""
import numpy as np
import pytest

import oracle
from paper_1807_06507_gb300 import workloads as W
from tests.gpu_util import score, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    from paper_1807_06507_gb300 import swcorr
    swcorr.load()
    return swcorr


def run(sw, x, y, k, stride=None):
    p = sw.Plan(x.shape, k, stride, dtype="f32")
    c = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    p.check_status()
    fb = p.fallbacks()
    out = c.cpu().numpy()
    p.close()
    return out, fb


def check(c, x, y, k, stride=None):
    ref, rx, ry = oracle.corr(x, y, k, stride, relvar=True)
    return score(c, ref, rx, ry, exact_nan=False)


@pytest.mark.parametrize("spike", [1e6, 1e30])
@pytest.mark.parametrize("dist", ["uniform", "normal"])
def test_2d_bright_cell_in_lane(sw, spike, dist):
    rng = np.random.default_rng(int(np.log10(spike)) + (dist == "normal"))
    shape = (150, 520)
    if dist == "uniform":
        x = rng.random(shape).astype(np.float32)
    else:
        x = rng.standard_normal(shape).astype(np.float32)
    y = (0.7 * x + 0.3 * rng.standard_normal(shape)).astype(np.float32)
    # one bright cell in x (inside lane 3 of strip 0), one in y elsewhere
    x[40, 27] = np.float32(spike)
    y[101, 300] = np.float32(spike)
    c, fb = run(sw, x, y, 7)
    m, n_sc, _ = check(c, x, y, 7)
    assert n_sc > 70_000
    assert fb > 0, "the recomputation path did not run"


def test_2d_bright_cells_strided_and_wide_window(sw):
    rng = np.random.default_rng(11)
    x = rng.random((130, 400)).astype(np.float32)
    y = (x + 0.5 * rng.random((130, 400))).astype(np.float32)
    x[::37, ::53] = np.float32(3e7)
    for k, st in (((9, 15), (2, 3)), ((21, 31), None)):
        c, fb = run(sw, x, y, k, st)
        check(c, x, y, k, st)
        assert fb > 0


@pytest.mark.parametrize("spike", [1e6, 1e30])
def test_1d_bright_cell_in_chunk(sw, spike):
    rng = np.random.default_rng(3 + int(np.log10(spike)))
    n = 60_000
    x = rng.random(n).astype(np.float32)
    y = (0.5 * x + rng.random(n)).astype(np.float32)
    x[20_000] = np.float32(spike)
    y[45_123] = np.float32(-spike)
    c, fb = run(sw, x, y, 1001)
    check(c, x, y, 1001)
    assert fb > 0


@pytest.mark.parametrize("k", [1055, 2015])
def test_1d_windows_over_1023_cells_on_offset_walk(sw, k):
    # flip every 4096 samples: chunks that span a sign flip of y do not
    # convert exactly at the chunk's 20 bits
    x, y = W.random_walk_pair(120_000, seed=k, flip=4096)
    c, fb = run(sw, x, y, k)
    m, n_sc, _ = check(c, x, y, k)
    assert n_sc > 50_000


def test_1d_offset_walk_converts_exactly(sw):
    x, y = W.random_walk_pair(200_000, seed=5, flip=1 << 30)  # no flip: every chunk exact
    c, fb = run(sw, x, y, 1001)
    check(c, x, y, 1001)
    assert fb == 0


@pytest.mark.parametrize("spike", [1e6, 1e30])
def test_3d_bright_cell_in_item(sw, spike):
    rng = np.random.default_rng(int(np.log10(spike)))
    shape = (24, 40, 150)
    x = rng.standard_normal(shape).astype(np.float32)
    y = (0.5 * x + rng.standard_normal(shape)).astype(np.float32)
    x[12, 20, 60] = np.float32(spike)
    c, fb = run(sw, x, y, 9)
    check(c, x, y, 9)
    assert fb > 0


def test_3d_11_cubed_on_offset_data(sw):
    rng = np.random.default_rng(21)
    shape = (26, 30, 140)
    x = (1e4 + rng.standard_normal(shape)).astype(np.float32)
    y = (-3e3 + 0.3 * x + rng.standard_normal(shape)).astype(np.float32)
    for st in (1, 2):
        c, fb = run(sw, x, y, 11, st)
        check(c, x, y, 11, st)


def test_3d_halfspace_full_size_no_fallback(sw):
    """The 9^3 half-space volume certifies at 22 bits without recomputation
    (sampled windows against the oracle)."""
    x, y = W.halfspace_volume_pair((256, 512, 512))
    c, fb = run(sw, x, y, 9)
    rng = np.random.default_rng(4)
    idx = rng.integers(0, c.size, 40_000)
    ref, rx, ry = oracle.corr(x, y, 9, idx=idx, relvar=True)
    score(c.ravel()[idx], ref, rx, ry, exact_nan=False)
    assert fb == 0


def test_2d_integer_data_converts_exactly(sw):
    vis, ir = W.night_scene((600, 1100), seed=12)
    x, y = vis.astype(np.float32), ir.astype(np.float32)
    c, fb = run(sw, x, y, 7)
    check(c, x, y, 7)
    assert fb == 0


@pytest.mark.parametrize("k", [7, (31, 31), (9, 3)])
def test_2d_off_integer_night_scene(sw, k):
    """A night scene scaled off the integers (lights thousands of times the
    dark level): the lane maps leave most dark windows uncertified, so the
    lanes' second tier (the finer re-march) carries them."""
    vis, ir = W.night_scene((300, 700), seed=17)
    x, y = vis.astype(np.float32) * np.float32(0.37), ir.astype(np.float32)
    c, fb = run(sw, x, y, k)
    m, n_sc, _ = check(c, x, y, k)
    assert n_sc > 150_000
    assert fb > 0


def test_2d_smooth_radiance_field(sw):
    """A smooth log-normal field with 1% noise: windows of 31 x 31 cells whose
    spread is small next to the lane's range."""
    rng = np.random.default_rng(19)
    yy, xx = np.mgrid[0:260, 0:640].astype(np.float32)
    field = np.exp(2.0 * np.sin(xx / 97.0) * np.cos(yy / 61.0)).astype(np.float32)
    x = (field * (1 + 0.01 * rng.standard_normal(field.shape))).astype(np.float32)
    y = (0.5 * field + 0.02 * rng.standard_normal(field.shape)).astype(np.float32)
    for k in (7, 31):
        c, _ = run(sw, x, y, k)
        check(c, x, y, k)


@pytest.mark.parametrize("k,stride", [(9, 1), (5, 2)])
def test_3d_smooth_field_and_sparse_spots(sw, k, stride):
    """A smooth log-normal volume with 1% noise, and N(0, 1) data with sparse
    spots of 1e3: most items need the wide second tier."""
    rng = np.random.default_rng(23 + k)
    shape = (20, 44, 150)
    zz, yy, xx = np.meshgrid(*(np.arange(n, dtype=np.float32) for n in shape), indexing="ij")
    field = np.exp(2.0 * np.sin(xx / 37.0) * np.cos(yy / 23.0) * np.cos(zz / 17.0)).astype(np.float32)
    fx = (field * (1 + 0.01 * rng.standard_normal(shape))).astype(np.float32)
    fy = (0.5 * field + 0.02 * rng.standard_normal(shape)).astype(np.float32)
    sx = rng.standard_normal(shape).astype(np.float32)
    sy = (0.5 * sx + rng.standard_normal(shape)).astype(np.float32)
    sx.reshape(-1)[rng.integers(0, sx.size, sx.size // 5000)] = np.float32(1e3)
    for x, y in ((fx, fy), (sx, sy)):
        c, fb = run(sw, x, y, k, stride)
        check(c, x, y, k, stride)
        assert fb > 0
