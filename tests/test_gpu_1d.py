"""GPU parity of the fused 1-D kernel (long windows) against the CPU oracle."""
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


def run1(sw, x, y, k, stride=None, dtype=None):
    dtype = dtype or ("u16" if x.dtype == np.uint16 else "f32")
    p = sw.Plan(x.shape, k, stride, dtype=dtype)
    c = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    p.check_status()
    out = c.cpu().numpy()
    p.close()
    return out


@pytest.mark.parametrize("n,k", [(50_000, 1001), (20_011, 101), (9_000, 7), (3_000, 2001), (70_000, 1)])
def test_random_walk_f32(sw, n, k):
    x, y = W.random_walk_pair(n, seed=n + k, flip=4096)
    ref, rx, ry = oracle.corr(x, y, k, relvar=True)
    score(run1(sw, x, y, k), ref, rx, ry, exact_nan=False)


@pytest.mark.parametrize("n,k,stride", [(40_000, 101, 1), (40_000, 101, 3), (5_555, 64, 2), (777, 1001, 1),
                                        (70_000, 2015, 1), (33_333, 4000, 5), (20_000, 31, 9),
                                        (1, 5, 1), (2, 1, 1), (100, 100, 7)])
def test_u16_series_exact_nan(sw, n, k, stride):
    rng = np.random.default_rng(n + k)
    x = rng.integers(0, 65536, n).astype(np.uint16)
    y = (rng.integers(0, 65536, n) // 2 + x // 2).astype(np.uint16)
    x[n // 3: n // 3 + 300] = 17
    c = run1(sw, x, y, k, stride)
    score(c, oracle.corr(x, y, k, stride))


def test_f32_offsets_and_constant_runs(sw):
    rng = np.random.default_rng(5)
    n = 30_000
    x = (1e7 + rng.integers(0, 50, n)).astype(np.float32)
    y = (200.0 + rng.random(n)).astype(np.float32)
    x[1000:4000] = np.float32(1e7 + 3)
    c = run1(sw, x, y, 301)
    ref, rx, ry = oracle.corr(x, y, 301, relvar=True)
    assert np.isnan(ref).sum() > 1000
    score(c, ref, rx, ry, exact_nan=False)


def test_full_length_series_sampled(sw):
    # 2^26 samples, window 1001: sampled windows (both ends, chunk seams, uniform)
    x, y = W.random_walk_pair()
    c = run1(sw, x, y, 1001)
    n = x.size
    rng = np.random.default_rng(0)
    L = 32 * 63
    seams = (np.arange(1, 200) * L * 97) % n
    idx = np.unique(np.concatenate([np.arange(3000), np.arange(n - 3000, n), rng.integers(0, n, 1 << 18),
                                    (seams[:, None] + np.arange(-2, 3)[None, :]).ravel() % n]))
    ref, rx, ry = oracle.corr(x, y, 1001, idx=idx, relvar=True)
    score(c[idx], ref, rx, ry, exact_nan=False)


def test_unaligned_base_plain_loads(sw):
    rng = np.random.default_rng(7)
    buf_x = rng.random(10_001).astype(np.float32)
    buf_y = rng.random(10_001).astype(np.float32)
    xd = to_dev(buf_x, torch)[1:]
    yd = to_dev(buf_y, torch)[1:]
    p = sw.Plan((10_000,), 51, dtype="f32")
    c = p.run(xd, yd)
    torch.cuda.synchronize()
    ref, rx, ry = oracle.corr(buf_x[1:].copy(), buf_y[1:].copy(), 51, relvar=True)
    score(c.cpu().numpy(), ref, rx, ry, exact_nan=False)


@pytest.mark.parametrize("n,k,stride", [(30_000, 301, 2), (50_000, 1001, 1), (9_000, 2015, 1), (12_345, 500, 7)])
def test_f32_strides_and_chunk_seams(sw, n, k, stride):
    # chunks of 4 warps x 2016 outputs: seams between warps and between chunks
    x, y = W.random_walk_pair(n, seed=n + 3 * k, flip=1500)
    c = run1(sw, x, y, k, stride)
    ref, rx, ry = oracle.corr(x, y, k, stride, relvar=True)
    score(c, ref, rx, ry, exact_nan=False)


def test_host_run_1d(sw):
    x, y = W.random_walk_pair(30_001, seed=41, flip=5000)
    p = sw.Plan(x.shape, 301, 2, dtype="f32")
    ref = p.run(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    ch = p.run_host(x, y)
    assert np.array_equal(ch, ref.cpu().numpy(), equal_nan=True)
    p.check_status()



@pytest.mark.parametrize("n,k,stride", [(40_000, 1001, 1), (20_011, 64, 3), (300_000, 18001, 9), (5_000, 2015, 1)])
def test_u16_sums_bit_exact(sw, n, k, stride):
    """The exact window sums (Section 1, steps 1-3) of a 1-D uint16 plan on
    full-range 16-bit data, up to windows of 18001 cells (the 1-D span of a
    chunk bounds k by its shared memory)."""
    rng = np.random.default_rng(n + k)
    x = rng.integers(0, 65536, n).astype(np.uint16)
    y = rng.integers(0, 65536, n).astype(np.uint16)
    x[n // 2: n // 2 + 3000] = 65535
    p = sw.Plan(x.shape, k, stride, dtype="u16", flags=sw.FLAG_EMIT_SUMS)
    s = torch.zeros((p.outputs(), 5), dtype=torch.int64, device="cuda")
    c = p.run(to_dev(x, torch), to_dev(y, torch), sums=s)
    torch.cuda.synchronize()
    p.check_status()
    got = s.cpu().numpy()
    p.close()
    assert np.array_equal(got, oracle.sums_u16(x, y, k, stride))
    score(c.cpu().numpy(), oracle.corr(x, y, k, stride))
