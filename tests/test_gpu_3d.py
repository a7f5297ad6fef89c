"""GPU parity of the fused 3-D kernel against the CPU oracle."""
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


def run3(sw, x, y, k, stride=None):
    dtype = "u16" if x.dtype == np.uint16 else "f32"
    p = sw.Plan(x.shape, k, stride, dtype=dtype)
    c = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    p.check_status()
    out = c.cpu().numpy()
    p.close()
    return out


@pytest.mark.parametrize("stride", [1, 2])
def test_halfspace_volume_small(sw, stride):
    x, y = W.halfspace_volume_pair((40, 70, 300), seed=11)
    ref, rx, ry = oracle.corr(x, y, 9, stride, relvar=True)
    score(run3(sw, x, y, 9, stride), ref, rx, ry, exact_nan=False)


@pytest.mark.parametrize("shape,k", [((12, 33, 260), (3, 5, 5)), ((9, 20, 140), (5, 3, 3)), ((1, 1, 1), 3),
                                     ((5, 3, 200), 7), ((17, 9, 129), (1, 1, 1)), ((6, 30, 64), (9, 15, 15)),
                                     ((7, 11, 131), (3, 5, 5)), ((40, 17, 250), (15, 3, 3))])
def test_u16_volumes_exact(sw, shape, k):
    rng = np.random.default_rng(sum(shape))
    x = rng.integers(0, 65536, shape).astype(np.uint16)
    y = rng.integers(0, 65536, shape).astype(np.uint16)
    x[:, : shape[1] // 2, : shape[2] // 3] = 9
    score(run3(sw, x, y, k), oracle.corr(x, y, k))


@pytest.mark.parametrize("stride", [(2, 1, 3), (1, 2, 2)])
def test_f32_strides_and_offsets(sw, stride):
    rng = np.random.default_rng(3)
    x = (1e4 + rng.standard_normal((20, 40, 150))).astype(np.float32)
    y = (0.5 * x + rng.standard_normal((20, 40, 150))).astype(np.float32)
    ref, rx, ry = oracle.corr(x, y, (5, 7, 7), stride, relvar=True)
    score(run3(sw, x, y, (5, 7, 7), stride), ref, rx, ry, exact_nan=False)


def test_full_volume_stride2_and_sampled_stride1(sw):
    x, y = W.halfspace_volume_pair()
    c2 = run3(sw, x, y, 9, 2)
    ref, rx, ry = oracle.corr(x, y, 9, 2, relvar=True)
    score(c2, ref, rx, ry, exact_nan=False)
    c1 = run3(sw, x, y, 9, 1)
    rng = np.random.default_rng(0)
    idx = rng.integers(0, c1.size, 1 << 18)
    ref, rx, ry = oracle.corr(x, y, 9, 1, idx=idx, relvar=True)
    score(c1.ravel()[idx], ref, rx, ry, exact_nan=False)


def test_f32_padded_rows_ragged_edge(sw):
    # rows of 150 floats in a 152-float pitch (TMA path, ragged last 16-byte
    # group): the padding holds 1e30, which must stay out of every range
    rng = np.random.default_rng(5)
    shape = (18, 27, 150)
    x = (3e3 + rng.standard_normal(shape)).astype(np.float32)
    y = (0.3 * x + rng.standard_normal(shape)).astype(np.float32)
    xp = np.full(shape[:2] + (152,), 1e30, np.float32)
    yp = np.full(shape[:2] + (152,), -1e30, np.float32)
    xp[..., :150], yp[..., :150] = x, y
    p = sw.Plan(shape, (5, 9, 9), dtype="f32")
    c = p.run(torch.from_numpy(xp).cuda()[..., :150], torch.from_numpy(yp).cuda()[..., :150])
    torch.cuda.synchronize()
    p.check_status()
    ref, rx, ry = oracle.corr(x, y, (5, 9, 9), relvar=True)
    score(c.cpu().numpy(), ref, rx, ry, exact_nan=False)


@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_host_run_3d(sw, dtype):
    rng = np.random.default_rng(8)
    shape = (12, 30, 136)
    if dtype == "u16":
        x = rng.integers(0, 4096, shape).astype(np.uint16)
        y = rng.integers(0, 4096, shape).astype(np.uint16)
    else:
        x = (50 + rng.standard_normal(shape)).astype(np.float32)
        y = (0.5 * x + rng.standard_normal(shape)).astype(np.float32)
    p = sw.Plan(shape, (3, 5, 5), dtype=dtype)
    ref = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    ch = p.run_host(x, y)
    assert np.array_equal(ch, ref.cpu().numpy(), equal_nan=True)
    p.check_status()



@pytest.mark.parametrize("shape,k,stride", [((40, 50, 130), (9, 9, 9), None), ((33, 40, 70), (5, 7, 7), (2, 3, 1)),
                                            ((150, 20, 40), (145, 15, 15), None)])
def test_u16_sums_bit_exact(sw, shape, k, stride):
    """The exact window sums of a 3-D uint16 plan on full-range 16-bit data,
    up to windows of 145 x 15 x 15 = 32625 cells."""
    rng = np.random.default_rng(sum(shape))
    x = rng.integers(0, 65536, shape).astype(np.uint16)
    y = rng.integers(0, 65536, shape).astype(np.uint16)
    x[:, :5, :9] = 65535
    p = sw.Plan(x.shape, k, stride, dtype="u16", flags=sw.FLAG_EMIT_SUMS)
    s = torch.zeros((p.outputs(), 5), dtype=torch.int64, device="cuda")
    c = p.run(to_dev(x, torch), to_dev(y, torch), sums=s)
    torch.cuda.synchronize()
    p.check_status()
    got = s.cpu().numpy().reshape(p.oshape + (5,))
    p.close()
    assert np.array_equal(got, oracle.sums_u16(x, y, k, stride))
    score(c.cpu().numpy(), oracle.corr(x, y, k, stride))
