"""Window shapes outside the fused kernels' instances.

The paper defines the method for windows "of a given size" and step
(Introduction) and for any number of dimensions (Section 1); the fused 1-D,
2-D and 3-D kernels are instantiated for odd widths up to 31 (2-D), equal
odd in-plane sizes up to 15 (3-D) and 1-D windows up to 2016 strides.
Every other shape runs on the general path (one sum pass per dimension over
materialised integer streams).  Each case is compared with the oracle: the
uint16 window sums bit for bit, c within 1e-5 on scored windows.
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


def run(sw, x, y, k, stride=None, sums=False):
    dtype = "u16" if x.dtype == np.uint16 else "f32"
    p = sw.Plan(x.shape, k, stride, dtype=dtype, flags=sw.FLAG_EMIT_SUMS if sums else 0)
    s = torch.zeros((p.outputs(), 5), dtype=torch.int64, device="cuda") if sums else None
    c = p.run(to_dev(x, torch), to_dev(y, torch), sums=s)
    torch.cuda.synchronize()
    p.check_status()
    out = c.cpu().numpy()
    ss = s.cpu().numpy().reshape(p.oshape + (5,)) if sums else None
    p.close()
    return out, ss


def pair(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == "u16":
        x = rng.integers(0, 16384, shape).astype(np.uint16)
        y = ((x // 2) + rng.integers(0, 8192, shape)).astype(np.uint16)
        x.reshape(-1)[::61] = 100
    else:
        x = rng.standard_normal(shape).astype(np.float32)
        y = (0.5 * x + rng.standard_normal(shape)).astype(np.float32)
    return x, y


CASES = [
    ((60, 130), (4, 4), None), ((45, 101), (6, 2), (2, 1)), ((31, 90), (3, 8), None), ((40, 150), (2, 32), (1, 3)),
    ((50, 120), (3, 41), None), ((70, 64), (9, 64), None),
    ((12, 20, 60), (3, 5, 7), None), ((10, 25, 70), (5, 3, 9), (2, 1, 2)), ((9, 40, 50), (3, 21, 21), None),
    ((5, 40, 45), (1, 31, 31), None), ((8, 16, 40), (4, 4, 4), None), ((7, 14, 33), (2, 6, 2), (1, 2, 3)),
    ((12_000,), 5000, None), ((9_000,), 4001, (3,)),
]


@pytest.mark.parametrize("shape,k,stride", CASES)
@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_shape_matches_oracle(sw, shape, k, stride, dtype):
    x, y = pair(shape, dtype, len(shape) * 100 + sum(np.atleast_1d(k)))
    c, s = run(sw, x, y, k, stride, sums=(dtype == "u16"))
    if dtype == "u16":
        assert np.array_equal(s, oracle.sums_u16(x, y, k, stride))
        score(c, oracle.corr(x, y, k, stride))
    else:
        ref, rx, ry = oracle.corr(x, y, k, stride, relvar=True)
        score(c, ref, rx, ry, exact_nan=False)


def hdr_pair(shape, seed):
    """float32 off the integers with sparse cells 10^4 times the background:
    most blocks need the second tier, at every border geometry."""
    rng = np.random.default_rng(seed)
    x = (0.37 * (100.0 + rng.standard_normal(shape))).astype(np.float32)
    y = (0.5 * x + 0.3 * rng.standard_normal(shape)).astype(np.float32)
    flat = x.reshape(-1)
    flat[rng.integers(0, flat.size, max(1, flat.size // 3000))] = np.float32(3.7e5)
    return x, y


HDR_CASES = [((1, 500), (7, 7), None), ((3, 701), (7, 7), None), ((17, 2049), (9, 31), (2, 3)),
             ((40, 263), (5, 13), None), ((2, 9, 131), (9, 9, 9), None), ((6, 21, 77), (5, 5, 5), (2, 2, 2)),
             ((1500,), 1001, None), ((20_000,), 999, (3,))]


@pytest.mark.parametrize("shape,k,stride", HDR_CASES)
def test_fused_float32_second_tier_at_edges(sw, shape, k, stride):
    x, y = hdr_pair(shape, len(shape) * 7 + sum(np.atleast_1d(k)))
    c, _ = run(sw, x, y, k, stride)
    ref, rx, ry = oracle.corr(x, y, k, stride, relvar=True)
    score(c, ref, rx, ry, exact_nan=False)
