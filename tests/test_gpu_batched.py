"""GPU parity of the batched persistent launch (many uneven uint16 scenes)."""
import numpy as np
import pytest

import oracle
from paper_1807_06507_gb300 import workloads as W
from tests.gpu_util import score, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def padded(a, pad_to=8):
    """Copy with rows padded to a multiple of pad_to elements (TMA pitch rule)."""
    h, w = a.shape
    wp = -(-w // pad_to) * pad_to
    out = np.zeros((h, wp), dtype=a.dtype)
    out[:, :w] = a
    return out


def test_batched_matches_oracle_and_plain_plans():
    from paper_1807_06507_gb300 import swcorr
    swcorr.load()
    scenes = W.batched_scenes(12, scale=0.08)
    dev = []
    for s in scenes:
        h, w = s.x.shape
        xd = to_dev(padded(s.x), torch)[:, :w]
        yd = to_dev(padded(s.y), torch)[:, :w]
        c = torch.full((h, w), -5.0, dtype=torch.float32, device="cuda")
        dev.append((xd, yd, c, s.k))
    bp = swcorr.BatchedPlan(dev)
    for rep in range(2):  # graph replay reuses the reset counter
        for _, _, c, _ in dev:
            c.fill_(-5.0)
        bp.run()
        torch.cuda.synchronize()
        bp.check_status()
        for (xd, yd, c, k), s in zip(dev, scenes):
            got = c.cpu().numpy()
            assert not np.any(got == -5.0)
            score(got, oracle.corr(s.x, s.y, k))
    # same results as one plain plan per scene
    for (xd, yd, c, k), s in zip(dev[:4], scenes[:4]):
        p = swcorr.Plan(s.x.shape, k, dtype="u16")
        cp = p.run(xd, yd)
        torch.cuda.synchronize()
        assert np.allclose(cp.cpu().numpy(), c.cpu().numpy(), rtol=0, atol=2e-7, equal_nan=True)
    bp.close()


def test_batched_rejects_unaligned_pitch():
    from paper_1807_06507_gb300 import swcorr
    x = torch.zeros((10, 13), dtype=torch.int16, device="cuda")
    c = torch.zeros((10, 13), dtype=torch.float32, device="cuda")
    with pytest.raises(swcorr.SwcorrError) as ei:
        swcorr.BatchedPlan([(x, x, c, 3)])
    assert ei.value.status == swcorr.ERR_ALIGNMENT


@pytest.mark.parametrize("ks", [(3, 5, 7), (15, 31), ((3, 9), (9, 3), 1)])
def test_batched_single_engine_and_rectangular(ks):
    # only the 32-bit engine, only the 64-bit engine, rectangular windows
    from paper_1807_06507_gb300 import swcorr
    swcorr.load()
    rng = np.random.default_rng(len(ks))
    dev, ref = [], []
    for i, k in enumerate(ks):
        h, w = int(rng.integers(40, 300)), int(rng.integers(30, 700))
        x, y = W.night_scene((h, w), seed=100 + i)
        xd = to_dev(padded(x), torch)[:, :w]
        yd = to_dev(padded(y), torch)[:, :w]
        c = torch.full((h, w), -5.0, dtype=torch.float32, device="cuda")
        dev.append((xd, yd, c, k))
        ref.append(oracle.corr(x, y, k))
    bp = swcorr.BatchedPlan(dev)
    bp.run()
    torch.cuda.synchronize()
    bp.check_status()
    for (_, _, c, _), r in zip(dev, ref):
        score(c.cpu().numpy(), r)
    bp.close()
