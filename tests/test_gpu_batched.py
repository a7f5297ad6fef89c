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


def f32_scene(rng, h, w, kind):
    if kind == "integer":  # converts exactly: the same results whatever the tiling
        x, y = W.night_scene((h, w), seed=int(rng.integers(1 << 30)))
        return x.astype(np.float32), y.astype(np.float32) - np.float32(900.0)
    x = rng.standard_normal((h, w)).astype(np.float32)
    y = (0.6 * x + rng.standard_normal((h, w))).astype(np.float32)
    if kind == "spiked":  # bright cells force the per-window recomputation
        x[h // 3, w // 2] = np.float32(1e6)
        y[(2 * h) // 3, w // 5] = np.float32(-1e30)
    return x, y


def test_batched_f32_matches_oracle_and_plain_plans():
    from paper_1807_06507_gb300 import swcorr
    swcorr.load()
    rng = np.random.default_rng(31)
    ks = [3, (5, 9), 7, 13, (3, 17), 31, 1, (21, 11), 9]
    kinds = ["integer", "normal", "spiked"]
    dev, host = [], []
    for i, k in enumerate(ks):
        h, w = int(rng.integers(40, 260)), int(rng.integers(30, 600))
        x, y = f32_scene(rng, h, w, kinds[i % 3])
        xd = to_dev(padded(x), torch)[:, :w]
        yd = to_dev(padded(y), torch)[:, :w]
        c = torch.full((h, w), -5.0, dtype=torch.float32, device="cuda")
        dev.append((xd, yd, c, k))
        host.append((x, y, k))
    bp = swcorr.BatchedPlan(dev)
    for rep in range(2):
        for _, _, c, _ in dev:
            c.fill_(-5.0)
        bp.run()
        torch.cuda.synchronize()
        bp.check_status()
        for (_, _, c, _), (x, y, k) in zip(dev, host):
            got = c.cpu().numpy()
            assert not np.any(got == -5.0)
            ref, rx, ry = oracle.corr(x, y, k, relvar=True)
            score(got, ref, rx, ry, exact_nan=False)
    assert bp.fallbacks() > 0, "the spiked scenes took no recomputation"
    # integer-valued scenes: the same results as one plain plan per scene
    for (xd, yd, c, k), (x, y, _) in zip(dev[::3], host[::3]):
        p = swcorr.Plan(x.shape, k, dtype="f32")
        cp = p.run(xd, yd)
        torch.cuda.synchronize()
        p.check_status()
        assert np.allclose(cp.cpu().numpy(), c.cpu().numpy(), rtol=0, atol=2e-6, equal_nan=True)
        p.close()
    bp.close()


def test_batched_rejects_mixed_dtypes():
    from paper_1807_06507_gb300 import swcorr
    xf = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    xu = torch.zeros((16, 16), dtype=torch.int16, device="cuda")
    c = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises((swcorr.SwcorrError, ValueError)):
        swcorr.BatchedPlan([(xf, xf, c, 3), (xu, xu, c, 3)])
