"""Failure path on the GPU without a fault: a bounded device wait that runs
out (the test hook withholds one row's copy) must end its kernel with a
status the host reads, leave every other work item correct and the context
usable."""
import time

import numpy as np
import pytest

import oracle
from paper_1807_06507_gb300 import workloads as W
from tests.gpu_util import score, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_the_rest_completes():
    from paper_1807_06507_gb300 import swcorr
    swcorr.load()
    x, y = W.night_scene((256, 1024), seed=31)
    xd, yd = to_dev(x, torch), to_dev(y, torch)
    p = swcorr.Plan(x.shape, 7, dtype="u16", flags=swcorr.FLAG_TEST_STALL)
    c = torch.full(x.shape, -7.0, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    p.run(xd, yd, c=c)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert p.status() == swcorr.ERR_TIMEOUT
    assert p.status() == swcorr.OK  # reading the status resets it
    assert 0.2 < waited < 30.0
    # every strip but the stalled item's (columns 0..255, first row block) is right
    ref = oracle.corr(x, y, 7)
    got = c.cpu().numpy()
    score(got[:, 256:], ref[:, 256:])
    p.close()
    # the context is still usable: a plain plan on the same data
    q = swcorr.Plan(x.shape, 7, dtype="u16")
    c2 = q.run(xd, yd)
    torch.cuda.synchronize()
    q.check_status()
    score(c2.cpu().numpy(), ref)


def test_stall_hook_rejected_outside_2d_u16():
    from paper_1807_06507_gb300 import swcorr
    for shape, dt in (((1000,), "u16"), ((64, 64), "f32"), ((4, 8, 8), "u16")):
        with pytest.raises(swcorr.SwcorrError) as ei:
            swcorr.Plan(shape, 3, dtype=dt, flags=swcorr.FLAG_TEST_STALL)
        assert ei.value.status == swcorr.ERR_INVALID_ARG
