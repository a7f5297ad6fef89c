"""The no-allocation 2-D uint16 entry point, called through the C ABI.

Callers whose device memory belongs to their own pool allocator, or that
must not call cudaMalloc in a latency-critical loop, use
swcorr_run2d_u16_noalloc: its kernel keeps its scratch in a static device
array of the library.  This file checks, on two calls in a row with different
inputs, that its output equals the plan path's output (same kernel, same
tolerance as every parity test), and that the second call is not disturbed by
what the first one left in the shared array.  It is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1807_06507_gb300 import workloads as W
from tests.gpu_util import score, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def noalloc_run(lib, x, y, k):
    rows, cols = x.shape
    xd, yd = to_dev(x, torch), to_dev(y, torch)
    c = torch.full((rows, cols), -7.0, dtype=torch.float32, device="cuda")
    st = lib.swcorr_run2d_u16_noalloc(rows, cols, k, k, ctypes.c_void_p(xd.data_ptr()),
                                      ctypes.c_void_p(yd.data_ptr()), cols, ctypes.c_void_p(c.data_ptr()), cols,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.swcorr_last_error().decode()
    torch.cuda.synchronize()
    return c.cpu().numpy()


def plan_run(sw, x, y, k):
    p = sw.Plan(x.shape, k, dtype="u16")
    c = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    p.check_status()
    out = c.cpu().numpy()
    p.close()
    return out


def test_noalloc_matches_plan_path_twice():
    from paper_1807_06507_gb300 import swcorr
    lib = swcorr.load()
    cases = [(W.night_scene((301, 1040), seed=31), 7), (W.night_scene((257, 777), seed=32), 5)]
    for (x, y), k in cases:
        got = noalloc_run(lib, x, y, k)
        ref = plan_run(swcorr, x, y, k)
        assert not np.any(got == -7.0)
        score(got, ref.astype(np.float64), tol=1e-5)


def test_noalloc_rejects_bad_sizes():
    from paper_1807_06507_gb300 import swcorr
    lib = swcorr.load()
    null = ctypes.c_void_p(0)
    st = lib.swcorr_run2d_u16_noalloc(1 << 31, 8, 7, 7, null, null, 0, null, 0, null)
    assert st == swcorr.ERR_UNSUPPORTED and b"32-bit" in lib.swcorr_last_error()
    assert lib.swcorr_run2d_u16_noalloc(0, 8, 7, 7, null, null, 0, null, 0, null) == swcorr.ERR_INVALID_ARG
