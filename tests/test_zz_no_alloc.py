"""The no-allocation 2-D uint16 entry point, called through the C ABI.

Callers whose device memory belongs to their own pool allocator, or that
must not call cudaMalloc in a latency-critical loop, use
swcorr_run2d_u16_noalloc: its kernel keeps its scratch in a static device
array of the library.  This file checks, on two calls in a row with different
inputs, that its output equals the plan path's output and the CPU oracle's
(same tolerance as every parity test), that the second call is not disturbed
by what the first one left in the shared array, that padded row pitches are
honoured (the plain-load row loader) with the padding of c untouched, and
that swcorr_noalloc_status reports a clean run.  It is collected last so that
a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1807_06507_gb300 import workloads as W
from tests.gpu_util import score, to_dev

torch = pytest.importorskip("torch")

SENTINEL = -7.0


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def noalloc_run(lib, x, y, k, pad_in=0, pad_out=0):
    """Run the entry point on (optionally row-padded) device copies of x, y."""
    rows, cols = x.shape
    ip, op = cols + pad_in, cols + pad_out
    xp = np.zeros((rows, ip), np.uint16)
    yp = np.zeros((rows, ip), np.uint16)
    xp[:, :cols], yp[:, :cols] = x, y
    xd, yd = to_dev(xp, torch), to_dev(yp, torch)
    c = torch.full((rows, op), SENTINEL, dtype=torch.float32, device="cuda")
    st = lib.swcorr_run2d_u16_noalloc(rows, cols, k, k, ctypes.c_void_p(xd.data_ptr()),
                                      ctypes.c_void_p(yd.data_ptr()), ip, ctypes.c_void_p(c.data_ptr()), op,
                                      _stream())
    assert st == 0, lib.swcorr_last_error().decode()
    fb = ctypes.c_int64(-5)
    st = lib.swcorr_noalloc_status(_stream(), ctypes.byref(fb))
    assert st == 0, lib.swcorr_last_error().decode()
    assert fb.value >= 0
    out = c.cpu().numpy()
    assert np.all(out[:, cols:] == SENTINEL), "padding columns of c were written"
    return out[:, :cols]


def plan_run(sw, x, y, k):
    p = sw.Plan(x.shape, k, dtype="u16")
    c = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    p.check_status()
    out = c.cpu().numpy()
    p.close()
    return out


@pytest.mark.gpu
def test_noalloc_matches_plan_path_and_oracle_twice():
    from paper_1807_06507_gb300 import swcorr
    lib = swcorr.load()
    cases = [(W.night_scene((301, 1040), seed=31), 7), (W.night_scene((257, 777), seed=32), 5)]
    for (x, y), k in cases:
        got = noalloc_run(lib, x, y, k)
        assert not np.any(got == SENTINEL)
        ref = plan_run(swcorr, x, y, k)
        score(got, ref.astype(np.float64), tol=1e-5)
        score(got, oracle.corr(x, y, k), tol=1e-5)


@pytest.mark.gpu
def test_noalloc_padded_pitches():
    from paper_1807_06507_gb300 import swcorr
    lib = swcorr.load()
    x, y = W.night_scene((97, 301), seed=33)
    got = noalloc_run(lib, x, y, 7, pad_in=3, pad_out=5)
    score(got, oracle.corr(x, y, 7), tol=1e-5)


def test_noalloc_rejects_bad_sizes():
    from paper_1807_06507_gb300 import swcorr
    lib = swcorr.load()
    null = ctypes.c_void_p(0)
    st = lib.swcorr_run2d_u16_noalloc(1 << 31, 8, 7, 7, null, null, 0, null, 0, null)
    assert st == swcorr.ERR_UNSUPPORTED and b"32-bit" in lib.swcorr_last_error()
    assert lib.swcorr_run2d_u16_noalloc(0, 8, 7, 7, null, null, 0, null, 0, null) == swcorr.ERR_INVALID_ARG


def test_noalloc_rejects_misaligned_output():
    """A c pointer that is not 4-byte aligned is refused on the host, before
    any device work (these pointers are never dereferenced)."""
    from paper_1807_06507_gb300 import swcorr
    lib = swcorr.load()
    p16 = ctypes.c_void_p(1 << 20)
    st = lib.swcorr_run2d_u16_noalloc(64, 64, 7, 7, p16, p16, 0, ctypes.c_void_p((1 << 20) + 2), 0, None)
    assert st == swcorr.ERR_ALIGNMENT and b"4-byte" in lib.swcorr_last_error()
