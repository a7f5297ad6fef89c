"""GPU parity of the fused 2-D uint16 kernel against the CPU oracle.

Calls go through the C ABI (ctypes binding).  The integer window sums are
compared bit-exactly with the oracle's brute-force int64 sums; c within 1e-5
on every finite window, with identical NaN masks (the zero-variance test is
exact on both sides).
"""
import numpy as np
import pytest

import oracle
from paper_1807_06507_gb300 import workloads as W
from tests.gpu_util import score, to_dev, sample_indices

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    from paper_1807_06507_gb300 import swcorr
    swcorr.load()
    return swcorr


def run_u16(sw, x, y, k, stride=None, sums=False, **kw):
    p = sw.Plan(x.shape, k, stride, dtype="u16", flags=sw.FLAG_EMIT_SUMS if sums else 0)
    xd, yd = to_dev(x, torch), to_dev(y, torch)
    s = torch.zeros(p.outputs() * 5, dtype=torch.int64, device="cuda") if sums else None
    c = p.run(xd, yd, sums=s, **kw)
    torch.cuda.synchronize()
    p.check_status()
    fb = p.fallbacks()
    out = (c.cpu().numpy(), s.cpu().numpy().reshape(tuple(p.oshape) + (5,)) if sums else None, fb)
    p.close()
    return out


@pytest.mark.parametrize("shape,k", [((257, 530), 7), ((100, 1100), 3), ((64, 97), 5), ((300, 515), 15),
                                     ((200, 300), 31), ((41, 600), (7, 3)), ((90, 128), (3, 9)),
                                     ((33, 40), (1, 7)), ((20, 530), (9, 1))])
def test_night_scene_parity_and_exact_sums(sw, shape, k):
    x, y = W.night_scene(shape, seed=W.seed_for(2) + shape[0])
    c, s, _ = run_u16(sw, x, y, k, sums=True)
    assert np.array_equal(s, oracle.sums_u16(x, y, k))
    score(c, oracle.corr(x, y, k))


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (3, 700), (700, 3), (5, 5), (2, 513), (17, 1025)])
def test_tiny_and_ragged(sw, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.integers(0, 65536, shape).astype(np.uint16)
    y = rng.integers(0, 65536, shape).astype(np.uint16)
    for k in (1, 3, 7):
        c, s, _ = run_u16(sw, x, y, k, sums=True)
        assert np.array_equal(s, oracle.sums_u16(x, y, k))
        score(c, oracle.corr(x, y, k))


def test_full_range_forces_exact_fallback(sw):
    # bright, wide windows: second moments beyond 2^32 must take the exact path
    rng = np.random.default_rng(77)
    x = rng.integers(40000, 65536, (120, 600)).astype(np.uint16)
    y = rng.integers(0, 65536, (120, 600)).astype(np.uint16)
    c, s, fb = run_u16(sw, x, y, 7, sums=True)
    assert fb > 0
    assert np.array_equal(s, oracle.sums_u16(x, y, 7))
    score(c, oracle.corr(x, y, 7))


@pytest.mark.parametrize("shape,k", [((140, 700), 15), ((120, 530), 31), ((90, 600), (3, 31)), ((150, 300), (31, 3)),
                                     ((70, 515), (9, 9)), ((61, 333), (5, 13)), ((40, 260), (65, 1))])
def test_wide_windows_full_range_exact(sw, shape, k):
    # windows of more than 64 cells run the 64-bit engine: exact sums and c
    # on full 16-bit data, with no per-window fallback
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    x = rng.integers(0, 65536, shape).astype(np.uint16)
    y = (x // 2 + rng.integers(0, 32768, shape)).astype(np.uint16)
    c, s, fb = run_u16(sw, x, y, k, sums=True)
    assert fb == 0
    assert np.array_equal(s, oracle.sums_u16(x, y, k))
    score(c, oracle.corr(x, y, k))


def test_wide_windows_strides_pitch_and_nan(sw):
    x, y = W.night_scene((133, 611), seed=21)
    x[10:70, 40:300] = 65535
    y[80:130, 200:600] = 7
    k = (11, 13)
    c, s, fb = run_u16(sw, x, y, k, stride=(2, 3), sums=True)
    assert fb == 0
    assert np.array_equal(s, oracle.sums_u16(x, y, k, (2, 3)))
    ref = oracle.corr(x, y, k, (2, 3))
    assert np.isnan(ref).sum() > 1000
    score(c, ref)
    # a row pitch of 613 elements (not a multiple of 16 bytes): plain loads
    xp = np.zeros((133, 613), np.uint16)
    yp = np.zeros((133, 613), np.uint16)
    xp[:, :611], yp[:, :611] = x, y
    p = sw.Plan(x.shape, k, dtype="u16")
    cp = p.run(to_dev(xp, torch), to_dev(yp, torch), in_pitch=(613, 1))
    torch.cuda.synchronize()
    p.check_status()
    score(cp.cpu().numpy(), oracle.corr(x, y, k))


def test_largest_uint16_window(sw):
    # 1057 x 31 = 32767 cells of full-range data: the window sums reach
    # 2^31 - 2^15 and the variances about 2^61, all still exact
    rng = np.random.default_rng(1057)
    shape = (1100, 40)
    x = rng.integers(0, 65536, shape).astype(np.uint16)
    x[:, :20] = 65535
    y = rng.integers(0, 65536, shape).astype(np.uint16)
    k = (1057, 31)
    c, s, fb = run_u16(sw, x, y, k, sums=True)
    assert fb == 0
    assert np.array_equal(s, oracle.sums_u16(x, y, k))
    score(c, oracle.corr(x, y, k))
    # one row more is beyond the fused kernel's 32768 cells: the plan runs on
    # the general path, whose 64-bit sums are exact too
    c2, s2, _ = run_u16(sw, x, y, (1058, 31), sums=True)
    assert np.array_equal(s2, oracle.sums_u16(x, y, (1058, 31)))
    score(c2, oracle.corr(x, y, (1058, 31)))
    # the limit counts in-bounds cells: a window taller than the grid is fine
    sw.Plan((600, 40), (5001, 31), dtype="u16").close()


@pytest.mark.parametrize("stride", [(2, 2), (3, 1), (1, 2), (2, 3)])
def test_strides(sw, stride):
    x, y = W.night_scene((123, 700), seed=5)
    c, s, _ = run_u16(sw, x, y, 7, stride=stride, sums=True)
    assert c.shape == (-(-123 // stride[0]), -(-700 // stride[1]))
    assert np.array_equal(s, oracle.sums_u16(x, y, 7, stride))
    score(c, oracle.corr(x, y, 7, stride))


def test_constant_patches_are_nan(sw):
    x, y = W.night_scene((150, 400), seed=9)
    x[20:60, 30:200] = 4242
    y[100:140, 100:390] = 0
    c, _, _ = run_u16(sw, x, y, 7)
    ref = oracle.corr(x, y, 7)
    assert np.isnan(ref).sum() > 1000
    score(c, ref)


def test_pitched_input_and_output(sw):
    x, y = W.night_scene((130, 500), seed=11)
    xp = np.zeros((130, 520), np.uint16)
    yp = np.zeros((130, 520), np.uint16)
    xp[:, :500], yp[:, :500] = x, y
    p = sw.Plan(x.shape, 7, dtype="u16")
    xd, yd = to_dev(xp, torch), to_dev(yp, torch)
    cbig = torch.full((130, 512), 7.0, dtype=torch.float32, device="cuda")
    p.run(xd, yd, c=cbig, in_pitch=(520, 1), out_pitch=(512, 1))
    torch.cuda.synchronize()
    p.check_status()
    cb = cbig.cpu().numpy()
    assert np.all(cb[:, 500:] == 7.0)
    score(cb[:, :500], oracle.corr(x, y, 7))


def test_unaligned_pitch_uses_plain_loads(sw):
    # a row pitch of 51 uint16 (102 B) cannot be described to TMA; the
    # plain-load row loader must give the same results
    rng = np.random.default_rng(4)
    x = rng.integers(0, 16384, (40, 51)).astype(np.uint16)
    y = rng.integers(0, 16384, (40, 51)).astype(np.uint16)
    c, s, _ = run_u16(sw, x, y, 5, sums=True)
    assert np.array_equal(s, oracle.sums_u16(x, y, 5))
    score(c, oracle.corr(x, y, 5))
    xs, ys = x[:, :50], y[:, :50]
    p = sw.Plan((40, 50), 5, dtype="u16")
    cp = p.run(to_dev(x, torch), to_dev(y, torch), in_pitch=(51, 1))
    torch.cuda.synchronize()
    score(cp.cpu().numpy(), oracle.corr(np.ascontiguousarray(xs), np.ascontiguousarray(ys), 5))


def test_odd_base_address_rejected(sw):
    p = sw.Plan((10, 48), 3, dtype="u16")
    buf = torch.zeros(10 * 48 * 2 + 16, dtype=torch.uint8, device="cuda")
    c = torch.empty((10, 48), dtype=torch.float32, device="cuda")

    class Odd:
        def __init__(self, ptr):
            self.ptr = ptr

        def data_ptr(self):
            return self.ptr

        def is_contiguous(self):
            return True

        device = buf.device

    with pytest.raises(sw.SwcorrError) as ei:
        p.run(Odd(buf.data_ptr() + 1), Odd(buf.data_ptr() + 1), c=c)
    assert ei.value.status == sw.ERR_ALIGNMENT


def test_night_scene_full_size(sw):
    # 12 Mpx night scene, 7x7: every window against the oracle.
    x, y = W.night_scene((3000, 4000), seed=W.seed_for(2))
    c, s, fb = run_u16(sw, x, y, 7, sums=True)
    assert np.array_equal(s, oracle.sums_u16(x, y, 7))
    m, n_sc, _ = score(c, oracle.corr(x, y, 7))
    assert n_sc > 11_000_000


def _pinned(a, torch):
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).pin_memory()
    v = t.numpy()
    return (v.view(np.uint16) if a.dtype == np.uint16 else v), t


@pytest.mark.parametrize("stride", [None, (2, 3)])
def test_host_run_pinned_graph(sw, stride):
    # page-locked buffers take the recorded-graph path: a replay must read the
    # buffers' current contents, and new buffers must re-record
    import torch
    shape = (530, 1000)
    x0, y0 = W.night_scene(shape, seed=21)
    x1, y1 = W.night_scene(shape, seed=22)
    p = sw.Plan(shape, 7, stride, dtype="u16")
    hx, tx = _pinned(x0, torch)
    hy, ty = _pinned(y0, torch)
    c = torch.empty(p.oshape, dtype=torch.float32).pin_memory().numpy()

    def dev(x, y):
        r = p.run(to_dev(x, torch), to_dev(y, torch))
        torch.cuda.synchronize()
        return r.cpu().numpy()

    p.run_host(hx, hy, c)
    assert np.array_equal(c, dev(x0, y0), equal_nan=True)
    hx[...] = x1
    hy[...] = y1
    c[...] = 7.0
    p.run_host(hx, hy, c)  # replay
    assert np.array_equal(c, dev(x1, y1), equal_nan=True)
    hx2, tx2 = _pinned(x0, torch)
    c2 = torch.empty(p.oshape, dtype=torch.float32).pin_memory().numpy()
    p.run_host(hx2, hy, c2)  # new buffers: re-recorded
    assert np.array_equal(c2, dev(x0, y1), equal_nan=True)
    score(c2, oracle.corr(x0, y1, 7, stride=stride))
    p.check_status()


def test_host_run_mixed_page_locking(sw):
    # only all-page-locked buffers take the recorded graph; every mix takes
    # the stream path, and all give the device run's result
    import torch
    shape = (300, 512)
    x, y = W.night_scene(shape, seed=23)
    p = sw.Plan(shape, 5, dtype="u16")
    ref = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    hx, tx = _pinned(x, torch)
    hy, ty = _pinned(y, torch)
    pinned_c = torch.empty(p.oshape, dtype=torch.float32).pin_memory().numpy()
    for xx, yy, cc in ((hx, hy, np.empty(p.oshape, np.float32)), (x.copy(), y.copy(), pinned_c),
                       (hx, y.copy(), pinned_c), (hx, hy, pinned_c)):
        cc[...] = 5.0
        p.run_host(xx, yy, cc)
        assert np.array_equal(cc, ref, equal_nan=True)
    p.check_status()


@pytest.mark.parametrize("shape,k,stride", [((230, 640), 31, None), ((180, 512), (31, 3), None),
                                             ((200, 520), (3, 31), (2, 1)), ((150, 600), 9, (1, 3))])
def test_host_run_tall_windows_and_wide_engine(sw, shape, k, stride):
    # band halos reach into earlier bands' rows; k >= 9 runs the 64-bit engine
    import torch
    x, y = W.night_scene(shape, seed=31)
    p = sw.Plan(shape, k, stride, dtype="u16")
    ref = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    hx, tx = _pinned(x, torch)
    hy, ty = _pinned(y, torch)
    c = torch.empty(p.oshape, dtype=torch.float32).pin_memory().numpy()
    p.run_host(hx, hy, c)  # recorded graph, direct output
    assert np.array_equal(c, ref, equal_nan=True)
    assert np.array_equal(p.run_host(x, y), ref, equal_nan=True)  # stream path
    p.check_status()


def test_host_run_matches_device_run(sw):
    x, y = W.night_scene((200, 640), seed=13)
    p = sw.Plan(x.shape, 7, dtype="u16")
    ch = p.run_host(x, y)
    cd = p.run(to_dev(x, torch), to_dev(y, torch))
    torch.cuda.synchronize()
    assert np.array_equal(ch, cd.cpu().numpy(), equal_nan=True)
    score(ch, oracle.corr(x, y, 7))
