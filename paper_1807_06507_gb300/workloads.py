"""Seeded synthetic workloads for the sliding-window correlation.

These generators stand in for the paper's VIIRS visible/infrared night
images (Section 3 tests on a 4064x3072 pair that is not available here) and
for the other workload shapes the library is measured on.  They hold none of
the correlation method's arithmetic: they only synthesise input grids, so the
tests and the benchmark can feed the same arrays to the CUDA path and to the
CPU oracle.  numpy only; every generator takes an explicit seed.

Shapes are C order: dimension 0 is the outermost (rows for 2-D, planes for
3-D), the last dimension is contiguous.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 180706507


def seed_for(config_index: int) -> int:
    return BASE_SEED + int(config_index)


# ---------------------------------------------------------------- 2-D, U(0,1)
def uniform_pair(shape=(512, 512), seed=seed_for(1)):
    """x ~ U(0,1); y = -0.8 x + 0.2 N(0,1), float32 (2-D 512x512 by default)."""
    rng = np.random.default_rng(seed)
    x = rng.random(shape, dtype=np.float64)
    y = -0.8 * x + 0.2 * rng.standard_normal(shape)
    return x.astype(np.float32), y.astype(np.float32)


# ------------------------------------------------------ 2-D night scene (u16)
def _value_noise(rng, shape, period):
    """Bilinear upsampling of a random lattice with the given period (pixels),
    interpolated along columns first, then along rows (float32)."""
    h, w = shape
    gh, gw = h // period + 2, w // period + 2
    lat = rng.random((gh, gw), dtype=np.float32)
    ry = np.arange(h, dtype=np.float32) / np.float32(period)
    rx = np.arange(w, dtype=np.float32) / np.float32(period)
    iy = ry.astype(np.int64)
    ix = rx.astype(np.int64)
    fy = (ry - iy)[:, None]
    fx = (rx - ix)[None, :]
    lx = lat[:, ix] * (1 - fx) + lat[:, ix + 1] * fx
    return lx[iy] * (1 - fy) + lx[iy + 1] * fy


def _upsample(a, factor, shape):
    """Bilinear upsampling of a coarse grid by an integer factor, cropped to shape."""
    h, w = shape
    ry = np.arange(h, dtype=np.float32) / np.float32(factor)
    rx = np.arange(w, dtype=np.float32) / np.float32(factor)
    iy = np.minimum(ry.astype(np.int64), a.shape[0] - 2)
    ix = np.minimum(rx.astype(np.int64), a.shape[1] - 2)
    fy = (ry - iy)[:, None]
    fx = (rx - ix)[None, :]
    lx = a[:, ix] * (1 - fx) + a[:, ix + 1] * fx
    return lx[iy] * (1 - fy) + lx[iy + 1] * fy


def cloud_field(rng, shape, coverage=0.30, coarse=4):
    """Smooth multi-octave value noise mapped to a [0,1] cloud opacity.

    Octaves at periods 512/256/128/64 px with halving amplitudes, evaluated on
    a grid `coarse` times sparser (the field is smooth at that scale) and
    normalised to [0,1]; the top `coverage` fraction becomes cloud with a
    linear ramp; the result is upsampled bilinearly to full resolution.
    """
    h, w = shape
    cs = (h // coarse + 2, w // coarse + 2)
    p = np.zeros(cs, dtype=np.float32)
    amp = np.float32(1.0)
    for period in (512, 256, 128, 64):
        p += amp * _value_noise(rng, cs, period // coarse)
        amp *= np.float32(0.5)
    p = (p - p.min()) / max(float(p.max() - p.min()), 1e-12)
    q = np.quantile(p, 1.0 - coverage)
    f = np.clip((p - q) / max(1.0 - q, 1e-12), 0.0, 1.0).astype(np.float32)
    return _upsample(f, coarse, shape)


def night_scene(shape=(3000, 4000), seed=seed_for(2), n_sources=None,
                vis_mean=200.0, ir_mean=4000.0, sd=20.0):
    """Visible/infrared night-scene pair, uint16 with 14-bit values.

    Dark Gaussian background (visible mean 200, infrared mean 4000, sd 20),
    point sources (Gaussian PSF sigma = 1 px, peak U(8000, 16000), 7x7
    footprint) in the visible channel only (about 2000 per 12 Mpx), and a
    smooth 30%-coverage cloud field that raises visible by up to 3000 and
    lowers infrared by up to 2500.  Rounded and clipped to [0, 16383].
    """
    rng = np.random.default_rng(seed)
    h, w = shape
    if n_sources is None:
        n_sources = int(round(2000 * h * w / 12e6))
    vis = np.float32(vis_mean) + np.float32(sd) * rng.standard_normal(shape, dtype=np.float32)
    ir = np.float32(ir_mean) + np.float32(sd) * rng.standard_normal(shape, dtype=np.float32)
    if n_sources > 0:
        ys = rng.integers(0, h, n_sources)
        xs = rng.integers(0, w, n_sources)
        peak = rng.uniform(8000.0, 16000.0, n_sources)
        for dy in range(-3, 4):
            for dx in range(-3, 4):
                yy, xx = ys + dy, xs + dx
                ok = (yy >= 0) & (yy < h) & (xx >= 0) & (xx < w)
                np.add.at(vis, (yy[ok], xx[ok]), (peak[ok] * np.exp(-0.5 * (dy * dy + dx * dx))).astype(np.float32))
    f = cloud_field(rng, shape)
    vis += np.float32(3000.0) * f
    ir -= np.float32(2500.0) * f
    vis = np.clip(np.rint(vis), 0, 16383).astype(np.uint16)
    ir = np.clip(np.rint(ir), 0, 16383).astype(np.uint16)
    return vis, ir


# ----------------------------------------------------- 1-D random-walk series
def random_walk_pair(n=1 << 26, seed=seed_for(3), offset=1e4, flip=1 << 20, phi=0.9):
    """Two float32 series: x a unit-step random walk from 1e4; y = s(t)*0.5*x + e.

    e is AR(1) noise (phi = 0.9, N(0,1) innovations) and the sign s(t) flips
    every `flip` samples.  In-window spread is tiny next to the 1e4 offset,
    the hard case for cancellation.
    """
    rng = np.random.default_rng(seed)
    steps = rng.standard_normal(n)
    steps[0] = 0.0
    x = offset + np.cumsum(steps)
    innov = rng.standard_normal(n)
    e = np.empty(n)
    # AR(1) by blocks of a linear filter: e_t = phi e_{t-1} + u_t
    try:
        from scipy.signal import lfilter
        e[:] = lfilter([1.0], [1.0, -phi], innov)
    except Exception:  # pragma: no cover - scipy is normally present
        acc = 0.0
        for t in range(n):
            acc = phi * acc + innov[t]
            e[t] = acc
    sign = np.where((np.arange(n) // flip) % 2 == 0, 1.0, -1.0)
    y = sign * 0.5 * x + e
    return x.astype(np.float32), y.astype(np.float32)


# ------------------------------------------------------------ 3-D volumes
def _box3_mean_inbounds(a):
    """3x3x3 box mean over in-bounds cells (input smoothing, not the method)."""
    s = np.zeros_like(a)
    cnt = np.zeros_like(a)
    ones = np.ones_like(a)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                for ax, d in enumerate((dz, dy, dx)):
                    n = a.shape[ax]
                    if d > 0:
                        dst[ax], src[ax] = slice(0, n - d), slice(d, n)
                    elif d < 0:
                        dst[ax], src[ax] = slice(-d, n), slice(0, n + d)
                s[tuple(dst)] += a[tuple(src)]
                cnt[tuple(dst)] += ones[tuple(src)]
    return s / cnt


def halfspace_volume_pair(shape=(256, 512, 512), seed=seed_for(4)):
    """x = 3x3x3 box mean of N(0,1); y = x inside a random half-space, N(0,1) outside."""
    rng = np.random.default_rng(seed)
    x = _box3_mean_inbounds(rng.standard_normal(shape).astype(np.float32))
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    p0 = rng.random(3) * np.asarray(shape)
    zz = (np.arange(shape[0]) - p0[0]) * u[0]
    yy = (np.arange(shape[1]) - p0[1]) * u[1]
    xx = (np.arange(shape[2]) - p0[2]) * u[2]
    mask = (zz[:, None, None] + yy[None, :, None] + xx[None, None, :]) >= 0
    noise = rng.standard_normal(shape).astype(np.float32)
    y = np.where(mask, x, noise)
    return x.astype(np.float32), y.astype(np.float32)


# ----------------------------------------------------------- batched scenes
@dataclass
class Scene:
    x: np.ndarray
    y: np.ndarray
    k: int
    seed: int = 0
    meta: dict = field(default_factory=dict)


def batched_scenes(n_scenes=64, seed=seed_for(5), w_range=(1024, 6000), h_range=(1024, 4000),
                   k_choices=(3, 5, 7, 15, 31), scale=1.0):
    """Uneven uint16 scene pairs for the batched launch.

    Per scene: width ~ U{1024..6000}, height ~ U{1024..4000} (both multiplied
    by `scale` for small test runs), square window k ~ U{3,5,7,15,31}, pixels
    from night_scene with its own seed.
    """
    rng = np.random.default_rng(seed)
    scenes = []
    for i in range(n_scenes):
        w = int(rng.integers(w_range[0], w_range[1] + 1))
        h = int(rng.integers(h_range[0], h_range[1] + 1))
        k = int(rng.choice(k_choices))
        w = max(1, int(round(w * scale)))
        h = max(1, int(round(h * scale)))
        vis, ir = night_scene((h, w), seed=seed + 1000 + i)
        scenes.append(Scene(vis, ir, k, seed + 1000 + i, {"h": h, "w": w}))
    return scenes


# ---------------------------------------------------- float data off the grid
def smooth_field_pair(shape, seed=seed_for(7), noise=0.01):
    """A smooth log-normal field f = exp(2 prod_d trig(i_d / L_d)) on a grid of
    any dimension (L = 97, 61, 43, ... cells; sin on the last axis, cos on
    the others), x = f (1 + noise N(0,1)), y = f / 2 + 2 noise N(0,1)
    (float32): radiance-like data whose windows have a spread small next to
    the range of the tile they sit in."""
    rng = np.random.default_rng(seed)
    scales = (97.0, 61.0, 43.0, 37.0, 29.0, 23.0, 19.0, 17.0)
    arg = np.ones(shape, dtype=np.float64)
    for d, n in enumerate(shape):
        ax = np.arange(n, dtype=np.float64) / scales[len(shape) - 1 - d]
        trig = np.sin(ax) if d == len(shape) - 1 else np.cos(ax)
        arg = arg * trig.reshape((1,) * d + (n,) + (1,) * (len(shape) - 1 - d))
    f = np.exp(2.0 * arg).astype(np.float32)
    x = (f * (1 + noise * rng.standard_normal(shape))).astype(np.float32)
    y = (0.5 * f + 2 * noise * rng.standard_normal(shape)).astype(np.float32)
    return x, y


# ------------------------------------------------------- n-dimensional grids
def correlated_grid_pair(shape, seed=seed_for(6), rho=0.5):
    """x ~ N(0,1) iid on a grid of any dimension; y = rho x + N(0,1) noise
    (float32): the general n-dimensional path's workload."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape, dtype=np.float32)
    y = np.float32(rho) * x + rng.standard_normal(shape, dtype=np.float32)
    return x, y.astype(np.float32)
