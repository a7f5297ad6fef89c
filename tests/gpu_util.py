"""Helpers shared by the GPU parity tests (host-side marshalling and scoring)."""
import numpy as np

import oracle

TOL = 1e-5          # max |c_gpu - c_oracle| on scored windows
RELVAR_MIN = 1e-6   # scored: relative variance of both channels above this


def to_dev(a, torch):
    """numpy -> CUDA tensor with the same bits (uint16 travels as int16)."""
    if a.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def score(c_gpu, c_ref, rvx=None, rvy=None, tol=TOL, exact_nan=True):
    """Compare GPU float32 c with the oracle's float64 c.

    Oracle NaN => GPU NaN is required everywhere.  With exact_nan the NaN
    masks must be identical (exact integer paths).  Scored windows (both
    relative variances > RELVAR_MIN, or all finite windows when no relvar is
    given) must agree within tol.  Returns (max_err, n_scored, n_unscored).
    """
    c_gpu = np.asarray(c_gpu, dtype=np.float64)
    ref_nan = np.isnan(c_ref)
    gpu_nan = np.isnan(c_gpu)
    assert np.all(gpu_nan[ref_nan]), f"{int((~gpu_nan[ref_nan]).sum())} windows finite on GPU but NaN in oracle"
    if exact_nan:
        assert np.array_equal(ref_nan, gpu_nan), f"{int((gpu_nan & ~ref_nan).sum())} extra GPU NaNs"
    if rvx is None:
        scored = ~ref_nan
    else:
        scored = (~ref_nan) & (rvx > RELVAR_MIN) & (rvy > RELVAR_MIN)
    assert not np.any(gpu_nan[scored]), "GPU NaN on a scored window"
    err = np.abs(c_gpu[scored] - c_ref[scored])
    m = float(err.max()) if err.size else 0.0
    assert m <= tol, f"max |dc| = {m:.3e} > {tol:g} ({int((err > tol).sum())} of {err.size} windows)"
    assert np.all(np.abs(c_gpu[~gpu_nan]) <= 1.0)
    return m, int(scored.sum()), int((~ref_nan & ~scored).sum())


def sample_indices(oshape, n, rng, borders=True):
    """Flat output indices: n uniform ones plus (optionally) every border window
    within 40 cells of an edge along the first/last rows/cols of a 2-D grid."""
    total = int(np.prod(oshape))
    idx = [rng.integers(0, total, n)]
    if borders and len(oshape) == 2:
        H, W = oshape
        rr = np.r_[0:min(40, H), max(0, H - 40):H]
        cc = np.r_[0:min(40, W), max(0, W - 40):W]
        g = np.concatenate([(rr[:, None] * W + np.arange(W)[None, :]).ravel(),
                            (np.arange(H)[:, None] * W + cc[None, :]).ravel()])
        idx.append(g)
    return np.unique(np.concatenate(idx))
