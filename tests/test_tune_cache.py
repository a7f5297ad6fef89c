"""Tune cache: JSON parsing and lookup in the C library (no GPU needed), and
tuned plans on the GPU (same results as the defaults)."""
import json

import numpy as np
import pytest

from paper_1807_06507_gb300 import swcorr


@pytest.fixture()
def sw(tmp_path):
    swcorr.load()
    yield swcorr
    # back to the package's own cache (or none)
    swcorr.set_tune_file(swcorr.DEFAULT_TUNE_FILE if __import__("os").path.exists(swcorr.DEFAULT_TUNE_FILE)
                         else None)


def _write(tmp_path, doc):
    p = tmp_path / "tune.json"
    p.write_text(doc if isinstance(doc, str) else json.dumps(doc))
    return str(p)


DOC = {"format": "swcorr-tune-1", "entries": [
    {"device": "GPU A", "kind": "plain", "ndim": 2, "dtype": "u16", "k": [7, 7], "prefetch": 3, "tile_rows": 21,
     "ctas_per_sm": 12, "us": 50.0},
    {"device": "GPU A", "ndim": 1, "dtype": "f32", "k": [1001], "ctas_per_sm": 4},
    {"device": "GPU B", "kind": "plain", "ndim": 2, "dtype": "u16", "k": [7, 7], "prefetch": 5},
    {"device": "GPU A", "kind": "batched", "ndim": 2, "dtype": "u16", "k": [0, 0], "prefetch": 6, "tile_rows": 32},
]}


def test_lookup_by_device_window_and_dtype(sw, tmp_path):
    sw.set_tune_file(_write(tmp_path, DOC))
    assert sw.tune_lookup(2, 7, "u16", device="GPU A") == {"prefetch": 3, "tile_rows": 21, "ctas_per_sm": 12}
    assert sw.tune_lookup(2, 7, "u16", device="GPU B") == {"prefetch": 5, "tile_rows": 0, "ctas_per_sm": 0}
    assert sw.tune_lookup(1, 1001, "f32", device="GPU A") == {"prefetch": 0, "tile_rows": 0, "ctas_per_sm": 4}
    assert sw.tune_lookup(2, 7, "f32", device="GPU A") is None       # other dtype
    assert sw.tune_lookup(2, (7, 5), "u16", device="GPU A") is None  # other window
    assert sw.tune_lookup(2, 7, "u16", device="GPU C") is None       # other device
    assert sw.tune_lookup(2, 0, "u16", device="GPU A", batched=True) == {"prefetch": 6, "tile_rows": 32,
                                                                          "ctas_per_sm": 0}
    # the batched entry serves any window
    assert sw.tune_lookup(2, 31, "u16", device="GPU A", batched=True)["prefetch"] == 6


@pytest.mark.parametrize("bad", [
    "{not json",
    '{"format": "swcorr-tune-1"}',
    '{"format": "other", "entries": []}',
    json.dumps({"format": "swcorr-tune-1", "entries": [{"device": "A", "ndim": 2, "dtype": "u16", "k": [7]}]}),
    json.dumps({"format": "swcorr-tune-1", "entries": [{"device": "A", "ndim": 2, "dtype": "u8", "k": [7, 7]}]}),
    json.dumps({"format": "swcorr-tune-1", "entries": [{"device": "A", "ndim": 2, "dtype": "u16", "k": [7, 7],
                                                         "prefetch": 99}]}),
    json.dumps({"format": "swcorr-tune-1", "entries": [{"device": "A", "ndim": 2, "dtype": "u16", "k": [7, 7],
                                                         "tile_rows": 1.5}]}),
])
def test_bad_file_is_ignored_as_a_whole(sw, tmp_path, bad):
    sw.set_tune_file(_write(tmp_path, DOC))
    assert sw.tune_lookup(2, 7, "u16", device="GPU A") is not None
    with pytest.raises(sw.SwcorrError) as ei:
        sw.set_tune_file(_write(tmp_path, bad))
    assert ei.value.status == sw.ERR_INVALID_ARG
    assert sw.tune_lookup(2, 7, "u16", device="GPU A") is None


def test_missing_file_and_no_cache(sw, tmp_path):
    with pytest.raises(sw.SwcorrError):
        sw.set_tune_file(str(tmp_path / "does_not_exist.json"))
    sw.set_tune_file(None)
    assert sw.tune_lookup(2, 7, "u16") is None


def test_unknown_tune_field_rejected_by_binding(sw):
    with pytest.raises(KeyError):
        swcorr._tune_struct({"warps": 4})


def test_shipped_cache_parses(sw):
    import os
    if not os.path.exists(sw.DEFAULT_TUNE_FILE):
        pytest.skip("no tune cache shipped")
    sw.set_tune_file(sw.DEFAULT_TUNE_FILE)
    with open(sw.DEFAULT_TUNE_FILE) as f:
        doc = json.load(f)
    for e in doc["entries"]:
        got = sw.tune_lookup(e["ndim"], e["k"], e["dtype"], device=e["device"], batched=e["kind"] == "batched")
        assert got == {k: e.get(k, 0) for k in swcorr.TUNE_FIELDS}


# ------------------------------------------------------------------ GPU
@pytest.mark.gpu
@pytest.mark.parametrize("tune", [{"prefetch": 2}, {"prefetch": 6, "tile_rows": 16}, {"tile_rows": 40},
                                  {"ctas_per_sm": 5}, {"prefetch": 8, "tile_rows": 100, "ctas_per_sm": 1}])
def test_tuned_plans_give_the_default_results(sw, tune):
    import torch
    from paper_1807_06507_gb300 import workloads as W
    from tests.gpu_util import to_dev
    x, y = W.night_scene((300, 1100), seed=4)
    d = sw.Plan(x.shape, 7, dtype="u16", tune={})
    t = sw.Plan(x.shape, 7, dtype="u16", tune=tune)
    got = t.tune()
    for k, v in tune.items():
        assert got[k] == v or (k == "ctas_per_sm" and got[k] <= v)
    xd, yd = to_dev(x, torch), to_dev(y, torch)
    c0 = d.run(xd, yd)
    c1 = t.run(xd, yd)
    torch.cuda.synchronize()
    d.check_status()
    t.check_status()
    assert np.array_equal(c0.cpu().numpy(), c1.cpu().numpy(), equal_nan=True)


@pytest.mark.gpu
def test_out_of_range_tune_rejected(sw):
    for bad in ({"prefetch": 9}, {"tile_rows": -1}, {"ctas_per_sm": 33}):
        with pytest.raises(sw.SwcorrError) as ei:
            sw.Plan((100, 100), 7, dtype="u16", tune=bad)
        assert ei.value.status == sw.ERR_INVALID_ARG


@pytest.mark.gpu
def test_plan_reads_the_cache(sw, tmp_path):
    import torch
    dev = torch.cuda.get_device_name()
    doc = {"format": "swcorr-tune-1", "entries": [
        {"device": dev, "kind": "plain", "ndim": 2, "dtype": "u16", "k": [5, 5], "prefetch": 7, "tile_rows": 33}]}
    sw.set_tune_file(_write(tmp_path, doc))
    p = sw.Plan((500, 600), 5, dtype="u16")
    assert p.tune()["prefetch"] == 7 and p.tune()["tile_rows"] == 33
    q = sw.Plan((500, 600), 3, dtype="u16")
    assert q.tune()["prefetch"] != 7
