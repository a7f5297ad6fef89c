"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects bad arguments without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "swcorr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(swcorr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_06507_gb300 import build, swcorr
    build.build()
    return swcorr.load()


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    from paper_1807_06507_gb300 import swcorr
    assert sorted(swcorr.EXPORTS) == declared_symbols()


def test_status_strings(lib):
    for st in range(8):
        assert lib.swcorr_status_string(st)
    assert b"sm_103a" in lib.swcorr_version()


def test_argument_errors_without_gpu(lib):
    from paper_1807_06507_gb300 import swcorr
    h = ctypes.c_void_p()
    shape = (ctypes.c_int64 * 2)(10, 10)
    k = (ctypes.c_int32 * 2)(3, 3)
    bad_k = (ctypes.c_int32 * 2)(0, 3)
    assert lib.swcorr_plan_create(None, 2, shape, k, None, swcorr.U16, 0, 0) == swcorr.ERR_INVALID_ARG
    shape9 = (ctypes.c_int64 * 9)(*([4] * 9))
    k9 = (ctypes.c_int32 * 9)(*([3] * 9))
    assert lib.swcorr_plan_create(ctypes.byref(h), 9, shape9, k9, None, swcorr.U16, 0, 0) == swcorr.ERR_UNSUPPORTED
    assert lib.swcorr_plan_create(ctypes.byref(h), 0, shape9, k9, None, swcorr.U16, 0, 0) == swcorr.ERR_UNSUPPORTED
    assert lib.swcorr_plan_create(ctypes.byref(h), 2, shape, bad_k, None, swcorr.U16, 0, 0) == swcorr.ERR_INVALID_ARG
    assert lib.swcorr_plan_create(ctypes.byref(h), 2, shape, k, None, 7, 0, 0) == swcorr.ERR_INVALID_ARG
    assert lib.swcorr_plan_create(ctypes.byref(h), 2, shape, k, None, swcorr.U16, 3, 0) == swcorr.ERR_INVALID_ARG
    assert lib.swcorr_plan_create(ctypes.byref(h), 2, shape, k, None, swcorr.U16, 0, 64) == swcorr.ERR_INVALID_ARG
    # sums are defined for clipped windows only
    assert lib.swcorr_plan_create(ctypes.byref(h), 2, shape, k, None, swcorr.U16, swcorr.BORDER_PAPER,
                                  swcorr.FLAG_EMIT_SUMS) == swcorr.ERR_INVALID_ARG
    assert lib.swcorr_plan_create(ctypes.byref(h), 2, shape, k, None, swcorr.F32, 0, 1) == swcorr.ERR_INVALID_ARG
    assert lib.swcorr_last_error()
    assert lib.swcorr_run(None, None, None, None, None, None, None, None) == swcorr.ERR_INVALID_ARG
    assert lib.swcorr_plan_outputs(None) == -1
    lib.swcorr_plan_destroy(None)


def test_plan_without_device_reports_no_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1807_06507_gb300 import swcorr
    h = ctypes.c_void_p()
    shape = (ctypes.c_int64 * 2)(10, 10)
    k = (ctypes.c_int32 * 2)(3, 3)
    assert lib.swcorr_plan_create(ctypes.byref(h), 2, shape, k, None, swcorr.U16, 0, 0) == swcorr.ERR_NO_DEVICE


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1807_06507_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
