"""The C ABI library builds, loads without a GPU and exports every symbol
include/lv.h declares; argument errors come back as status codes before any
device work (CPU only)."""
import ctypes

import numpy as np
import pytest

from paper_2002_02481_gb300 import build, lv


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lv.load()


def test_exports_every_declared_symbol(lib):
    names = lv.exported_names()
    assert "lv_surface_create" in names and "lv_price_greeks" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _create(lib, spot, time, sigma):
    h = ctypes.c_void_p()
    spot = np.ascontiguousarray(spot, dtype=np.float64)
    time = np.ascontiguousarray(time, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.lv_surface_create(dp(spot), len(spot), dp(time), len(time), dp(sigma), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("spot,time,sigma,why", [
    ([100.0], [0.0], [0.2], "one spot node"),
    ([100.0, 90.0], [0.0], [0.2, 0.2], "decreasing spot nodes"),
    ([0.0, 90.0], [0.0], [0.2, 0.2], "non-positive spot node"),
    ([80.0, 120.0], [0.5, 0.5], [0.2] * 4, "repeated time node"),
    ([80.0, 120.0], [-1.0, 0.5], [0.2] * 4, "negative time node"),
    ([80.0, 120.0], [0.0], [0.2, float("nan")], "NaN sigma"),
    ([80.0, 120.0], [0.0], [0.2, 0.0], "zero sigma"),
    ([80.0, 120.0], [0.0], [0.2, -0.1], "negative sigma"),
])
def test_create_rejects_bad_grids(lib, spot, time, sigma, why):
    st, h = _create(lib, spot, time, sigma)
    assert st == lv.LV_EINVAL, why
    assert not h.value
    assert lib.lv_last_error()


def test_null_arguments_are_rejected(lib):
    p = ctypes.c_double()
    assert lib.lv_price(None, 100.0, 0.0, 100.0, 1.0, 10, 100, 1, ctypes.byref(p), None) == lv.LV_EINVAL
    assert lib.lv_price_greeks(None, 100.0, 0.0, 100.0, 1.0, 10, 100, 1, None, None, None) == lv.LV_EINVAL
    assert lib.lv_set_option_type(None, 1) == lv.LV_EINVAL
    assert lib.lv_set_launch(None, 256, 8, 0) == lv.LV_EINVAL
    out = ctypes.c_void_p()
    assert lib.lv_surface_create(None, 2, None, 1, None, ctypes.byref(out)) == lv.LV_EINVAL
    lib.lv_surface_destroy(None)   # ignored
