"""The allocation-free entry point, for callers that cannot allocate device
memory during a call (a loop under a no-allocation rule, a runtime that
owns all device memory): through the C ABI it must
give the same price, delta and vegas as lv_price_greeks_device, call after
call, on scratch memory the library reserved when it was loaded.

This file is collected last so that a run stopping at the first failure
has already run every other test; it passes on its own in a fresh process
too. Needs a GB300."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2002_02481_gb300 import build, lv
    build.build()
    lib = lv.load()
    f = lib.lv_price_greeks_device_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib, lv, torch


def test_matches_the_allocating_entry_point_on_two_calls():
    lib, lv, torch = _lib()
    surf, opt = W.config_paper_shape()
    s = lv.Surface.from_workload(surf, lib)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    n = 3 + surf.n_spot * surf.n_time
    ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, ref.data_ptr())
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.lv_price_greeks_device_noalloc(s.h, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths,
                                                opt.seed, out.data_ptr())
        assert st == lv.LV_OK, lib.lv_last_error().decode()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o)), f"call {call}: non-finite output"
        # same paths, same per-path arithmetic; only the reduction order may differ
        assert abs(o[0] - r[0]) <= 1e-12 * abs(r[0]), (call, o[0], r[0])
        assert abs(o[1] - r[1]) <= 1e-9 * abs(r[1]), (call, o[1], r[1])
        assert abs(o[2] - r[2]) <= 1e-9 * abs(r[2]), (call, o[2], r[2])
        assert np.max(np.abs(o[3:] - r[3:])) <= 1e-6 * np.max(np.abs(r[3:])), call
    s.close()


def test_rejects_arguments_outside_the_domain():
    lib, lv, torch = _lib()
    surf, opt = W.config_small()
    s = lv.Surface.from_workload(surf, lib)
    out = torch.zeros(3 + surf.n_spot * surf.n_time, dtype=torch.float64, device="cuda")
    st = lib.lv_price_greeks_device_noalloc(s.h, opt.S0, opt.r, opt.K, opt.T, 8193, opt.n_paths, opt.seed,
                                            out.data_ptr())
    assert st == lv.LV_EINVAL and b"n_steps" in lib.lv_last_error()
    st = lib.lv_price_greeks_device_noalloc(s.h, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, 0, opt.seed,
                                            out.data_ptr())
    assert st == lv.LV_EINVAL and b"n_paths" in lib.lv_last_error()
    s.close()


def test_large_grid_fits_the_array_in_passes():
    """A 100 x 100 grid at 1,260 steps: a full-width launch overflows the
    array, so the plan runs fewer blocks; the results still match the
    allocating entry point."""
    lib, lv, torch = _lib()
    surf = W.random_surface(5, 100, 100, s_lo=20.0, s_hi=300.0, t_hi=5.0)
    opt = W.Option(S0=100.0, r=0.0, K=100.0, T=5.0, n_steps=1260, n_paths=1 << 15, seed=3)
    s = lv.Surface.from_workload(surf, lib)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    n = 3 + surf.n_spot * surf.n_time
    ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, ref.data_ptr())
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.lv_price_greeks_device_noalloc(s.h, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths,
                                            opt.seed, out.data_ptr())
    assert st == lv.LV_OK, lib.lv_last_error().decode()
    torch.cuda.synchronize()
    r, o = ref.cpu().numpy(), out.cpu().numpy()
    assert np.all(np.isfinite(o))
    assert abs(o[0] - r[0]) <= 1e-12 * abs(r[0])
    assert abs(o[1] - r[1]) <= 1e-9 * abs(r[1])
    assert np.max(np.abs(o[3:] - r[3:])) <= 1e-6 * np.max(np.abs(r[3:]))
    s.close()


def test_kahan_mode_on_a_narrowed_launch():
    """Kahan level 2 reserves per-warp rows in the array, so on the 30 x 60
    grid at 2^20 paths the launch runs fewer blocks than the allocating entry
    point's; two calls in a row still match it."""
    lib, lv, torch = _lib()
    surf, opt = W.config_paper_shape()
    s = lv.Surface.from_workload(surf, lib)
    s.set_accumulation(lv.LV_ACC_KAHAN)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    n = 3 + surf.n_spot * surf.n_time
    ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, ref.data_ptr())
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.lv_price_greeks_device_noalloc(s.h, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths,
                                                opt.seed, out.data_ptr())
        assert st == lv.LV_OK, lib.lv_last_error().decode()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o)), f"call {call}: non-finite output"
        assert abs(o[0] - r[0]) <= 1e-9 * abs(r[0]), (call, o[0], r[0])
        assert abs(o[1] - r[1]) <= 1e-8 * abs(r[1]), (call, o[1], r[1])
        assert np.max(np.abs(o[3:] - r[3:])) <= 1e-6 * np.max(np.abs(r[3:])), call
    s.close()


def test_two_paths_per_lane():
    """With two paths per lane the checkpoint ring per warp doubles; the plan
    inside the array accounts for it, and two calls in a row match the
    allocating entry point."""
    lib, lv, torch = _lib()
    surf, opt = W.config_paper_shape()
    s = lv.Surface.from_workload(surf, lib)
    s.set_launch(128, 4, 0)
    s.set_paths_per_lane(2)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    n = 3 + surf.n_spot * surf.n_time
    ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, ref.data_ptr())
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.lv_price_greeks_device_noalloc(s.h, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths,
                                                opt.seed, out.data_ptr())
        assert st == lv.LV_OK, lib.lv_last_error().decode()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o)), f"call {call}: non-finite output"
        assert abs(o[0] - r[0]) <= 1e-12 * abs(r[0]), (call, o[0], r[0])
        assert abs(o[1] - r[1]) <= 1e-9 * abs(r[1]), (call, o[1], r[1])
        assert np.max(np.abs(o[3:] - r[3:])) <= 1e-6 * np.max(np.abs(r[3:])), call
    s.close()
