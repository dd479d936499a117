"""The tangent-ratio adjoint (LV_ADJ_TANGENT: x_bar_{n+1} = x_bar_N D_N /
D_{n+1} with the tangent D_n = d x_n / d x_0) against the FP64 oracle's
reverse-mode adjoint, element by element on the same seeded inputs, with the
same tolerances as the checkpointed reverse sweep; and against that sweep on
the same paths. Needs a GB300."""
import json
import os

import numpy as np
import pytest

import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G
from .test_gpu_parity import EDGE

pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LV_PARITY_REPORT")
T = lv.LV_ADJ_TANGENT


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


def _report(name, d):
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": "tangent: " + name, **d}) + "\n")


@pytest.mark.parametrize("case", EDGE, ids=[c[0] for c in EDGE])
def test_edge_cases(case, lib):
    name, surf, opt = case
    _report(name, G.full_parity(surf, opt, lib, label=name, method=T))


def test_small_config(lib):
    surf, opt = W.config_small()
    _report("20x10 grid, 52 steps, 2^14 paths", G.full_parity(surf, opt, lib, label="small", method=T))


def test_paper_shape_full_size(lib):
    surf, opt = W.config_paper_shape()
    _report("30x60 grid, 156 steps, 2^20 paths", G.full_parity(surf, opt, lib, label="paper", method=T))


@pytest.mark.parametrize("acc", [0, 1])
def test_both_level2_modes(lib, acc):
    surf, opt = W.config_precision("paper")
    opt = W.Option(**{**opt.__dict__, "n_paths": 1 << 16})
    _report(f"precision paper 2^16 acc={acc}",
            G.full_parity(surf, opt, lib, accumulation=acc, label=f"acc={acc}", method=T))


@pytest.mark.parametrize("case", ["20x10", "30x60 2^18 binary64", "30x60 2^18 Kahan", "edge: 33 paths",
                                  "edge: put, uneven grid"])
def test_two_paths_per_lane(case, lib):
    """Pass 1 on two paths per lane, their binary32 arithmetic in packed
    pairs (tangent_forward2): the same per-path arithmetic, checked against
    the oracle path for path in both level-2 modes, with the binary search
    for the cell (uneven grid) and a ragged last tile."""
    acc = 0
    if case == "20x10":
        surf, opt = W.config_small()
    elif case.startswith("30x60"):
        surf, opt = W.config_paper_shape()
        opt.n_paths = 1 << 18
        acc = 1 if case.endswith("Kahan") else 0
    elif case == "edge: 33 paths":
        _, surf, opt = EDGE[5]
    else:
        _, surf, opt = EDGE[2]
    s = G.make_surface(surf, opt, lib, accumulation=acc, method=T, ppl=2)
    assert s.get_paths_per_lane(opt.n_steps, opt.n_paths) == 2
    s.close()
    _report(f"two paths per lane: {case}",
            G.full_parity(surf, opt, lib, accumulation=acc, label=case, method=T, ppl=2))


def test_matches_the_reverse_sweep_on_the_same_paths(lib):
    """Same paths, same payoffs: the two forms differ only in rounding and
    reduction order."""
    surf, opt = W.config_large()
    opt = W.Option(**{**opt.__dict__, "r": 0.01, "K": 110.0, "n_paths": 1 << 14, "seed": 4})
    out = {}
    for m in (lv.LV_ADJ_REVERSE, T):
        s = G.make_surface(surf, opt, lib, method=m)
        out[m] = s.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
        s.close()
    (p0, d0, v0), (p1, d1, v1) = out[lv.LV_ADJ_REVERSE], out[T]
    assert abs(p1 - p0) <= 1e-12 * abs(p0)
    assert abs(d1 - d0) <= 1e-6 * abs(d0), (d0, d1)
    assert np.max(np.abs(v1 - v0)) <= 1e-5 * np.max(np.abs(v0))


def test_device_and_noalloc_entry_points(lib):
    import ctypes
    import torch
    surf, opt = W.config_small()
    s = G.make_surface(surf, opt, lib, method=T)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    n = 3 + surf.n_spot * surf.n_time
    p, d, v = s.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    dev = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    s.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, dev.data_ptr())
    f = lib.lv_price_greeks_device_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    na = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    assert f(s.h, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, na.data_ptr()) == lv.LV_OK
    torch.cuda.synchronize()
    for o in (dev.cpu().numpy(), na.cpu().numpy()):
        assert np.all(np.isfinite(o))
        assert abs(o[0] - p) <= 1e-12 * abs(p)
        assert abs(o[1] - d) <= 1e-9 * abs(d)
        assert np.max(np.abs(o[3:].reshape(v.shape) - v)) <= 1e-6 * np.max(np.abs(v))
    s.close()


def test_rejects_an_unknown_method(lib):
    surf, opt = W.config_small()
    s = lv.Surface.from_workload(surf, lib)
    with pytest.raises(lv.LVError):
        s.set_adjoint_method(2)
    s.close()


def test_vanishing_factor_is_flagged(lib):
    """On a fine grid with sigma drawn i.i.d. per node, S d sigma / d S reaches
    ~25, so 1 + g_n = 1 + h_n S d sigma / d S comes within 2^-20 of zero on
    some live paths among 2^20: the tangent-ratio form must refuse (NaN device
    outputs, LV_ENUMERIC with the host outputs untouched), the reverse sweep
    on the same paths must not, and the next tangent call on a benign grid
    must succeed (the flag is reset)."""
    import ctypes

    import torch
    surf = W.random_surface(22, 128, 128, s_lo=40.0, s_hi=250.0, t_hi=1.5)
    opt = W.Option(S0=100.0, r=0.0, K=95.0, T=1.5, n_steps=64, n_paths=1 << 20, seed=22)
    gs = G.make_surface(surf, opt, lib, method=T)
    n = 3 + gs.IJ
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    gs.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
    torch.cuda.synchronize()
    assert np.all(np.isnan(d.cpu().numpy()))
    price, delta = ctypes.c_double(-7.0), ctypes.c_double(-7.0)
    vega = np.full(gs.IJ, -7.0)
    st = lib.lv_price_greeks(gs.h, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed,
                             ctypes.byref(price), ctypes.byref(delta),
                             vega.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == lv.LV_ENUMERIC
    assert price.value == -7.0 and delta.value == -7.0 and np.all(vega == -7.0)
    # the raw-sums path (what a path-range shard returns) carries the flag as NaN
    # sums, and finalizing them keeps every output NaN, the standard error included
    sums = torch.zeros(n, dtype=torch.float64, device="cuda")
    gs.set_stream(torch.cuda.current_stream().cuda_stream)
    gs.price_greeks_sums_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, 0, opt.n_paths, opt.seed, 0,
                                sums.data_ptr())
    fin = torch.zeros(n, dtype=torch.float64, device="cuda")
    gs.finalize_sums_device(sums.data_ptr(), opt.n_paths, opt.S0, fin.data_ptr())
    torch.cuda.synchronize()
    assert np.all(np.isnan(sums.cpu().numpy()))
    assert np.all(np.isnan(fin.cpu().numpy())), fin.cpu().numpy()[:3]
    gs.set_stream(0)
    gs.set_adjoint_method(lv.LV_ADJ_REVERSE)
    p, dl, v = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert np.isfinite(p) and np.isfinite(dl) and np.all(np.isfinite(v))
    gs.close()
    s2, o2 = W.config_small()
    g2 = G.make_surface(s2, o2, lib, method=T)
    p2, d2, v2 = g2.price_greeks(o2.S0, o2.r, o2.K, o2.T, o2.n_steps, o2.n_paths, o2.seed)
    assert np.isfinite(p2) and np.all(np.isfinite(v2))
    g2.close()
