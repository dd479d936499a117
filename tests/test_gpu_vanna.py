"""Second-order buckets d^2 price / (d S0 d sigma_ij) on the GPU against the
FP64 oracle (needs a GB300), path for path on the same seeds, with the
kernel's near-node decisions checked and imposed (the kernel's two forward
passes run the same path arithmetic as the reverse sweep's forward pass, so
the diagnostics kernel's decision log holds for them).

Tolerances: price and delta 1e-5 relative; every bucket within 1e-4 of the
larger of the largest |bucket| and that bucket's per-path RMS (the
per-path terms of a second derivative cancel in the mean, while binary32
rounding scales with the terms themselves)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G
from .test_gpu_parity import EDGE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


def _parity(surf, opt, lib, label, ppl=0):
    gs = G.make_surface(surf, opt, lib, ppl=ppl)
    dec, stats = G.per_path(gs, surf, opt)
    ref = oracle.run_vanna(surf, opt, decisions=dec)
    p, d, vn = gs.price_greeks_vanna(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    gs.close()
    base = oracle.finalize(oracle.run_sums(surf, opt, decisions=dec), opt.n_paths, opt.S0,
                           surf.n_spot * surf.n_time)
    assert abs(p - base[0]) <= G.PRICE_RTOL * max(abs(base[0]), 1e-300), (label, p, base[0])
    assert abs(d - ref["delta"]) <= G.DELTA_RTOL * max(abs(ref["delta"]), 1e-300), (label, d, ref["delta"])
    P = opt.n_paths
    rms = np.sqrt(ref["sums"][oracle.VN_NSCAL + surf.n_spot * surf.n_time:] / P).reshape(surf.n_spot, surf.n_time)
    scale = np.maximum(np.max(np.abs(ref["vanna"])), rms)
    err = np.abs(vn - ref["vanna"])
    assert np.all(err <= 1e-4 * scale + 1e-300), (label, float(np.max(err / np.maximum(scale, 1e-300))))
    return float(np.max(err / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("case", EDGE, ids=[c[0] for c in EDGE])
def test_vanna_edge_cases(case, lib):
    name, surf, opt = case
    _parity(surf, opt, lib, name)


def test_vanna_small_grid(lib):
    surf, opt = W.config_small()
    _parity(surf, opt, lib, "20x10")


def test_vanna_paper_grid(lib):
    surf, opt = W.config_paper_shape()
    opt.n_paths = 1 << 18
    _parity(surf, opt, lib, "30x60, 2^18 paths")


@pytest.mark.parametrize("case", ["20x10", "30x60, 2^18 paths", "edge: 33 paths", "edge: put, uneven grid"])
def test_vanna_two_paths_per_lane(case, lib):
    """Pass 1 on two paths per lane, their binary32 arithmetic in packed
    pairs (tangent_forward2): the same per-path values, so the same parity
    with the oracle; and the same results as one path per lane up to
    reduction order."""
    if case == "20x10":
        surf, opt = W.config_small()
    elif case == "30x60, 2^18 paths":
        surf, opt = W.config_paper_shape()
        opt.n_paths = 1 << 18
    elif case == "edge: 33 paths":
        _, surf, opt = EDGE[5]
    else:
        _, surf, opt = EDGE[2]
    _parity(surf, opt, lib, case + " (two paths per lane)", ppl=2)
    a = G.make_surface(surf, opt, lib, ppl=1)
    b = G.make_surface(surf, opt, lib, ppl=2)
    assert b.get_paths_per_lane(opt.n_steps, opt.n_paths) == 2
    pa, da, va = a.price_greeks_vanna(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    pb, db, vb = b.price_greeks_vanna(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(pb - pa) <= 1e-12 * max(abs(pa), 1e-300) and abs(db - da) <= 1e-9 * max(abs(da), 1e-300)
    assert np.max(np.abs(vb - va)) <= 1e-6 * max(np.max(np.abs(va)), 1e-300)
    a.close()
    b.close()


def test_vanna_device_entry_point_and_readings(lib):
    import torch
    surf, opt = W.config_small()
    gs = G.make_surface(surf, opt, lib)
    gs.set_stream(torch.cuda.current_stream().cuda_stream)
    d = torch.zeros(3 + gs.IJ, dtype=torch.float64, device="cuda")
    gs.price_greeks_vanna_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
    torch.cuda.synchronize()
    p, dl, vn = gs.price_greeks_vanna(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    o = d.cpu().numpy()
    assert abs(o[0] - p) <= 1e-12 * abs(p) and abs(o[1] - dl) <= 1e-9 * abs(dl)
    assert np.max(np.abs(o[3:].reshape(vn.shape) - vn)) <= 1e-6 * np.max(np.abs(vn))
    # the price and delta are those of the first-order call
    p1, d1, _ = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(p1 - p) <= 1e-12 * abs(p) and abs(d1 - dl) <= 1e-6 * abs(dl)
    for setter in (lambda: gs.set_scheme(lv.LV_SCHEME_S), lambda: gs.set_interpolation(lv.LV_INTERP_LOGS)):
        gs.set_scheme(lv.LV_SCHEME_LOG)
        gs.set_interpolation(lv.LV_INTERP_S)
        setter()
        with pytest.raises(lv.LVError) as e:
            gs.price_greeks_vanna(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
        assert e.value.status == lv.LV_EINVAL
    gs.close()
