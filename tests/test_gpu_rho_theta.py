"""Rho and d price / d T from the GPU's reverse sweep (lv_price_greeks_ext)
against the FP64 oracle's pathwise sums on the same seeded inputs, under
every reading, with the near-node decisions of the kernel imposed on the
oracle as in the vega parity tests; the extended call's price, delta and
vegas equal the plain call's. Needs a GB300."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G
from .test_gpu_parity import EDGE

pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LV_PARITY_REPORT")
# rho and d V / d T: within 1e-5 of the larger of |mean| and the per-path RMS
# (a mean can be a near cancellation of per-path values, e.g. the rho of a
# call struck at 0, while rounding scales with the per-path values)
RTOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


def _check(surf, opt, lib, label):
    gs = G.make_surface(surf, opt, lib)
    decisions, _ = G.per_path(gs, surf, opt)
    sums = oracle.run_sums(surf, opt, decisions=decisions)
    P = opt.n_paths
    ref_rho, ref_dvdt = sums[oracle.SUM_RHO] / P, sums[oracle.SUM_DVDT] / P
    rms_rho, rms_dvdt = np.sqrt(sums[oracle.SUM_RHO_2] / P), np.sqrt(sums[oracle.SUM_DVDT_2] / P)
    p, d, v, rho, dvdt = gs.price_greeks_ext(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    e_r = abs(rho - ref_rho) / max(abs(ref_rho), rms_rho, 1e-12)
    e_t = abs(dvdt - ref_dvdt) / max(abs(ref_dvdt), rms_dvdt, 1e-12)
    assert e_r <= RTOL and e_t <= RTOL, f"{label}: rho {rho} vs {ref_rho} ({e_r:.2e}), dV/dT {dvdt} vs {ref_dvdt} ({e_t:.2e})"
    # the rest of the extended call equals the plain call (same paths; reduction order)
    p0, d0, v0 = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(p - p0) <= 1e-12 * max(abs(p0), 1e-300) and abs(d - d0) <= 1e-9 * max(abs(d0), 1e-12)
    assert np.max(np.abs(v - v0)) <= 1e-6 * max(np.max(np.abs(v0)), 1e-12)
    gs.close()
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": "rho, dV/dT: " + label, "rho_rel": e_r, "dvdt_rel": e_t}) + "\n")


@pytest.mark.parametrize("case", EDGE, ids=[c[0] for c in EDGE])
def test_edge_cases(case, lib):
    name, surf, opt = case
    if opt.r == 0.0:
        opt = W.Option(**{**opt.__dict__, "r": 0.015})   # a nonzero rate exercises every term
    _check(surf, opt, lib, name)


@pytest.mark.parametrize("interp,scheme", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_small_config_every_reading(interp, scheme, lib):
    surf, opt = W.config_small()
    surf = W.Surface(surf.spot, surf.time, surf.sigma, interp=interp)
    opt = W.Option(**{**opt.__dict__, "r": 0.02, "scheme": scheme})
    _check(surf, opt, lib, f"20x10 grid, reading ({interp}, {scheme})")


def test_paper_shape(lib):
    surf, opt = W.config_paper_shape()
    opt = W.Option(**{**opt.__dict__, "n_paths": 1 << 18, "r": 0.01})
    _check(surf, opt, lib, "30x60 grid, 156 steps, 2^18 paths")


def test_device_layout(lib):
    import torch
    surf, opt = W.config_small()
    s = lv.Surface.from_workload(surf, lib)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    IJ = surf.n_spot * surf.n_time
    out = torch.full((5 + IJ,), float("nan"), dtype=torch.float64, device="cuda")
    s.price_greeks_ext_device(opt.S0, 0.02, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, out.data_ptr())
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    p, d, v, rho, dvdt = s.price_greeks_ext(opt.S0, 0.02, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert np.all(np.isfinite(o))
    assert abs(o[3 + IJ] - rho) <= 1e-9 * abs(rho) and abs(o[4 + IJ] - dvdt) <= 1e-9 * abs(dvdt)
    assert abs(o[0] - p) <= 1e-12 * abs(p)
    s.close()
