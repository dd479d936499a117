"""Bump-and-reprice baseline (Sec. III) on the GPU against the oracle's
binary64 central differences with the same bump and common random numbers,
and against the adjoint (needs a GB300)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G

pytestmark = pytest.mark.gpu
REPORT = os.environ.get("LV_PARITY_REPORT")


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_bump_against_oracle_bump_and_adjoint(eps, lib):
    surf = W.random_surface(8, 4, 3, s_lo=80, s_hi=125, t_hi=1.0)
    opt = W.Option(S0=100.0, r=0.01, K=100.0, T=0.9, n_steps=12, n_paths=8192, seed=5)
    gs = G.make_surface(surf, opt, lib)
    p, d, v = gs.bump_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, eps)
    vo, do = oracle.bump(surf, opt, eps, 1e-4 * opt.S0)
    ref = oracle.price_greeks(surf, opt)
    pa, da, va = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    vmax = np.max(np.abs(vo))
    stats = dict(eps=eps, price_rel=abs(p - ref["price"]) / ref["price"],
                 bump_vs_oracle_bump_vega_of_max=float(np.max(np.abs(v - vo)) / vmax),
                 bump_vs_oracle_bump_delta_rel=abs(d - do) / abs(do),
                 oracle_bump_vs_oracle_adjoint_vega_of_max=float(np.max(np.abs(vo - ref["vega"])) / vmax),
                 gpu_bump_vs_gpu_adjoint_vega_of_max=float(np.max(np.abs(v - va)) / vmax))
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": f"bump eps={eps}", **stats}) + "\n")
    assert stats["price_rel"] <= 1e-5
    # binary32 paths: the bumped and unbumped trajectories round differently, which puts
    # noise of order ulp(x) / eps on every path's difference quotient
    assert stats["bump_vs_oracle_bump_vega_of_max"] <= (2e-2 if eps < 1e-3 else 5e-3)
    assert stats["bump_vs_oracle_bump_delta_rel"] <= 2e-2
    gs.close()
