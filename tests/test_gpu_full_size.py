"""Full-size checks through a property that holds exactly at any size:
pathwise put-call parity. On the same paths, a call and a put at strike K
have terminal adjoints that differ by e^{-rT} S_N on every path (the
indicator of one or the other is 1, except at a tie), which is the terminal
adjoint of a call at K = 0 (every path live). The reverse sweep is linear in
x_bar_N, so the deltas and the vegas obey

    delta_call - delta_put = delta_(K=0),   vega_call - vega_put = vega_(K=0),

and the prices price_call - price_put = price_(K=0) - e^{-rT} K, up to the
rounding of the sums. Run at the sizes and launch shapes bench.py times:
the 100x100 grid with 1,260 steps and 2^26 paths at k = 4, and the 30x60
grid with 156 steps and 2^20 paths at the default shape. The oracle cannot
run these sizes; the per-path parity tests cover the arithmetic itself."""
import math

import numpy as np
import pytest

import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


def _three(lib, surf, opt, launch):
    out = {}
    for name, K, phi in (("call", opt.K, 1), ("put", opt.K, -1), ("fwd", 0.0, 1)):
        gs = G.make_surface(surf, opt, lib, launch=launch)
        gs.set_option_type(phi)
        out[name] = gs.price_greeks(opt.S0, opt.r, K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
        gs.close()
    return out


@pytest.mark.parametrize("config", ["large 100x100, 1260 steps, 2^26 paths, k=4",
                                    "paper shape 30x60, 156 steps, 2^20 paths"])
def test_pathwise_put_call_parity_at_full_size(config, lib):
    if config.startswith("large"):
        surf, opt = W.config_large()
        launch = (128, 4, 0)
    else:
        surf, opt = W.config_paper_shape()
        launch = None
    r = _three(lib, surf, opt, launch)
    (pc, dc, vc), (pp, dp, vp), (p0, d0, v0) = r["call"], r["put"], r["fwd"]
    disc = math.exp(-opt.r * opt.T)
    assert np.all(np.isfinite(vc)) and np.all(np.isfinite(vp)) and np.all(np.isfinite(v0))
    assert abs((pc - pp) - (p0 - disc * opt.K)) <= 1e-6 * p0
    assert abs((dc - dp) - d0) <= 1e-9 * abs(d0)
    assert np.max(np.abs((vc - vp) - v0)) <= 1e-5 * np.max(np.abs(v0))
    # and the forward's price is S0 within Monte Carlo error (martingale)
    assert abs(p0 - disc * opt.S0 * math.exp(opt.r * opt.T)) <= 5e-3 * opt.S0
