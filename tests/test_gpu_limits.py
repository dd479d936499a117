"""The CUDA path against the oracle at the documented limits: the largest
step count (LV_MAX_STEPS, whose time table is the biggest shared-memory
array), the largest grid (LV_MAX_NODES nodes, read through L1), and path
indices at the top of the 48-bit counter space with a nonzero stream id
(the high counter words of Philox)."""
import numpy as np
import pytest

import oracle
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


def test_largest_step_count(lib):
    opt = W.Option(S0=100.0, r=0.01, K=100.0, T=2.0, n_steps=8192, n_paths=1024, seed=21)
    G.full_parity(W.small_skew_surface(), opt, lib, label="8192 steps")


def test_largest_grid(lib):
    """A smooth 128x128 surface. (On i.i.d. sigma per node at this spacing,
    S d sigma / d S reaches ~25, the Euler map amplifies any difference in the
    state by up to 1 + 25 sqrt(dt) |Z| per step, and binary32 and binary64
    paths separate: the comparison would measure the conditioning of the
    surface, not the kernel.)"""
    surf = W.seeded_skew_surface(22, n_spot=128, n_time=128, t_hi=1.5)
    assert surf.n_spot * surf.n_time == 16384
    opt = W.Option(S0=100.0, r=0.0, K=95.0, T=1.5, n_steps=64, n_paths=4096, seed=22)
    G.full_parity(surf, opt, lib, label="128x128 grid")


def test_top_of_the_path_index_space(lib):
    import torch
    surf = W.small_skew_surface()
    opt = W.Option(S0=100.0, r=0.02, K=105.0, T=1.0, n_steps=52, n_paths=4096, seed=23)
    m = 4096
    pb = (1 << 48) - m
    gs = G.make_surface(surf, opt, lib)
    decisions, _ = G.per_path(gs, surf, opt, m=m, path_begin=pb)
    ref = oracle.run_sums(surf, opt, pb, pb + m, decisions=decisions)
    d = torch.zeros(3 + gs.IJ, dtype=torch.float64, device="cuda")
    gs.price_greeks_sums_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, pb, pb + m, opt.seed, 0, d.data_ptr())
    s = d.cpu().numpy()
    assert abs(s[0] - ref[oracle.SUM_V]) <= G.PRICE_RTOL * abs(ref[oracle.SUM_V])
    assert abs(s[2] - ref[oracle.SUM_XBAR0]) <= G.DELTA_RTOL * abs(ref[oracle.SUM_XBAR0])
    v_ref = ref[oracle.NSCAL:oracle.NSCAL + gs.IJ]
    assert np.max(np.abs(s[3:] - v_ref)) <= G.VEGA_TOL_OF_MAX * np.max(np.abs(v_ref))
    # the largest stream id (the top 16 bits of counter word 2) against the oracle,
    # path for path with the kernel's near-node decisions checked and imposed
    o2 = W.Option(**{**opt.__dict__, "stream_id": 65535})
    dec2, _ = G.per_path(gs, surf, o2, m=m, path_begin=pb)
    ref2 = oracle.run_sums(surf, o2, pb, pb + m, decisions=dec2)
    d2 = torch.zeros_like(d)
    gs.price_greeks_sums_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, pb, pb + m, opt.seed, 65535,
                                d2.data_ptr())
    s2 = d2.cpu().numpy()
    assert abs(s2[0] - ref2[oracle.SUM_V]) <= G.PRICE_RTOL * abs(ref2[oracle.SUM_V])
    assert abs(s2[2] - ref2[oracle.SUM_XBAR0]) <= G.DELTA_RTOL * abs(ref2[oracle.SUM_XBAR0])
    v2 = ref2[oracle.NSCAL:oracle.NSCAL + gs.IJ]
    assert np.max(np.abs(s2[3:] - v2)) <= G.VEGA_TOL_OF_MAX * np.max(np.abs(v2))
