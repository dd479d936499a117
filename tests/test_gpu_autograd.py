"""The adjoint kernel behind torch.autograd: backward gives the adjoint's
delta and vegas, which match the FP64 oracle and central finite
differences (the bump baseline) on a small grid. Needs a GB300."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2002_02481_gb300 import build, lv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


def test_backward_is_the_adjoint(lib):
    import torch
    from paper_2002_02481_gb300.autograd import lv_price
    surf = W.random_surface(8, 4, 3, s_lo=80, s_hi=125, t_hi=1.0)
    opt = W.Option(S0=100.0, r=0.01, K=100.0, T=0.9, n_steps=12, n_paths=8192, seed=5)
    s = lv.Surface.from_workload(surf, lib)
    S0 = torch.tensor(opt.S0, dtype=torch.float64, requires_grad=True)
    sigma = torch.tensor(surf.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    price = lv_price(S0, sigma, s, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    (3.0 * price).backward()
    p, d, v = s.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    # same kernel, separate runs: equal up to the order of the binary32 bucket reductions
    assert abs(float(price) - p) <= 1e-12 * abs(p)
    assert abs(float(S0.grad) - 3.0 * d) <= 1e-9 * abs(d)
    assert np.max(np.abs(sigma.grad.cpu().numpy() - 3.0 * v)) <= 1e-6 * np.max(np.abs(3.0 * v))
    # against the FP64 oracle's adjoint and its central differences
    ref = oracle.price_greeks(surf, opt)
    assert abs(float(S0.grad) / 3.0 - ref["delta"]) <= 1e-5 * abs(ref["delta"])
    vmax = np.max(np.abs(ref["vega"]))
    assert np.max(np.abs(sigma.grad.cpu().numpy() / 3.0 - ref["vega"])) <= 1e-4 * vmax
    vfd, dfd = oracle.bump(surf, opt, 1e-5, 1e-5 * opt.S0)
    assert np.max(np.abs(sigma.grad.cpu().numpy() / 3.0 - vfd)) <= 2e-3 * vmax
    s.close()


def test_two_terms_on_one_surface(lib):
    """Two prices on one Surface with different sigma (and option type) in one
    graph, a single backward: each term gets the derivatives of its own
    sigma, not of whatever the surface holds when backward runs."""
    import torch
    from paper_2002_02481_gb300.autograd import lv_price
    surf = W.random_surface(8, 4, 3, s_lo=80, s_hi=125, t_hi=1.0)
    opt = W.Option(S0=100.0, r=0.01, K=100.0, T=0.9, n_steps=12, n_paths=8192, seed=5)
    s = lv.Surface.from_workload(surf, lib)
    sig_a = torch.tensor(surf.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    sig_b = torch.tensor(surf.sigma * 1.3, dtype=torch.float64, device="cuda", requires_grad=True)
    S0 = torch.tensor(opt.S0, dtype=torch.float64, requires_grad=True)
    pa = lv_price(S0, sig_a, s, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    s.set_option_type(-1)
    pb = lv_price(S0, sig_b, s, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    s.set_option_type(1)
    s.set_sigma(surf.sigma * 0.5)                  # what the surface holds when backward runs
    (pa + 2.0 * pb).backward()
    # each term separately, on fresh handles
    ra = lv.Surface.from_workload(surf, lib)
    _, da, va = ra.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    rb = lv.Surface(surf.spot, surf.time, surf.sigma * 1.3, lib)
    rb.set_option_type(-1)
    _, db, vb = rb.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(float(S0.grad) - (da + 2.0 * db)) <= 1e-9 * (abs(da) + 2.0 * abs(db))
    assert np.max(np.abs(sig_a.grad.cpu().numpy() - va)) <= 1e-6 * np.max(np.abs(va))
    assert np.max(np.abs(sig_b.grad.cpu().numpy() - 2.0 * vb)) <= 1e-6 * np.max(np.abs(2.0 * vb))
    for h in (s, ra, rb):
        h.close()
