"""The binary64 kernels against the FP64 oracle (needs a GB300).

lv_price_greeks_fp64_device runs every path in binary64 and follows the
same definition as the oracle, so the two differ only by the rounding of
CUDA's and the C library's binary64 functions and by summation order: the
aggregates are held to 1e-10 (price, delta; relative) and 1e-10 of the
largest bucket. The binary64 bump baseline (lv_bump_greeks_fp64) is held
to the oracle's own central bump-and-reprice with common random numbers
(Sec. III) on the same paths at 1e-7 of the largest bucket: the
differences (V+ - V-) / eps amplify rounding of V by 1 / eps."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2002_02481_gb300 import build, lv

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


def _fp64(lib, surf, opt):
    import torch
    s = lv.Surface.from_workload(surf, lib)
    s.set_option_type(opt.phi)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    d = torch.zeros(3 + surf.n_spot * surf.n_time, dtype=torch.float64, device="cuda")
    s.price_greeks_fp64_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
    torch.cuda.synchronize()
    s.close()
    return d.cpu().numpy()


CASES = [
    ("20x10 grid, 52 steps, 2^14 paths", *W.config_small()),
    ("30x60 grid, 156 steps, 2^16 paths", W.config_paper_shape()[0],
     W.Option(**{**W.config_paper_shape()[1].__dict__, "n_paths": 1 << 16})),
    ("2x1 grid, one time node", W.random_surface(1, 2, 1, s_lo=80, s_hi=125),
     W.Option(S0=100.0, r=0.0, K=100.0, T=1.0, n_steps=13, n_paths=3000, seed=3)),
    ("3x2 grid, paths leave both sides, r > 0", W.random_surface(2, 3, 2, s_lo=97, s_hi=103, t_hi=0.5),
     W.Option(S0=100.0, r=0.01, K=99.0, T=0.5, n_steps=8, n_paths=5000, seed=4)),
    ("uneven 7x5 grid, put", W.random_surface(3, 7, 5, s_lo=75, s_hi=130, t_hi=1.0, uneven=True),
     W.Option(S0=100.0, r=0.02, K=101.0, T=0.8, n_steps=10, n_paths=4097, seed=5, phi=-1)),
    ("K = 0, every path live", W.small_skew_surface(),
     W.Option(S0=100.0, r=0.04, K=0.0, T=1.0, n_steps=20, n_paths=8192, seed=10)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_adjoint_matches_the_oracle(case, lib):
    name, surf, opt = case
    g = _fp64(lib, surf, opt)
    ref = oracle.finalize(oracle.run_sums(surf, opt), opt.n_paths, opt.S0, surf.n_spot * surf.n_time)
    assert abs(g[0] - ref[0]) <= TOL * abs(ref[0]), (name, g[0], ref[0])
    assert abs(g[1] - ref[1]) <= TOL * abs(ref[1]), (name, g[1], ref[1])
    assert abs(g[2] - ref[2]) <= 1e-8 * abs(ref[2]), (name, g[2], ref[2])
    vmax = np.max(np.abs(ref[3:]))
    assert np.max(np.abs(g[3:] - ref[3:])) <= TOL * vmax, (name, np.max(np.abs(g[3:] - ref[3:])) / vmax)


def test_fp64_rejects_the_other_readings(lib):
    import torch
    surf, opt = W.config_small()
    s = lv.Surface.from_workload(surf, lib)
    s.set_scheme(lv.LV_SCHEME_S)
    d = torch.zeros(3 + s.IJ, dtype=torch.float64, device="cuda")
    with pytest.raises(lv.LVError) as e:
        s.price_greeks_fp64_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
    assert e.value.status == lv.LV_EINVAL
    s.close()


def test_fp64_bump_matches_the_oracle_bump(lib):
    surf, opt = W.config_small()
    opt = W.Option(**{**opt.__dict__, "n_paths": 2048, "r": 0.01})
    s = lv.Surface.from_workload(surf, lib)
    for eps in (1e-4, 1e-6):
        p, d, v = s.bump_greeks_fp64(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, eps)
        vref, dref = oracle.bump(surf, opt, eps, eps * opt.S0)       # the spot bump scales with eps
        vmax = np.max(np.abs(vref))
        assert np.max(np.abs(v - vref)) <= 1e-7 * vmax * (1e-4 / eps), eps
        assert abs(d - dref) <= 1e-7 * abs(dref) * (1e-4 / eps), (eps, d, dref)
    # and the price of the unbumped scenario is the plain estimator's
    ref = oracle.price_greeks(surf, opt)
    assert abs(p - ref["price"]) <= TOL * abs(ref["price"])
    s.close()


def test_fp64_bump_converges_to_the_pathwise_adjoint(lib):
    """Central differences of the binary64 estimator at eps = 1e-6 against the
    oracle's pathwise adjoint on the same paths: the same derivative up to
    O(eps^2) and the paths whose payoff or cell decision the bump moves."""
    surf, opt = W.config_small()
    opt = W.Option(**{**opt.__dict__, "n_paths": 8192})
    s = lv.Surface.from_workload(surf, lib)
    _, d, v = s.bump_greeks_fp64(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, 1e-6)
    ref = oracle.price_greeks(surf, opt)
    vmax = np.max(np.abs(ref["vega"]))
    assert np.max(np.abs(v - ref["vega"])) <= 1e-4 * vmax
    assert abs(d - ref["delta"]) <= 1e-4 * abs(ref["delta"])
    s.close()


def test_fp64_follows_set_sigma(lib):
    """lv_surface_set_sigma uploads the binary64 copy of sigma only when a
    binary64 call needs it: a handle created with one grid and then given
    another gives the binary64 results of a handle created with the second,
    also after a binary32 call in between and with two grid changes before
    the binary64 call."""
    import dataclasses
    import torch
    surf, opt = W.config_small()
    opt.n_paths = 1 << 12
    rng = np.random.default_rng(11)
    sig2 = surf.sigma * (1.0 + 0.2 * rng.random(surf.sigma.shape))
    sig3 = surf.sigma * (1.0 - 0.1 * rng.random(surf.sigma.shape))
    ref = _fp64(lib, dataclasses.replace(surf, sigma=sig3), opt)
    s = lv.Surface.from_workload(surf, lib)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    d = torch.zeros(3 + surf.n_spot * surf.n_time, dtype=torch.float64, device="cuda")
    s.set_sigma(sig2)
    s.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    s.set_sigma(sig3)
    s.price_greeks_fp64_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
    torch.cuda.synchronize()
    got = d.cpu().numpy()
    s.close()
    assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0]) and abs(got[1] - ref[1]) <= 1e-12 * abs(ref[1])
    assert np.max(np.abs(got[3:] - ref[3:])) <= 1e-12 * np.max(np.abs(ref[3:]))
