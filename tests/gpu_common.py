"""Shared GPU-parity machinery: run the CUDA path and the FP64 oracle on the
same seeded inputs and compare.

Tolerances (written here, used by every parity test): price and delta within
1e-5 relative, every vega bucket within 1e-4 of the largest |bucket|.

The payoff indicator 1{phi (S_N - K) > 0} is an integer decided in floating
point: a path whose terminal spot lies within binary32 rounding of K can be
decided differently by the kernel (binary32 path) and the oracle (binary64
path). Such paths are found from the per-path outputs, checked to lie at the
kink (|S_N - K| <= KINK_REL * K), and the kernel's decision is imposed on the
oracle for exactly those paths before the aggregates are compared.
"""
import numpy as np

import oracle
from paper_2002_02481_gb300 import lv

PRICE_RTOL = 1e-5
DELTA_RTOL = 1e-5
VEGA_TOL_OF_MAX = 1e-4
KINK_REL = 1e-4          # a decision may differ only this close to the strike
X_ATOL = 1e-4            # per-path |x_N(binary32) - x_N(binary64)|


def make_surface(w_surf, opt, lib, launch=None, accumulation=0):
    s = lv.Surface.from_workload(w_surf, lib)
    s.set_option_type(opt.phi)
    s.set_accumulation(accumulation)
    if launch:
        s.set_launch(*launch)
    return s


def per_path(gs, w_surf, opt, m=None, path_begin=0):
    """Per-path comparison on paths [path_begin, path_begin + m); returns the
    kernel's payoff decisions for the paths where the two sides differ."""
    m = opt.n_paths if m is None else m
    gx, gV, gxb = gs.debug_paths(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.seed, path_begin, m)
    ox, oV, oxb = oracle.paths(w_surf, opt, path_begin, m)
    dx = np.abs(gx.astype(np.float64) - ox)
    assert np.all(np.isfinite(gx)) and dx.max() <= X_ATOL, f"max |dx_N| = {dx.max():.3e}"
    g_itm, o_itm = gV > 0, oV > 0
    flipped = np.nonzero(g_itm != o_itm)[0]
    if flipped.size:
        SN = np.exp(ox[flipped])
        assert np.all(np.abs(SN - opt.K) <= KINK_REL * opt.K), "decision differs away from the kink"
    # payoffs: continuous in S_N, so they differ by about S_N |dx_N|
    disc = np.exp(-opt.r * opt.T)
    np.testing.assert_array_less(np.abs(gV - oV), X_ATOL * disc * np.exp(ox) + 1e-6)
    both = g_itm & o_itm
    if both.any():
        rel = np.abs(gxb[both] - oxb[both]) / np.maximum(np.abs(oxb[both]), 1e-12)
        # most paths match to binary32 rounding; a path whose spot sits within rounding
        # of a node may pick the neighbouring cell's slope d sigma/d S for that step
        assert np.median(rel) < 1e-5, np.median(rel)
        assert np.quantile(rel, 0.99) < 1e-3, np.quantile(rel, 0.99)
        assert rel.max() < 0.1, rel.max()
    stats = dict(max_dx=float(dx.max()), n_flipped=int(flipped.size))
    return {int(path_begin + p): bool(g_itm[p]) for p in flipped}, stats


def _rel(a, b):
    # relative error; exact zeros (e.g. every path out of the money) must match exactly
    return abs(a - b) / abs(b) if b != 0 else abs(a - b)


def compare_aggregates(gpu_price, gpu_delta, gpu_vega, ref, label=""):
    price, delta, vega = ref[0], ref[1], ref[3:].reshape(gpu_vega.shape)
    e_p = _rel(gpu_price, price)
    e_d = _rel(gpu_delta, delta)
    vmax = np.max(np.abs(vega))
    e_v = np.max(np.abs(gpu_vega - vega)) / vmax if vmax > 0 else np.max(np.abs(gpu_vega))
    msg = f"{label}: price rel {e_p:.2e}, delta rel {e_d:.2e}, vega/max {e_v:.2e}"
    assert e_p <= PRICE_RTOL, msg
    assert e_d <= DELTA_RTOL, msg
    assert e_v <= VEGA_TOL_OF_MAX, msg
    return dict(price_rel=e_p, delta_rel=e_d, vega_of_max=e_v)


def full_parity(w_surf, opt, lib, launch=None, accumulation=0, label=""):
    """Per-path check on every path, then aggregates against the oracle with
    the kernel's kink decisions imposed."""
    gs = make_surface(w_surf, opt, lib, launch, accumulation)
    overrides, stats = per_path(gs, w_surf, opt)
    ref = oracle.finalize(oracle.run_sums(w_surf, opt, itm_overrides=overrides), opt.n_paths, opt.S0,
                          w_surf.n_spot * w_surf.n_time)
    p, d, v = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    errs = compare_aggregates(p, d, v, ref, label)
    gs.close()
    return {**stats, **errs}
