"""Shared GPU-parity machinery: run the CUDA path and the FP64 oracle on the
same seeded inputs and compare.

Tolerances (written here, used by every parity test): price and delta within
1e-5 relative, every vega bucket within 1e-4 of the largest |bucket|.

Two integers of the method are decided in floating point, so a binary32
path (kernel) and a binary64 path (oracle) can decide them differently when
the value sits within rounding of the threshold:
  - the payoff indicator 1{phi (S_N - K) > 0}, for S_N within rounding of K;
  - the spot cell of a step and whether S lies inside the grid (which picks
    the side of d sigma / d S), for S within rounding of a node.
The kernel's debug entry point reports its per-path results and logs every
step whose spot lies within NODE_BAND of a node together with the decision
it took there; the oracle takes the kernel's decisions for exactly those
steps and for the paths whose payoff decision differs (checked to lie at the
kink), and the comparison then runs path for path.
"""
import numpy as np

import oracle
from paper_2002_02481_gb300 import lv

PRICE_RTOL = 1e-5
DELTA_RTOL = 1e-5
VEGA_TOL_OF_MAX = 1e-4
KINK_REL = 1e-4          # a payoff decision may differ only this close to the strike
X_ATOL = 1e-4            # per-path |x_N(binary32) - x_N(binary64)|
NODE_BAND = 2e-4         # logged steps: |S - s| <= NODE_BAND * s for a node s of the cell


def make_surface(w_surf, opt, lib, launch=None, accumulation=0, method=lv.LV_ADJ_REVERSE):
    s = lv.Surface.from_workload(w_surf, lib)
    s.set_option_type(opt.phi)
    s.set_accumulation(accumulation)
    s.set_adjoint_method(method)
    s.set_interpolation(getattr(w_surf, "interp", 0))
    s.set_scheme(getattr(opt, "scheme", 0))
    if launch:
        s.set_launch(*launch)
    return s


def per_path(gs, w_surf, opt, m=None, path_begin=0):
    """Per-path comparison on paths [path_begin, path_begin + m); returns the
    decisions for the oracle (the kernel's, where they can differ)."""
    m = opt.n_paths if m is None else m
    cap = min(1 << 27, 64 * m + 65536)
    gx, gV, gxb, cells = gs.debug_paths(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.seed, path_begin, m,
                                        node_band=NODE_BAND, ev_cap=cap)
    ox, oV, oxb = oracle.paths(w_surf, opt, path_begin, m, decisions=oracle.Decisions(cells=cells))
    dx = np.abs(gx.astype(np.float64) - ox)
    assert np.all(np.isfinite(gx)) and dx.max() <= X_ATOL, f"max |dx_N| = {dx.max():.3e}"
    assert dx.max() <= 0.25 * NODE_BAND, "the paths drift further apart than the logged band"
    g_itm, o_itm = gV > 0, oV > 0
    flipped = np.nonzero(g_itm != o_itm)[0]
    if flipped.size:
        SN = np.exp(ox[flipped])
        assert np.all(np.abs(SN - opt.K) <= KINK_REL * opt.K), "decision differs away from the kink"
    # payoffs: continuous in S_N, so they differ by about S_N |dx_N|
    disc = np.exp(-opt.r * opt.T)
    np.testing.assert_array_less(np.abs(gV - oV), X_ATOL * disc * np.exp(ox) + 1e-6)
    both = g_itm & o_itm
    xb_stats = {}
    if both.any():
        rel = np.abs(gxb[both] - oxb[both]) / np.maximum(np.abs(oxb[both]), 1e-12)
        assert np.median(rel) < 1e-5, np.median(rel)
        assert np.quantile(rel, 0.99) < 1e-3, np.quantile(rel, 0.99)
        assert rel.max() < 1e-2, rel.max()
        xb_stats = dict(xbar0_rel_median=float(np.median(rel)), xbar0_rel_q99=float(np.quantile(rel, 0.99)),
                        xbar0_rel_max=float(rel.max()))
    stats = dict(max_dx=float(dx.max()), n_flipped=int(flipped.size), n_cell_decisions=int(len(cells[0])),
                 **xb_stats)
    itm = {int(path_begin + p): bool(g_itm[p]) for p in flipped}
    return oracle.Decisions(itm=itm, cells=cells), stats


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


def full_parity(w_surf, opt, lib, launch=None, accumulation=0, label="", method=lv.LV_ADJ_REVERSE):
    """Per-path check on every path, then aggregates against the oracle with
    the kernel's kink decisions imposed. The per-path check and the decisions
    come from the reverse sweep's diagnostics kernel, whose forward arithmetic
    the tangent-ratio kernel shares."""
    gs = make_surface(w_surf, opt, lib, launch, accumulation, method)
    decisions, stats = per_path(gs, w_surf, opt)
    ref = oracle.finalize(oracle.run_sums(w_surf, opt, decisions=decisions), opt.n_paths, opt.S0,
                          w_surf.n_spot * w_surf.n_time)
    p, d, v = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    errs = compare_aggregates(p, d, v, ref, label)
    gs.close()
    return {**stats, **errs}
