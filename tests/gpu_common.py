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
step whose spot lies within NODE_BAND of a node of its cell, with the
decision it took there. The harness first measures how far the binary32
paths drift from the oracle's (max |dx_N| over the paths) and sets the
decision band to DRIFT_FACTOR times that drift plus the rounding of the
kernel's cell index. The oracle then takes the kernel's logged cell
decisions and its payoff decisions where they differ from its own, and
checks each one: a decision other than its own is accepted only when the
oracle's own spot lies within the band of the node (or strike) that
separates the two choices, and the cell is the neighbour across that node;
anything else is refused (oracle.DecisionRefused). The comparison then runs
path for path, each path held to the bound its own drift implies:
  |V - V_o|        <= disc (S_N (dx_N + 2^-20) + K 2^-22)
  |xbar_0 - xbar_0o| <= |xbar_0o| (dx_N + amp band + N 2^-21 + 2^-20),
with amp the oracle's per-path bound on how a relative error in every spot
moves ln |xbar_0| (lv_oracle.c), and N 2^-21 eight binary32 roundings a step.
"""
import numpy as np

import oracle
from paper_2002_02481_gb300 import lv

PRICE_RTOL = 1e-5
DELTA_RTOL = 1e-5
VEGA_TOL_OF_MAX = 1e-4
NODE_BAND = 5e-4         # logged steps: |S - s| <= NODE_BAND * s for a node s of the cell
DRIFT_FACTOR = 4.0       # decision band = DRIFT_FACTOR * max |dx_N| + INDEX_ROUNDING
INDEX_ROUNDING = 2.0 ** -20   # relative error of the kernel's binary32 cell index, in S


def make_surface(w_surf, opt, lib, launch=None, accumulation=0, method=lv.LV_ADJ_REVERSE, ppl=0):
    s = lv.Surface.from_workload(w_surf, lib)
    s.set_option_type(opt.phi)
    s.set_accumulation(accumulation)
    s.set_adjoint_method(method)
    s.set_interpolation(getattr(w_surf, "interp", 0))
    s.set_scheme(getattr(opt, "scheme", 0))
    if launch:
        s.set_launch(*launch)
    if ppl:
        s.set_paths_per_lane(ppl)
    return s


def per_path(gs, w_surf, opt, m=None, path_begin=0):
    """Per-path comparison on paths [path_begin, path_begin + m); returns the
    decisions for the oracle (the kernel's, checked by the oracle) and the
    statistics of the comparison."""
    m = opt.n_paths if m is None else m
    cap = min(1 << 27, 64 * m + 65536)
    gx, gV, gxb, cells = gs.debug_paths(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.seed, path_begin, m,
                                        node_band=NODE_BAND, ev_cap=cap, stream_id=opt.stream_id)
    assert np.all(np.isfinite(gx)), "non-finite binary32 path"
    # drift of the binary32 paths from the oracle's own, before any decision is taken
    ox0, oV0, _ = oracle.paths(w_surf, opt, path_begin, m)
    dx0 = np.abs(gx.astype(np.float64) - ox0)
    band = DRIFT_FACTOR * float(dx0.max()) + INDEX_ROUNDING
    # every step where the two sides could decide a cell differently lies within band of
    # a node for the oracle, so within band + drift < NODE_BAND for the kernel: it was logged
    assert band <= 0.5 * NODE_BAND, f"drift {dx0.max():.3e} too large for the logged band"
    flipped = np.nonzero((gV > 0) != (oV0 > 0))[0]
    itm = {int(path_begin + p): bool(gV[p] > 0) for p in flipped}
    dec = oracle.Decisions(itm=itm, cells=cells, band=band)
    ox, oV, oxb, amp = oracle.paths(w_surf, opt, path_begin, m, decisions=dec, amp=True)
    overrides = dec.overrides
    dx = np.abs(gx.astype(np.float64) - ox)
    SN = np.exp(ox)
    disc = np.exp(-opt.r * opt.T)
    # payoffs: continuous in S_N (binary32: exp2 and a subtraction)
    v_bound = disc * (SN * (dx + 2.0 ** -20) + abs(opt.K) * 2.0 ** -22) + 1e-300
    v_err = np.abs(gV.astype(np.float64) - oV)
    assert np.all(v_err <= v_bound), f"payoff off its bound by {np.max(v_err / v_bound):.2f}x"
    both = (gV > 0) & (oV > 0)
    xb_stats = {}
    if both.any():
        ref = np.abs(oxb[both])
        err = np.abs(gxb[both].astype(np.float64) - oxb[both])
        bound = ref * (dx[both] + amp[both] * band + opt.n_steps * 2.0 ** -21 + 2.0 ** -20)
        ratio = err / np.maximum(bound, 1e-300)
        assert np.all(ratio <= 1.0), f"xbar_0 off its per-path bound by {ratio.max():.2f}x"
        rel = err / np.maximum(ref, 1e-300)
        xb_stats = dict(xbar0_rel_median=float(np.median(rel)), xbar0_rel_q99=float(np.quantile(rel, 0.99)),
                        xbar0_rel_max=float(rel.max()), xbar0_err_of_bound_max=float(ratio.max()))
    stats = dict(path_steps=int(m) * int(opt.n_steps), max_dx=float(dx.max()), band=band,
                 logged_steps=int(len(cells[0])), cell_overrides=overrides["cell"],
                 payoff_overrides=overrides["payoff"], **xb_stats)
    return dec, stats


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


def full_parity(w_surf, opt, lib, launch=None, accumulation=0, label="", method=lv.LV_ADJ_REVERSE, ppl=0):
    """Per-path check on every path, then aggregates against the oracle with
    the kernel's kink decisions imposed. The per-path check and the decisions
    come from the reverse sweep's diagnostics kernel, whose forward arithmetic
    the tangent-ratio kernel shares."""
    gs = make_surface(w_surf, opt, lib, launch, accumulation, method, ppl)
    decisions, stats = per_path(gs, w_surf, opt)
    ref = oracle.finalize(oracle.run_sums(w_surf, opt, decisions=decisions), opt.n_paths, opt.S0,
                          w_surf.n_spot * w_surf.n_time)
    p, d, v = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    errs = compare_aggregates(p, d, v, ref, label)
    gs.close()
    return {**stats, **errs}
