"""Decisions imposed on the oracle (payoff indicator, spot cell) behave as
specified: imposing the oracle's own decisions changes nothing, and
imposing a different one changes exactly the affected path (CPU only)."""
import numpy as np

import oracle
import workloads as W


def _setup():
    surf, _ = W.config_small()
    opt = W.Option(S0=100.0, r=0.02, K=100.0, T=1.0, n_steps=20, n_paths=64, seed=4)
    return surf, opt


def test_own_decisions_change_nothing():
    surf, opt = _setup()
    base = oracle.run_sums(surf, opt, n_threads=1)
    xN, V, _ = oracle.paths(surf, opt, 0, opt.n_paths)
    # the oracle's own payoff decisions for every path, and its own cells at a few steps
    itm = {p: bool(V[p] > 0) for p in range(opt.n_paths)}
    cells_p, cells_n, cells_c = [], [], []
    for p in range(8):
        z = oracle.normals(opt.seed, p, opt.n_steps)
        x = np.log(opt.S0)
        dt = opt.T / opt.n_steps
        for n in range(opt.n_steps):
            e = oracle.sigma_eval(surf, np.exp(x), n * dt)
            inside = int(surf.spot[0] <= np.exp(x) <= surf.spot[-1])
            cells_p.append(p); cells_n.append(n); cells_c.append(2 * e["i"] + inside)
            x = x + (opt.r - 0.5 * e["sigma"] ** 2) * dt + e["sigma"] * np.sqrt(dt) * z[n]
    dec = oracle.Decisions(itm=itm, cells=(cells_p, cells_n, cells_c))
    again = oracle.run_sums(surf, opt, n_threads=1, decisions=dec)
    np.testing.assert_array_equal(base, again)


def test_flipped_payoff_decision_moves_one_path():
    surf, opt = _setup()
    xN, V, xb = oracle.paths(surf, opt, 0, opt.n_paths)
    p = int(np.nonzero(V > 0)[0][0])
    base = oracle.run_sums(surf, opt, n_threads=1)
    flipped = oracle.run_sums(surf, opt, n_threads=1, decisions=oracle.Decisions(itm={p: False}))
    one = oracle.run_sums(surf, opt, p, p + 1, n_threads=1)
    assert abs((base[oracle.SUM_XBAR0] - flipped[oracle.SUM_XBAR0]) - one[oracle.SUM_XBAR0]) < 1e-9
    IJ = surf.n_spot * surf.n_time
    np.testing.assert_allclose(base[oracle.NSCAL:oracle.NSCAL + IJ] - flipped[oracle.NSCAL:oracle.NSCAL + IJ],
                               one[oracle.NSCAL:oracle.NSCAL + IJ], atol=1e-9)
    assert base[oracle.SUM_V] == flipped[oracle.SUM_V]      # the payoff itself is not a decision


def test_forced_neighbour_cell_changes_only_the_slope_side():
    """Forcing the left neighbour cell at a step where S sits exactly on a
    node keeps sigma (continuous) and the bucket weights, and changes the
    sensitivity only through the slope d sigma / d S."""
    surf = W.random_surface(6, 4, 2, s_lo=90, s_hi=112, t_hi=1.0)
    node = float(surf.spot[2])
    right = oracle.sigma_eval(surf, node, 0.3)
    assert right["i"] == 2
    opt = W.Option(S0=node, r=0.0, K=node * 0.5, T=0.5, n_steps=3, n_paths=1, seed=2)
    own = oracle.sigma_eval(surf, float(np.exp(np.log(node))), 0.0)["i"]   # S_0 as the path sees it
    other = 1 if own == 2 else 2
    base = oracle.run_sums(surf, opt, n_threads=1)
    forced = oracle.run_sums(surf, opt, n_threads=1,
                             decisions=oracle.Decisions(cells=([0], [0], [2 * other + 1])))
    assert abs(forced[oracle.SUM_V] - base[oracle.SUM_V]) < 1e-12 * base[oracle.SUM_V]  # sigma continuous
    assert forced[oracle.SUM_XBAR0] != base[oracle.SUM_XBAR0]
