"""Decisions imposed on the oracle (payoff indicator, spot cell) behave as
specified: imposing the oracle's own decisions changes nothing, imposing a
different one changes exactly the affected path, and the oracle refuses any
imposed decision that rounding of the path could not have produced (CPU
only). Also pins the per-path bound ``amp`` the GPU parity harness uses."""
import numpy as np
import pytest
import torch

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
    # a band wide enough to admit this path's flip (it is not at the strike)
    band = abs(np.exp(xN[p]) - opt.K) / opt.K * (1 + 1e-9)
    dec = oracle.Decisions(itm={p: False}, band=band)
    flipped = oracle.run_sums(surf, opt, n_threads=1, decisions=dec)
    assert dec.overrides == {"cell": 0, "payoff": 1}
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
    dec = oracle.Decisions(cells=([0], [0], [2 * other + 1]), band=1e-12)
    forced = oracle.run_sums(surf, opt, n_threads=1, decisions=dec)
    assert dec.overrides == {"cell": 1, "payoff": 0}
    assert abs(forced[oracle.SUM_V] - base[oracle.SUM_V]) < 1e-12 * base[oracle.SUM_V]  # sigma continuous
    assert forced[oracle.SUM_XBAR0] != base[oracle.SUM_XBAR0]


def _trajectory(surf, opt, p):
    """ln S_0 .. ln S_N of path p, restated in numpy from the oracle's normals
    and its pinned sigma lookup (log-Euler, main reading)."""
    z = oracle.normals(opt.seed, p, opt.n_steps)
    dt = opt.T / opt.n_steps
    x = [np.log(opt.S0)]
    for n in range(opt.n_steps):
        e = oracle.sigma_eval(surf, np.exp(x[-1]), n * dt)
        x.append(x[-1] + (opt.r - 0.5 * e["sigma"] ** 2) * dt + e["sigma"] * np.sqrt(dt) * z[n])
    return np.array(x), z


def _far_step(surf, opt, p, margin=1e-3):
    """A step of path p whose spot lies more than margin (relative) from every
    node, with the oracle's own cell code there."""
    x, _ = _trajectory(surf, opt, p)
    for n in range(1, opt.n_steps):
        S = np.exp(x[n])
        if np.min(np.abs(S - surf.spot) / surf.spot) > margin:
            i = oracle.sigma_eval(surf, S, n * opt.T / opt.n_steps)["i"]
            inside = int(surf.spot[0] <= S <= surf.spot[-1])
            return n, i, inside, S
    raise AssertionError("no step away from the nodes")


def test_non_adjacent_cell_is_refused():
    surf, opt = _setup()
    n, i, inside, _ = _far_step(surf, opt, 0)
    j = i + 2 if i + 2 <= surf.n_spot - 2 else i - 2
    with pytest.raises(oracle.DecisionRefused):
        oracle.run_sums(surf, opt, n_threads=1, decisions=oracle.Decisions(cells=([0], [n], [2 * j + inside]),
                                                                          band=1.0))


def test_neighbour_cell_away_from_its_node_is_refused():
    surf, opt = _setup()
    n, i, inside, S = _far_step(surf, opt, 0)
    j = i + 1 if i + 1 <= surf.n_spot - 2 else i - 1
    node = surf.spot[max(i, j)]
    tight = 0.5 * abs(S - node) / node
    with pytest.raises(oracle.DecisionRefused):
        oracle.run_sums(surf, opt, n_threads=1, decisions=oracle.Decisions(cells=([0], [n], [2 * j + inside]),
                                                                          band=tight))
    # the same decision inside a band that reaches the node is applied
    dec = oracle.Decisions(cells=([0], [n], [2 * j + inside]), band=4 * tight)
    oracle.run_sums(surf, opt, n_threads=1, decisions=dec)
    assert dec.overrides == {"cell": 1, "payoff": 0}


def test_inside_flag_away_from_the_edge_is_refused():
    surf, opt = _setup()
    n, i, inside, S = _far_step(surf, opt, 0)
    edge = min(abs(S - surf.spot[0]) / surf.spot[0], abs(S - surf.spot[-1]) / surf.spot[-1])
    with pytest.raises(oracle.DecisionRefused):
        oracle.run_sums(surf, opt, n_threads=1,
                        decisions=oracle.Decisions(cells=([0], [n], [2 * i + (1 - inside)]), band=0.5 * edge))


def test_cell_code_out_of_range_is_refused():
    surf, opt = _setup()
    with pytest.raises(oracle.DecisionRefused):
        oracle.run_sums(surf, opt, n_threads=1,
                        decisions=oracle.Decisions(cells=([0], [3], [2 * (surf.n_spot - 1) + 1]), band=1.0))
    with pytest.raises(RuntimeError):          # a negative code is malformed input
        oracle.run_sums(surf, opt, n_threads=1, decisions=oracle.Decisions(cells=([0], [3], [-2]), band=1.0))


def test_payoff_flip_away_from_the_strike_is_refused():
    surf, opt = _setup()
    xN, V, _ = oracle.paths(surf, opt, 0, opt.n_paths)
    p = int(np.argmax(np.abs(np.exp(xN) - opt.K)))
    d = abs(np.exp(xN[p]) - opt.K) / opt.K
    with pytest.raises(oracle.DecisionRefused):
        oracle.paths(surf, opt, 0, opt.n_paths, decisions=oracle.Decisions(itm={p: not bool(V[p] > 0)},
                                                                           band=0.5 * d))


def _amp_bound_check(surf, opt, scheme, interp):
    """d ln |prod_n (1 + g_n)| / d e, with every spot S_n of the path scaled by
    (1 + e) inside its own cell (normals and cells fixed), by torch.autograd,
    against the oracle's amp: the bound must hold path by path."""
    s = W.Surface(**{**surf.__dict__, "interp": interp})
    o = W.Option(**{**opt.__dict__, "scheme": scheme})
    m = 24
    _, V, _, amp = oracle.paths(s, o, 0, m, amp=True)
    dt = o.T / o.n_steps
    sqdt = np.sqrt(dt)
    spot = torch.tensor(s.spot, dtype=torch.float64)
    checked = 0
    for p in range(m):
        if not V[p] > 0:
            continue
        z = oracle.normals(o.seed, p, o.n_steps)
        # the path in binary64, as the oracle runs it (state ln S, or S on scheme 1)
        st = np.log(o.S0) if scheme == 0 else o.S0
        e = torch.zeros((), dtype=torch.float64, requires_grad=True)
        logprod = torch.zeros((), dtype=torch.float64)
        for n in range(o.n_steps):
            S = float(np.exp(st)) if scheme == 0 else float(st)
            pt = oracle.sigma_eval(s, S, n * dt)
            i, j, v = pt["i"], pt["j"], pt["v"]
            Se = S * (1 + e)
            lo, hi = spot[i], spot[i + 1]
            if interp == 0:
                u = torch.clamp((Se - lo) / (hi - lo), 0.0, 1.0)
            else:
                u = torch.clamp((torch.log(Se) - torch.log(lo)) / (torch.log(hi) - torch.log(lo)), 0.0, 1.0)
            J = s.n_time
            sg = np.asarray(s.sigma).reshape(s.n_spot, J)
            c0 = (1 - v) * sg[i, j] + (v * sg[i, j + 1] if J > 1 else 0.0)
            c1 = (1 - v) * sg[i + 1, j] + (v * sg[i + 1, j + 1] if J > 1 else 0.0)
            sigma = c0 + (c1 - c0) * u
            inside = s.spot[0] <= S <= s.spot[-1]
            # d sigma / d S is constant inside the cell (linear in S or in ln S)
            if not inside:
                dsig = torch.zeros((), dtype=torch.float64)
            elif interp == 0:
                dsig = torch.tensor((c1 - c0) / (s.spot[i + 1] - s.spot[i]), dtype=torch.float64)
            else:
                dsig = (c1 - c0) / (Se * float(np.log(s.spot[i + 1] / s.spot[i])))
            if scheme == 0:
                h = sqdt * z[n] - sigma * dt
                factor = 1 + h * Se * dsig
            else:
                h = Se * sqdt * z[n]
                factor = 1 + o.r * dt + sigma * sqdt * z[n] + h * dsig
            logprod = logprod + torch.log(torch.abs(factor))
            sv = pt["sigma"]
            st = st + (o.r - 0.5 * sv * sv) * dt + sv * sqdt * z[n] if scheme == 0 else \
                st + o.r * st * dt + sv * st * sqdt * z[n]
        (d,) = torch.autograd.grad(logprod, [e])
        assert abs(float(d)) <= amp[p] * (1 + 1e-9) + 1e-15, (p, float(d), amp[p])
        checked += 1
    assert checked > 3


@pytest.mark.parametrize("scheme,interp", [(0, 0), (0, 1), (1, 0)], ids=["log-S", "log-S ln-weight", "Euler on S"])
def test_amp_bounds_the_spot_sensitivity(scheme, interp):
    surf = W.random_surface(11, 6, 4, s_lo=85, s_hi=118, t_hi=1.0)
    opt = W.Option(S0=100.0, r=0.02, K=98.0, T=0.8, n_steps=12, n_paths=24, seed=12)
    _amp_bound_check(surf, opt, scheme, interp)


def test_amp_is_zero_on_a_flat_grid():
    surf = W.flat_surface(0.2)
    opt = W.Option(S0=100.0, r=0.0, K=100.0, T=1.0, n_steps=10, n_paths=64, seed=3)
    _, _, _, amp = oracle.paths(surf, opt, 0, 64, amp=True)
    assert np.all(amp == 0.0)
