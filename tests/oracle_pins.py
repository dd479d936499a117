"""Pins that tie the FP64 oracle to facts outside itself.

Each pin takes an oracle library handle, so the same battery runs against
the real oracle (tests/test_oracle_pins.py) and against copies with a
planted mistake (tests/test_oracle_mutants.py), where at least one pin must
fail. None of them retypes the oracle's own formulas: they compare with
cuRAND's Philox, with distribution laws, with Black-Scholes closed forms,
with identities that hold path by path, with central differences of the
oracle's own forward estimator, and with torch.autograd on an independent
restatement of the forward (tests/torch_lv.py).
"""
import math

import numpy as np
from scipy import stats
from scipy.special import ndtr

import oracle
import workloads as W

from . import _curand_host
from . import torch_lv


# ---------------------------------------------------------------- helpers

def bs_call_put(S0, K, T, r, sigma, phi):
    """Black-Scholes price, delta and vega (textbook closed forms)."""
    sd = sigma * math.sqrt(T)
    d1 = (math.log(S0 / K) + (r + 0.5 * sigma * sigma) * T) / sd
    d2 = d1 - sd
    disc = math.exp(-r * T)
    if phi > 0:
        price = S0 * ndtr(d1) - K * disc * ndtr(d2)
        delta = ndtr(d1)
    else:
        price = K * disc * ndtr(-d2) - S0 * ndtr(-d1)
        delta = ndtr(d1) - 1.0
    vega = S0 * math.exp(-0.5 * d1 * d1) / math.sqrt(2 * math.pi) * math.sqrt(T)
    return price, delta, vega


def se_of(sum1, sum2, n):
    mean = sum1 / n
    var = max(sum2 / n - mean * mean, 0.0) * n / max(n - 1, 1)
    return math.sqrt(var / n)


# ------------------------------------------------------------------- RNG

def pin_philox_curand(lib):
    """Philox4x32-10 block function == cuRAND's host generator, over
    counters with nonzero c0, c1 and c2 and several keys."""
    cu = _curand_host.load()
    if cu is None:
        import pytest
        pytest.skip("libcurand not available")
    seeds = [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF]
    offsets = [0, 4 * (5 * 65536 + 123), 4 * (1 << 48), 4 * (((1 << 32) + 7) * 65536 + 65530)]
    for seed in seeds:
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for off in offsets:
            words = _curand_host.generate(cu, seed, off, 4 * 12).reshape(-1, 4)
            for t in range(words.shape[0]):
                ctr = _curand_host.counter_of(off // 4 + t)
                got = oracle.philox4x32_10(ctr, key, lib=lib)
                assert np.array_equal(got, words[t]), (seed, off, t, got, words[t])


def pin_normals_from_curand_words(lib):
    """The oracle's normals for (seed, stream, path, step) are Box-Muller of
    the uniforms of the Philox words at counter (step/4, path low, path high
    | stream << 16, 0); words taken from cuRAND, transform by Python's math."""
    cu = _curand_host.load()
    if cu is None:
        import pytest
        pytest.skip("libcurand not available")
    seed = 0x00000000DEADBEEF
    # cuRAND tuple p sits at counter (p >> 16 over c0:c1, p & 0xffff, 0); with stream 0 and
    # path < 2^14 the oracle's counter (blk, path, 0, 0) is tuple ((path << 32 | blk) << 16)
    for path in (0, 3, 9000):
        z = oracle.normals(seed, path, 12, lib=lib)
        for blk in range(3):
            p = ((path << 32) | blk) << 16
            w = _curand_host.generate(cu, seed, 4 * p, 4)
            u = [((int(x) >> 9) + 0.5) * 2.0 ** -23 for x in w]
            expect = []
            for a, b in ((u[0], u[1]), (u[2], u[3])):
                rad = math.sqrt(-2.0 * math.log(a))
                expect += [rad * math.cos(2 * math.pi * b), rad * math.sin(2 * math.pi * b)]
            np.testing.assert_allclose(z[4 * blk:4 * blk + 4], expect, rtol=1e-13, atol=1e-13)


def pin_uniform_exact(lib):
    """Every uniform lies in (0, 1) and is exactly representable in binary32
    (both precisions see the same value); the extremes are 2^-24, 1 - 2^-24."""
    rng = np.random.Generator(np.random.PCG64(11))
    ws = list(rng.integers(0, 2 ** 32, size=2000, dtype=np.uint64)) + [0, 0xFFFFFFFF, 1 << 31]
    for w in ws:
        u = oracle.uniform(int(w), lib=lib)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
    assert oracle.uniform(0, lib=lib) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF, lib=lib) == 1.0 - 2.0 ** -24


def pin_normal_law(lib):
    """2^18 normals: moments within 4 SE of N(0, 1), KS test, radius^2 of
    each Box-Muller pair ~ Exp(mean 2), no lag-1 correlation."""
    n_paths, n_steps = 4096, 64
    z = np.concatenate([oracle.normals(7, p, n_steps, lib=lib) for p in range(n_paths)])
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)
    assert abs(stats.skew(z)) < 4 * math.sqrt(6 / n)
    assert abs(stats.kurtosis(z)) < 4 * math.sqrt(24 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    pairs = z.reshape(-1, 2)
    r2 = (pairs ** 2).sum(1)
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-4
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 4 / math.sqrt(n)


# ------------------------------------------------------------ flat surface

def pin_black_scholes(lib):
    """Flat sigma: log-Euler is exact in law, so price, delta and the sum of
    all vega buckets match Black-Scholes within 3.5 standard errors."""
    sig = 0.2
    cases = [(1.0, 0.0, 1, 100.0), (3.0, 0.0, 1, 100.0), (5.0, 0.0, 1, 100.0),
             (1.0, 0.03, -1, 110.0), (2.0, 0.03, 1, 90.0)]
    surf = W.flat_surface(sig, n_spot=6, n_time=4, s_lo=30.0, s_hi=400.0, t_hi=5.0)
    for T, r, phi, K in cases:
        opt = W.Option(S0=100.0, r=r, K=K, T=T, n_steps=26, n_paths=1 << 15, seed=3, phi=phi)
        s = oracle.run_sums(surf, opt, lib=lib)
        P = opt.n_paths
        price, delta, vega = bs_call_put(100.0, K, T, r, sig, phi)
        got_p = s[oracle.SUM_V] / P
        got_d = s[oracle.SUM_XBAR0] / (P * 100.0)
        got_v = s[oracle.SUM_VTOT] / P
        assert abs(got_p - price) < 3.5 * se_of(s[oracle.SUM_V], s[oracle.SUM_V2], P), (T, got_p, price)
        se_d = se_of(s[oracle.SUM_XBAR0], s[oracle.SUM_XBAR0_2], P) / 100.0
        assert abs(got_d - delta) < 3.5 * se_d, (T, got_d, delta)
        se_v = se_of(s[oracle.SUM_VTOT], s[oracle.SUM_VTOT_2], P)
        assert abs(got_v - vega) < 3.5 * se_v, (T, got_v, vega)
        # the bucket array sums to the same total
        vb = s[oracle.NSCAL:oracle.NSCAL + surf.n_spot * surf.n_time].sum() / P
        assert abs(vb - got_v) <= 1e-10 * max(1.0, abs(got_v))


def pin_flat_closed_form_paths(lib):
    """Flat sigma, per path: x_N = ln S0 + (r - sigma^2/2) T + sigma sqrt(dt)
    sum Z exactly, and the path's bucket total equals the flat pathwise vega
    e^{-rT} 1{phi(S_N-K)>0} phi S_N (sqrt(dt) sum Z - sigma T) (partition of
    unity of the bilinear weights)."""
    sig, r, T, N, K = 0.25, 0.02, 2.0, 24, 100.0
    surf = W.flat_surface(sig, n_spot=4, n_time=3, s_lo=50.0, s_hi=200.0, t_hi=2.0)
    for phi in (1, -1):
        opt = W.Option(S0=100.0, r=r, K=K, T=T, n_steps=N, n_paths=64, seed=9, phi=phi)
        xN, V, xb = oracle.paths(surf, opt, 0, 64, lib=lib)
        dt = T / N
        for p in range(64):
            zs = oracle.normals(9, p, N, lib=lib).sum()
            x_exact = math.log(100.0) + (r - 0.5 * sig * sig) * T + sig * math.sqrt(dt) * zs
            assert abs(xN[p] - x_exact) < 1e-12
            SN = math.exp(x_exact)
            itm = phi * (SN - K) > 0
            s = oracle.run_sums(surf, opt, p, p + 1, lib=lib, n_threads=1)
            vpath = math.exp(-r * T) * phi * SN * (math.sqrt(dt) * zs - sig * T) if itm else 0.0
            assert abs(s[oracle.SUM_VTOT] - vpath) <= 1e-11 * max(1.0, abs(vpath)), (p, s[oracle.SUM_VTOT], vpath)
            # flat grid: d x_N / d x_0 = 1, so xbar_0 = e^{-rT} phi S_N on in-the-money paths
            assert abs(xb[p] - (math.exp(-r * T) * phi * SN if itm else 0.0)) < 1e-10


# --------------------------------------------------------------- invariants

def pin_martingale(lib):
    """Any grid: E[e^{-rT} S_N] = S0 under log-Euler, so a call struck at 0
    prices S0 with delta 1 and zero total vega, within 3.5 SE."""
    surf, _ = W.config_small()
    for r in (0.0, 0.04):
        opt = W.Option(S0=100.0, r=r, K=0.0, T=1.0, n_steps=52, n_paths=1 << 15, seed=5)
        s = oracle.run_sums(surf, opt, lib=lib)
        P = opt.n_paths
        assert abs(s[oracle.SUM_V] / P - 100.0) < 3.5 * se_of(s[oracle.SUM_V], s[oracle.SUM_V2], P)
        se_d = se_of(s[oracle.SUM_XBAR0], s[oracle.SUM_XBAR0_2], P) / 100.0
        assert abs(s[oracle.SUM_XBAR0] / (P * 100.0) - 1.0) < 3.5 * se_d
        se_v = se_of(s[oracle.SUM_VTOT], s[oracle.SUM_VTOT_2], P)
        assert abs(s[oracle.SUM_VTOT] / P) < 3.5 * se_v


def pin_put_call_parity(lib):
    """Path by path, call - put = e^{-rT}(S_N - K); with the same seeds the
    price, delta and every bucket of (call - put) equal those of a call
    struck at 0 minus K e^{-rT}, to rounding."""
    surf, _ = W.config_small()
    r, T, K = 0.03, 1.0, 104.0
    base = dict(S0=100.0, r=r, T=T, n_steps=40, n_paths=4096, seed=21)
    c = oracle.run_sums(surf, W.Option(K=K, phi=1, **base), lib=lib)
    p = oracle.run_sums(surf, W.Option(K=K, phi=-1, **base), lib=lib)
    f = oracle.run_sums(surf, W.Option(K=0.0, phi=1, **base), lib=lib)
    P = base["n_paths"]
    IJ = surf.n_spot * surf.n_time
    assert abs((c[0] - p[0]) - (f[0] - P * K * math.exp(-r * T))) < 1e-9 * f[0]
    assert abs((c[oracle.SUM_XBAR0] - p[oracle.SUM_XBAR0]) - f[oracle.SUM_XBAR0]) < 1e-9 * f[oracle.SUM_XBAR0]
    vc, vp, vf = (a[oracle.NSCAL:oracle.NSCAL + IJ] for a in (c, p, f))
    assert np.max(np.abs((vc - vp) - vf)) < 1e-9 * np.max(np.abs(vf))


# ------------------------------------------------------------- the adjoint

ADJOINT_CASES = [
    # name, surface, S0, r, K, T, N, phi, P, seed
    ("2x1 constant-in-time", W.random_surface(1, 2, 1, s_lo=80, s_hi=125), 100.0, 0.0, 100.0, 1.0, 6, 1, 24, 3),
    ("3x2 leaves grid both sides", W.random_surface(2, 3, 2, s_lo=92, s_hi=108, t_hi=0.5), 100.0, 0.01, 99.0, 0.5, 8, 1, 32, 4),
    ("uneven 5x4 put, K at node", None, 100.0, 0.02, None, 0.8, 10, -1, 32, 5),
    ("4x3 T mid-cell", W.random_surface(4, 4, 3, s_lo=70, s_hi=140, t_hi=2.0), 100.0, 0.0, 95.0, 1.3, 9, 1, 32, 6),
    ("small skew r>0", W.config_small()[0], 100.0, 0.05, 100.0, 1.0, 13, 1, 32, 7),
]


def _case(c):
    name, surf, S0, r, K, T, N, phi, P, seed = c
    if surf is None:
        surf = W.random_surface(3, 5, 4, s_lo=75, s_hi=130, t_hi=1.0, uneven=True)
        K = float(surf.spot[2])
    return name, surf, W.Option(S0=S0, r=r, K=K, T=T, n_steps=N, n_paths=P, seed=seed, phi=phi)


def pin_adjoint_vs_autograd(lib):
    """The hand-written reverse sweep equals torch.autograd of an independent
    FP64 restatement of the forward, on tiny grids covering a one-column
    grid, paths leaving the grid on both sides, irregular nodes, a strike at
    a node, a maturity inside a time cell, puts and a nonzero rate."""
    for c in ADJOINT_CASES:
        name, surf, opt = _case(c)
        Z = np.stack([oracle.normals(opt.seed, p, opt.n_steps, lib=lib) for p in range(opt.n_paths)])
        price, delta, vega, _ = torch_lv.autograd_greeks(
            surf.spot, surf.time, surf.sigma, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.phi, Z)
        res = oracle.finalize(oracle.run_sums(surf, opt, lib=lib), opt.n_paths, opt.S0,
                              surf.n_spot * surf.n_time, lib=lib)
        scale = max(1e-3, np.max(np.abs(vega)))
        assert abs(res[0] - price) <= 1e-11 * max(1.0, abs(price)), name
        assert abs(res[1] - delta) <= 1e-11 * max(1.0, abs(delta)), (name, res[1], delta)
        np.testing.assert_allclose(res[3:].reshape(vega.shape), vega, rtol=0, atol=1e-11 * scale,
                                   err_msg=name)


def pin_adjoint_vs_bump(lib):
    """Adjoint delta and buckets equal central bump-and-reprice (Sec. III)
    with common random numbers and eps = 1e-6, to O(eps^2), on a small grid
    where no path sits within the bump of a payoff or cell kink."""
    surf = W.random_surface(8, 3, 2, s_lo=85, s_hi=118, t_hi=0.6)
    opt = W.Option(S0=100.0, r=0.01, K=101.0, T=0.6, n_steps=4, n_paths=64, seed=12, phi=1)
    xN, _, _ = oracle.paths(surf, opt, 0, opt.n_paths, lib=lib)
    assert np.min(np.abs(np.exp(xN) - opt.K)) > 1e-3   # no path near the payoff kink
    res = oracle.finalize(oracle.run_sums(surf, opt, lib=lib), opt.n_paths, opt.S0, 6, lib=lib)
    vfd, dfd = oracle.bump(surf, opt, 1e-6, 1e-6 * opt.S0, lib=lib)
    scale = np.max(np.abs(vfd))
    np.testing.assert_allclose(res[3:].reshape(3, 2), vfd, rtol=0, atol=2e-6 * scale)
    assert abs(res[1] - dfd) < 2e-6 * max(1.0, abs(dfd))


def pin_bilinear(lib):
    """Bilinear sigma: exact node values at nodes, flat outside the grid,
    weights a partition of unity, d sigma/d S equal to a central difference
    inside a cell and 0 outside, and the cell rule max{i : s_i <= S}."""
    surf = W.random_surface(5, 4, 3, s_lo=80, s_hi=120, t_hi=1.0, uneven=True)
    s, t, g = surf.spot, surf.time, surf.sigma
    for i in range(4):
        for j in range(3):
            e = oracle.sigma_eval(surf, s[i], t[j], lib=lib)
            assert abs(e["sigma"] - g[i, j]) < 1e-15
            assert e["i"] == min(i, 2) and e["j"] == min(j, 1)
    lo = oracle.sigma_eval(surf, 10.0, 0.5, lib=lib)
    hi = oracle.sigma_eval(surf, 1000.0, 0.5, lib=lib)
    assert lo["dsigma_dS"] == 0.0 and hi["dsigma_dS"] == 0.0
    edge_lo = oracle.sigma_eval(surf, s[0], 0.5, lib=lib)
    edge_hi = oracle.sigma_eval(surf, s[-1], 0.5, lib=lib)
    assert abs(lo["sigma"] - edge_lo["sigma"]) < 1e-15 and abs(hi["sigma"] - edge_hi["sigma"]) < 1e-15
    late = oracle.sigma_eval(surf, 100.0, 7.0, lib=lib)
    last = oracle.sigma_eval(surf, 100.0, t[-1], lib=lib)
    assert abs(late["sigma"] - last["sigma"]) < 1e-15
    rng = np.random.Generator(np.random.PCG64(4))
    for _ in range(50):
        S = rng.uniform(s[0], s[-1])
        tt = rng.uniform(0.0, t[-1])
        e = oracle.sigma_eval(surf, S, tt, lib=lib)
        assert abs(sum(e["w"]) - 1.0) < 1e-14
        assert s[e["i"]] <= S < s[e["i"] + 1] or (e["i"] == 2 and S <= s[3])
        h = 1e-6
        if min(abs(S - x) for x in s) > 10 * h:
            fd = (oracle.sigma_eval(surf, S + h, tt, lib=lib)["sigma"]
                  - oracle.sigma_eval(surf, S - h, tt, lib=lib)["sigma"]) / (2 * h)
            assert abs(fd - e["dsigma_dS"]) < 1e-7
        # value from scipy's regular-grid linear interpolator
        from scipy.interpolate import RegularGridInterpolator
        ref = RegularGridInterpolator((s, t), g, method="linear")([[S, tt]])[0]
        assert abs(ref - e["sigma"]) < 1e-13


# ------------------------------------------- the other readings of Sec. IV

def pin_flat_closed_form_paths_euler_x(lib):
    """Euler on X, flat sigma, per path: X_N = S0 prod_n (1 + r dt + sigma
    sqrt(dt) Z_n); d V / d ln S0 = e^{-rT} phi X_N on in-the-money paths
    (X_N is linear in S0); the bucket total is d V / d sigma =
    e^{-rT} phi X_N sum_n sqrt(dt) Z_n / (1 + r dt + sigma sqrt(dt) Z_n)."""
    sig, r, T, N, K = 0.3, 0.03, 1.5, 18, 100.0
    surf = W.flat_surface(sig, n_spot=4, n_time=3, s_lo=40.0, s_hi=250.0, t_hi=1.5)
    dt = T / N
    for phi in (1, -1):
        opt = W.Option(S0=100.0, r=r, K=K, T=T, n_steps=N, n_paths=48, seed=13, phi=phi, scheme=oracle.SCHEME_X)
        xN, V, xb = oracle.paths(surf, opt, 0, 48, lib=lib)
        for p in range(48):
            z = oracle.normals(13, p, N, lib=lib)
            f = 1.0 + r * dt + sig * math.sqrt(dt) * z
            XN = 100.0 * np.prod(f)
            assert abs(math.exp(xN[p]) - XN) < 1e-12 * XN
            itm = phi * (XN - K) > 0
            disc = math.exp(-r * T)
            assert abs(V[p] - (disc * phi * (XN - K) if itm else 0.0)) < 1e-11 * XN
            assert abs(xb[p] - (disc * phi * XN if itm else 0.0)) < 1e-11 * XN
            s = oracle.run_sums(surf, opt, p, p + 1, lib=lib, n_threads=1)
            vpath = disc * phi * XN * np.sum(math.sqrt(dt) * z / f) if itm else 0.0
            assert abs(s[oracle.SUM_VTOT] - vpath) <= 1e-11 * max(1.0, abs(vpath)), (p, s[oracle.SUM_VTOT], vpath)


def pin_martingale_euler_x(lib):
    """Euler on X on any grid: E[X_N] = S0 (1 + r dt)^N, so a call struck at
    0 prices e^{-rT} S0 (1 + r dt)^N with delta e^{-rT} (1 + r dt)^N, within
    3.5 standard errors."""
    surf, _ = W.config_small()
    for r in (0.0, 0.05):
        opt = W.Option(S0=100.0, r=r, K=0.0, T=1.0, n_steps=26, n_paths=1 << 15, seed=6, scheme=oracle.SCHEME_X)
        s = oracle.run_sums(surf, opt, lib=lib)
        P, dt = opt.n_paths, opt.T / opt.n_steps
        grow = math.exp(-r * opt.T) * (1.0 + r * dt) ** opt.n_steps
        assert abs(s[oracle.SUM_V] / P - 100.0 * grow) < 3.5 * se_of(s[oracle.SUM_V], s[oracle.SUM_V2], P)
        se_d = se_of(s[oracle.SUM_XBAR0], s[oracle.SUM_XBAR0_2], P) / 100.0
        assert abs(s[oracle.SUM_XBAR0] / (P * 100.0) - grow) < 3.5 * se_d


def pin_log_interpolation(lib):
    """Spot weight linear in ln S: a grid with sigma_ij = a_j + b_j ln s_i is
    reproduced exactly inside the grid, (1-v)(a_j + b_j ln S) + v(a_{j+1} +
    b_{j+1} ln S), with d sigma / d S = ((1-v) b_j + v b_{j+1}) / S; values
    equal scipy's linear interpolator on (ln s, t); flat and slope 0 outside."""
    from scipy.interpolate import RegularGridInterpolator
    s = np.array([60.0, 75.0, 97.0, 120.0, 155.0])
    t = np.array([0.0, 0.4, 1.1])
    a, b = np.array([0.9, 1.1, 0.7]), np.array([-0.12, -0.16, -0.09])
    g = a[None, :] + b[None, :] * np.log(s)[:, None]
    surf = W.Surface(s, t, g, interp=oracle.INTERP_LOGS)
    rng = np.random.Generator(np.random.PCG64(8))
    ref = RegularGridInterpolator((np.log(s), t), g, method="linear")
    for _ in range(60):
        S = rng.uniform(s[0], s[-1])
        tt = rng.uniform(0.0, t[-1])
        e = oracle.sigma_eval(surf, S, tt, lib=lib)
        j = min(int(np.searchsorted(t, tt, side="right")) - 1, 1)
        v = (tt - t[j]) / (t[j + 1] - t[j])
        exact = (1 - v) * (a[j] + b[j] * math.log(S)) + v * (a[j + 1] + b[j + 1] * math.log(S))
        assert abs(e["sigma"] - exact) < 1e-13
        assert abs(e["dsigma_dS"] - ((1 - v) * b[j] + v * b[j + 1]) / S) < 1e-13
        assert abs(e["sigma"] - ref([[math.log(S), tt]])[0]) < 1e-13
        assert abs(sum(e["w"]) - 1.0) < 1e-14
    for S in (10.0, 1000.0):
        e = oracle.sigma_eval(surf, S, 0.5, lib=lib)
        edge = oracle.sigma_eval(surf, s[0] if S < s[0] else s[-1], 0.5, lib=lib)
        assert e["dsigma_dS"] == 0.0 and abs(e["sigma"] - edge["sigma"]) < 1e-15


def _model_cases():
    out = []
    for interp, scheme, tag in ((oracle.INTERP_LOGS, oracle.SCHEME_LOG, "ln-S weight"),
                                (oracle.INTERP_S, oracle.SCHEME_X, "Euler on X"),
                                (oracle.INTERP_LOGS, oracle.SCHEME_X, "both")):
        for c in ADJOINT_CASES[:4]:
            name, surf, opt = _case(c)
            surf = W.Surface(surf.spot, surf.time, surf.sigma, interp=interp)
            out.append((f"{tag}: {name}", surf, W.Option(**{**opt.__dict__, "scheme": scheme})))
    return out


def pin_adjoint_vs_autograd_readings(lib):
    """The reverse sweep against torch.autograd of the independent
    restatement, under the ln-S spot weight, the Euler scheme on X and both,
    on the same tiny grids as pin_adjoint_vs_autograd."""
    for name, surf, opt in _model_cases():
        Z = np.stack([oracle.normals(opt.seed, p, opt.n_steps, lib=lib) for p in range(opt.n_paths)])
        price, delta, vega, _ = torch_lv.autograd_greeks(
            surf.spot, surf.time, surf.sigma, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.phi, Z,
            interp=surf.interp, scheme=opt.scheme)
        res = oracle.finalize(oracle.run_sums(surf, opt, lib=lib), opt.n_paths, opt.S0,
                              surf.n_spot * surf.n_time, lib=lib)
        scale = max(1e-3, np.max(np.abs(vega)))
        assert abs(res[0] - price) <= 1e-11 * max(1.0, abs(price)), name
        assert abs(res[1] - delta) <= 1e-11 * max(1.0, abs(delta)), (name, res[1], delta)
        np.testing.assert_allclose(res[3:].reshape(vega.shape), vega, rtol=0, atol=1e-11 * scale, err_msg=name)


def pin_adjoint_vs_bump_readings(lib):
    """Central bump-and-reprice (Sec. III) against the adjoint under the
    other readings, as in pin_adjoint_vs_bump."""
    for interp, scheme in ((oracle.INTERP_LOGS, oracle.SCHEME_LOG), (oracle.INTERP_S, oracle.SCHEME_X)):
        base = W.random_surface(8, 3, 2, s_lo=85, s_hi=118, t_hi=0.6)
        surf = W.Surface(base.spot, base.time, base.sigma, interp=interp)
        opt = W.Option(S0=100.0, r=0.01, K=101.0, T=0.6, n_steps=4, n_paths=64, seed=12, phi=1, scheme=scheme)
        xN, _, _ = oracle.paths(surf, opt, 0, opt.n_paths, lib=lib)
        assert np.min(np.abs(np.exp(xN) - opt.K)) > 1e-3
        res = oracle.finalize(oracle.run_sums(surf, opt, lib=lib), opt.n_paths, opt.S0, 6, lib=lib)
        vfd, dfd = oracle.bump(surf, opt, 1e-6, 1e-6 * opt.S0, lib=lib)
        scale = np.max(np.abs(vfd))
        np.testing.assert_allclose(res[3:].reshape(3, 2), vfd, rtol=0, atol=2e-6 * scale)
        assert abs(res[1] - dfd) < 2e-6 * max(1.0, abs(dfd))


# ------------------------------------------------------ rho and d V / d T

def pin_black_scholes_rho_dvdt(lib):
    """Flat sigma (log-Euler is exact in law): the pathwise rho and d V / d T
    equal Black-Scholes' rho and -theta (d V / d T at fixed S0) within 3.5
    standard errors, for a call and a put."""
    from scipy.stats import norm
    sig, r, T, S0, K = 0.22, 0.04, 1.3, 100.0, 104.0
    surf = W.flat_surface(sig, n_spot=3, n_time=4, s_lo=30.0, s_hi=400.0, t_hi=2.0)
    d1 = (math.log(S0 / K) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    for phi in (1, -1):
        opt = W.Option(S0=S0, r=r, K=K, T=T, n_steps=16, n_paths=1 << 16, seed=31, phi=phi)
        s = oracle.run_sums(surf, opt, lib=lib)
        P = opt.n_paths
        rho = phi * K * T * math.exp(-r * T) * norm.cdf(phi * d2)
        dvdt = S0 * norm.pdf(d1) * sig / (2 * math.sqrt(T)) + phi * r * K * math.exp(-r * T) * norm.cdf(phi * d2)
        assert abs(s[oracle.SUM_RHO] / P - rho) < 3.5 * se_of(s[oracle.SUM_RHO], s[oracle.SUM_RHO_2], P), phi
        assert abs(s[oracle.SUM_DVDT] / P - dvdt) < 3.5 * se_of(s[oracle.SUM_DVDT], s[oracle.SUM_DVDT_2], P), phi


def pin_rho_dvdt_vs_bump(lib):
    """Pathwise rho and d V / d T equal central differences of the oracle's
    own price in r and in T (same normals, n_steps fixed) to O(eps^2), on a
    grid that varies in time, where no path and no step time sits within the
    bump of a payoff, cell or time-node kink."""
    surf = W.random_surface(9, 4, 3, s_lo=86, s_hi=116, t_hi=0.9)
    for scheme in (oracle.SCHEME_LOG, oracle.SCHEME_X):
        opt = W.Option(S0=100.0, r=0.02, K=101.0, T=0.7, n_steps=5, n_paths=64, seed=14, phi=1, scheme=scheme)
        xN, _, _ = oracle.paths(surf, opt, 0, opt.n_paths, lib=lib)
        assert np.min(np.abs(np.exp(xN) - opt.K)) > 1e-3
        tn = np.arange(opt.n_steps) * opt.T / opt.n_steps
        assert np.min(np.abs(tn[:, None] - surf.time[None, :])[1:]) > 1e-4   # t_0 = 0 sits on a node in both bumps
        s = oracle.run_sums(surf, opt, lib=lib)
        P = opt.n_paths

        def price(**kw):
            o = W.Option(**{**opt.__dict__, **kw})
            return oracle.run_sums(surf, o, greeks=False, lib=lib)[oracle.SUM_V] / P

        e = 1e-6
        rho_fd = (price(r=opt.r + e / 2) - price(r=opt.r - e / 2)) / e
        dvdt_fd = (price(T=opt.T + e / 2) - price(T=opt.T - e / 2)) / e
        assert abs(s[oracle.SUM_RHO] / P - rho_fd) < 2e-6 * max(1.0, abs(rho_fd)), (scheme, s[oracle.SUM_RHO] / P, rho_fd)
        assert abs(s[oracle.SUM_DVDT] / P - dvdt_fd) < 2e-6 * max(1.0, abs(dvdt_fd)), (scheme, s[oracle.SUM_DVDT] / P, dvdt_fd)


def pin_rho_dvdt_vs_autograd(lib):
    """Pathwise rho and d V / d T against torch.autograd of the independent
    restatement with r and T as inputs, on the tiny grids of the adjoint pins
    under every reading."""
    cases = [_case(c) for c in ADJOINT_CASES] + [(n, s, o) for n, s, o in _model_cases()]
    for name, surf, opt in cases:
        Z = np.stack([oracle.normals(opt.seed, p, opt.n_steps, lib=lib) for p in range(opt.n_paths)])
        ref = torch_lv.autograd_all(surf.spot, surf.time, surf.sigma, opt.S0, opt.r, opt.K, opt.T, opt.n_steps,
                                    opt.phi, Z, interp=getattr(surf, "interp", 0), scheme=opt.scheme)
        s = oracle.run_sums(surf, opt, lib=lib)
        P = opt.n_paths
        assert abs(s[oracle.SUM_RHO] / P - ref["rho"]) <= 1e-10 * max(1.0, abs(ref["rho"])), (name, ref["rho"])
        assert abs(s[oracle.SUM_DVDT] / P - ref["dVdT"]) <= 1e-10 * max(1.0, abs(ref["dVdT"])), (name, ref["dVdT"])


# ------------------------------------------------ second-order buckets

def _path_and_cells(surf, opt, p, lib):
    """ln S_0 .. ln S_N of path p (numpy restatement of the log-Euler step on
    the oracle's normals and its pinned bilinear lookup) and, per step, the
    cell and weights (i, j, u, v, inside)."""
    z = oracle.normals(opt.seed, p, opt.n_steps, lib=lib)
    dt = opt.T / opt.n_steps
    x, cells = [math.log(opt.S0)], []
    for n in range(opt.n_steps):
        S = math.exp(x[-1])
        e = oracle.sigma_eval(surf, S, n * dt, lib=lib)
        cells.append((e["i"], e["j"], e["u"], e["v"], bool(surf.spot[0] <= S <= surf.spot[-1])))
        x.append(x[-1] + (opt.r - 0.5 * e["sigma"] * e["sigma"]) * dt + e["sigma"] * math.sqrt(dt) * z[n])
    return np.array(x), cells


def pin_vanna_vs_autograd(lib):
    """Per path, the oracle's second-order buckets equal torch.autograd of
    the definitions: the gradient of the pathwise delta at the fixed path
    plus the delta times the gradient of the path's log density, on tiny
    grids (paths leaving the grid, one time node, a put, r > 0)."""
    cases = [(W.random_surface(2, 3, 2, s_lo=92, s_hi=108, t_hi=0.5), 100.0, 0.01, 99.0, 0.5, 8, 1, 9),
             (W.random_surface(1, 3, 1, s_lo=80, s_hi=125), 100.0, 0.0, 100.0, 1.0, 6, 1, 3),
             (W.random_surface(4, 4, 3, s_lo=70, s_hi=140, t_hi=2.0), 100.0, 0.03, 104.0, 1.3, 9, -1, 6)]
    checked = 0
    for surf, S0, r, K, T, N, phi, seed in cases:
        opt = W.Option(S0=S0, r=r, K=K, T=T, n_steps=N, n_paths=12, seed=seed, phi=phi)
        for p in range(opt.n_paths):
            x, cells = _path_and_cells(surf, opt, p, lib)
            ref = torch_lv.vanna_at_fixed_path(surf.spot, surf.time, surf.sigma, S0, r, K, T, phi, x, cells)
            got = oracle.run_vanna(surf, opt, p, p + 1, n_threads=1, lib=lib)["vanna"]
            scale = max(1e-9, float(np.max(np.abs(ref))))
            assert np.max(np.abs(got - ref)) <= 1e-9 * scale, (p, np.max(np.abs(got - ref)), scale)
            checked += int(np.any(ref != 0.0))
    assert checked >= 8


def pin_vanna_flat_black_scholes(lib):
    """On a flat grid log-Euler is exact in law, so the buckets summed over
    the grid (a partition of unity) estimate Black-Scholes vanna
    d^2 C / d S0 d sigma = -phi(d1) d2 / sigma, within 4 standard errors."""
    sig, S0, K, T = 0.2, 100.0, 100.0, 1.0
    surf = W.flat_surface(sig)
    opt = W.Option(S0=S0, r=0.0, K=K, T=T, n_steps=4, n_paths=1 << 20, seed=31)
    res = oracle.run_vanna(surf, opt, lib=lib)
    sd = sig * math.sqrt(T)
    d1 = (math.log(S0 / K) + 0.5 * sig * sig * T) / sd
    d2 = d1 - sd
    vanna = -math.exp(-0.5 * d1 * d1) / math.sqrt(2 * math.pi) * d2 / sig
    assert abs(res["total"] - vanna) <= 4 * res["total_se"], (res["total"], vanna, res["total_se"])
    assert res["total_se"] < 0.1 * abs(vanna)
    _, delta, _ = bs_call_put(S0, K, T, 0.0, sig, 1)
    assert abs(res["delta"] - delta) <= 0.01, (res["delta"], delta)


def pin_vanna_one_step_closed_form(lib):
    """One Euler step from inside a cell is exactly Black-Scholes with
    sigma_0 = sigma(S0, 0), which depends on S0 and on the two nodes of the
    cell: each bucket's estimate equals central differences (in S0 and in
    sigma_ij) of that closed form, within 4 standard errors."""
    surf = W.random_surface(7, 4, 3, s_lo=90, s_hi=111, t_hi=1.0)
    S0, K, T, r = 100.0, 101.0, 0.4, 0.02
    opt = W.Option(S0=S0, r=r, K=K, T=T, n_steps=1, n_paths=1 << 21, seed=17)
    res = oracle.run_vanna(surf, opt, lib=lib)

    def price(s0, sg):
        i = int(np.searchsorted(surf.spot, s0, side="right") - 1)
        u = (s0 - surf.spot[i]) / (surf.spot[i + 1] - surf.spot[i])
        sigma0 = sg[i, 0] * (1 - u) + sg[i + 1, 0] * u
        return bs_call_put(s0, K, T, r, sigma0, 1)[0]

    hs, he = 1e-3, 1e-4
    base = np.array(surf.sigma, dtype=np.float64)
    ref = np.zeros_like(base)
    for (i, j) in np.ndindex(base.shape):
        def d_price_d_sig(s0):
            up, dn = base.copy(), base.copy()
            up[i, j] += he
            dn[i, j] -= he
            return (price(s0, up) - price(s0, dn)) / (2 * he)
        ref[i, j] = (d_price_d_sig(S0 + hs) - d_price_d_sig(S0 - hs)) / (2 * hs)
    assert np.count_nonzero(np.abs(ref) > 1e-6) == 2        # the two nodes of the cell, time row 0
    err = np.abs(res["vanna"] - ref)
    assert np.all(err <= 4 * res["vanna_se"] + 1e-5), (res["vanna"], ref, res["vanna_se"])


ALL_PINS = [pin_philox_curand, pin_normals_from_curand_words, pin_uniform_exact, pin_normal_law,
            pin_black_scholes, pin_flat_closed_form_paths, pin_martingale, pin_put_call_parity,
            pin_adjoint_vs_autograd, pin_adjoint_vs_bump, pin_bilinear,
            pin_flat_closed_form_paths_euler_x, pin_martingale_euler_x, pin_log_interpolation,
            pin_adjoint_vs_autograd_readings, pin_adjoint_vs_bump_readings,
            pin_black_scholes_rho_dvdt, pin_rho_dvdt_vs_bump, pin_rho_dvdt_vs_autograd,
            pin_vanna_vs_autograd, pin_vanna_flat_black_scholes, pin_vanna_one_step_closed_form]
