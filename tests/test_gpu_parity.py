"""CUDA path against the FP64 oracle, element by element on the same seeded
inputs, through the C ABI (needs a GB300)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G

pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LV_PARITY_REPORT")


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


def _report(name, d):
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": name, **d}) + "\n")


EDGE = [
    # name, surface, option
    ("2x1 grid, one time node", W.random_surface(1, 2, 1, s_lo=80, s_hi=125),
     W.Option(S0=100.0, r=0.0, K=100.0, T=1.0, n_steps=13, n_paths=3000, seed=3)),
    ("3x2 grid, paths leave both sides", W.random_surface(2, 3, 2, s_lo=97, s_hi=103, t_hi=0.5),
     W.Option(S0=100.0, r=0.01, K=99.0, T=0.5, n_steps=8, n_paths=5000, seed=4)),
    ("uneven 7x5 grid (binary search), put", W.random_surface(3, 7, 5, s_lo=75, s_hi=130, t_hi=1.0, uneven=True),
     W.Option(S0=100.0, r=0.02, K=101.0, T=0.8, n_steps=10, n_paths=4097, seed=5, phi=-1)),
    ("strike at a node, maturity inside a time cell", W.random_surface(4, 6, 4, s_lo=70, s_hi=140, t_hi=2.0),
     W.Option(S0=100.0, r=0.0, K=float(W.random_surface(4, 6, 4, s_lo=70, s_hi=140, t_hi=2.0).spot[2]),
              T=1.3, n_steps=9, n_paths=2500, seed=6)),
    ("one path", W.small_skew_surface(), W.Option(S0=100.0, r=0.0, K=90.0, T=1.0, n_steps=52, n_paths=1, seed=2)),
    ("ragged tail 33 paths, 1 step", W.small_skew_surface(),
     W.Option(S0=100.0, r=0.03, K=100.0, T=0.1, n_steps=1, n_paths=33, seed=8)),
    ("deep OTM call (few live paths)", W.small_skew_surface(),
     W.Option(S0=100.0, r=0.0, K=160.0, T=1.0, n_steps=52, n_paths=20000, seed=9)),
    ("K = 0 (every path live)", W.small_skew_surface(),
     W.Option(S0=100.0, r=0.04, K=0.0, T=1.0, n_steps=20, n_paths=8192, seed=10)),
]


@pytest.mark.parametrize("case", EDGE, ids=[c[0] for c in EDGE])
def test_edge_cases(case, lib):
    name, surf, opt = case
    _report(name, G.full_parity(surf, opt, lib, label=name))


def test_small_skew_16384_paths(lib):
    surf, opt = W.config_small()
    _report("20x10 grid, 52 steps, 2^14 paths", G.full_parity(surf, opt, lib, label="small"))


def test_paper_shape_full_size(lib):
    """30x60 grid, 156 steps, 2^20 paths: every path checked, aggregates at
    full size in the default launch shape, which is the one the benchmark's
    tuner picks on GB300 (block 128, checkpoints every 4 steps, two paths per
    lane in packed pairs)."""
    surf, opt = W.config_paper_shape()
    s = G.make_surface(surf, opt, lib)
    assert s.get_launch(opt.n_steps, True)[:2] == (128, 4)
    assert s.get_paths_per_lane(opt.n_steps, opt.n_paths) == 2
    s.close()
    _report("30x60 grid, 156 steps, 2^20 paths", G.full_parity(surf, opt, lib, label="paper shape"))


@pytest.mark.parametrize("acc", [0, 1], ids=["fp64", "kahan"])
def test_precision_subset(acc, lib):
    """2^24-path precision workload: its first 2^18 paths against the oracle
    with both level-2 accumulations."""
    for which in ("small", "paper"):
        surf, opt = W.config_precision(which)
        opt.n_paths = 1 << 18
        _report(f"precision {which} 2^18 acc={acc}", G.full_parity(surf, opt, lib, accumulation=acc,
                                                                    label=f"precision {which}"))


def test_large_grid_sample(lib):
    """100x100 grid, 1,260 steps, checkpoints every 32 steps: the first 2^14
    paths against the oracle."""
    surf, opt = W.config_large()
    opt.n_paths = 1 << 14
    _report("100x100 grid, 1260 steps, 2^14 paths, k=32",
            G.full_parity(surf, opt, lib, launch=(128, 32, 0), label="large"))


def test_large_grid_timed_shape(lib):
    """100x100 grid, 1,260 steps, in the launch shape the benchmark times it
    at (block 128, checkpoints every 4 steps, the grid read through L1): the
    first 2^14 paths against the oracle."""
    surf, opt = W.config_large()
    opt.n_paths = 1 << 14
    s = G.make_surface(surf, opt, lib, launch=(128, 4, 0))
    assert s.get_launch(opt.n_steps, True)[:2] == (128, 4)
    s.close()
    _report("100x100 grid, 1260 steps, 2^14 paths, k=4",
            G.full_parity(surf, opt, lib, launch=(128, 4, 0), label="large k=4"))


@pytest.mark.parametrize("ppl_case", ["small", "paper 2^18", "edge: 33 paths", "edge: put, uneven grid",
                                      "large 100x100, grid through L1"])
def test_two_paths_per_lane(ppl_case, lib):
    """Two paths per lane in the forward tiles (a warp claims two tiles and
    runs them interleaved): the same per-path arithmetic, checked against the
    oracle path for path, at k = 4 and 8 and in both level-2 modes. Every
    instantiation but (k = 4, binary64, grid in shared memory) runs the two
    paths' binary32 arithmetic in packed pairs; the cases cover both forms, the
    binary search for the cell (uneven grid) and the grid read through L1."""
    if ppl_case == "small":
        surf, opt = W.config_small()
        cases = [((128, 4, 0), 0), ((128, 8, 0), 1)]
    elif ppl_case == "paper 2^18":
        surf, opt = W.config_paper_shape()
        opt.n_paths = 1 << 18
        cases = [((128, 4, 0), 0), ((128, 4, 0), 1), ((128, 8, 0), 0)]
    elif ppl_case == "large 100x100, grid through L1":
        surf, opt = W.config_large()
        opt.n_paths = 1 << 14
        cases = [((128, 4, 0), 0)]
    elif ppl_case == "edge: 33 paths":
        _, surf, opt = EDGE[5]
        cases = [((64, 4, 0), 0)]
    else:
        _, surf, opt = EDGE[2]
        cases = [((128, 8, 0), 1)]
    for launch, acc in cases:
        s = G.make_surface(surf, opt, lib, launch=launch, accumulation=acc, ppl=2)
        assert s.get_paths_per_lane(opt.n_steps, opt.n_paths) == 2
        s.close()
        _report(f"two paths per lane: {ppl_case} {launch} acc={acc}",
                G.full_parity(surf, opt, lib, launch=launch, accumulation=acc, ppl=2, label=ppl_case))


def test_two_paths_per_lane_equals_one(lib):
    """Same paths, same per-path arithmetic: one or two paths per lane agree to
    reduction-order rounding, with the two paths in scalar registers (k = 4,
    binary64 level 2) and in packed pairs (k = 8, and Kahan level 2); where two
    paths per lane do not exist the call runs one."""
    surf, opt = W.config_paper_shape()
    opt.n_paths = 1 << 17
    for launch, acc in [((128, 4, 0), 0), ((128, 8, 0), 0), ((128, 4, 0), 1)]:
        a = G.make_surface(surf, opt, lib, launch=launch, accumulation=acc, ppl=1)
        b = G.make_surface(surf, opt, lib, launch=launch, accumulation=acc, ppl=2)
        assert a.get_paths_per_lane(opt.n_steps, opt.n_paths) == 1
        assert b.get_paths_per_lane(opt.n_steps, opt.n_paths) == 2
        pa, da, va = a.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
        pb, db, vb = b.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
        # Kahan level 2 keeps each thread's scalar sums as compensated binary32
        # pairs (within about 2^-23 of that thread's sum), and which paths share
        # a thread depends on the paths per lane: the binary64 totals of the two
        # runs then differ by about 1e-10 relative (the binary64 mode: 1e-14)
        tp, td = (1e-12, 1e-9) if acc == 0 else (1e-8, 1e-8)
        assert abs(pb - pa) <= tp * abs(pa) and abs(db - da) <= td * abs(da), (launch, acc)
        assert np.max(np.abs(vb - va)) <= 1e-6 * np.max(np.abs(va)), (launch, acc)
        a.close()
        b.close()
    # the default: two where they exist, for calls that give every warp two pairs of tiles
    b = G.make_surface(surf, opt, lib, launch=(128, 4, 0))
    assert b.get_paths_per_lane(opt.n_steps, 1 << 22) == 2
    assert b.get_paths_per_lane(opt.n_steps, 1 << 12) == 1
    b.set_launch(128, 16, 0)
    assert b.get_paths_per_lane(opt.n_steps, 1 << 22) == 1       # checkpoints every 16 steps: one
    b.set_launch(128, 4, 0)
    b.set_scheme(lv.LV_SCHEME_S)
    assert b.get_paths_per_lane(opt.n_steps, 1 << 22) == 2       # every reading's reverse sweep
    b.set_adjoint_method(lv.LV_ADJ_TANGENT)
    assert b.get_paths_per_lane(opt.n_steps, 1 << 22) == 1       # the main reading's tangent ratio only
    with pytest.raises(lv.LVError):
        b.get_paths_per_lane(opt.n_steps, 0)
    with pytest.raises(lv.LVError):
        b.set_paths_per_lane(3)
    b.close()


@pytest.mark.parametrize("case", ["paper 2^18", "uneven 7x5 grid (binary search), put", "large 100x100"])
def test_price_only_matches_adjoint_price(case, lib):
    """The forward-only kernel (two paths per lane in packed binary32 pairs)
    and the adjoint kernel at one path per lane (scalar arithmetic) compute the
    same paths bit for bit: their prices agree to binary64 reduction order."""
    if case == "paper 2^18":
        surf, opt = W.config_paper_shape()
        opt.n_paths = 1 << 18
    elif case == "large 100x100":
        surf, opt = W.config_large()
        opt.n_paths = 1 << 16
    else:
        _, surf, opt = next(e for e in EDGE if e[0] == case)
    gs = G.make_surface(surf, opt, lib, launch=(128, 4, 0), ppl=1)
    p, d, v = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    pp, se = gs.price(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(pp - p) <= 1e-11 * max(abs(p), 1e-300) and se >= 0
    gs.close()


@pytest.mark.parametrize("launch", [(128, 4, 0), (96, 8, 0), (128, 16, 0), (128, 32, 1), (64, 8, 2), (32, 4, 0)])
def test_launch_shape_invariance(launch, lib):
    """Per-path arithmetic does not depend on the launch shape; results agree
    to reduction-order rounding."""
    surf, opt = W.config_small()
    opt.n_paths = 20000
    base = G.make_surface(surf, opt, lib)
    p0, d0, v0 = base.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    alt = G.make_surface(surf, opt, lib, launch=launch)
    p1, d1, v1 = alt.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(p1 - p0) <= 1e-12 * abs(p0)
    assert abs(d1 - d0) <= 1e-9 * abs(d0)
    assert np.max(np.abs(v1 - v0)) <= 1e-6 * np.max(np.abs(v0))


def test_more_than_1024_level2_rows(lib):
    """One-warp blocks on 2^16 paths give more than 1,024 level-2 rows, so the
    level-3 finalize sums its chunks in several groups of 32."""
    import torch
    surf, opt = W.config_small()
    opt.n_paths = 1 << 16
    base = G.make_surface(surf, opt, lib)
    p0, d0, v0 = base.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    alt = G.make_surface(surf, opt, lib, launch=(32, 4, 0))
    block, _, bps = alt.get_launch(opt.n_steps, True)
    rows = min(opt.n_paths // 32, bps * torch.cuda.get_device_properties(0).multi_processor_count)
    assert block == 32 and rows > 1024, (block, bps, rows)
    p1, d1, v1 = alt.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(p1 - p0) <= 1e-12 * abs(p0)
    assert abs(d1 - d0) <= 1e-9 * abs(d0)
    assert np.max(np.abs(v1 - v0)) <= 1e-6 * np.max(np.abs(v0))


@pytest.mark.parametrize("ppl", [1, 2], ids=["one path per lane", "two paths per lane"])
def test_path_range_sharding(ppl, lib):
    """Sums over [0, P/3), [P/3, P) add up to the sums over [0, P): the
    path-range split a multi-GPU run would use (a range that starts off a
    tile boundary; each rank's range at the benchmark's size runs two paths
    per lane)."""
    import torch
    surf, opt = W.config_paper_shape()
    P = 1 << 16
    gs = G.make_surface(surf, opt, lib, ppl=ppl)
    n = 3 + surf.n_spot * surf.n_time
    whole = torch.zeros(n, dtype=torch.float64, device="cuda")
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    gs.set_stream(torch.cuda.current_stream().cuda_stream)
    args = (opt.S0, opt.r, opt.K, opt.T, opt.n_steps)
    gs.price_greeks_sums_device(*args, 0, P, opt.seed, 0, whole.data_ptr())
    gs.price_greeks_sums_device(*args, 0, P // 3, opt.seed, 0, a.data_ptr())
    gs.price_greeks_sums_device(*args, P // 3, P, opt.seed, 0, b.data_ptr())
    torch.cuda.synchronize()
    w, s = whole.cpu().numpy(), (a + b).cpu().numpy()
    assert abs(w[0] - s[0]) <= 1e-12 * abs(w[0])
    assert abs(w[2] - s[2]) <= 1e-10 * abs(w[2])
    assert np.max(np.abs(w[3:] - s[3:])) <= 1e-6 * np.max(np.abs(w[3:]))
    # and the raw sums agree with the oracle's
    ref = oracle.run_sums(surf, opt, 0, P)
    assert abs(w[0] - ref[oracle.SUM_V]) <= 1e-5 * abs(ref[oracle.SUM_V])
    # finalizing the combined sums on the device gives the single-call result
    fin = torch.zeros(n, dtype=torch.float64, device="cuda")
    gs.finalize_sums_device((a + b).data_ptr(), P, opt.S0, fin.data_ptr())
    one = torch.zeros(n, dtype=torch.float64, device="cuda")
    gs.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed, one.data_ptr())
    torch.cuda.synchronize()
    f, o = fin.cpu().numpy(), one.cpu().numpy()
    assert abs(f[0] - o[0]) <= 1e-12 * abs(o[0]) and abs(f[1] - o[1]) <= 1e-9 * abs(o[1])
    assert abs(f[2] - o[2]) <= 1e-9 * abs(o[2])
    assert np.max(np.abs(f[3:] - o[3:])) <= 1e-6 * np.max(np.abs(o[3:]))
    # and the sharded helper (one rank here) agrees too
    from paper_2002_02481_gb300.shard import price_greeks_sharded
    sh = price_greeks_sharded(gs, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed).cpu().numpy()
    assert abs(sh[0] - o[0]) <= 1e-12 * abs(o[0]) and np.max(np.abs(sh[3:] - o[3:])) <= 1e-6 * np.max(np.abs(o[3:]))


def test_device_output_matches_host_output(lib):
    import torch
    surf, opt = W.config_small()
    gs = G.make_surface(surf, opt, lib)
    gs.set_stream(torch.cuda.current_stream().cuda_stream)
    out = torch.zeros(3 + surf.n_spot * surf.n_time, dtype=torch.float64, device="cuda")
    gs.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, out.data_ptr())
    torch.cuda.synchronize()
    p, d, v = gs.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    o = out.cpu().numpy()
    assert abs(o[0] - p) <= 1e-12 * abs(p)
    assert abs(o[1] - d) <= 1e-9 * abs(d)
    np.testing.assert_allclose(o[3:].reshape(v.shape), v, rtol=0, atol=1e-6 * np.max(np.abs(v)))
    # the price-only entry point agrees with the price of the adjoint call
    pp, se = gs.price(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    assert abs(pp - p) <= 1e-12 * abs(p) and se > 0


def test_stream_switch_between_calls(lib):
    """Calls on one handle alternate between two streams: the library waits
    for the old stream before switching, and every call gives the same result
    (the level-2 rows, the counters and the staging buffers are shared)."""
    import torch
    surf, opt = W.config_small()
    gs = G.make_surface(surf, opt, lib)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    n = 3 + surf.n_spot * surf.n_time
    outs = []
    for k in range(4):
        s = streams[k % 2]
        gs.set_stream(s.cuda_stream)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(s):
            out.fill_(float("nan"))
        gs.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, out.data_ptr())
        outs.append(out)
    torch.cuda.synchronize()
    ref = outs[0].cpu().numpy()
    assert np.all(np.isfinite(ref))
    for o in (x.cpu().numpy() for x in outs[1:]):
        # the same paths; only the order of the binary32 bucket reductions differs
        assert abs(o[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert abs(o[1] - ref[1]) <= 1e-9 * abs(ref[1])
        np.testing.assert_allclose(o[3:], ref[3:], rtol=0, atol=1e-6 * np.max(np.abs(ref[3:])))
    gs.set_stream(0)


def test_gpu_argument_errors(lib):
    surf, opt = W.config_small()
    gs = G.make_surface(surf, opt, lib)
    bad = [
        dict(S0=-1.0), dict(T=0.0), dict(K=-5.0), dict(n_steps=0), dict(n_steps=lv_max_steps() + 1),
        dict(n_paths=0), dict(r=float("inf")),
    ]
    for b in bad:
        a = dict(S0=100.0, r=0.0, K=100.0, T=1.0, n_steps=10, n_paths=100, seed=1)
        a.update(b)
        with pytest.raises(lv.LVError) as e:
            gs.price_greeks(**a)
        assert e.value.status == lv.LV_EINVAL, b
    with pytest.raises(lv.LVError):
        gs.set_launch(100, 8, 0)
    with pytest.raises(lv.LVError):
        gs.set_launch(256, 4, 0)
    with pytest.raises(lv.LVError):
        gs.set_launch(256, 12, 0)


def lv_max_steps():
    return 8192
