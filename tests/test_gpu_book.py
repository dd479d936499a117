"""A book of options in one persistent, graph-captured launch (needs a
GB300): every option equals the single-option sums call with the same
Philox stream (up to reduction order), graph replays with new parameters
equal uncaptured runs, the autotuner keeps a working shape, and options on
nonzero streams match the FP64 oracle."""
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


def _book_inputs():
    surfs = [W.small_skew_surface(), W.seeded_skew_surface(3, n_spot=12, n_time=7, t_hi=2.0),
             W.random_surface(5, 6, 1, s_lo=70, s_hi=140), W.random_surface(6, 9, 4, s_lo=60, s_hi=150, uneven=True)]
    rng = np.random.Generator(np.random.PCG64(11))
    items = []
    for o in range(14):
        T = float(rng.choice([0.25, 0.5, 1.0, 2.0]))
        items.append(W.BookItem(surface=int(rng.integers(0, len(surfs))), phi=int(rng.choice([-1, 1])),
                                K=float(rng.uniform(80, 120)), T=T, n_steps=max(1, int(round(26 * T))),
                                n_paths=int(rng.integers(1, 9000)), stream_id=o + 3))
    items[0].n_paths = 1
    items[1].n_paths = 33
    return surfs, items


def _single(lib, surf, it, S0, r, seed):
    import torch
    s = lv.Surface.from_workload(surf, lib)
    s.set_option_type(it.phi)
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    n = 3 + surf.n_spot * surf.n_time
    sums = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.price_greeks_sums_device(S0, r, it.K, it.T, it.n_steps, 0, it.n_paths, seed, it.stream_id, sums.data_ptr())
    s.finalize_sums_device(sums.data_ptr(), it.n_paths, S0, out.data_ptr())
    torch.cuda.synchronize()
    s.close()
    return out.cpu().numpy()


def _close(a, b, label):
    # same per-path arithmetic; the binary32 level-1 bucket sums run in a different
    # order (the book sums up to 8,192 paths per work item before its binary64 atomics)
    assert abs(a[0] - b[0]) <= 1e-12 * max(abs(b[0]), 1e-300), (label, a[0], b[0])
    assert abs(a[1] - b[1]) <= 1e-9 * max(abs(b[1]), 1e-12) + 1e-15, (label, a[1], b[1])
    vmax = np.max(np.abs(b[3:]))
    assert np.max(np.abs(a[3:] - b[3:])) <= 1e-5 * vmax + 1e-15, label


def test_book_matches_single_option_calls(lib):
    import torch
    surfs, items = _book_inputs()
    handles = [lv.Surface.from_workload(s, lib) for s in surfs]
    book = lv.Book(handles, items, lib)
    for h in handles:
        h.close()                                  # the book keeps its own copy of the grids
    S0, r, seed = 100.0, 0.02, 9
    out = book.run(S0, r, seed)                    # captures the graph
    for o, it in enumerate(items):
        ref = _single(lib, surfs[it.surface], it, S0, r, seed)
        _close(out[book.offsets[o]:book.offsets[o + 1]], ref, f"option {o}")
    # replay with other parameters against an uncaptured run
    out2 = book.run(95.0, 0.0, 12345)
    d = torch.zeros(book.offsets[-1], dtype=torch.float64, device="cuda")
    book.run_device(95.0, 0.0, 12345, d.data_ptr())
    torch.cuda.synchronize()
    dd = d.cpu().numpy()
    for o in range(len(items)):
        _close(out2[book.offsets[o]:book.offsets[o + 1]], dd[book.offsets[o]:book.offsets[o + 1]], f"replay {o}")
    assert not np.allclose(out2, out)          # other S0, r and seed: other results
    # autotuner: keeps a shape that still reproduces the results
    blk, k, item_paths, ms = book.tune(S0, r, seed)
    assert blk in (64, 128) and k in (4, 8) and item_paths > 0 and ms > 0
    assert book.paths_per_lane() in (1, 2)
    out3 = book.run(S0, r, seed)
    for o in range(len(items)):
        _close(out3[book.offsets[o]:book.offsets[o + 1]], out[book.offsets[o]:book.offsets[o + 1]], f"tuned {o}")
    book.close()


def test_book_options_against_oracle(lib):
    surfs, items = _book_inputs()
    handles = [lv.Surface.from_workload(s, lib) for s in surfs]
    book = lv.Book(handles, items, lib)
    S0, r, seed = 100.0, 0.02, 9
    out = book.run(S0, r, seed)
    for o in (1, 4, 7, 11):
        it = items[o]
        opt = W.Option(S0=S0, r=r, K=it.K, T=it.T, n_steps=it.n_steps, n_paths=it.n_paths, seed=seed,
                       phi=it.phi, stream_id=it.stream_id)
        ref = oracle.price_greeks(surfs[it.surface], opt)
        p, dlt, _, v = book.result(out, o)
        assert abs(p - ref["price"]) <= 1e-5 * max(abs(ref["price"]), 1e-12), (o, p, ref["price"])
        assert abs(dlt - ref["delta"]) <= 1e-5 * max(abs(ref["delta"]), 1e-12), (o, dlt, ref["delta"])
        vm = np.max(np.abs(ref["vega"]))
        assert np.max(np.abs(v - ref["vega"].reshape(-1))) <= 1e-4 * max(vm, 1e-12), o
    book.close()


def test_aggregated_risk_is_the_weighted_sum_of_the_options(lib):
    """Per surface: the weighted sums of the options' prices, deltas and vega
    buckets (and the independent-stream standard error), accumulated inside
    the persistent kernel; graph replay and the device entry point agree."""
    import torch
    surfs, items = _book_inputs()
    handles = [lv.Surface.from_workload(s, lib) for s in surfs]
    book = lv.Book(handles, items, lib)
    S0, r, seed = 100.0, 0.02, 9
    per_option = book.run(S0, r, seed)
    for weights in (np.ones(len(items)), np.random.Generator(np.random.PCG64(3)).normal(size=len(items))):
        book.set_weights(weights)
        risk = book.run_risk(S0, r, seed)
        for s in range(len(surfs)):
            mine = [o for o, it in enumerate(items) if it.surface == s]
            p = sum(weights[o] * book.result(per_option, o)[0] for o in mine)
            d = sum(weights[o] * book.result(per_option, o)[1] for o in mine)
            e = np.sqrt(sum((weights[o] * book.result(per_option, o)[2]) ** 2 for o in mine))
            v = sum(weights[o] * book.result(per_option, o)[3] for o in mine) if mine else 0.0
            rp, rd, re, rv = book.risk(risk, s)
            scale = max(sum(abs(weights[o] * book.result(per_option, o)[0]) for o in mine), 1e-12)
            assert abs(rp - p) <= 1e-12 * scale, (s, rp, p)
            dscale = max(sum(abs(weights[o] * book.result(per_option, o)[1]) for o in mine), 1e-12)
            assert abs(rd - d) <= 1e-9 * dscale, (s, rd, d)
            assert abs(re - e) <= 1e-9 * max(e, 1e-12), (s, re, e)
            vscale = max(sum(np.max(np.abs(weights[o] * book.result(per_option, o)[3])) for o in mine), 1e-12)
            assert np.max(np.abs(rv - v)) <= 1e-5 * vscale, s
        dev = torch.zeros(book.risk_offsets[-1], dtype=torch.float64, device="cuda")
        book.run_risk_device(S0, r, seed, dev.data_ptr())
        torch.cuda.synchronize()
        dd = dev.cpu().numpy()
        for s in range(len(surfs)):
            a, b = book.risk(dd, s), book.risk(risk, s)
            assert abs(a[0] - b[0]) <= 1e-12 * max(abs(b[0]), 1e-12)
            assert np.max(np.abs(a[3] - b[3])) <= 1e-5 * max(np.max(np.abs(b[3])), 1e-12)
    with pytest.raises(lv.LVError):
        book.set_weights(np.full(len(items), np.nan))
    book.close()


def test_aggregated_risk_against_the_oracle(lib):
    """One surface's aggregated vega buckets against the weighted sum of the
    FP64 oracle's per-option buckets."""
    surfs, items = _book_inputs()
    handles = [lv.Surface.from_workload(s, lib) for s in surfs]
    book = lv.Book(handles, items, lib)
    S0, r, seed = 100.0, 0.02, 9
    weights = np.linspace(-1.0, 2.0, len(items))
    book.set_weights(weights)
    risk = book.run_risk(S0, r, seed)
    s = items[4].surface
    ref_p, ref_v = 0.0, 0.0
    for o, it in enumerate(items):
        if it.surface != s:
            continue
        opt = W.Option(S0=S0, r=r, K=it.K, T=it.T, n_steps=it.n_steps, n_paths=it.n_paths, seed=seed,
                       phi=it.phi, stream_id=it.stream_id)
        ref = oracle.price_greeks(surfs[s], opt)
        ref_p = ref_p + weights[o] * ref["price"]
        ref_v = ref_v + weights[o] * ref["vega"].reshape(-1)
    p, _, _, v = book.risk(risk, s)
    assert abs(p - ref_p) <= 1e-5 * max(abs(ref_p), 1e-12)
    assert np.max(np.abs(v - ref_v)) <= 1e-4 * max(np.max(np.abs(ref_v)), 1e-12)
    book.close()


def test_benchmark_book_against_oracle(lib):
    """The benchmark's book (8 seeded 30x60 surfaces x 64 options, uneven
    maturities and path counts up to 2^20) in the launch shape its autotuner
    picks: four options of surface 0 at their real path counts against the
    oracle, path for path with the kernel's near-node decisions checked and
    imposed (the book runs the single-option kernel's per-path code)."""
    surfs_w = W.book_surfaces()
    items = W.book_items()
    handles = [lv.Surface.from_workload(s, lib) for s in surfs_w]
    book = lv.Book(handles, items, lib)
    for h in handles:
        h.close()
    book.tune(100.0, 0.0, 1)
    out = book.run(100.0, 0.0, 1)
    mine = [o for o, it in enumerate(items) if it.surface == 0]
    # the longest maturity, the most paths, a put and a short call
    pick = {max(mine, key=lambda o: items[o].T), max(mine, key=lambda o: items[o].n_paths),
            next(o for o in mine if items[o].phi < 0), next(o for o in mine if items[o].phi > 0 and items[o].T <= 0.5)}
    for o in sorted(pick):
        it = items[o]
        opt = W.Option(S0=100.0, r=0.0, K=it.K, T=it.T, n_steps=it.n_steps, n_paths=it.n_paths, seed=1,
                       phi=it.phi, stream_id=it.stream_id)
        gs = G.make_surface(surfs_w[0], opt, lib)
        dec, _ = G.per_path(gs, surfs_w[0], opt)
        gs.close()
        ref = oracle.finalize(oracle.run_sums(surfs_w[0], opt, decisions=dec), opt.n_paths, opt.S0,
                              surfs_w[0].n_spot * surfs_w[0].n_time)
        p, d, _, v = book.result(out, o)
        G.compare_aggregates(p, d, v, ref, label=f"book option {o} (T={it.T}, P={it.n_paths}, phi={it.phi})")
    book.close()


def test_book_two_paths_per_lane_against_single_calls(lib):
    """The book at two paths per lane equals the single-option sums calls
    option by option, at small item sizes so that many items end with a
    single tile (the second tile of a claim then lies beyond the item and
    belongs to another block's item), at k = 4 and 8."""
    surfs, items = _book_inputs()
    handles = [lv.Surface.from_workload(s, lib) for s in surfs]
    book = lv.Book(handles, items, lib)
    for h in handles:
        h.close()
    S0, r, seed = 100.0, 0.02, 9
    for blk, k, item_paths in ((128, 4, 96), (64, 8, 2048)):
        book.set_launch(blk, k, item_paths, 2)
        assert book.paths_per_lane() == 2
        out = book.run(S0, r, seed)
        for o, it in enumerate(items):
            ref = _single(lib, surfs[it.surface], it, S0, r, seed)
            _close(out[book.offsets[o]:book.offsets[o + 1]], ref, f"option {o} ({blk}, {k}, {item_paths})")
    with pytest.raises(lv.LVError):
        book.set_launch(128, 4, 96, 3)
    book.close()
