"""The other readings of the scheme on the GPU (needs a GB300): the spot
weight linear in ln S (LV_INTERP_LOGS), the Euler scheme on S
(LV_SCHEME_S) and both, each against the FP64 oracle under the same
reading, element by element on the same seeded inputs, with the tolerances
of the main reading; through the reverse sweep and the tangent-ratio form.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G
from .test_gpu_parity import EDGE

pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LV_PARITY_REPORT")
READINGS = [(lv.LV_INTERP_LOGS, lv.LV_SCHEME_LOG, "ln-S weight"),
            (lv.LV_INTERP_S, lv.LV_SCHEME_S, "Euler on S"),
            (lv.LV_INTERP_LOGS, lv.LV_SCHEME_S, "both")]


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


def _with(surf, opt, interp, scheme):
    return (W.Surface(surf.spot, surf.time, surf.sigma, interp=interp),
            W.Option(**{**opt.__dict__, "scheme": scheme}))


@pytest.mark.parametrize("reading", READINGS, ids=[r[2] for r in READINGS])
@pytest.mark.parametrize("case", EDGE, ids=[c[0] for c in EDGE])
def test_edge_cases(case, reading, lib):
    name, surf, opt = case
    interp, scheme, tag = reading
    s, o = _with(surf, opt, interp, scheme)
    _report(f"{tag}: {name}", G.full_parity(s, o, lib, label=f"{tag}: {name}"))


@pytest.mark.parametrize("reading", READINGS, ids=[r[2] for r in READINGS])
def test_paper_shape(reading, lib):
    interp, scheme, tag = reading
    surf, opt = W.config_paper_shape()
    opt = W.Option(**{**opt.__dict__, "n_paths": 1 << 18})
    s, o = _with(surf, opt, interp, scheme)
    _report(f"{tag}: 30x60 grid, 156 steps, 2^18 paths", G.full_parity(s, o, lib, label=tag))


@pytest.mark.parametrize("reading", READINGS, ids=[r[2] for r in READINGS])
def test_tangent_ratio_and_kahan(reading, lib):
    interp, scheme, tag = reading
    surf, opt = W.config_small()
    s, o = _with(surf, opt, interp, scheme)
    G.full_parity(s, o, lib, label=f"{tag} tangent", method=lv.LV_ADJ_TANGENT)
    G.full_parity(s, o, lib, label=f"{tag} Kahan", accumulation=1, launch=(128, 8, 0))


@pytest.mark.parametrize("reading", READINGS, ids=[r[2] for r in READINGS])
def test_two_paths_per_lane(reading, lib):
    """Two paths per lane in the forward tiles under every reading (packed
    pairs under the ln-S weight, scalar pairs for Euler on S): the oracle path for path
    at k = 4 (binary64) and k = 8 (Kahan), on the paper's grid, an uneven
    grid with a put and a ragged tile; and the same results as one path per
    lane up to reduction order."""
    interp, scheme, tag = reading
    surf, opt = W.config_paper_shape()
    opt = W.Option(**{**opt.__dict__, "n_paths": 1 << 17})
    s, o = _with(surf, opt, interp, scheme)
    for launch, acc in [((128, 4, 0), 0), ((128, 8, 0), 1)]:
        g = G.make_surface(s, o, lib, launch=launch, accumulation=acc, ppl=2)
        assert g.get_paths_per_lane(o.n_steps, o.n_paths) == 2
        g.close()
        _report(f"{tag}: two paths per lane {launch} acc={acc}",
                G.full_parity(s, o, lib, launch=launch, accumulation=acc, ppl=2, label=f"{tag} ppl2"))
    for name, es, eo in (EDGE[2], EDGE[5]):
        s2, o2 = _with(es, eo, interp, scheme)
        G.full_parity(s2, o2, lib, launch=(128, 4, 0), ppl=2, label=f"{tag} ppl2: {name}")
    a = G.make_surface(s, o, lib, launch=(128, 4, 0), ppl=1)
    b = G.make_surface(s, o, lib, launch=(128, 4, 0), ppl=2)
    args = (o.S0, o.r, o.K, o.T, o.n_steps, o.n_paths, o.seed)
    pa, da, va = a.price_greeks(*args)
    pb, db, vb = b.price_greeks(*args)
    assert abs(pb - pa) <= 1e-12 * abs(pa) and abs(db - da) <= 1e-9 * abs(da)
    assert np.max(np.abs(vb - va)) <= 1e-6 * np.max(np.abs(va))
    a.close()
    b.close()


def test_large_k_is_capped_and_the_bump_and_book_refuse(lib):
    surf, opt = W.config_small()
    s = lv.Surface.from_workload(surf, lib)
    s.set_scheme(lv.LV_SCHEME_S)
    s.set_launch(128, 32, 0)
    assert s.get_launch(opt.n_steps, True)[1] == 8
    with pytest.raises(lv.LVError):
        s.bump_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, 1024, opt.seed, 1e-4)
    with pytest.raises(lv.LVError):
        lv.Book([s], [W.BookItem(surface=0, phi=1, K=100.0, T=1.0, n_steps=10, n_paths=64, stream_id=0)], lib)
    with pytest.raises(lv.LVError):
        s.set_scheme(7)
    with pytest.raises(lv.LVError):
        s.set_interpolation(-1)
    s.close()
