"""The packed binary32 pairs (.f32x2) give every path the same value, bit for
bit, as the scalar code (needs a GB300).

With at most a few hundred paths, summing their binary64 payoffs in another
order moves the price by less than 1e-13 relative, while a single path whose
binary32 payoff differed by one ulp would move it by about 1e-8 / n_paths.
So the price of a packed kernel (two paths per lane) agreeing with the scalar
kernel's (one path per lane) to 1e-13 on the same paths checks each path.
Kernels compared: the forward-only kernel (always packed) and the adjoint at
two paths per lane (packed forward and paired reverse normals) against the
adjoint at one path per lane, under every reading of the scheme (the
adjoint packs under the log-Euler readings and keeps scalar pairs for Euler
on S, whose forward-only kernel packs); the tangent-ratio adjoint (main
reading) at two against one."""
import pytest

import workloads as W
from paper_2002_02481_gb300 import build, lv

from . import gpu_common as G
from .test_gpu_parity import EDGE

pytestmark = pytest.mark.gpu

TOL = 1e-13

CASES = [
    ("30x60 grid, 156 steps", W.config_paper_shape()),
    ("20x10 grid, 52 steps", W.config_small()),
    ("uneven 7x5 grid (binary search), put", EDGE[2][1:]),
    ("3x2 grid, paths leave both sides", EDGE[1][1:]),
]


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


READINGS = [(lv.LV_INTERP_S, lv.LV_SCHEME_LOG, "main reading"), (lv.LV_INTERP_LOGS, lv.LV_SCHEME_LOG, "ln-S weight"),
            (lv.LV_INTERP_S, lv.LV_SCHEME_S, "Euler on S"), (lv.LV_INTERP_LOGS, lv.LV_SCHEME_S, "both")]


@pytest.mark.parametrize("reading", READINGS, ids=[r[2] for r in READINGS])
@pytest.mark.parametrize("n_paths", [1, 33, 64, 97, 256])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_packed_pairs_match_scalar_paths(case, n_paths, reading, lib):
    interp, scheme, _ = reading
    name, (surf, opt) = case
    opt = W.Option(**{**opt.__dict__, "n_paths": n_paths})
    args = (opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    one = G.make_surface(surf, opt, lib, launch=(128, 4, 0), ppl=1)
    two = G.make_surface(surf, opt, lib, launch=(128, 4, 0), ppl=2)
    for s in (one, two):
        s.set_interpolation(interp)
        s.set_scheme(scheme)
    p1, _, _ = one.price_greeks(*args)
    p2, _, _ = two.price_greeks(*args)
    pf, _ = two.price(*args)
    got = [("adjoint, two paths per lane", p2), ("forward only", pf)]
    if reading[2] == "main reading":           # the tangent-ratio form pairs the main reading
        for s in (one, two):
            s.set_adjoint_method(lv.LV_ADJ_TANGENT)
        t1, _, _ = one.price_greeks(*args)
        t2, _, _ = two.price_greeks(*args)
        got += [("tangent ratio, one path per lane", t1), ("tangent ratio, two paths per lane", t2)]
    assert two.get_paths_per_lane(opt.n_steps, opt.n_paths) == 2
    one.close()
    two.close()
    scale = max(abs(p1), 1e-300)
    for label, p in got:
        assert abs(p - p1) <= TOL * scale, (name, n_paths, label, p, p1)
