"""The device entry points inside a CUDA graph: a call captured on a stream
after one warm-up call (so that the handle's scratch exists) replays to the
same outputs as an eager call, replay after replay. This covers the
launches the path makes: the memory clear, the adjoint kernel and the two
level-3 stages chained by programmatic dependent launch."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("ext", [False, True], ids=["price_greeks", "price_greeks_ext"])
def test_captured_call_replays_to_the_eager_result(ext, lib):
    import torch
    surf, opt = W.config_small()
    gs = G.make_surface(surf, opt, lib)
    s = torch.cuda.Stream()
    gs.set_stream(s.cuda_stream)
    n = (5 if ext else 3) + surf.n_spot * surf.n_time
    call = gs.price_greeks_ext_device if ext else gs.price_greeks_device
    eager = torch.zeros(n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        call(opt.S0, 0.01, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, eager.data_ptr())
    s.synchronize()
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call(opt.S0, 0.01, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, out.data_ptr())
    ref = eager.cpu().numpy()
    for _ in range(3):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert abs(o[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert abs(o[1] - ref[1]) <= 1e-9 * abs(ref[1])
        np.testing.assert_allclose(o[3:], ref[3:], rtol=0, atol=1e-6 * np.max(np.abs(ref[3:])))
    gs.set_stream(0)
