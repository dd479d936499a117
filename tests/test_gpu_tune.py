"""Single-option autotuner (needs a GB300): picks a valid launch shape, keeps
the results (up to reduction order), and a new handle of the same grid size
and step count reads the shape back from the LV_TUNE_CACHE file."""
import os

import numpy as np
import pytest

import workloads as W
from paper_2002_02481_gb300 import build, lv

pytestmark = pytest.mark.gpu


def test_tune_and_cache(tmp_path, monkeypatch):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    lib = lv.load()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("LV_TUNE_CACHE", str(cache))
    surf, opt = W.config_small()
    a = lv.Surface.from_workload(surf, lib)
    args = (opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    p0, d0, v0 = a.price_greeks(*args)
    blk, k, ms = a.tune(*args)
    ppl = a.get_paths_per_lane(opt.n_steps, opt.n_paths)
    assert blk in (64, 128) and k in (4, 8, 16) and ms > 0
    assert ppl in (1, 2) and (ppl == 1 or k in (4, 8))
    assert a.get_launch(opt.n_steps, True)[:2] == (blk, k)
    p1, d1, v1 = a.price_greeks(*args)
    assert abs(p1 - p0) <= 1e-12 * abs(p0) and abs(d1 - d0) <= 1e-9 * abs(d0)
    assert np.max(np.abs(v1 - v0)) <= 1e-6 * np.max(np.abs(v0))
    assert cache.exists() and str(blk) in cache.read_text()
    b = lv.Surface.from_workload(surf, lib)          # fresh handle: shape from the cache
    assert b.get_launch(opt.n_steps, True)[:2] == (blk, k)
    assert b.get_paths_per_lane(opt.n_steps, opt.n_paths) == ppl
    a.close()
    b.close()
