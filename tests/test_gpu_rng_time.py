"""The integer work of the CUDA path against the oracle, exactly (needs a
GB300): the Philox4x32-10 words the kernels draw for a counter (Sec. IV-B,
read as Philox; the oracle's generator is pinned against cuRAND), and the
per-step time table (time cell and weight of sigma's left point t_n,
Sec. IV-A and IV-D). Also the binary32 normals derived from those words,
against the oracle's binary64 normals, within the bound the hardware
approximations allow."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2002_02481_gb300 import build, lv

pytestmark = pytest.mark.gpu

REPORT = os.environ.get("LV_PARITY_REPORT")


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return lv.load()


SEEDS = [0, 1, 0x9E3779B97F4A7C15, 0xFFFFFFFFFFFFFFFF]
STREAMS = [0, 1, 4097, 65535]


def _counters(rng, n):
    paths = np.concatenate([[0, 1, 31, 32, (1 << 32) - 1, 1 << 32, (1 << 32) + 5, (1 << 48) - 1],
                            rng.integers(0, 1 << 48, size=n - 8, dtype=np.int64)])
    blocks = np.concatenate([[0, 1, 38, 39, 314, 2047, 0, 1], rng.integers(0, 2048, size=n - 8)]).astype(np.uint32)
    return paths.astype(np.int64), blocks


@pytest.mark.parametrize("seed", SEEDS, ids=[hex(s) for s in SEEDS])
def test_philox_words_bit_exact(seed, lib):
    rng = np.random.Generator(np.random.PCG64(seed & 0xFFFF))
    for stream in STREAMS:
        paths, blocks = _counters(rng, 256)
        w, _ = lv.debug_normals(seed, stream, paths, blocks, lib)
        for e in range(paths.shape[0]):
            p = int(paths[e])
            ctr = [int(blocks[e]), p & 0xFFFFFFFF, ((p >> 32) & 0xFFFF) | (stream << 16), 0]
            ref = oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
            assert np.array_equal(w[e], ref), (hex(seed), stream, p, int(blocks[e]))


def test_normals_within_the_approximation_bound(lib):
    """Z = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b) in binary32 with the hardware's
    lg2 / sqrt / sin / cos approximations against binary64 libm on the same
    uniforms: |dZ| <= 2^-18 (1 + |Z|) + dr, where dr bounds the radius error
    2 ln 2 * 2^-21 / (rho_gpu + rho_oracle) that an absolute error of lg2
    near u_a = 1 (rho near 0) produces."""
    rng = np.random.Generator(np.random.PCG64(5))
    seed, stream = 1, 0
    paths, blocks = _counters(rng, 1 << 16)
    _, z = lv.debug_normals(seed, stream, paths, blocks, lib)
    worst = 0.0
    ref = np.zeros((paths.shape[0], 4))
    for e in range(paths.shape[0]):
        zz = oracle.normals(seed, int(paths[e]), 4 * (int(blocks[e]) + 1), stream)
        ref[e] = zz[4 * int(blocks[e]):]
    z = z.astype(np.float64)
    for a in (0, 2):
        rho_o = np.hypot(ref[:, a], ref[:, a + 1])
        rho_g = np.hypot(z[:, a], z[:, a + 1])
        dr = 2 * np.log(2) * 2.0 ** -21 / np.maximum(rho_o + rho_g, 1e-30)
        for q in (a, a + 1):
            err = np.abs(z[:, q] - ref[:, q])
            bound = 2.0 ** -18 * (1 + np.abs(ref[:, q])) + dr
            worst = max(worst, float(np.max(err / bound)))
            assert np.all(err <= bound), float(np.max(err / bound))
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": "normals vs oracle", "n": int(4 * paths.shape[0]),
                                "err_of_bound_max": worst}) + "\n")


def _time_table_case(surf, T, N, lib):
    h = lv.Surface.from_workload(surf, lib)
    j, v = h.time_table(T, N)
    h.close()
    dt = T / N
    J = surf.n_time
    for n in range(N):
        t = n * dt
        if J == 1:
            jr, vr = 0, 0.0
        else:
            pt = oracle.sigma_eval(surf, float(surf.spot[0]), t)   # the time cell does not depend on S
            jr, vr = pt["j"], pt["v"]
        assert j[n] == jr, (n, int(j[n]), jr)
        assert np.float32(vr) == v[n], (n, float(v[n]), vr)         # the same binary64 value, rounded once


@pytest.mark.parametrize("which", ["small", "paper", "large", "past the last node", "uneven", "one time node"])
def test_time_table_exact(which, lib):
    if which == "small":
        surf, opt = W.config_small()
        _time_table_case(surf, opt.T, opt.n_steps, lib)
    elif which == "paper":
        surf, opt = W.config_paper_shape()
        _time_table_case(surf, opt.T, opt.n_steps, lib)
    elif which == "large":
        surf, opt = W.config_large()
        _time_table_case(surf, opt.T, opt.n_steps, lib)
    elif which == "past the last node":
        _time_table_case(W.small_skew_surface(), 2.5, 130, lib)
    elif which == "uneven":
        _time_table_case(W.random_surface(3, 7, 5, s_lo=75, s_hi=130, t_hi=1.0, uneven=True), 0.8, 10, lib)
    else:
        _time_table_case(W.random_surface(1, 2, 1, s_lo=80, s_hi=125), 1.0, 13, lib)
