"""Seeded synthetic inputs for the local-volatility Monte Carlo workloads.

This module only builds inputs: local-vol grids (spot nodes, time nodes,
sigma values) and option books. It holds none of the method's arithmetic
(no random normals, no interpolation, no Euler steps, no payoffs), so the
CPU oracle and the CUDA path can both be fed from it without sharing code.

The paper (Sec. IV-A, IV-C) uses a 30 x 60 spot x time grid whose
calibrated values come from an external book; those values are not
available, so the grids here are smooth, seeded skews of the same shape.
Every sigma array is spot-major: ``sigma[i, j]`` belongs to spot node
``i`` and time node ``j`` (flattened index ``i * n_time + j``).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np


@dataclasses.dataclass
class Surface:
    spot: np.ndarray   # [I] strictly increasing, > 0
    time: np.ndarray   # [J] strictly increasing, >= 0
    sigma: np.ndarray  # [I, J] float64, spot-major
    interp: int = 0    # spot weight linear in S (0) or in ln S (1)

    @property
    def n_spot(self) -> int:
        return int(self.spot.shape[0])

    @property
    def n_time(self) -> int:
        return int(self.time.shape[0])


@dataclasses.dataclass
class Option:
    S0: float
    r: float
    K: float
    T: float
    n_steps: int
    n_paths: int
    seed: int = 1
    phi: int = 1          # +1 call, -1 put
    stream_id: int = 0
    scheme: int = 0       # Euler on ln S (0) or on S (1)


def log_spaced(lo: float, hi: float, n: int) -> np.ndarray:
    """n nodes with equal ratios from lo to hi."""
    return lo * (hi / lo) ** (np.arange(n, dtype=np.float64) / (n - 1))


def small_skew_surface() -> Surface:
    """20 spot nodes log-spaced over 50-200, 10 time nodes uniform over 0-1y,
    sigma = 0.20 - 0.10 ln(S/100) + 0.02 t clipped to [0.05, 0.6]."""
    s = log_spaced(50.0, 200.0, 20)
    t = np.arange(10, dtype=np.float64) / 9.0
    sig = 0.20 - 0.10 * np.log(s[:, None] / 100.0) + 0.02 * t[None, :]
    return Surface(s, t, np.clip(sig, 0.05, 0.6))


def seeded_skew_surface(surface_seed: int, n_spot: int = 30, n_time: int = 60,
                        s_lo: float = 20.0, s_hi: float = 300.0,
                        t_hi: float = 3.0) -> Surface:
    """Seeded smooth skew: base ~ U[0.15, 0.30], slope ~ U[-0.15, -0.05] per
    unit ln(S/100), iid N(0, 0.005^2) noise per node, clipped to [0.05, 0.6].
    Spot nodes are log-spaced over [s_lo, s_hi], time nodes uniform on
    [0, t_hi]."""
    rng = np.random.Generator(np.random.PCG64(surface_seed))
    base = rng.uniform(0.15, 0.30)
    slope = rng.uniform(-0.15, -0.05)
    noise = rng.normal(0.0, 0.005, size=(n_spot, n_time))
    s = log_spaced(s_lo, s_hi, n_spot)
    t = np.linspace(0.0, t_hi, n_time)
    sig = base + slope * np.log(s[:, None] / 100.0) + noise
    return Surface(s, t, np.clip(sig, 0.05, 0.6))


def flat_surface(sigma: float, n_spot: int = 5, n_time: int = 3,
                 s_lo: float = 40.0, s_hi: float = 250.0,
                 t_hi: float = 5.0) -> Surface:
    """Constant sigma on a small grid (Black-Scholes special case)."""
    s = log_spaced(s_lo, s_hi, n_spot)
    t = np.linspace(0.0, t_hi, n_time) if n_time > 1 else np.zeros(1)
    return Surface(s, t, np.full((n_spot, n_time), float(sigma)))


def random_surface(seed: int, n_spot: int, n_time: int, s_lo: float = 60.0,
                   s_hi: float = 160.0, t_hi: float = 1.0,
                   uneven: bool = False) -> Surface:
    """Arbitrary positive grid for edge-case tests; ``uneven`` draws
    irregular node spacings (not log-uniform)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if uneven:
        gaps = rng.uniform(0.2, 1.8, size=n_spot - 1)
        s = s_lo + (s_hi - s_lo) * np.concatenate([[0.0], np.cumsum(gaps)]) / gaps.sum()
        if n_time > 1:
            tg = rng.uniform(0.3, 1.7, size=n_time - 1)
            t = t_hi * np.concatenate([[0.0], np.cumsum(tg)]) / tg.sum()
        else:
            t = np.zeros(1)
    else:
        s = log_spaced(s_lo, s_hi, n_spot)
        t = np.linspace(0.0, t_hi, n_time) if n_time > 1 else np.zeros(1)
    sig = rng.uniform(0.1, 0.45, size=(n_spot, n_time))
    return Surface(s, t, sig)


# ---------------------------------------------------------------- workloads

def config_small() -> tuple[Surface, Option]:
    """20x10 grid, call K=100 T=1, 52 steps, 16,384 paths, seed 1."""
    return small_skew_surface(), Option(S0=100.0, r=0.0, K=100.0, T=1.0,
                                        n_steps=52, n_paths=16384, seed=1)


def config_paper_shape() -> tuple[Surface, Option]:
    """The paper's workload shape (Sec. IV-C, IV-D): 30x60 grid (1,800
    sensitivities), 156 steps; 2^20 paths; call K=100 T=3."""
    return seeded_skew_surface(2), Option(S0=100.0, r=0.0, K=100.0, T=3.0,
                                          n_steps=156, n_paths=1 << 20, seed=1)


def config_precision(surface: str = "small") -> tuple[Surface, Option]:
    """2^24 paths, 156 steps, on the 20x10 grid (or the 30x60 one)."""
    if surface == "small":
        return small_skew_surface(), Option(S0=100.0, r=0.0, K=100.0, T=1.0,
                                            n_steps=156, n_paths=1 << 24, seed=1)
    return seeded_skew_surface(2), Option(S0=100.0, r=0.0, K=100.0, T=3.0,
                                          n_steps=156, n_paths=1 << 24, seed=1)


def config_large() -> tuple[Surface, Option]:
    """100x100 grid over 20-300 x [0, 5], call K=100 T=5, 1,260 steps,
    2^26 paths."""
    surf = seeded_skew_surface(5, n_spot=100, n_time=100, t_hi=5.0)
    return surf, Option(S0=100.0, r=0.0, K=100.0, T=5.0, n_steps=1260,
                        n_paths=1 << 26, seed=1)


@dataclasses.dataclass
class BookItem:
    surface: int
    phi: int
    K: float
    T: float
    n_steps: int
    n_paths: int
    stream_id: int


def book_surfaces(n_surf: int = 8) -> List[Surface]:
    return [seeded_skew_surface(100 + s) for s in range(n_surf)]


def book_items(n_surf: int = 8, per_surface: int = 64, seed: int = 7,
               log2_lo: float = 14.0, log2_hi: float = 20.0) -> List[BookItem]:
    """Calls/puts 50/50, K ~ U[60, 140], T uniform over {0.25, 0.5, 1, 2, 3},
    weekly steps N = round(52 T), paths floor(2^U[log2_lo, log2_hi])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mats = np.array([0.25, 0.5, 1.0, 2.0, 3.0])
    items: List[BookItem] = []
    for s in range(n_surf):
        for _ in range(per_surface):
            phi = 1 if rng.uniform() < 0.5 else -1
            K = float(rng.uniform(60.0, 140.0))
            T = float(mats[rng.integers(0, len(mats))])
            P = int(np.floor(2.0 ** rng.uniform(log2_lo, log2_hi)))
            items.append(BookItem(surface=s, phi=phi, K=K, T=T,
                                  n_steps=int(round(52 * T)), n_paths=P,
                                  stream_id=len(items)))
    return items
