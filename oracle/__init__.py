"""FP64 CPU oracle for the local-volatility Monte Carlo price and its
pathwise adjoint -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package. The CUDA library never imports it and shares
no code with it. The arithmetic lives in ``lv_oracle.c`` (plain C, binary64,
libm); this module compiles it with gcc and marshals numpy arrays.

Every function cites the passage of arXiv 2002.02481 it follows in
``lv_oracle.c``. Readings where the paper is silent are listed there too.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lv_oracle.c")
_HDR = os.path.join(_HERE, "lv_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liblv_oracle.so")

NSCAL = 13
VN_DELTA, VN_DELTA_2, VN_TOT, VN_TOT_2, VN_TINY, VN_NSCAL = 0, 1, 2, 3, 4, 5
(SUM_V, SUM_V2, SUM_XBAR0, SUM_XBAR0_2, SUM_VTOT, SUM_VTOT_2, SUM_SN, KINK_COUNT, KINK_XBAR0,
 SUM_RHO, SUM_RHO_2, SUM_DVDT, SUM_DVDT_2) = range(13)

_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


INTERP_S, INTERP_LOGS = 0, 1      # spot weight linear in S / in ln S
SCHEME_LOG, SCHEME_X = 0, 1       # Euler on ln X / on X


class _Surface(ctypes.Structure):
    _fields_ = [("n_spot", ctypes.c_int32), ("n_time", ctypes.c_int32),
                ("spot", ctypes.POINTER(ctypes.c_double)),
                ("time", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.POINTER(ctypes.c_double)),
                ("interp", ctypes.c_int32)]


class _Option(ctypes.Structure):
    _fields_ = [("S0", ctypes.c_double), ("r", ctypes.c_double), ("K", ctypes.c_double),
                ("T", ctypes.c_double), ("n_steps", ctypes.c_int32), ("phi", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32), ("scheme", ctypes.c_int32)]


class _Decisions(ctypes.Structure):
    _fields_ = [("itm_path", ctypes.POINTER(ctypes.c_int64)), ("itm_val", ctypes.POINTER(ctypes.c_int8)),
                ("n_itm", ctypes.c_int64),
                ("cell_path", ctypes.POINTER(ctypes.c_int64)), ("cell_step", ctypes.POINTER(ctypes.c_int32)),
                ("cell_code", ctypes.POINTER(ctypes.c_int32)), ("n_cell", ctypes.c_int64),
                ("band", ctypes.c_double), ("out_overrides", ctypes.POINTER(ctypes.c_int64))]


class DecisionRefused(RuntimeError):
    """An imposed decision that rounding of the path could not have produced
    (status ORC_EDECISION of lv_oracle.c)."""


class Decisions:
    """Decisions taken from another implementation (see lv_oracle.c):
    ``itm`` maps path -> payoff indicator; ``cells`` is (paths, steps,
    codes) with code = 2 * spot_cell + inside_grid. A decision that differs
    from the oracle's own is applied only when the oracle's own value lies
    within ``band`` (relative) of the strike, of the node between the two
    cells, or of the grid's edge node; otherwise the call raises
    DecisionRefused. After a call, ``overrides`` holds how many cell and
    payoff decisions differed from the oracle's own and were applied."""

    def __init__(self, itm: Optional[dict] = None, cells=None, band: float = 0.0):
        keys = sorted((itm or {}).keys())
        self.itm_path = np.array(keys, dtype=np.int64)
        self.itm_val = np.array([1 if itm[k] else 0 for k in keys], dtype=np.int8)
        if cells is None:
            cells = (np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
        cp, cs, cc = (np.asarray(a) for a in cells)
        order = np.lexsort((cs, cp))
        self.cell_path = np.ascontiguousarray(cp[order], dtype=np.int64)
        self.cell_step = np.ascontiguousarray(cs[order], dtype=np.int32)
        self.cell_code = np.ascontiguousarray(cc[order], dtype=np.int32)
        self.band = float(band)
        self._ov = np.zeros(2, dtype=np.int64)
        P = ctypes.POINTER
        self.c = _Decisions(self.itm_path.ctypes.data_as(P(ctypes.c_int64)),
                            self.itm_val.ctypes.data_as(P(ctypes.c_int8)), len(keys),
                            self.cell_path.ctypes.data_as(P(ctypes.c_int64)),
                            self.cell_step.ctypes.data_as(P(ctypes.c_int32)),
                            self.cell_code.ctypes.data_as(P(ctypes.c_int32)), len(self.cell_path),
                            self.band, self._ov.ctypes.data_as(P(ctypes.c_int64)))

    @property
    def overrides(self) -> dict:
        return {"cell": int(self._ov[0]), "payoff": int(self._ov[1])}


class _Point(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("j", ctypes.c_int32), ("u", ctypes.c_double),
                ("v", ctypes.c_double), ("w", ctypes.c_double * 4),
                ("sigma", ctypes.c_double), ("dsigma_dS", ctypes.c_double), ("dsigma_dt", ctypes.c_double),
                ("inside", ctypes.c_int32), ("du_dS", ctypes.c_double)]


def build(src: str = _SRC, out: str = _LIB, extra: tuple = ()) -> str:
    """Compile the oracle (plain C11, no fast-math, no FMA contraction, so
    x86-64 and aarch64 hosts evaluate the same expressions)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-I", _HERE, *extra, src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _stale() -> bool:
    if not os.path.exists(_LIB):
        return True
    t = os.path.getmtime(_LIB)
    return t < os.path.getmtime(_SRC) or t < os.path.getmtime(_HDR)


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load (building first if needed) the oracle library, or a variant at
    ``path`` (used by the planted-mistake tests)."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if _stale():
                build()
            _lib = _declare(ctypes.CDLL(_LIB))
    return _lib


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    P = ctypes.POINTER
    u32p, f64p = P(ctypes.c_uint32), P(ctypes.c_double)
    lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.orc_philox4x32_10.restype = None
    lib.orc_uniform.argtypes = [ctypes.c_uint32]
    lib.orc_uniform.restype = ctypes.c_double
    lib.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, f64p]
    lib.orc_normals.restype = None
    lib.orc_sigma_eval.argtypes = [P(_Surface), ctypes.c_double, ctypes.c_double, P(_Point)]
    lib.orc_sigma_eval.restype = None
    lib.orc_run.argtypes = [P(_Surface), P(_Option), ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                            ctypes.c_double, ctypes.c_int32, f64p]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_run_ex.argtypes = [P(_Surface), P(_Option), ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_double, P(_Decisions), ctypes.c_int32, f64p]
    lib.orc_run_ex.restype = ctypes.c_int
    lib.orc_finalize.argtypes = [f64p, ctypes.c_int64, ctypes.c_double, ctypes.c_int64, f64p]
    lib.orc_finalize.restype = ctypes.c_int
    lib.orc_paths.argtypes = [P(_Surface), P(_Option), ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                              f64p, f64p, f64p]
    lib.orc_paths.restype = ctypes.c_int
    lib.orc_paths_ex.argtypes = [P(_Surface), P(_Option), ctypes.c_int64, ctypes.c_int64, P(_Decisions),
                                 ctypes.c_int32, f64p, f64p, f64p, f64p]
    lib.orc_paths_ex.restype = ctypes.c_int
    lib.orc_bump.argtypes = [P(_Surface), P(_Option), ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int32, f64p, f64p]
    lib.orc_bump.restype = ctypes.c_int
    lib.orc_run_vanna.argtypes = [P(_Surface), P(_Option), ctypes.c_int64, ctypes.c_int64, P(_Decisions),
                                  ctypes.c_int32, f64p]
    lib.orc_run_vanna.restype = ctypes.c_int
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Args:
    """Keeps the numpy buffers alive while C sees their pointers."""

    def __init__(self, spot, time, sigma, S0, r, K, T, n_steps, seed, phi=1, stream_id=0, interp=0, scheme=0):
        self.spot, self.time = _f64(spot), _f64(time)
        self.sigma = _f64(sigma).reshape(-1)
        I, J = self.spot.shape[0], self.time.shape[0]
        if self.sigma.shape[0] != I * J:
            raise ValueError("sigma must hold n_spot * n_time values")
        self.IJ = I * J
        self.surf = _Surface(I, J, _ptr(self.spot), _ptr(self.time), _ptr(self.sigma), int(interp))
        self.opt = _Option(float(S0), float(r), float(K), float(T), int(n_steps), int(phi),
                           int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream_id), int(scheme))


def _args(surface, opt) -> _Args:
    """C views of a workloads.Surface and workloads.Option (their interp and
    scheme fields select the reading; both default to the main one)."""
    return _Args(surface.spot, surface.time, surface.sigma, opt.S0, opt.r, opt.K, opt.T, opt.n_steps,
                 opt.seed, opt.phi, opt.stream_id, getattr(surface, "interp", 0), getattr(opt, "scheme", 0))


ORC_EDECISION = 5


def _check(st: int, what: str) -> None:
    if st == ORC_EDECISION:
        raise DecisionRefused(f"oracle {what}: an imposed decision lies outside its band")
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def philox4x32_10(ctr, key, lib=None) -> np.ndarray:
    lib = lib or load_library()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(w: int, lib=None) -> float:
    return float((lib or load_library()).orc_uniform(int(w) & 0xFFFFFFFF))


def normals(seed: int, path: int, n_steps: int, stream_id: int = 0, lib=None) -> np.ndarray:
    """Z_0 .. Z_{N-1} of one path."""
    lib = lib or load_library()
    z = np.zeros(n_steps, dtype=np.float64)
    lib.orc_normals(int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream_id), int(path), int(n_steps), _ptr(z))
    return z


def sigma_eval(surface, S: float, t: float, lib=None) -> dict:
    """Bilinear sigma, d sigma / d S, cell and node weights at (S, t)."""
    lib = lib or load_library()
    a = _Args(surface.spot, surface.time, surface.sigma, 1.0, 0.0, 1.0, 1.0, 1, 0,
              interp=getattr(surface, "interp", 0))
    p = _Point()
    lib.orc_sigma_eval(ctypes.byref(a.surf), float(S), float(t), ctypes.byref(p))
    return dict(i=p.i, j=p.j, u=p.u, v=p.v, w=list(p.w), sigma=p.sigma, dsigma_dS=p.dsigma_dS,
                dsigma_dt=p.dsigma_dt, inside=bool(p.inside), du_dS=p.du_dS)


def run_sums(surface, opt, path_begin: int = 0, path_end: Optional[int] = None,
             greeks: bool = True, kink_tol: float = 0.0, n_threads: Optional[int] = None,
             lib=None, decisions: Optional[Decisions] = None) -> np.ndarray:
    """Raw sums over paths [path_begin, path_end): NSCAL scalars, vega[IJ],
    kink_vega[IJ] (see lv_oracle.h for the layout). ``decisions`` imposes
    payoff-indicator and spot-cell decisions on listed paths / steps."""
    lib = lib or load_library()
    a = _args(surface, opt)
    if path_end is None:
        path_end = opt.n_paths
    out = np.zeros(NSCAL + 2 * a.IJ, dtype=np.float64)
    st = lib.orc_run_ex(ctypes.byref(a.surf), ctypes.byref(a.opt), int(path_begin), int(path_end),
                        int(bool(greeks)), float(kink_tol),
                        ctypes.byref(decisions.c) if decisions is not None else None,
                        int(n_threads or default_threads()), _ptr(out))
    _check(st, "run")
    return out


def finalize(sums: np.ndarray, n_paths: int, S0: float, IJ: int, lib=None) -> np.ndarray:
    """[price, delta, stderr, vega_0 .. vega_{IJ-1}]."""
    lib = lib or load_library()
    s = _f64(sums)
    res = np.zeros(3 + IJ, dtype=np.float64)
    _check(lib.orc_finalize(_ptr(s), int(n_paths), float(S0), int(IJ), _ptr(res)), "finalize")
    return res


def price_greeks(surface, opt, n_threads: Optional[int] = None, lib=None) -> dict:
    """Price, its standard error, delta and the vega grid [I, J]."""
    s = run_sums(surface, opt, 0, opt.n_paths, True, 0.0, n_threads, lib)
    IJ = surface.n_spot * surface.n_time
    res = finalize(s, opt.n_paths, opt.S0, IJ, lib)
    return dict(price=res[0], delta=res[1], stderr=res[2],
                vega=res[3:].reshape(surface.n_spot, surface.n_time), sums=s,
                rho=s[SUM_RHO] / opt.n_paths, dVdT=s[SUM_DVDT] / opt.n_paths)


def paths(surface, opt, path_begin: int, m: int, n_threads: Optional[int] = None, lib=None,
          decisions: Optional[Decisions] = None, amp: bool = False):
    """Per-path x_N, discounted payoff and d V / d x_0 for m paths (and, with
    ``amp``, each path's bound on d ln |xbar_0| / d e for a relative error e
    in every spot of the path)."""
    lib = lib or load_library()
    a = _args(surface, opt)
    xN, V, xb, am = (np.zeros(m) for _ in range(4))
    _check(lib.orc_paths_ex(ctypes.byref(a.surf), ctypes.byref(a.opt), int(path_begin), int(m),
                            ctypes.byref(decisions.c) if decisions is not None else None,
                            int(n_threads or default_threads()), _ptr(xN), _ptr(V), _ptr(xb),
                            _ptr(am) if amp else None), "paths")
    return (xN, V, xb, am) if amp else (xN, V, xb)


def bump(surface, opt, eps_sigma: float, eps_S0: float, n_paths: Optional[int] = None,
         n_threads: Optional[int] = None, lib=None):
    """Central bump-and-reprice with common random numbers (Sec. III):
    (vega grid [I, J], delta)."""
    lib = lib or load_library()
    a = _args(surface, opt)
    vega = np.zeros(a.IJ)
    delta = ctypes.c_double(0.0)
    _check(lib.orc_bump(ctypes.byref(a.surf), ctypes.byref(a.opt), int(n_paths or opt.n_paths),
                        float(eps_sigma), float(eps_S0), int(n_threads or default_threads()),
                        _ptr(vega), ctypes.byref(delta)), "bump")
    return vega.reshape(surface.n_spot, surface.n_time), delta.value


def run_vanna(surface, opt, path_begin: int = 0, path_end: Optional[int] = None,
              n_threads: Optional[int] = None, lib=None, decisions: Optional[Decisions] = None) -> dict:
    """Second-order buckets d^2 price / (d S0 d sigma_ij) over paths
    [path_begin, path_end) (lv_oracle.c, orc_run_vanna): dict with the raw
    sums and the estimates: 'delta', 'vanna' [I, J], 'vanna_se' [I, J],
    'total' (sum over buckets) and 'total_se'."""
    lib = lib or load_library()
    a = _args(surface, opt)
    if path_end is None:
        path_end = opt.n_paths
    out = np.zeros(VN_NSCAL + 2 * a.IJ, dtype=np.float64)
    st = lib.orc_run_vanna(ctypes.byref(a.surf), ctypes.byref(a.opt), int(path_begin), int(path_end),
                           ctypes.byref(decisions.c) if decisions is not None else None,
                           int(n_threads or default_threads()), _ptr(out))
    _check(st, "run_vanna")
    P = max(int(path_end - path_begin), 1)
    I, J = surface.n_spot, surface.n_time
    vs = out[VN_NSCAL:VN_NSCAL + a.IJ]
    vq = out[VN_NSCAL + a.IJ:]
    mean = vs / P
    se = np.sqrt(np.maximum(vq / P - mean * mean, 0.0) / max(P - 1, 1))
    tot = out[VN_TOT] / P
    tot_se = np.sqrt(max(out[VN_TOT_2] / P - tot * tot, 0.0) / max(P - 1, 1))
    return dict(sums=out, delta=out[VN_DELTA] / P, vanna=mean.reshape(I, J), vanna_se=se.reshape(I, J),
                total=tot, total_se=tot_se, tiny=int(out[VN_TINY]))
