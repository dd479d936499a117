"""Thin ctypes binding of the C ABI in include/lv.h (argument marshalling
only: every step of the Monte Carlo path and its adjoint runs in the CUDA
library). The functions keep the C names.

The library is loaded from the package's _lib/ directory; when it is missing
this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblv_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lv.h")

LV_OK, LV_EINVAL, LV_ENOMEM, LV_ECUDA, LV_EINTERNAL, LV_ENUMERIC = range(6)
LV_ACC_FP64, LV_ACC_KAHAN = 0, 1
LV_ADJ_REVERSE, LV_ADJ_TANGENT = 0, 1
LV_INTERP_S, LV_INTERP_LOGS = 0, 1
LV_SCHEME_LOG, LV_SCHEME_S = 0, 1
LV_OUT_PRICE, LV_OUT_DELTA, LV_OUT_STDERR, LV_OUT_VEGA = 0, 1, 2, 3
LV_SUM_V, LV_SUM_V2, LV_SUM_XBAR0, LV_SUM_VEGA = 0, 1, 2, 3

_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


class LVError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what} failed (status {status}): {msg}")
        self.status = status


def exported_names() -> list[str]:
    """Every function name declared in include/lv.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:lv_status|void|const char\*)\s+(lv_\w+)\s*\(", text, re.M)))


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the compiled library (no build, no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"CUDA library not built: {p} is missing "
                              "(run __graft_entry__.build() or python -m paper_2002_02481_gb300.build)")
        lib = _declare(ctypes.CDLL(p))
        if path is None:
            _lib = lib
        return lib


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    c = ctypes
    vp, d, i32, i64, u64, u32 = c.c_void_p, c.c_double, c.c_int32, c.c_int64, c.c_uint64, c.c_uint32
    dp, fp = c.POINTER(c.c_double), c.POINTER(c.c_float)
    sig = {
        "lv_surface_create": [dp, i32, dp, i32, dp, c.POINTER(vp)],
        "lv_surface_destroy": [vp],
        "lv_surface_set_sigma": [vp, dp],
        "lv_set_option_type": [vp, i32],
        "lv_set_stream": [vp, vp],
        "lv_set_accumulation": [vp, i32],
        "lv_set_adjoint_method": [vp, i32],
        "lv_surface_set_interpolation": [vp, i32],
        "lv_set_scheme": [vp, i32],
        "lv_set_launch": [vp, i32, i32, i32],
        "lv_set_kernel_events": [vp, vp, vp],
        "lv_set_paths_per_lane": [vp, i32],
        "lv_get_paths_per_lane": [vp, i32, i64, c.POINTER(i32)],
        "lv_tune": [vp, d, d, d, d, i32, i64, u64, c.POINTER(i32), c.POINTER(i32), c.POINTER(d)],
        "lv_get_launch": [vp, i32, i32, c.POINTER(i32), c.POINTER(i32), c.POINTER(i32)],
        "lv_price": [vp, d, d, d, d, i32, i64, u64, dp, dp],
        "lv_price_greeks": [vp, d, d, d, d, i32, i64, u64, dp, dp, dp],
        "lv_price_greeks_device": [vp, d, d, d, d, i32, i64, u64, vp],
        "lv_price_greeks_ext": [vp, d, d, d, d, i32, i64, u64, dp, dp, dp, dp, dp],
        "lv_price_greeks_ext_device": [vp, d, d, d, d, i32, i64, u64, vp],
        "lv_price_greeks_sums_device": [vp, d, d, d, d, i32, i64, i64, u64, u32, vp],
        "lv_finalize_sums_device": [vp, vp, i64, d, vp],
        "lv_debug_paths": [vp, d, d, d, d, i32, u64, u32, i64, i64, fp, fp, fp, d, i64,
                           c.POINTER(i32), c.POINTER(i64)],
        "lv_debug_normals": [u64, u32, c.POINTER(i64), c.POINTER(u32), i64, c.POINTER(u32), fp],
        "lv_debug_time_table": [vp, d, i32, c.POINTER(i32), fp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None if name == "lv_surface_destroy" else c.c_int
    lib.lv_last_error.argtypes = []
    lib.lv_last_error.restype = c.c_char_p
    for name, args in _optional_sigs(c).items():
        if hasattr(lib, name):
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = c.c_int
    return lib


def _optional_sigs(c):
    vp, d, i32, i64, u64 = c.c_void_p, c.c_double, c.c_int32, c.c_int64, c.c_uint64
    dp = c.POINTER(c.c_double)
    return {
        "lv_bump_greeks": [vp, d, d, d, d, i32, i64, u64, d, dp, dp, dp],
        "lv_bump_greeks_fp64": [vp, d, d, d, d, i32, i64, u64, d, dp, dp, dp],
        "lv_price_greeks_fp64_device": [vp, d, d, d, d, i32, i64, u64, vp],
        "lv_measure_pipe_peaks": [dp],
        "lv_price_greeks_vanna": [vp, d, d, d, d, i32, i64, u64, dp, dp, dp],
        "lv_price_greeks_vanna_device": [vp, d, d, d, d, i32, i64, u64, vp],
    }


def _check(lib, st: int, what: str) -> None:
    if st != LV_OK:
        raise LVError(st, what, lib.lv_last_error().decode(errors="replace"))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Surface:
    """A local-vol grid staged on the current CUDA device (lv_surface_t).

    The object mirrors the settings it last passed to the handle (sigma,
    option type, accumulation, adjoint method, interpolation, scheme) in
    attributes of the same names, so that a caller can restore them."""

    def __init__(self, spot, time, sigma, lib: Optional[ctypes.CDLL] = None):
        self.lib = lib or load()
        self.spot = np.ascontiguousarray(spot, dtype=np.float64)
        self.time = np.ascontiguousarray(time, dtype=np.float64)
        s = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1)
        self.n_spot, self.n_time = self.spot.shape[0], self.time.shape[0]
        # the handle's settings as last set through this object (read by autograd)
        self.sigma = s.copy()
        self.phi, self.accumulation, self.method = 1, LV_ACC_FP64, LV_ADJ_REVERSE
        self.interp, self.scheme = LV_INTERP_S, LV_SCHEME_LOG
        self.h = ctypes.c_void_p()
        _check(self.lib, self.lib.lv_surface_create(_dp(self.spot), self.n_spot, _dp(self.time), self.n_time,
                                                    _dp(s), ctypes.byref(self.h)), "lv_surface_create")

    @classmethod
    def from_workload(cls, surf, lib=None) -> "Surface":
        return cls(surf.spot, surf.time, surf.sigma, lib)

    @property
    def IJ(self) -> int:
        return self.n_spot * self.n_time

    def close(self) -> None:
        if self.h:
            self.lib.lv_surface_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # settings
    def set_sigma(self, sigma) -> None:
        s = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1)
        _check(self.lib, self.lib.lv_surface_set_sigma(self.h, _dp(s)), "lv_surface_set_sigma")
        self.sigma = s.copy()

    def set_option_type(self, phi: int) -> None:
        _check(self.lib, self.lib.lv_set_option_type(self.h, int(phi)), "lv_set_option_type")
        self.phi = int(phi)

    def set_stream(self, stream_ptr: int) -> None:
        _check(self.lib, self.lib.lv_set_stream(self.h, ctypes.c_void_p(stream_ptr or None)), "lv_set_stream")

    def state(self) -> dict:
        """The settings mirrored by this object (see the class docstring)."""
        return dict(sigma=self.sigma.copy(), phi=self.phi, accumulation=self.accumulation, method=self.method,
                    interp=self.interp, scheme=self.scheme)

    def restore(self, st: dict) -> None:
        """Passes the settings of state() back to the handle."""
        self.set_sigma(st["sigma"])
        self.set_option_type(st["phi"])
        self.set_accumulation(st["accumulation"])
        self.set_adjoint_method(st["method"])
        self.set_interpolation(st["interp"])
        self.set_scheme(st["scheme"])

    def set_accumulation(self, mode: int) -> None:
        _check(self.lib, self.lib.lv_set_accumulation(self.h, int(mode)), "lv_set_accumulation")
        self.accumulation = int(mode)

    def set_adjoint_method(self, method: int) -> None:
        """LV_ADJ_REVERSE (checkpointed reverse sweep) or LV_ADJ_TANGENT (tangent ratio)."""
        _check(self.lib, self.lib.lv_set_adjoint_method(self.h, int(method)), "lv_set_adjoint_method")
        self.method = int(method)

    def set_interpolation(self, interp: int) -> None:
        """LV_INTERP_S (spot weight linear in S) or LV_INTERP_LOGS (in ln S)."""
        _check(self.lib, self.lib.lv_surface_set_interpolation(self.h, int(interp)), "lv_surface_set_interpolation")
        self.interp = int(interp)

    def set_scheme(self, scheme: int) -> None:
        """LV_SCHEME_LOG (Euler on ln S) or LV_SCHEME_S (Euler on S)."""
        _check(self.lib, self.lib.lv_set_scheme(self.h, int(scheme)), "lv_set_scheme")
        self.scheme = int(scheme)

    def set_launch(self, block: int = 0, k: int = 0, blocks_per_sm: int = 0) -> None:
        _check(self.lib, self.lib.lv_set_launch(self.h, int(block), int(k), int(blocks_per_sm)), "lv_set_launch")

    def set_paths_per_lane(self, ppl: int) -> None:
        """1 or 2 paths per lane in the adjoint's forward tiles (0: tuned / default)."""
        _check(self.lib, self.lib.lv_set_paths_per_lane(self.h, int(ppl)), "lv_set_paths_per_lane")

    def get_paths_per_lane(self, n_steps: int, n_paths: int) -> int:
        p = ctypes.c_int32()
        _check(self.lib, self.lib.lv_get_paths_per_lane(self.h, int(n_steps), int(n_paths), ctypes.byref(p)),
               "lv_get_paths_per_lane")
        return p.value

    def set_kernel_events(self, start_ptr: int, end_ptr: int) -> None:
        _check(self.lib, self.lib.lv_set_kernel_events(self.h, ctypes.c_void_p(start_ptr or None),
                                                       ctypes.c_void_p(end_ptr or None)), "lv_set_kernel_events")

    def tune(self, S0, r, K, T, n_steps, n_paths, seed):
        b, k, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(self.lib, self.lib.lv_tune(self.h, S0, r, K, T, int(n_steps), int(n_paths), int(seed),
                                          ctypes.byref(b), ctypes.byref(k), ctypes.byref(ms)), "lv_tune")
        return b.value, k.value, ms.value

    def get_launch(self, n_steps: int, greeks: bool = True):
        b, k, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib, self.lib.lv_get_launch(self.h, int(n_steps), int(greeks), ctypes.byref(b),
                                                ctypes.byref(k), ctypes.byref(s)), "lv_get_launch")
        return b.value, k.value, s.value

    # pricing
    def price(self, S0, r, K, T, n_steps, n_paths, seed):
        p, e = ctypes.c_double(), ctypes.c_double()
        _check(self.lib, self.lib.lv_price(self.h, S0, r, K, T, int(n_steps), int(n_paths), int(seed),
                                           ctypes.byref(p), ctypes.byref(e)), "lv_price")
        return p.value, e.value

    def price_greeks(self, S0, r, K, T, n_steps, n_paths, seed):
        p, d = ctypes.c_double(), ctypes.c_double()
        vega = np.zeros(self.IJ, dtype=np.float64)
        _check(self.lib, self.lib.lv_price_greeks(self.h, S0, r, K, T, int(n_steps), int(n_paths), int(seed),
                                                  ctypes.byref(p), ctypes.byref(d), _dp(vega)), "lv_price_greeks")
        return p.value, d.value, vega.reshape(self.n_spot, self.n_time)

    def price_greeks_ext(self, S0, r, K, T, n_steps, n_paths, seed):
        """(price, delta, vega [I, J], rho, d price / d T)."""
        p, d, rho, dvdt = (ctypes.c_double() for _ in range(4))
        vega = np.zeros(self.IJ, dtype=np.float64)
        _check(self.lib, self.lib.lv_price_greeks_ext(self.h, S0, r, K, T, int(n_steps), int(n_paths), int(seed),
                                                      ctypes.byref(p), ctypes.byref(d), _dp(vega),
                                                      ctypes.byref(rho), ctypes.byref(dvdt)), "lv_price_greeks_ext")
        return p.value, d.value, vega.reshape(self.n_spot, self.n_time), rho.value, dvdt.value

    def price_greeks_ext_device(self, S0, r, K, T, n_steps, n_paths, seed, d_out_ptr: int) -> None:
        _check(self.lib, self.lib.lv_price_greeks_ext_device(self.h, S0, r, K, T, int(n_steps), int(n_paths),
                                                             int(seed), ctypes.c_void_p(d_out_ptr)),
               "lv_price_greeks_ext_device")

    def price_greeks_device(self, S0, r, K, T, n_steps, n_paths, seed, d_out_ptr: int) -> None:
        _check(self.lib, self.lib.lv_price_greeks_device(self.h, S0, r, K, T, int(n_steps), int(n_paths),
                                                         int(seed), ctypes.c_void_p(d_out_ptr)),
               "lv_price_greeks_device")

    def price_greeks_sums_device(self, S0, r, K, T, n_steps, path_begin, path_end, seed, stream_id,
                                 d_sums_ptr: int) -> None:
        _check(self.lib, self.lib.lv_price_greeks_sums_device(
            self.h, S0, r, K, T, int(n_steps), int(path_begin), int(path_end), int(seed), int(stream_id),
            ctypes.c_void_p(d_sums_ptr)), "lv_price_greeks_sums_device")

    def finalize_sums_device(self, d_sums_ptr: int, n_paths: int, S0: float, d_out_ptr: int) -> None:
        _check(self.lib, self.lib.lv_finalize_sums_device(self.h, ctypes.c_void_p(d_sums_ptr), int(n_paths),
                                                          float(S0), ctypes.c_void_p(d_out_ptr)),
               "lv_finalize_sums_device")

    def debug_paths(self, S0, r, K, T, n_steps, seed, path_begin, m, node_band=0.0, ev_cap=0, stream_id=0):
        """(x_N, V, xbar0) per path, plus the near-node decision log
        (paths, steps, codes) when ev_cap > 0."""
        xN, V, xb = (np.zeros(m, dtype=np.float32) for _ in range(3))
        ev = np.zeros((max(ev_cap, 1), 3), dtype=np.int32)
        n_ev = ctypes.c_int64(0)
        _check(self.lib, self.lib.lv_debug_paths(
            self.h, S0, r, K, T, int(n_steps), int(seed), int(stream_id), int(path_begin), int(m), _fp(xN), _fp(V),
            _fp(xb),
            float(node_band), int(ev_cap), ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            ctypes.byref(n_ev)), "lv_debug_paths")
        if ev_cap <= 0:
            return xN, V, xb
        if n_ev.value > ev_cap:
            raise LVError(LV_EINTERNAL, "lv_debug_paths", f"decision log holds {ev_cap} < {n_ev.value} entries")
        e = ev[:n_ev.value]
        return xN, V, xb, (e[:, 0].astype(np.int64) + int(path_begin), e[:, 1].copy(), e[:, 2].copy())

    def price_greeks_vanna(self, S0, r, K, T, n_steps, n_paths, seed):
        """(price, delta, d^2 price / (d S0 d sigma) [I, J]) (lv_price_greeks_vanna)."""
        p, d = ctypes.c_double(), ctypes.c_double()
        vn = np.zeros(self.IJ, dtype=np.float64)
        _check(self.lib, self.lib.lv_price_greeks_vanna(self.h, S0, r, K, T, int(n_steps), int(n_paths), int(seed),
                                                        ctypes.byref(p), ctypes.byref(d), _dp(vn)),
               "lv_price_greeks_vanna")
        return p.value, d.value, vn.reshape(self.n_spot, self.n_time)

    def price_greeks_vanna_device(self, S0, r, K, T, n_steps, n_paths, seed, d_out_ptr: int) -> None:
        _check(self.lib, self.lib.lv_price_greeks_vanna_device(self.h, S0, r, K, T, int(n_steps), int(n_paths),
                                                               int(seed), ctypes.c_void_p(d_out_ptr)),
               "lv_price_greeks_vanna_device")

    def price_greeks_fp64_device(self, S0, r, K, T, n_steps, n_paths, seed, d_out_ptr: int) -> None:
        """The binary64 reference run (lv_price_greeks_fp64_device)."""
        _check(self.lib, self.lib.lv_price_greeks_fp64_device(self.h, S0, r, K, T, int(n_steps), int(n_paths),
                                                              int(seed), ctypes.c_void_p(d_out_ptr)),
               "lv_price_greeks_fp64_device")

    def bump_greeks_fp64(self, S0, r, K, T, n_steps, n_paths, seed, eps):
        """Central bump-and-reprice with binary64 paths (lv_bump_greeks_fp64)."""
        p, d = ctypes.c_double(), ctypes.c_double()
        vega = np.zeros(self.IJ, dtype=np.float64)
        _check(self.lib, self.lib.lv_bump_greeks_fp64(self.h, S0, r, K, T, int(n_steps), int(n_paths), int(seed),
                                                      float(eps), ctypes.byref(p), ctypes.byref(d), _dp(vega)),
               "lv_bump_greeks_fp64")
        return p.value, d.value, vega.reshape(self.n_spot, self.n_time)

    def time_table(self, T, n_steps):
        """The kernels' (time cell j_n, binary32 weight v_n) for every step."""
        j = np.zeros(n_steps, dtype=np.int32)
        v = np.zeros(n_steps, dtype=np.float32)
        _check(self.lib, self.lib.lv_debug_time_table(self.h, float(T), int(n_steps),
                                                      j.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _fp(v)),
               "lv_debug_time_table")
        return j, v

    def bump_greeks(self, S0, r, K, T, n_steps, n_paths, seed, eps):
        p, d = ctypes.c_double(), ctypes.c_double()
        vega = np.zeros(self.IJ, dtype=np.float64)
        _check(self.lib, self.lib.lv_bump_greeks(self.h, S0, r, K, T, int(n_steps), int(n_paths), int(seed),
                                                 float(eps), ctypes.byref(p), ctypes.byref(d), _dp(vega)),
               "lv_bump_greeks")
        return p.value, d.value, vega.reshape(self.n_spot, self.n_time)


PIPES = ("ffma", "mufu_ex2", "mufu_lg2", "mufu_sin", "mufu_cos", "mufu_sqrt", "imad", "imad_wide", "lop3")


def measure_pipe_peaks(lib=None) -> dict:
    """Measured thread-instructions per second of each probed pipe operation
    on the current device (lv_measure_pipe_peaks)."""
    lib = lib or load()
    out = np.zeros(len(PIPES), dtype=np.float64)
    _check(lib, lib.lv_measure_pipe_peaks(_dp(out)), "lv_measure_pipe_peaks")
    return dict(zip(PIPES, out.tolist()))


def debug_normals(seed, stream_id, paths, blocks, lib=None):
    """The kernels' Philox words [n, 4] (uint32) and binary32 normals [n, 4]
    for the (path, block) counters listed."""
    lib = lib or load()
    p = np.ascontiguousarray(paths, dtype=np.int64)
    b = np.ascontiguousarray(blocks, dtype=np.uint32)
    n = p.shape[0]
    w = np.zeros((n, 4), dtype=np.uint32)
    z = np.zeros((n, 4), dtype=np.float32)
    _check(lib, lib.lv_debug_normals(int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream_id),
                                     p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), int(n),
                                     w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _fp(z)), "lv_debug_normals")
    return w, z


class Instrument(ctypes.Structure):
    """lv_instrument of include/lv.h."""
    _fields_ = [("surface", ctypes.c_int32), ("phi", ctypes.c_int32), ("K", ctypes.c_double),
                ("T", ctypes.c_double), ("n_steps", ctypes.c_int32), ("n_paths", ctypes.c_int64),
                ("stream_id", ctypes.c_uint32)]


def _declare_book(lib):
    c = ctypes
    vp, d, i32, i64, u64 = c.c_void_p, c.c_double, c.c_int32, c.c_int64, c.c_uint64
    sigs = {
        "lv_book_create": [c.POINTER(vp), i32, c.POINTER(Instrument), i32, c.POINTER(vp)],
        "lv_book_destroy": [vp],
        "lv_book_output_offsets": [vp, c.POINTER(i64)],
        "lv_book_set_stream": [vp, vp],
        "lv_book_run": [vp, d, d, u64, c.POINTER(d)],
        "lv_book_run_device": [vp, d, d, u64, vp],
        "lv_book_tune": [vp, d, d, u64, c.POINTER(i32), c.POINTER(i32), c.POINTER(i32), c.POINTER(d)],
        "lv_book_set_weights": [vp, c.POINTER(d)],
        "lv_book_risk_offsets": [vp, c.POINTER(i64)],
        "lv_book_run_risk": [vp, d, d, u64, c.POINTER(d)],
        "lv_book_run_risk_device": [vp, d, d, u64, vp],
        "lv_book_paths_per_lane": [vp, c.POINTER(i32)],
        "lv_book_set_launch": [vp, i32, i32, i32, i32],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None if name == "lv_book_destroy" else c.c_int
    return lib


class Book:
    """A book of options on several surfaces (lv_book_t)."""

    def __init__(self, surfaces, items, lib: Optional[ctypes.CDLL] = None):
        self.lib = _declare_book(lib or load())
        arr = (ctypes.c_void_p * len(surfaces))(*[s.h.value for s in surfaces])
        ins = (Instrument * len(items))(*[Instrument(it.surface, it.phi, it.K, it.T, it.n_steps, it.n_paths,
                                                     it.stream_id) for it in items])
        self.n = len(items)
        self.h = ctypes.c_void_p()
        _check(self.lib, self.lib.lv_book_create(arr, len(surfaces), ins, self.n, ctypes.byref(self.h)),
               "lv_book_create")
        off = (ctypes.c_int64 * (self.n + 1))()
        _check(self.lib, self.lib.lv_book_output_offsets(self.h, off), "lv_book_output_offsets")
        self.offsets = list(off)
        self.n_surfaces = len(surfaces)
        roff = (ctypes.c_int64 * (self.n_surfaces + 1))()
        _check(self.lib, self.lib.lv_book_risk_offsets(self.h, roff), "lv_book_risk_offsets")
        self.risk_offsets = list(roff)

    def close(self) -> None:
        if self.h:
            self.lib.lv_book_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, S0, r, seed) -> np.ndarray:
        out = np.zeros(self.offsets[-1], dtype=np.float64)
        _check(self.lib, self.lib.lv_book_run(self.h, S0, r, int(seed), _dp(out)), "lv_book_run")
        return out

    def run_device(self, S0, r, seed, d_out_ptr: int) -> None:
        _check(self.lib, self.lib.lv_book_run_device(self.h, S0, r, int(seed), ctypes.c_void_p(d_out_ptr)),
               "lv_book_run_device")

    def set_stream(self, stream_ptr: int) -> None:
        _check(self.lib, self.lib.lv_book_set_stream(self.h, ctypes.c_void_p(stream_ptr or None)),
               "lv_book_set_stream")

    def tune(self, S0, r, seed):
        b, k, p, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(self.lib, self.lib.lv_book_tune(self.h, S0, r, int(seed), ctypes.byref(b), ctypes.byref(k),
                                               ctypes.byref(p), ctypes.byref(ms)), "lv_book_tune")
        return b.value, k.value, p.value, ms.value

    def set_launch(self, block: int, k: int, item_paths: int, ppl: int) -> None:
        _check(self.lib, self.lib.lv_book_set_launch(self.h, int(block), int(k), int(item_paths), int(ppl)),
               "lv_book_set_launch")

    def paths_per_lane(self) -> int:
        p = ctypes.c_int32()
        _check(self.lib, self.lib.lv_book_paths_per_lane(self.h, ctypes.byref(p)), "lv_book_paths_per_lane")
        return p.value

    def set_weights(self, weights) -> None:
        """Position weight per option for the aggregated risk."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.shape != (self.n,):
            raise ValueError(f"need {self.n} weights")
        _check(self.lib, self.lib.lv_book_set_weights(self.h, _dp(w)), "lv_book_set_weights")

    def run_risk(self, S0, r, seed) -> np.ndarray:
        """Aggregated risk per surface: [sum w price, sum w delta, stderr, sum w vega...] blocks."""
        out = np.zeros(self.risk_offsets[-1], dtype=np.float64)
        _check(self.lib, self.lib.lv_book_run_risk(self.h, S0, r, int(seed), _dp(out)), "lv_book_run_risk")
        return out

    def run_risk_device(self, S0, r, seed, d_out_ptr: int) -> None:
        _check(self.lib, self.lib.lv_book_run_risk_device(self.h, S0, r, int(seed), ctypes.c_void_p(d_out_ptr)),
               "lv_book_run_risk_device")

    def risk(self, out: np.ndarray, s: int):
        """(price, delta, stderr, vega flat) of surface s from a risk run's output."""
        r = out[self.risk_offsets[s]:self.risk_offsets[s + 1]]
        return r[0], r[1], r[2], r[3:]

    def result(self, out: np.ndarray, o: int):
        """(price, delta, stderr, vega flat) of option o from a run's output."""
        r = out[self.offsets[o]:self.offsets[o + 1]]
        return r[0], r[1], r[2], r[3:]
