"""Benchmark: adjoint path-steps/s (price + delta + every vega bucket) of the
local-volatility Monte Carlo on one GB300, on the paper's workload shape
(30 x 60 grid = 1,800 buckets, 156 Euler steps, call K=100 T=3, 2^20 paths).

One step = one lv_price_greeks_device call: forward, compaction, reverse
sweep with checkpoint recompute, bucket accumulation and the fixed-order
finalize, inputs resident on the device. Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on this host's cores on a
bounded sample of the same workload (the reference arm of the comparison).
Under torchrun (N > 1) every rank runs its own contiguous range of 2^20
paths of one N x 2^20-path estimate (weak scaling): the step is the
sharded call, the adjoint on the rank's range, one all-reduce of the
3 + 1,800 raw sums over the ranks and the finalize; rank 0 reports the
aggregate with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "adjoint path-steps/s (price+delta+all vegas)"
WORKLOAD = "30x60 local-vol grid, 156 steps, 2^20 paths, European call K=100 T=3, price+delta+1800 vegas"

# Algorithmic thread-operations of one path-step of the method: one forward
# step (Philox share, uniforms, Box-Muller share, exp, cell, bilinear sigma,
# Euler) for every path, plus one reverse step (sigma adjoint, x adjoint,
# bucket scatter) for the paths that end in the money (the others have a
# zero adjoint everywhere and are not swept back); the checkpoint recompute
# is overhead and is not counted.
FWD_OPS_PER_PATH_STEP = 36.0
REV_OPS_PER_PATH_STEP = 19.0
# Issue rate of an SM: 4 schedulers x 32 lanes per clock (the fallback peak
# when the pipe probe cannot run).
LANES_PER_SM_CLOCK = 128
# ncu pipe -> the probed instruction whose rate is that pipe's issue rate (one warp instruction
# per pipe issue): fma.rn.f32 on either FMA half, mad.lo.u32 on the heavy half, lop3 on the ALU,
# lg2 on the transcendental unit (ex2 issues at twice that rate; the 64-bit mad.wide takes two
# issues of the heavy half)
PIPE_OF_PROBE = {"fma": "ffma", "fmaheavy": "imad", "alu": "lop3", "xu": "mufu_lg2"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lr


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def time_oracle(surf, opt, n_paths: int, n_threads: int) -> float:
    """Seconds the FP64 oracle takes for price + delta + vegas over n_paths."""
    import oracle
    o = W.Option(**{**opt.__dict__, "n_paths": n_paths})
    t0 = time.perf_counter()
    oracle.run_sums(surf, o, 0, n_paths, greeks=True, n_threads=n_threads)
    return time.perf_counter() - t0


def run_reference(args):
    ws, rk, _ = dist_env()
    if rk != 0:
        return 0
    import oracle
    oracle.load_library()
    surf, opt = W.config_paper_shape()
    threads = oracle.default_threads()
    sample = opt.n_paths                  # the whole 2^20-path workload each step (~22 CPU-seconds)
    for _ in range(args.warmup):
        time_oracle(surf, opt, sample, threads)
    secs = [time_oracle(surf, opt, sample, threads) for _ in range(args.steps)]
    t = sum(secs) / len(secs)
    value = sample * opt.n_steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "path-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "30x60", "n_steps": opt.n_steps,
                   "n_paths_timed_per_step": sample, "cpu": cpu_model()},
        "cpu_baseline": {"value": value, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
                         "sample": f"all {sample} paths of the workload per step, 156 steps, "
                                   "price+delta+1800 vegas"},
        "e2e": {"value": value, "unit": "path-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def sigma_upload_bytes(surf) -> int:
    """Bytes lv_surface_set_sigma copies to the device per call: the binary32
    pairs (sigma_ij, sigma_{i+1,j} - sigma_ij), [max(J, 2)][I - 1] float2 (the
    binary64 copy goes only with the binary64 reference calls)."""
    return 8 * max(surf.n_time, 2) * (surf.n_spot - 1)


def kernel_source_hash() -> str:
    """Hash of the source files the adjoint kernel is built from (any edit to
    them invalidates a recorded traffic figure)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2002_02481_gb300", "csrc")
    text = "".join(open(os.path.join(csrc, f)).read()
                   for f in ("lv_device.cuh", "lv_mc.cuh", "lv_kernels.cu", "lv_internal.h"))
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def profiled_record():
    """The committed ncu record of one adjoint launch on the bench workload
    (DRAM bytes, warp instructions per pipe), or None when the kernel changed
    since it was taken."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "adjoint_kernel_paper_shape.json")))
    except (OSError, ValueError):
        return None
    return rec if rec.get("source_hash") == kernel_source_hash() else None


def profiled_traffic():
    rec = profiled_record()
    return rec["dram_bytes_per_launch"] if rec else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except (OSError, ValueError):
        return {"sm_max_mhz": 2070.0}, "fallback"


def time_call(fn, ev0, ev1, reps=3, warm=1):
    """Median kernel time (ms, from the library's kernel events) of fn()."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        fn()
        ev1.synchronize()
        ts.append(ev0.elapsed_time(ev1))
    return statistics.median(ts)


def other_workloads(lib, dev, ev0, ev1):
    """Kernel times of the other configurations (a few runs each)."""
    import torch

    from paper_2002_02481_gb300 import lv

    res = {}
    stream = torch.cuda.current_stream(dev)

    def single(name, surf, opt, launch=None, acc=0, method=lv.LV_ADJ_REVERSE, interp=0, scheme=0):
        S = lv.Surface.from_workload(surf, lib)
        S.set_stream(stream.cuda_stream)
        S.set_accumulation(acc)
        S.set_adjoint_method(method)
        S.set_interpolation(interp)
        S.set_scheme(scheme)
        if launch:
            S.set_launch(*launch)
        S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
        d = torch.zeros(3 + surf.n_spot * surf.n_time, dtype=torch.float64, device=dev)
        ms = time_call(lambda: S.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths,
                                                      opt.seed, d.data_ptr()), ev0, ev1)
        res[name] = {"adjoint_kernel_ms": ms, "path_steps_per_s": opt.n_paths * opt.n_steps / (ms * 1e-3),
                     "launch": list(S.get_launch(opt.n_steps, True)),
                     "paths_per_lane": S.get_paths_per_lane(opt.n_steps, opt.n_paths)}
        S.close()

    single("small 20x10, 52 steps, 2^14 paths", *W.config_small())
    # the other readings of the scheme, on the bench workload
    for interp, scheme, tag in ((lv.LV_INTERP_LOGS, lv.LV_SCHEME_LOG, "spot weight linear in ln S"),
                                (lv.LV_INTERP_S, lv.LV_SCHEME_S, "Euler on S"),
                                (lv.LV_INTERP_LOGS, lv.LV_SCHEME_S, "Euler on S, weight in ln S")):
        single(f"reading: {tag}, 30x60, 156 steps, 2^20 paths", *W.config_paper_shape(), interp=interp,
               scheme=scheme)
    # price, delta, vegas, rho and d price / d T in one reverse sweep
    S = lv.Surface.from_workload(W.config_paper_shape()[0], lib)
    S.set_stream(stream.cuda_stream)
    S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
    _, o = W.config_paper_shape()
    d = torch.zeros(5 + S.IJ, dtype=torch.float64, device=dev)
    ms = time_call(lambda: S.price_greeks_ext_device(o.S0, 0.01, o.K, o.T, o.n_steps, o.n_paths, o.seed,
                                                      d.data_ptr()), ev0, ev1)
    res["with rho and dV/dT (lv_price_greeks_ext), 30x60, 156 steps, 2^20 paths"] = {
        "adjoint_kernel_ms": ms, "path_steps_per_s": o.n_paths * o.n_steps / (ms * 1e-3), "r": 0.01}
    S.close()
    # second-order buckets d^2 price / (d S0 d sigma_ij) (two forward passes)
    S = lv.Surface.from_workload(W.config_paper_shape()[0], lib)
    S.set_stream(stream.cuda_stream)
    S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
    d = torch.zeros(3 + S.IJ, dtype=torch.float64, device=dev)
    ms = time_call(lambda: S.price_greeks_vanna_device(o.S0, o.r, o.K, o.T, o.n_steps, o.n_paths, o.seed,
                                                        d.data_ptr()), ev0, ev1)
    res["second-order buckets (lv_price_greeks_vanna), 30x60, 156 steps, 2^20 paths"] = {
        "kernel_ms": ms, "path_steps_per_s": o.n_paths * o.n_steps / (ms * 1e-3)}
    S.close()
    # the tangent-ratio form of the adjoint (two forward passes, no checkpoints)
    single("tangent-ratio adjoint, 30x60, 156 steps, 2^20 paths", *W.config_paper_shape(),
           method=lv.LV_ADJ_TANGENT)
    single("tangent-ratio adjoint, 30x60, 156 steps, 2^24 paths", *W.config_precision("paper"),
           method=lv.LV_ADJ_TANGENT)
    single("tangent-ratio adjoint, 100x100, 1260 steps, 2^26 paths", *W.config_large(), method=lv.LV_ADJ_TANGENT)
    for which in ("small", "paper"):
        surf, opt = W.config_precision(which)
        for acc, nm in ((0, "binary64"), (1, "Kahan")):
            single(f"precision {which} grid, 156 steps, 2^24 paths, level 2 {nm}", surf, opt, acc=acc)
    surf, opt = W.config_large()
    for k in (4, 32):
        single(f"large 100x100, 1260 steps, 2^26 paths, k={k}", surf, opt, launch=(128, k, 0))
    # the book: 8 grids x 64 options, one persistent launch, graph replay
    handles = [lv.Surface.from_workload(sf, lib) for sf in W.book_surfaces()]
    items = W.book_items()
    book = lv.Book(handles, items, lib)
    for h in handles:
        h.close()
    blk, k, item_paths, tune_ms = book.tune(100.0, 0.0, 1)
    book.run(100.0, 0.0, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for rep in range(reps):
        book.run(100.0, 0.0, 1 + rep)
    wall = (time.perf_counter() - t0) / reps
    ps = sum(it.n_paths * it.n_steps for it in items)
    res["book 8 grids x 64 options, graph replay"] = {
        "ms_per_run_wall": wall * 1e3, "path_steps": ps, "path_steps_per_s": ps / wall,
        "paths": sum(it.n_paths for it in items), "tuned": {"block": blk, "k": k, "item_paths": item_paths,
                                                            "paths_per_lane": book.paths_per_lane(),
                                                            "kernel_ms": tune_ms}}
    # the same book as aggregated risk per surface (position weights +-1)
    book.set_weights([1.0 if it.phi > 0 else -1.0 for it in items])
    book.run_risk(100.0, 0.0, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for rep in range(reps):
        book.run_risk(100.0, 0.0, 1 + rep)
    wall = (time.perf_counter() - t0) / reps
    res["book aggregated risk per surface, graph replay"] = {
        "ms_per_run_wall": wall * 1e3, "path_steps": ps, "path_steps_per_s": ps / wall,
        "outputs": book.risk_offsets[-1], "per_option_outputs": book.offsets[-1]}
    book.close()
    return res


def live_fraction(S, opt, m=1 << 16):
    """Fraction of paths that end in the money (nonzero terminal adjoint), from
    the kernel's per-path diagnostics on the first m paths."""
    _, V, _ = S.debug_paths(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.seed, 0, m)
    return float(np.mean(V > 0))


def roofline_block(kern_ms, path_steps, live, peaks, mhz, n_sm, rec):
    """Counted algorithmic work of the adjoint kernel against the measured
    issue rate, and, from the committed ncu record, each pipe's busy fraction
    against its measured rate."""
    counted = FWD_OPS_PER_PATH_STEP + REV_OPS_PER_PATH_STEP * live
    t = kern_ms * 1e-3
    if peaks and peaks.get("ffma", 0) > 0:
        peak = peaks["ffma"] / 1e9
        src = "measured: lv_measure_pipe_peaks, fma.rn.f32 rate (one thread-instruction per lane per clock)"
    else:
        peak = n_sm * LANES_PER_SM_CLOCK * mhz * 1e6 / 1e9
        src = f"derived: {n_sm} SMs x {LANES_PER_SM_CLOCK} lanes/clk x {mhz:.0f} MHz (pipe probe unavailable)"
    achieved = counted * path_steps / t / 1e9
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
           "traffic": rec["dram_bytes_per_launch"] if rec else None, "kernel_ms": kern_ms, "peak_source": src,
           "ops_per_path_step": {"forward": FWD_OPS_PER_PATH_STEP, "reverse": REV_OPS_PER_PATH_STEP,
                                 "live_fraction": live, "counted": counted},
           "frac_if_every_path_were_swept_back":
               (FWD_OPS_PER_PATH_STEP + REV_OPS_PER_PATH_STEP) * path_steps / t / 1e9 / peak}
    if rec and peaks and "pipe_warp_inst_per_launch" in rec:
        wi = rec["pipe_warp_inst_per_launch"]
        pipes = {}
        for pipe, probe in PIPE_OF_PROBE.items():
            if pipe in wi and peaks.get(probe, 0) > 0:
                rate = wi[pipe] * 32.0 / t
                pipes[pipe] = {"thread_ops_per_path_step": wi[pipe] * 32.0 / path_steps,
                               "achieved_gops": rate / 1e9, "peak_gops": peaks[probe] / 1e9,
                               "frac": rate / peaks[probe], "peak_probe": probe}
        if "all" in wi:
            issue = wi["all"] / (4.0 * n_sm * mhz * 1e6 * t)
            pipes["issue_slots"] = {"warp_inst_per_launch": wi["all"], "frac": issue,
                                    "thread_ops_per_path_step": wi["all"] * 32.0 / path_steps}
        if pipes:
            bind = max((k for k in pipes if k != "issue_slots"), key=lambda k: pipes[k]["frac"])
            out["pipes"] = pipes
            out["binding_pipe"] = bind
    return out


def equal_accuracy_bump(S, opt, errors, adjoint_err, kern_ms, bump32_ms, sample):
    """The bump baseline's variants on the accuracy sample (error against the
    FP64 oracle's pathwise estimator) with their time on the full workload,
    and the speed-up of the adjoint over the cheapest variant that is at
    least as accurate as the adjoint on every output."""
    import torch
    variants = []
    for eps in (1e-4, 1e-3, 1e-2):
        e = errors(*S.bump_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, sample, opt.seed, eps))
        variants.append({"name": f"binary32 paths, eps={eps:g}", "ms_full": bump32_ms, "timed_paths": opt.n_paths,
                         **e})
    eps64 = 1e-6
    e = errors(*S.bump_greeks_fp64(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, sample, opt.seed, eps64))
    timed = 1 << 16
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ev0.record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
    S.bump_greeks_fp64(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, timed, opt.seed, eps64)
    ms = ev0.elapsed_time(ev1) * opt.n_paths / timed
    variants.append({"name": f"binary64 paths, eps={eps64:g} (spot bump eps*S0)", "ms_full": ms,
                     "timed_paths": timed, "ms_full_is": f"kernel time on {timed} paths x {opt.n_paths // timed} "
                                                          "(linear in paths)", **e})
    keys = ("delta_rel", "vega_max_abs_of_max")
    ok = [v for v in variants if all(v[k] <= adjoint_err[k] for k in keys)]
    best = min(ok, key=lambda v: v["ms_full"]) if ok else None
    return {"sample": f"first {sample} paths", "adjoint": {k: adjoint_err[k] for k in keys},
            "variants": variants, "cheapest_at_adjoint_accuracy": best["name"] if best else None,
            "speedup_vs_adjoint_kernel": best["ms_full"] / kern_ms if best else None}


def large_record(lib, dev, peaks, n_sm, mhz, reps=3):
    """The 100 x 100 grid, 1,260 steps, 2^26 paths (the largest single-GPU
    configuration): device time, e2e through the host API, roofline and the
    oracle on a sample, at the tuned launch shape (k = 4) and, for the
    configured checkpoint interval, at k = 32."""
    import torch

    from paper_2002_02481_gb300 import lv

    import oracle
    surf, opt = W.config_large()
    S = lv.Surface.from_workload(surf, lib)
    stream = torch.cuda.current_stream(dev)
    S.set_stream(stream.cuda_stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev:
        e.record(stream)
    torch.cuda.synchronize(dev)
    d = torch.zeros(3 + S.IJ, dtype=torch.float64, device=dev)
    res = {"workload": "100x100 local-vol grid, 1260 steps, 2^26 paths, European call K=100 T=5, "
                       "price+delta+10000 vegas", "metric": METRIC, "unit": "path-steps/s"}
    ps = opt.n_paths * opt.n_steps
    for k in (4, 32):
        S.set_launch(128, k, 0)
        S.set_kernel_events(ev[2].cuda_event, ev[3].cuda_event)
        S.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
        step_ms, kern_ms = [], []
        for _ in range(reps):
            ev[0].record(stream)
            S.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
            ev[1].record(stream)
            ev[1].synchronize()
            step_ms.append(ev[0].elapsed_time(ev[1]))
            kern_ms.append(ev[2].elapsed_time(ev[3]))
        ms = statistics.median(step_ms)
        res[f"k={k}"] = {"ms_per_step": ms, "value": ps / (ms * 1e-3), "kernel_ms": statistics.median(kern_ms)}
    S.set_launch(128, 4, 0)
    res["launch"] = {"block": 128, "k": 4, "paths_per_lane": S.get_paths_per_lane(opt.n_steps, opt.n_paths),
                     "source": "tuned (k=4 fastest of 4, 8, 16; two paths per lane, packed pairs); k=32 is the "
                               "configured interval, reported beside it"}
    res["value"] = res["k=4"]["value"]
    res["ms_per_step"] = res["k=4"]["ms_per_step"]
    live = live_fraction(S, opt, 1 << 14)
    res["roofline"] = roofline_block(res["k=4"]["kernel_ms"], ps, live, peaks, mhz, n_sm, None)
    # end to end through the host API: sigma from pinned host memory, results to host memory
    sig_host = torch.from_numpy(np.ascontiguousarray(surf.sigma)).pin_memory().numpy()
    S.set_kernel_events(0, 0)
    S.set_sigma(sig_host)
    S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    t0 = time.perf_counter()
    for _ in range(reps):
        S.set_sigma(sig_host)
        S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    e2e_s = (time.perf_counter() - t0) / reps
    res["e2e"] = {"value": ps / e2e_s, "unit": "path-steps/s", "h2d_bytes_per_step": sigma_upload_bytes(surf),
                  "d2h_bytes_per_step": int(8 * (3 + S.IJ)), "ms_per_step": e2e_s * 1e3}
    threads = oracle.default_threads()
    sample = 1 << 14
    t0 = time.perf_counter()
    oracle.run_sums(surf, W.Option(**{**opt.__dict__, "n_paths": sample}), 0, sample, greeks=True, n_threads=threads)
    cpu_s = time.perf_counter() - t0
    res["cpu_baseline"] = {"value": sample * opt.n_steps / cpu_s, "unit": "path-steps/s", "cores": threads,
                           "kind": "oracle", "sample": f"first {sample} of the 2^26 paths, 1260 steps, price+delta+"
                           f"10000 vegas; extrapolated linearly in paths ({cpu_model()})"}
    S.close()
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2002_02481_gb300 import lv
    from paper_2002_02481_gb300.shard import price_greeks_sharded

    ws, rk, lr = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(lr)
    dev = torch.device("cuda", lr)
    lib = lv.load()
    surf, opt = W.config_paper_shape()
    P = opt.n_paths                       # per rank (weak scaling)
    S = lv.Surface.from_workload(surf, lib)
    stream = torch.cuda.current_stream(dev)
    S.set_stream(stream.cuda_stream)
    # launch shape from the project's autotuner, on this workload (or fixed by --launch)
    if args.launch:
        vals = [int(v) for v in args.launch.split(",")]
        S.set_launch(vals[0], vals[1], 0)
        S.set_paths_per_lane(vals[2] if len(vals) > 2 else 1)
        tuned = (vals[0], vals[1], None)
    else:
        tuned = S.tune(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed)
    n_out = 3 + surf.n_spot * surf.n_time
    d_out = torch.zeros(n_out, dtype=torch.float64, device=dev)
    d_sums = torch.zeros(n_out, dtype=torch.float64, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)      # torch creates the underlying CUDA events on first record
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
    # a buffer larger than L2 (129 MB), rewritten between timed steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        if ws == 1:
            S.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed, d_out.data_ptr())
        else:
            # this rank's 2^20 paths of one ws x 2^20-path estimate: the adjoint on the
            # range, one all-reduce of the raw sums, the finalize
            price_greeks_sharded(S, opt.S0, opt.r, opt.K, opt.T, opt.n_steps, ws * P, opt.seed, device=dev,
                                 sums=d_sums, out=d_out)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)

    step_ms, kern_ms = [], []
    with ClockSampler(lr) as clk:
        # the sampler reads every 200 ms: keep the GPU loaded for 0.6 s first so that
        # samples land on the same kind of load as the timed region that follows
        t_end = time.perf_counter() + 0.6
        while time.perf_counter() < t_end:
            step()
            torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        # the steps are queued without a host wait between them, so the host is
        # ahead of the device and every s0 -> s1 interval is device work only.
        # An event recorded between the adjoint kernel and the level-3 stages
        # that follow it by programmatic dependent launch costs about 6 us per
        # call, so the K timed steps run without kernel events, and an
        # identical run of K steps right after them records the adjoint
        # kernel's own duration (for the roofline)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        for e in evs:
            for x in e:
                x.record(stream)
        torch.cuda.synchronize(dev)
        S.set_kernel_events(0, 0)
        for e in evs:
            flush.fill_(1)
            e[0].record(stream)
            step()
            e[1].record(stream)
        torch.cuda.synchronize(dev)
        for e in evs:
            flush.fill_(1)
            S.set_kernel_events(e[2].cuda_event, e[3].cuda_event)
            step()
        torch.cuda.synchronize(dev)
        for e in evs:
            step_ms.append(e[0].elapsed_time(e[1]))
            kern_ms.append(e[2].elapsed_time(e[3]))
        S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = ws * P * opt.n_steps / (ms_per_step * 1e-3)

    # forward only (price without Greeks) and the bump-and-reprice baseline, same workload
    fwd_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        S.price(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed)
        fwd_ms.append(ev0.elapsed_time(ev1))
    bump = None
    bump32_ms = None
    if rk == 0 and not args.no_bump:
        pa, da, va = S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed)
        flush.fill_(1)
        pb, db, vb = S.bump_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed, 1e-4)
        bump32_ms = ev0.elapsed_time(ev1)
        bump = {"ms": bump32_ms, "scenarios": 3 + 2 * surf.n_spot * surf.n_time, "eps": 1e-4,
                "speedup_vs_adjoint_kernel": bump32_ms / statistics.mean(kern_ms),
                "max_vega_diff_vs_adjoint_of_max": float(np.max(np.abs(vb - va)) / np.max(np.abs(va))),
                "delta_diff_vs_adjoint_rel": abs(db - da) / abs(da)}

    # end to end through the public host API: sigma from pinned host memory in,
    # price/delta/vega out to host memory, every step
    e2e = None
    if rk == 0:
        sig_host = torch.from_numpy(np.ascontiguousarray(surf.sigma)).pin_memory()
        sig_np = sig_host.numpy()
        S.set_kernel_events(0, 0)
        for _ in range(2):
            S.set_sigma(sig_np)
            S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            S.set_sigma(sig_np)
            S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed)
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": P * opt.n_steps / e2e_s, "unit": "path-steps/s",
               "h2d_bytes_per_step": sigma_upload_bytes(surf), "d2h_bytes_per_step": int(8 * n_out),
               "ms_per_step": e2e_s * 1e3}

    if rk == 0:
        peaks_file, src = load_peaks()
        clocks = clk.summary()
        kern = statistics.mean(kern_ms)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks["sm_mhz"] or peaks_file.get("sm_max_mhz", 2070.0)
        try:
            pipe_peaks = lv.measure_pipe_peaks(lib)
        except lv.LVError:
            pipe_peaks = None
        live = live_fraction(S, opt)
        roofline = roofline_block(kern, P * opt.n_steps, live, pipe_peaks, mhz, n_sm, profiled_record())
        blk, kk, bps = S.get_launch(opt.n_steps, True)
        ppl = S.get_paths_per_lane(opt.n_steps, opt.n_paths)
        roofline["kernel"] = (f"adjoint_kernel<k={kk},binary64 level 2,{ppl} path(s) per lane> "
                              f"(block {blk}, {bps} blocks/SM)")
        roofline["clock_mhz"] = mhz
        workloads = None
        if not args.no_extra:
            S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
            workloads = other_workloads(lib, dev, ev0, ev1)
        large = None if args.no_large else large_record(lib, dev, pipe_peaks, n_sm, mhz)
        S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
        import oracle
        threads = oracle.default_threads()
        cpu_s = time_oracle(surf, opt, P, threads)
        cpu = {"value": P * opt.n_steps / cpu_s, "unit": "path-steps/s", "cores": threads,
               "kind": "oracle", "sample": f"all {P} paths of the workload, 156 steps, price+delta+1800 vegas, "
                                           f"{cpu_s:.1f} s on {threads} threads ({cpu_model()})"}
        sample = 1 << 13
        o_s = W.Option(**{**opt.__dict__, "n_paths": sample})
        ref = oracle.price_greeks(surf, o_s, n_threads=threads)
        # accuracy of the adjoint and of the bump baseline against the FP64 oracle's
        # pathwise estimator on the same paths (same counters)
        vmax = float(np.max(np.abs(ref["vega"])))

        def errors(p_, d_, v_):
            return {"price_rel": abs(p_ - ref["price"]) / abs(ref["price"]),
                    "delta_rel": abs(d_ - ref["delta"]) / abs(ref["delta"]),
                    "vega_max_abs_of_max": float(np.max(np.abs(v_ - ref["vega"]))) / vmax}
        adj_err = errors(*S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, sample, opt.seed))
        accuracy = {"sample": f"first {sample} of the 2^20 paths", "reference": "FP64 oracle, pathwise adjoint",
                    "adjoint": adj_err}
        if not args.no_bump:
            accuracy["bump_eps_1e-4"] = errors(*S.bump_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, sample,
                                                              opt.seed, 1e-4))
            bump["equal_accuracy"] = equal_accuracy_bump(S, opt, errors, adj_err, kern, bump32_ms, sample)
        line = {
            "metric": METRIC, "value": value, "unit": "path-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "30x60", "n_steps": opt.n_steps, "n_paths_per_gpu": P,
                       "launch": {"block": tuned[0], "k": tuned[1], "paths_per_lane": ppl,
                                  "source": "--launch" if args.launch else "lv_tune"},
                       "l2": "256 MB buffer rewritten between timed steps (outside the timed region)",
                       "parallelism": f"path-range shards x{ws}" + (", one all-reduce of 3+1800 sums per step"
                                                                     if ws > 1 else "")},
            "clocks": clocks, "gpu_launches": (3 if ws == 1 else 4) * args.steps, "roofline": roofline,
            "pipe_peaks_gops": {k: v / 1e9 for k, v in pipe_peaks.items()} if pipe_peaks else None,
            "cpu_baseline": cpu, "accuracy": accuracy, "e2e": e2e,
            "forward_only": {"kernel_ms": statistics.mean(fwd_ms),
                             "value": P * opt.n_steps / (statistics.mean(fwd_ms) * 1e-3), "unit": "path-steps/s"},
            "bump_reprice": bump,
            "large": large,
            "workloads": workloads,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def precision_study():
    """Config-3 study: binary32 paths with binary64 or Kahan binary32 level-2
    accumulation, each output's error stated against (a) the FP64 oracle on
    the first 2^18 paths (same counters) and (b) the full-FP64 GPU run
    (lv_price_greeks_fp64_device) over all 2^24 paths, on both config-3
    grids (reading C9). Prints one JSON line."""
    import torch

    import oracle
    from paper_2002_02481_gb300 import lv

    lib = lv.load()
    sub = 1 << 18

    def errs(p, d, v, rp, rd, rv):
        vm = float(np.max(np.abs(rv)))
        return {"price_rel": abs(p - rp) / abs(rp), "delta_rel": abs(d - rd) / abs(rd),
                "vega_max_abs_err_of_max": float(np.max(np.abs(v - rv))) / vm,
                "vega_rms_err_of_max": float(np.sqrt(np.mean((v - rv) ** 2))) / vm}

    out = {"study": "precision", "paths": 1 << 24, "oracle_paths": sub, "n_steps": 156,
           "references": {"oracle": "FP64 CPU oracle on the first 2^18 paths (same counters)",
                          "fp64_gpu": "lv_price_greeks_fp64_device, every path in binary64, all 2^24 paths"}}
    for which in ("small", "paper"):
        surf, opt = W.config_precision(which)
        o_sub = W.Option(**{**opt.__dict__, "n_paths": sub})
        t0 = time.perf_counter()
        ref = oracle.price_greeks(surf, o_sub)
        row = {"oracle_s": time.perf_counter() - t0, "oracle_threads": oracle.default_threads()}
        S = lv.Surface.from_workload(surf, lib)
        d = torch.zeros(3 + S.IJ, dtype=torch.float64, device="cuda")

        def fp64(n):
            torch.cuda.synchronize()
            t = time.perf_counter()
            S.price_greeks_fp64_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, n, opt.seed, d.data_ptr())
            torch.cuda.synchronize()
            o = d.cpu().numpy()
            return o[0], o[1], o[3:].reshape(surf.n_spot, surf.n_time), time.perf_counter() - t

        p64s, d64s, v64s, _ = fp64(sub)
        row["fp64_gpu_vs_oracle_2^18"] = errs(p64s, d64s, v64s, ref["price"], ref["delta"], ref["vega"])
        p64, d64, v64, t64 = fp64(opt.n_paths)
        row["fp64_gpu_s"] = t64
        for acc, nm in ((0, "binary64"), (1, "Kahan")):
            S.set_accumulation(acc)
            pf, df, vf = S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed)
            ps, ds, vs = S.price_greeks(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, sub, opt.seed)
            row[nm] = {"vs_oracle_2^18": errs(ps, ds, vs, ref["price"], ref["delta"], ref["vega"]),
                       "vs_fp64_gpu_2^24": errs(pf, df, vf, p64, d64, v64), "price": pf, "delta": df}
        S.close()
        row["fp64_gpu_2^24"] = {"price": p64, "delta": d64}
        row["oracle_2^18"] = {"price": ref["price"], "delta": ref["delta"], "stderr": ref["stderr"]}
        out[f"{which} grid {surf.n_spot}x{surf.n_time}"] = row
    print(json.dumps(out), flush=True)
    return 0


def path_sweep():
    """Adjoint kernel time and path-steps/s on the 30x60 / 156-step workload
    for 2^16 ... 2^24 paths at the bench's launch shape: how the end-of-kernel
    tail amortises. Prints one JSON line."""
    import torch

    from paper_2002_02481_gb300 import lv

    lib = lv.load()
    surf, opt = W.config_paper_shape()
    S = lv.Surface.from_workload(surf, lib)
    stream = torch.cuda.current_stream()
    S.set_stream(stream.cuda_stream)
    S.set_launch(128, 4, 0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
    d = torch.zeros(3 + S.IJ, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"study": "path sweep", "workload": "30x60 grid, 156 steps", "launch": [128, 4], "points": []}
    for lg in range(16, 25):
        P = 1 << lg
        ts = []
        for rep in range(6):
            flush.fill_(1)
            S.price_greeks_device(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, P, opt.seed, d.data_ptr())
            ev1.synchronize()
            if rep:
                ts.append(ev0.elapsed_time(ev1))
        ms = statistics.median(ts)
        out["points"].append({"paths": P, "kernel_ms": ms, "path_steps_per_s": P * opt.n_steps / (ms * 1e-3)})
    S.close()
    print(json.dumps(out), flush=True)
    return 0


def only(which: str, launch: str, reps: int, paths: int = 0):
    """One workload alone at a fixed shape (for profiling and quick timing):
    'book' (8 x 64 options, per-option outputs, graph replay), 'vanna' (the
    second-order buckets on the bench workload), 'large' (100 x 100, 1,260
    steps, 2^26 paths) or 'fp64' (the binary64 reference run, 2^20 paths).
    `paths` > 0 replaces the workload's path count (a smaller case of the same
    kernel for profiling). Prints one JSON line with the kernel (or replay)
    times."""
    import torch

    from paper_2002_02481_gb300 import lv

    lib = lv.load()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    vals = [int(v) for v in launch.split(",")] if launch else []
    out = {"only": which, "launch": vals, "paths": paths or None, "ms": []}
    if which == "book":
        handles = [lv.Surface.from_workload(sf, lib) for sf in W.book_surfaces()]
        book = lv.Book(handles, W.book_items(), lib)
        for h in handles:
            h.close()
        if vals:
            book.set_launch(*vals)
        for rep in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            book.run(100.0, 0.0, 1 + rep)
            out["ms"].append((time.perf_counter() - t0) * 1e3)
        book.close()
    else:
        surf, opt = W.config_large() if which == "large" else W.config_paper_shape()
        if paths > 0:
            opt = W.Option(**{**opt.__dict__, "n_paths": paths})
        S = lv.Surface.from_workload(surf, lib)
        S.set_stream(stream.cuda_stream)
        if vals:
            S.set_launch(vals[0], vals[1], 0)
            S.set_paths_per_lane(vals[2] if len(vals) > 2 else 1)
        S.set_kernel_events(ev0.cuda_event, ev1.cuda_event)
        d = torch.zeros(3 + S.IJ, dtype=torch.float64, device="cuda")
        call = {"vanna": S.price_greeks_vanna_device, "large": S.price_greeks_device,
                "fp64": S.price_greeks_fp64_device}[which]
        for _ in range(reps):
            call(opt.S0, opt.r, opt.K, opt.T, opt.n_steps, opt.n_paths, opt.seed, d.data_ptr())
            ev1.synchronize()
            out["ms"].append(ev0.elapsed_time(ev1))
        S.close()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-bump", action="store_true", help="skip the bump-and-reprice timing")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-large", action="store_true", help="skip the 100x100 / 1260-step / 2^26-path record")
    ap.add_argument("--only", default="", choices=["", "book", "vanna", "large", "fp64"],
                    help="time one workload alone at a fixed shape (for profiling)")
    ap.add_argument("--paths", type=int, default=0, help="with --only: the path count (profiling a smaller case)")
    ap.add_argument("--launch", default="",
                    help="fix the adjoint's launch shape as BLOCK,K[,PATHS_PER_LANE] instead of tuning it")
    ap.add_argument("--precision-study", action="store_true",
                    help="2^24-path precision workloads: binary64 vs Kahan level 2 against the FP64 oracle")
    ap.add_argument("--path-sweep", action="store_true",
                    help="adjoint kernel throughput for 2^16 ... 2^24 paths on the bench workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.precision_study:
        return precision_study()
    if args.path_sweep:
        return path_sweep()
    if args.only:
        return only(args.only, args.launch, max(1, args.steps), args.paths)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
