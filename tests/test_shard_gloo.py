"""Multi-rank path-range sharding on the CPU (gloo, world size 2): the
partition covers every path once and the cross-rank sum of per-range raw
sums equals the single-process sums. The oracle stands in for each rank's
per-range sums (the GPU side of the same call is tested on a GPU by the
path-range sharding parity test)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2002_02481_gb300.shard import path_range, price_greeks_sharded, sharded_sums


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import oracle
    import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        surf, opt = W.config_small()
        opt.n_paths = 3001
        IJ = surf.n_spot * surf.n_time

        def fn(b, e):
            s = oracle.run_sums(surf, opt, b, e, n_threads=1)
            return torch.from_numpy(np.concatenate([s[[oracle.SUM_V, oracle.SUM_V2, oracle.SUM_XBAR0]],
                                                    s[oracle.NSCAL:oracle.NSCAL + IJ]]))

        tot = sharded_sums(fn, opt.n_paths)
        q.put((rank, tot.numpy()))
    finally:
        dist.destroy_process_group()


def test_path_range_partition():
    for world in (1, 2, 3, 8):
        for P in (0, 1, 7, 1000, 1 << 20):
            ranges = [path_range(r, world, P) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == P
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
    with pytest.raises(ValueError):
        path_range(2, 2, 10)


def test_two_rank_sum_equals_single_process():
    import oracle
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    surf, opt = W.config_small()
    opt.n_paths = 3001
    s = oracle.run_sums(surf, opt, 0, opt.n_paths, n_threads=1)
    IJ = surf.n_spot * surf.n_time
    whole = np.concatenate([s[[oracle.SUM_V, oracle.SUM_V2, oracle.SUM_XBAR0]], s[oracle.NSCAL:oracle.NSCAL + IJ]])
    for r in (0, 1):
        np.testing.assert_allclose(res[r], whole, rtol=1e-12, atol=1e-12 * np.max(np.abs(whole)))
    np.testing.assert_array_equal(res[0], res[1])


class _OracleSurface:
    """Stands in for lv.Surface on the CPU: the raw sums of a path range and
    their finalize come from the FP64 oracle, written through data pointers
    as the device entry points write them."""

    def __init__(self, surf, opt):
        self.surf, self.opt = surf, opt
        self.n_spot, self.n_time = surf.n_spot, surf.n_time

    def _write(self, ptr, arr):
        import ctypes
        a = np.ascontiguousarray(arr, dtype=np.float64)
        ctypes.memmove(ptr, a.ctypes.data, a.nbytes)

    def price_greeks_sums_device(self, S0, r, K, T, n_steps, b, e, seed, stream_id, ptr):
        import oracle
        s = oracle.run_sums(self.surf, self.opt, b, e, n_threads=1)
        IJ = self.n_spot * self.n_time
        self._write(ptr, np.concatenate([s[[oracle.SUM_V, oracle.SUM_V2, oracle.SUM_XBAR0]],
                                         s[oracle.NSCAL:oracle.NSCAL + IJ]]))

    def finalize_sums_device(self, sums_ptr, n_paths, S0, out_ptr):
        import ctypes
        import oracle
        n = 3 + self.n_spot * self.n_time
        sums = np.frombuffer((ctypes.c_double * n).from_address(sums_ptr), dtype=np.float64).copy()
        full = np.zeros(oracle.NSCAL + 2 * (n - 3))
        full[[oracle.SUM_V, oracle.SUM_V2, oracle.SUM_XBAR0]] = sums[:3]
        full[oracle.NSCAL:oracle.NSCAL + n - 3] = sums[3:]
        self._write(out_ptr, oracle.finalize(full, n_paths, S0, n - 3))


def _sharded_worker(rank, world, port, q):
    import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        surf, opt = W.config_small()
        opt.n_paths = 3001
        n = 3 + surf.n_spot * surf.n_time
        sums = torch.zeros(n, dtype=torch.float64)
        out = torch.zeros(n, dtype=torch.float64)
        res = price_greeks_sharded(_OracleSurface(surf, opt), opt.S0, opt.r, opt.K, opt.T, opt.n_steps,
                                   opt.n_paths, opt.seed, device="cpu", sums=sums, out=out)
        assert res is out
        q.put((rank, out.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_price_greeks_sharded_equals_single_process():
    """The whole sharded call on two gloo ranks: each rank's range, the
    all-reduce and the finalize give every rank the single-process price,
    standard error, delta and vegas."""
    import oracle
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    surf, opt = W.config_small()
    opt.n_paths = 3001
    ref = oracle.finalize(oracle.run_sums(surf, opt, 0, opt.n_paths, n_threads=1), opt.n_paths, opt.S0,
                          surf.n_spot * surf.n_time)
    for r in (0, 1):
        np.testing.assert_allclose(res[r], ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))
    np.testing.assert_array_equal(res[0], res[1])
