"""Multi-process paths on CPU with the gloo backend (world size 2).

The build runs one process per GPU as independent replicas (no collective on
the data path).  Two things cross ranks and are checked here without a GPU:

* the job-level timing of ``bench.py``: the slowest replica's time and the
  units of all replicas (max over ranks, whole-job throughput);
* the data-parallel SCF reduction the method admits (Sec. 3.1: every process
  sums the coefficient contributions of its own particles, one sum of the
  (n_max+1)(l_max+1)^2 partial coefficients follows), simulated with the FP64
  oracle: the all-reduced shard coefficients equal the coefficients of all
  particles, and a fixed-order reduce-then-broadcast gives bit-identical
  coefficients on every rank.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)


def _bench_worker(rank, port, out):
    import bench
    _init(rank, port)
    try:
        ms = [3.5, 7.25][rank]
        got = bench.max_over_ranks(ms, dist)
        out[rank] = (got, bench.job_throughput(1000, WORLD, got))
    finally:
        dist.destroy_process_group()


def _scf_worker(rank, port, out):
    import oracle
    from paper_1406_4254_gb300 import inputs
    _init(rank, port)
    try:
        pm = inputs.hernquist(3001, seed=7, axes=(1.0, 0.8, 0.6))
        lo, hi = rank * len(pm) // WORLD, (rank + 1) * len(pm) // WORLD
        part = oracle.scf_coeffs(pm[lo:hi, :3], pm[lo:hi, 3], 6, 4)
        t = torch.tensor(part)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        # fixed order: gather the shards on rank 0, sum them in rank order, broadcast
        parts = [torch.zeros_like(t) for _ in range(WORLD)] if rank == 0 else None
        dist.gather(torch.tensor(part), parts, dst=0)
        fixed = sum(parts[1:], parts[0].clone()) if rank == 0 else torch.zeros_like(t)
        dist.broadcast(fixed, src=0)
        out[rank] = (t.numpy().copy(), fixed.numpy().copy())
    finally:
        dist.destroy_process_group()


def _run(worker):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=worker, args=(r, port, out)) for r in range(WORLD)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        assert codes == [0] * WORLD, codes
        return dict(out)


def test_bench_timing_is_the_slowest_replica():
    out = _run(_bench_worker)
    for r in range(WORLD):
        got, thr = out[r]
        assert got == 7.25
        assert thr == pytest.approx(1000 * WORLD / 7.25e-3)


def test_sharded_scf_coefficients_allreduce():
    import oracle
    from paper_1406_4254_gb300 import inputs
    out = _run(_scf_worker)
    pm = inputs.hernquist(3001, seed=7, axes=(1.0, 0.8, 0.6))
    full = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 6, 4)
    for r in range(WORLD):
        summed, fixed = out[r]
        np.testing.assert_allclose(summed, full, rtol=1e-12, atol=1e-15 * np.abs(full).max())
    assert np.array_equal(out[0][1], out[1][1])
