#!/usr/bin/env python3
"""Benchmark of the SCF + MEX expansion force calculation on GB300.

One step = one full SCF force calculation (coefficient pass + field pass,
(n_max, l_max) = (10, 6)) and one full MEX force calculation (radial sort,
inner/outer scans, field; l_max = 6) on the same N = 2^20 particles of a
Hernquist model stretched to axis ratios 1 : 0.8 : 0.6, in the mixed precision
path (FP32 arithmetic, FP64 coefficient reduction and scan carries).  The
metric is particle-forces per second: 2N per step (N by each method).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle (the
FP64 reference implementation written from the paper) on a bounded sample of
the same workload instead.  Multi-GPU (torchrun): independent replicas, one
per GPU (neither method is sharded across GPUs: each GPU runs the whole
workload on its own particles), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle forces/s at N=2^20 (SCF n10 l6; MEX l6), mixed vs FP64, same GB300"
UNIT = "particle-forces/s"
N_DEFAULT = 1 << 20
N_MAX, L_MAX = 10, 6
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (max SM clock)"


def workload_name(n):
    return f"hernquist-1:0.8:0.6 N={n} SCF(n_max=10,l_max=6)+MEX(l_max=6)"


# --- algorithmic work per particle (the useful-work counts of each kernel) ---
def scf_coeff_flops(n, l):
    # contraction 2(n+1)(l+1)^2 + Gegenbauer 3(n+1)(l+1) + angular 4(l+1)^2 + 30
    return 2 * (n + 1) * (l + 1) ** 2 + 3 * (n + 1) * (l + 1) + 4 * (l + 1) ** 2 + 30


def scf_field_flops(n, l):
    # contraction 4(n+1)(l+1)^2 + basis 6(n+1)(l+1) + angular+gradient 10(l+1)^2
    # + radial prefactors 8(l+1) + 80
    return 4 * (n + 1) * (l + 1) ** 2 + 6 * (n + 1) * (l + 1) + 10 * (l + 1) ** 2 \
        + 8 * (l + 1) + 80


def mex_flops(l):
    # per particle: harmonics 3(l+1)^2, their gradients 9(l+1)^2, inner and
    # outer moments 4(l+1)^2, scans 2(l+1)^2, potential 4(l+1)^2, gradient
    # terms 12(l+1)^2 (both sides) -> 34 (l+1)^2
    return 34 * (l + 1) ** 2


def kernel_traffic():
    """DRAM bytes per launch at N = 2^20 from the committed ncu summary, keyed
    by kernel and the hash of the source file it was captured from; a kernel
    whose source changed since reads as None."""
    import hashlib
    out = {}
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return out
    for line in open(path):
        parts = line.split()
        if len(parts) != 4 or parts[0].startswith("#"):
            continue
        kernel, src, digest, nbytes = parts
        f = os.path.join(ROOT, "paper_1406_4254_gb300", "csrc", src)
        if os.path.exists(f) and hashlib.sha256(open(f, "rb").read()).hexdigest()[:16] == digest:
            out[kernel] = float(nbytes)
    return out


def mex_bytes(fp64=False):
    # keys 16R+12W, 4 sort passes (8R+8W), tie pass 4R, gather 4R+16R+16W,
    # pass2 16R+4R+16W  (per particle, FP32 particles)
    b = 16 + 12 + 4 * 16 + 4 + (4 + 16 + 16) + (16 + 4 + 16)
    return b + (3 * 16 if fp64 else 0)


def fp32_peak_tflops():
    """FP32 CUDA-core peak derived from unit counts and the maximum SM clock."""
    return 152 * 128 * 2 * 2070.0 * 1e6 / 1e12


def measure_fma_peaks(dev, target_ms=5.0, reps=5, kinds=None):
    """FP32 and FP64 FMA rates of this GPU, in TFLOP/s, from the library's
    FMA-chain microbenchmark (etics_fma_peak): each kind is timed with CUDA
    events on the launching stream, best of `reps` launches of about
    `target_ms` each (a burst, as the step's kernels run).  'fp32' is the
    better of plain and paired FP32 FMAs."""
    import torch
    from paper_1406_4254_gb300 import etics
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 4
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kinds = kinds or {"ffma": etics.PEAK_FFMA, "ffma2": etics.PEAK_FFMA2, "dfma": etics.PEAK_DFMA}
    out = {}
    for name, kind in kinds.items():
        iters = 64
        for _ in range(8):   # calibrate the trip count to about target_ms
            e0.record(s)
            etics.fma_peak(kind, blocks, iters, sink)
            e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if ms > 0.5 * target_ms:
                break
            iters = int(iters * min(64.0, target_ms / max(ms, 1e-3)))
        iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
        best = 0.0
        for _ in range(reps):
            e0.record(s)
            flops = etics.fma_peak(kind, blocks, iters, sink)
            e1.record(s)
            torch.cuda.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[name] = best
    etics.check_error()
    if "ffma" in out and "ffma2" in out:
        out["fp32"] = max(out["ffma"], out["ffma2"])
    if "dfma" in out:
        out["fp64"] = out["dfma"]
    return out


MEX_L_LIMIT = 10   # compiled l_max limit of the MEX kernels (ETICS_MEX_LMAX_LIMIT)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# --- clocks sampling ---------------------------------------------------------
class Clocks:
    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# --- raw CUDA events (recorded inside the library on the call's stream) -------
class RawEvents:
    """cudaEvent_t handles created with the driver API, so that events the
    library records can be timed (torch only times events it recorded)."""

    def __init__(self, n):
        import ctypes
        self.ct = ctypes
        self.cu = ctypes.CDLL("libcuda.so.1")
        self.ev = []
        for _ in range(n):
            h = ctypes.c_void_p()
            rc = self.cu.cuEventCreate(ctypes.byref(h), 0)
            if rc != 0:
                raise RuntimeError(f"cuEventCreate failed ({rc})")
            self.ev.append(h)

    def handles(self, a, b):
        return [self.ct.c_void_p(h.value) for h in self.ev[a:b]]

    def ms(self, i, j):
        out = self.ct.c_float()
        rc = self.cu.cuEventElapsedTime(self.ct.byref(out), self.ev[i], self.ev[j])
        if rc != 0:
            raise RuntimeError(f"cuEventElapsedTime failed ({rc})")
        return float(out.value)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of one float over all ranks (the slowest replica sets the
    job's time); x itself with no process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units every replica processed over the
    slowest replica's time."""
    return units_per_rank * world / (ms * 1e-3)


# --- GPU arm -------------------------------------------------------------------
def run_etics(args, rank, world):
    import torch
    from paper_1406_4254_gb300 import etics, inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    pm = inputs.hernquist(n, seed=args.seed + rank, axes=(1.0, 0.8, 0.6))
    x = torch.tensor(pm, dtype=torch.float32, device=dev)
    x64 = torch.tensor(pm, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    coeffs = torch.empty((N_MAX + 1, (L_MAX + 1) ** 2), dtype=torch.float64, device=dev)
    out_scf = torch.empty_like(x)
    out_mex = torch.empty_like(x)
    ws_scf = etics.workspace(n, N_MAX, L_MAX, etics.SCF, etics.MIXED, dev)
    ws_mex = etics.workspace(n, 0, L_MAX, etics.MEX, etics.MIXED, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2

    # stage events: 0-2 scf coeffs (start, coefficient kernel end, end),
    # 3-4 scf field (start, end), 5-10 mex (start, keys, sorted, tile sums,
    # carries, end)
    rev = RawEvents(11)

    def step(timed_stages=False):
        if timed_stages:
            etics.set_stage_events(rev.handles(0, 3))
        etics.scf_coeffs(x, N_MAX, L_MAX, out=coeffs, ws=ws_scf)
        if timed_stages:
            etics.set_stage_events(rev.handles(3, 5))
        etics.scf_field(x, coeffs, N_MAX, L_MAX, out=out_scf)
        if timed_stages:
            etics.set_stage_events(rev.handles(5, 11))
        etics.mex_field(x, L_MAX, out=out_mex, ws=ws_mex)
        if timed_stages:
            etics.set_stage_events(None)

    # the two methods are independent: MEX (the longer chain) runs on a
    # high-priority stream and SCF on a normal one, so SCF's compute-bound
    # kernels fill the issue slots that MEX's latency-bound sort and scan
    # phases leave idle without delaying MEX's blocks
    side = torch.cuda.Stream(device=dev)
    hi = torch.cuda.Stream(device=dev, priority=-1)

    def step_concurrent():
        side.wait_stream(stream)
        hi.wait_stream(stream)
        with torch.cuda.stream(hi):
            etics.mex_field(x, L_MAX, out=out_mex, ws=ws_mex)
        with torch.cuda.stream(side):
            etics.scf_coeffs(x, N_MAX, L_MAX, out=coeffs, ws=ws_scf)
            etics.scf_field(x, coeffs, N_MAX, L_MAX, out=out_scf)
        stream.wait_stream(side)
        stream.wait_stream(hi)

    for _ in range(args.warmup):
        step()
        step_concurrent()
    torch.cuda.synchronize()
    etics.check_error()
    # the FP32 / FP64 FMA rates of this GPU, measured now (the roofline's
    # denominators for the arithmetic-bound kernels)
    peak_clocks = Clocks(local)
    peak_clocks.start()
    peaks_meas = measure_fma_peaks(dev)
    peaks_meas["clocks"] = peak_clocks.stop()

    clocks = Clocks(local)
    times, stage = [], {k: [] for k in ("coef_kernel", "finalize", "field_kernel", "mex_keys",
                                         "mex_sort", "mex_tile_sums", "mex_carry", "mex_pass2",
                                         "scf", "mex")}
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = etics.launch_count()
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1)                    # L2 flushed between timed steps
        t_start.record(stream)
        step_concurrent()
        t_end.record(stream)
        torch.cuda.synchronize()
        times.append(t_start.elapsed_time(t_end))
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = etics.launch_count() - l0
    if dist:
        dist.barrier()
    # per-kernel times: the same step with the two methods one after the other
    # on one stream, stage events between the kernels
    serial = []
    for _ in range(args.steps):
        flush.fill_(1)
        t_start.record(stream)
        step(timed_stages=True)
        t_end.record(stream)
        torch.cuda.synchronize()
        serial.append(t_start.elapsed_time(t_end))
        stage["coef_kernel"].append(rev.ms(0, 1))
        stage["finalize"].append(rev.ms(1, 2))
        stage["field_kernel"].append(rev.ms(3, 4))
        stage["scf"].append(rev.ms(0, 4))
        stage["mex_keys"].append(rev.ms(5, 6))
        stage["mex_sort"].append(rev.ms(6, 7))
        stage["mex_tile_sums"].append(rev.ms(7, 8))
        stage["mex_carry"].append(rev.ms(8, 9))
        stage["mex_pass2"].append(rev.ms(9, 10))
        stage["mex"].append(rev.ms(5, 10))
    # each method as one call with no events between its kernels (the stage
    # events above sit between the launches of a call and keep them from
    # overlapping): the per-method times and the SCF pass's roofline
    method = {"scf": [], "mex": []}
    for _ in range(args.steps):
        flush.fill_(1)
        t_start.record(stream)
        etics.scf_coeffs(x, N_MAX, L_MAX, out=coeffs, ws=ws_scf)
        etics.scf_field(x, coeffs, N_MAX, L_MAX, out=out_scf)
        t_end.record(stream)
        torch.cuda.synchronize()
        method["scf"].append(t_start.elapsed_time(t_end))
        flush.fill_(1)
        t_start.record(stream)
        etics.mex_field(x, L_MAX, out=out_mex, ws=ws_mex)
        t_end.record(stream)
        torch.cuda.synchronize()
        method["mex"].append(t_start.elapsed_time(t_end))
    etics.check_error()
    ms = max_over_ranks(statistics.mean(times), dist, dev)
    serial_ms = max_over_ranks(statistics.mean(serial), dist, dev)
    value = job_throughput(2 * n, world, ms)

    # ---- e2e: host (pinned) buffers through the public API ------------------
    host_in = torch.tensor(pm, dtype=torch.float32).pin_memory()
    host_scf = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    host_mex = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    dx = torch.empty_like(x)

    def e2e_step():
        dx.copy_(host_in, non_blocking=True)
        side.wait_stream(stream)
        hi.wait_stream(stream)
        with torch.cuda.stream(hi):
            etics.mex_field(dx, L_MAX, out=out_mex, ws=ws_mex)
            host_mex.copy_(out_mex, non_blocking=True)
        with torch.cuda.stream(side):
            etics.scf_coeffs(dx, N_MAX, L_MAX, out=coeffs, ws=ws_scf)
            etics.scf_field(dx, coeffs, N_MAX, L_MAX, out=out_scf)
            host_scf.copy_(out_scf, non_blocking=True)      # overlaps MEX
        stream.wait_stream(side)
        stream.wait_stream(hi)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1)
        t_start.record(stream)
        e2e_step()
        t_end.record(stream)
        torch.cuda.synchronize()
        e2e_t.append(t_start.elapsed_time(t_end))
    e2e_ms = max_over_ranks(statistics.mean(e2e_t), dist, dev)

    # ---- FP64 GPU path (same particles), a few steps -------------------------
    ws64s = etics.workspace(n, N_MAX, L_MAX, etics.SCF, etics.FP64, dev)
    ws64m = etics.workspace(n, 0, L_MAX, etics.MEX, etics.FP64, dev)
    o64 = torch.empty_like(x64)
    c64 = torch.empty_like(coeffs)
    def step64():
        etics.scf_coeffs(x64, N_MAX, L_MAX, out=c64, ws=ws64s)
        etics.scf_field(x64, c64, N_MAX, L_MAX, out=o64)
        t_mid.record(stream)
        etics.mex_field(x64, L_MAX, out=o64, ws=ws64m)
    t_mid = torch.cuda.Event(enable_timing=True)
    step64()
    torch.cuda.synchronize()
    f64_scf, f64_mex = [], []
    for _ in range(3):
        flush.fill_(1)
        t_start.record(stream)
        step64()
        t_end.record(stream)
        torch.cuda.synchronize()
        f64_scf.append(t_start.elapsed_time(t_mid))
        f64_mex.append(t_mid.elapsed_time(t_end))
    etics.check_error()

    result = None
    if rank == 0:
        result = {"ms": ms, "value": value, "stage": {k: statistics.mean(v) for k, v in stage.items()},
                  "method": {k: statistics.mean(v) for k, v in method.items()},
                  "launches": launches, "clocks": clk, "e2e_ms": e2e_ms, "serial_ms": serial_ms,
                  "f64": (statistics.mean(f64_scf), statistics.mean(f64_mex)),
                  "peaks": peaks_meas,
                  "out_scf": out_scf, "out_mex": out_mex, "x": x}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return result


def eps_stats(a, r):
    """median / p99 / max of eq. 23's relative force error |a - r| / |r|."""
    e = np.linalg.norm(a - r, axis=1) / np.linalg.norm(r, axis=1)
    return {"median": float(np.median(e)), "p99": float(np.quantile(e, 0.99)),
            "max": float(e.max()), "sample": int(len(e))}


def accuracy(x, out_scf, out_mex, sample=65536, seed=0):
    """eps~ of eq. 23 (Sec. 4.2) of the mixed path's forces:
      * against the FP64 oracle at the same (FP32-rounded) positions: SCF
        coefficients by the oracle from all N particles, its field on a
        seeded sample of `sample` particles; MEX by the oracle over all N
        particles (its field at a particle depends on every other), every
        particle compared;
      * against the library's FP64 GPU path at the same positions (every
        particle), which the parity tests tie to the oracle.
    The oracle runs on all host cores."""
    import oracle
    from paper_1406_4254_gb300 import etics
    xr = x.double()
    c = etics.scf_coeffs(xr, N_MAX, L_MAX)
    a_scf = etics.scf_field(xr, c, N_MAX, L_MAX)
    a_mex = etics.mex_field(xr, L_MAX)
    etics.check_error()
    pm = xr.cpu().numpy()
    o_scf = out_scf.double().cpu().numpy()[:, :3]
    o_mex = out_mex.double().cpu().numpy()[:, :3]
    t0 = time.perf_counter()
    c_or = oracle.scf_coeffs(pm[:, :3], pm[:, 3], N_MAX, L_MAX)
    idx = np.sort(np.random.default_rng(seed).choice(len(pm), min(sample, len(pm)),
                                                      replace=False))
    a_or, _ = oracle.scf_field(pm[idx, :3], N_MAX, L_MAX, c_or)
    t1 = time.perf_counter()
    m_or, _, _ = oracle.mex_field(pm[:, :3], pm[:, 3], L_MAX)
    t2 = time.perf_counter()
    scf = eps_stats(o_scf[idx], a_or)
    scf["what"] = (f"oracle coefficients from all {len(pm)} particles, field at "
                   f"{len(idx)} sampled particles")
    mex = eps_stats(o_mex, m_or)
    mex["what"] = f"oracle over all {len(pm)} particles, every particle compared"
    return {"vs_oracle": {"reference": "FP64 CPU oracle at the same positions",
                          "scf": scf, "mex": mex,
                          "oracle_seconds": {"scf": t1 - t0, "mex": t2 - t1},
                          "oracle_threads": oracle.default_threads()},
            "vs_fp64_gpu": {"reference": "the library's FP64 GPU path at the same positions",
                            "scf": eps_stats(o_scf, a_scf.cpu().numpy()[:, :3]),
                            "mex": eps_stats(o_mex, a_mex.cpu().numpy()[:, :3])}}


def oracle_step_time(pm_sample, nthreads=0):
    """Wall time of one oracle SCF (coeffs + field) and one MEX calculation
    on `nthreads` host threads (0 = all): the SCF coefficient sum in fixed
    particle chunks, the field loops per particle, MEX's moments and field
    terms per particle between serial cumulative sums."""
    import oracle
    x, m = pm_sample[:, :3], pm_sample[:, 3]
    t0 = time.perf_counter()
    c = oracle.scf_coeffs(x, m, N_MAX, L_MAX, nthreads=nthreads)
    oracle.scf_field(x, N_MAX, L_MAX, c, nthreads=nthreads)
    t1 = time.perf_counter()
    oracle.mex_field(x, m, L_MAX, nthreads=nthreads)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def cpu_baseline(n, n_single, seed=0):
    """The oracle on the host cores: one full step of the workload itself
    (all N particles) on all cores, and a sample of n_single particles on
    one core (the paper quotes one-core CPU figures, Sec. 3.4)."""
    import oracle
    from paper_1406_4254_gb300 import inputs
    pm = inputs.hernquist(n, seed=seed, axes=(1.0, 0.8, 0.6)).astype(np.float32).astype(np.float64)
    ts, tm = oracle_step_time(pm)
    t1 = sum(oracle_step_time(pm[:n_single], nthreads=1))
    return {"value": 2 * n / (ts + tm), "unit": UNIT, "cores": oracle.default_threads(),
            "kind": "oracle",
            "sample": (f"one step over all {n} particles of the workload (SCF {ts:.2f} s, "
                       f"MEX {tm:.2f} s) on all cores"),
            "single_core": {"value": 2 * n_single / t1, "unit": UNIT, "cores": 1,
                            "sample": f"{n_single} particles of the workload"}}


def run_leapfrog(args):
    """Plummer sphere (b = 1, AHW74 velocities), N = 2^20, SCF (10, 6), 100
    kick-drift-kick steps at dt = 0.01 (the paper's integrator, Secs. 3.4 and
    5.4), each step one CUDA-graph replay of etics_leapfrog_step.  Reports the
    energy drift |dE/E0| of the mixed and FP64 paths and, every 10th step, the
    relative force error (eq. 23) of the mixed path against the FP64 oracle
    and against the library's
    FP64 path at the same positions (coefficients from all particles, field
    on a 16384-particle sample)."""
    import torch
    from paper_1406_4254_gb300 import etics, inputs
    dev = torch.device("cuda", 0)
    n = args.n
    steps, dt, check_every = args.lf_steps, 0.01, 10
    pm, vel = inputs.plummer(n, seed=args.seed)
    v4 = np.zeros((n, 4))
    v4[:, :3] = vel
    res = {}
    for label, dtype in (("mixed", torch.float32), ("fp64", torch.float64)):
        x = torch.tensor(pm, dtype=dtype, device=dev)
        v = torch.tensor(v4, dtype=dtype, device=dev)
        prec = etics.MIXED if dtype == torch.float32 else etics.FP64
        extra = ((N_MAX + 1) * (L_MAX + 1) ** 2 * 8 + 255) // 256 * 256
        ws = torch.empty(etics.workspace_bytes(n, N_MAX, L_MAX, etics.SCF, prec) + extra + 256,
                         dtype=torch.uint8, device=dev)
        acc, _ = etics.scf_force(x, N_MAX, L_MAX)
        m = x[:, 3].double()

        def energy():
            kin = 0.5 * (m * (v[:, :3].double() ** 2).sum(1)).sum()
            return float(kin + 0.5 * (m * acc[:, 3].double()).sum())

        e0 = energy()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        # a throwaway copy warms up the library on the side stream
        xs, vs, accs = x.clone(), v.clone(), acc.clone()
        with torch.cuda.stream(side):
            etics.leapfrog_step(xs, vs, accs, dt, etics.SCF, N_MAX, L_MAX, ws=ws)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            etics.leapfrog_step(x, v, acc, dt, etics.SCF, N_MAX, L_MAX, ws=ws)
        errs, times = [], []
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for step in range(1, steps + 1):
            t0.record()
            graph.replay()
            t1.record()
            torch.cuda.synchronize()
            times.append(t0.elapsed_time(t1))
            if label == "mixed" and step % check_every == 0 and not args.no_accuracy:
                # eq. 23 against the FP64 oracle at the same positions:
                # coefficients from all particles, field on a 16384 sample;
                # and against the library's FP64 GPU path (same sample)
                import oracle
                xp = x.double()
                pm_now = xp.cpu().numpy()
                idx_np = np.sort(np.random.default_rng(step).choice(n, 16384, replace=False))
                c_or = oracle.scf_coeffs(pm_now[:, :3], pm_now[:, 3], N_MAX, L_MAX)
                a_or, _ = oracle.scf_field(pm_now[idx_np, :3], N_MAX, L_MAX, c_or)
                idx = torch.tensor(idx_np, device=dev)
                c = etics.scf_coeffs(xp, N_MAX, L_MAX)
                a_ref = etics.scf_field(xp[idx].contiguous(), c, N_MAX, L_MAX)
                a_ref = a_ref.cpu().numpy()[:, :3]
                a = acc.double()[idx].cpu().numpy()[:, :3]
                errs.append({"step": step, "vs_oracle": eps_stats(a, a_or),
                             "vs_fp64_gpu": eps_stats(a, a_ref)})
        etics.check_error()
        e1 = energy()
        ms = statistics.mean(times)
        res[label] = {"ms_per_step": ms, "particle_steps_per_s": n / (ms * 1e-3),
                      "energy_drift": abs(e1 / e0 - 1.0), "E0": e0, "E_end": e1}
        if errs:
            res[label]["force_error"] = errs
    return {"experiment": "leapfrog", "workload": f"plummer b=1 N={n} SCF(10,6) "
            f"{steps} KDK steps dt={dt}, graph-captured step", **res}


def run_batch(args):
    """256 independent Hernquist systems (N log-uniform in [2^12, 2^18], n_max
    in 6..14, l_max in 2..8, system i seeded with i): SCF coefficients and
    field of all systems in one graph-captured etics_scf_batch (three kernel
    nodes) with the autotuned launch shape, against one coefficient + one
    field call per system."""
    import torch
    from paper_1406_4254_gb300 import autotune, etics
    pm, sizes, nm, lm = autotune.ensemble(seed=args.seed)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    ntot = int(sum(sizes))
    tuning = autotune.lookup(nm, lm, sizes)
    tuned_now = False
    if tuning is None:
        best, _ = autotune.tune(x, sizes, nm, lm, reps=3, write=False)
        tuning = etics.BatchTuning(best["tile"], best["blocks_per_sm"], best["field_threads"],
                                   best["field_chunk"])
        tuned_now = True
    plan = etics.BatchPlan(sizes, nm, lm, tuning=tuning)
    coeffs = torch.empty(plan.coeff_count, dtype=torch.float64, device="cuda")
    out = torch.empty_like(x)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        etics.scf_batch(x, plan, coeffs=coeffs, out=out)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        etics.scf_batch(x, plan, coeffs=coeffs, out=out)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tb = []
    for _ in range(args.steps):
        t0.record()
        graph.replay()
        t1.record()
        torch.cuda.synchronize()
        tb.append(t0.elapsed_time(t1))
    # one call per system
    views = [x[plan.particle_offsets[i]:plan.particle_offsets[i + 1]] for i in range(len(sizes))]
    cs = [torch.empty((nm[i] + 1, (lm[i] + 1) ** 2), dtype=torch.float64, device="cuda")
          for i in range(len(sizes))]
    outs = [torch.empty_like(v) for v in views]
    ws = etics.workspace(max(sizes), 14, 8, etics.SCF, etics.MIXED)

    def loop():
        for i in range(len(sizes)):
            etics.scf_coeffs(views[i], nm[i], lm[i], out=cs[i], ws=ws)
            etics.scf_field(views[i], cs[i], nm[i], lm[i], out=outs[i])

    for _ in range(2):
        loop()
    torch.cuda.synchronize()
    tl = []
    for _ in range(max(3, args.steps // 2)):
        t0.record()
        loop()
        t1.record()
        torch.cuda.synchronize()
        tl.append(t0.elapsed_time(t1))
    # the same per-system calls captured into one graph (launch overhead removed)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2):
        loop()
    for _ in range(2):
        g2.replay()
    torch.cuda.synchronize()
    tg = []
    for _ in range(max(3, args.steps // 2)):
        t0.record()
        g2.replay()
        t1.record()
        torch.cuda.synchronize()
        tg.append(t0.elapsed_time(t1))
    # the plain FP64-GPU form: the same systems through the FP64 per-system
    # calls (eager and graph-captured) and through an FP64 batch
    x64 = x.double()
    views64 = [x64[plan.particle_offsets[i]:plan.particle_offsets[i + 1]]
               for i in range(len(sizes))]
    cs64 = [torch.empty_like(c) for c in cs]
    outs64 = [torch.empty_like(v) for v in views64]
    ws64 = etics.workspace(max(sizes), 14, 8, etics.SCF, etics.FP64)

    def loop64():
        for i in range(len(sizes)):
            etics.scf_coeffs(views64[i], nm[i], lm[i], out=cs64[i], ws=ws64)
            etics.scf_field(views64[i], cs64[i], nm[i], lm[i], out=outs64[i])

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0.record()
            fn()
            t1.record()
            torch.cuda.synchronize()
            ts.append(t0.elapsed_time(t1))
        return statistics.mean(ts)

    t64_eager = timed(loop64, max(3, args.steps // 2))
    g3 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g3):
        loop64()
    t64_graph = timed(g3.replay, max(3, args.steps // 2))
    plan64 = etics.BatchPlan(sizes, nm, lm, precision=etics.FP64)
    coeffs64b = torch.empty(plan64.coeff_count, dtype=torch.float64, device="cuda")
    out64b = torch.empty_like(x64)
    with torch.cuda.stream(side):
        etics.scf_batch(x64, plan64, coeffs=coeffs64b, out=out64b)
    torch.cuda.current_stream().wait_stream(side)
    g4 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g4):
        etics.scf_batch(x64, plan64, coeffs=coeffs64b, out=out64b)
    t64_batch = timed(g4.replay, max(3, args.steps // 2))
    etics.check_error()
    # eq. 23 force error of the batched mixed-precision forces against the
    # FP64 per-system forces, every particle of every system
    a_mixed = out[:, :3].double().cpu().numpy()
    a_fp64 = torch.cat(outs64)[:, :3].cpu().numpy()
    acc_vs_fp64 = eps_stats(a_mixed, a_fp64)
    # agreement of the two paths
    err = 0.0
    for i in range(0, len(sizes), 17):
        a = plan.coeffs_of(coeffs, i).cpu().numpy()
        b = cs[i].cpu().numpy()
        err = max(err, float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
    mb, ml = statistics.mean(tb), statistics.mean(tl)
    return {"experiment": "batch", "workload": f"{len(sizes)} Hernquist systems, N log-uniform "
            f"[2^12, 2^18] (total {ntot}), n_max 6..14, l_max 2..8", "total_particles": ntot,
            "batched_graph": {"ms": mb, "particle_forces_per_s": ntot / (mb * 1e-3),
                              "kernel_launches": 3},
            "one_call_per_system": {"ms": ml, "particle_forces_per_s": ntot / (ml * 1e-3),
                                    "kernel_launches": 3 * len(sizes)},
            "one_call_per_system_graph": {"ms": statistics.mean(tg),
                                          "particle_forces_per_s": ntot / (statistics.mean(tg) * 1e-3)},
            "fp64_one_call_per_system": {"ms": t64_eager,
                                         "particle_forces_per_s": ntot / (t64_eager * 1e-3)},
            "fp64_one_call_per_system_graph": {"ms": t64_graph,
                                               "particle_forces_per_s": ntot / (t64_graph * 1e-3)},
            "fp64_batched_graph": {"ms": t64_batch, "particle_forces_per_s": ntot / (t64_batch * 1e-3)},
            "speedup_vs_fp64_calls": t64_eager / mb, "speedup_vs_fp64_graph_of_calls": t64_graph / mb,
            "batched_mixed_force_error_vs_fp64_calls": acc_vs_fp64,
            "speedup": ml / mb, "speedup_vs_graph_of_calls": statistics.mean(tg) / mb,
            "tuning": tuning.as_dict(), "tuned_in_this_run": tuned_now,
            "max_rel_coeff_diff_batched_vs_single": err}


def run_surrogate(args):
    """Surrogate-accelerated SCF: a Hernquist sphere with a 5% l = 2, m = 2
    bar perturbation (N = 2^26 by default), SCF (14, 8), KDK at dt = 0.005.
    A plain-SCF run of --sur-steps steps produces the coefficient trajectory;
    on its first 75% the library's kernels fit, for each coefficient and each
    horizon k = 1..S (S = --sur-stride), a linear predictor of the vector k
    steps after a history of eight true vectors spaced S apart (least
    squares, FP64), and train the per-coefficient MLP (8 -> 256 -> 256 -> S,
    bf16 weights, FP32 accumulation) on what those miss; both are validated
    on the rest.  From the final state four continuations of --sur-eval steps
    are timed: plain SCF every step; the coefficient pass on every S-th step
    only and the forecast on the others (judging, on each recompute step, the
    forecast it would have used against the force-error budget: median <=
    1e-5, 99th percentile <= 1e-4, on 4096 particles; a miss makes the next
    block plain SCF); the same with the fitted predictors alone (no network);
    and plain reuse of the last coefficients on the other steps (judged the
    same way).  An
    untimed pass then measures each forecast step's relative force error (eq. 23)
    against plain SCF at the same positions on a 65536-particle sample."""
    import torch
    from paper_1406_4254_gb300 import etics, inputs, surrogate
    dev = torch.device("cuda", 0)
    n, n_max, l_max, dt = args.sur_n, 14, 8, 0.005
    t0 = time.time()
    pm, vel = inputs.hernquist_bar(n, seed=args.seed, eps=0.05)
    t_ic = time.time() - t0
    x = torch.tensor(pm, dtype=torch.float32, device=dev)
    v = torch.zeros_like(x)
    v[:, :3] = torch.tensor(vel, dtype=torch.float32, device=dev)
    del pm, vel
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    traj, acc = surrogate.coefficient_trajectory(x, v, args.sur_steps, dt, n_max, l_max)
    ev1.record()
    torch.cuda.synchronize()
    ms_traj = ev0.elapsed_time(ev1) / args.sur_steps
    T = traj.shape[0]
    n_train = int(0.75 * T)
    S = args.sur_stride
    fc = surrogate.Forecaster(n_max, l_max, stride=S, hidden=256, seed=args.seed)
    ev0.record()
    losses = fc.fit(traj[:n_train], iters=args.sur_iters, batch=16, lr=1e-3, seed=args.seed,
                    log_every=max(1, args.sur_iters // 10))
    ev1.record()
    torch.cuda.synchronize()
    ms_train = ev0.elapsed_time(ev1)
    he = fc.horizon_errors(traj, n_train)
    med = lambda a: float(np.median(a))  # noqa: E731
    m = x[:, 3].double()

    def energy(vv, aa):
        return float(0.5 * (m * (vv[:, :3].double() ** 2).sum(1)).sum()
                     + 0.5 * (m * aa[:, 3].double()).sum())

    modes = {}
    for mode in ("plain", "forecast", "fitted", "hold"):
        xs, vs, accs = x.clone(), v.clone(), acc.clone()
        fc.reset(traj)
        e0 = energy(vs, accs)
        torch.cuda.synchronize()
        ev0.record()
        if mode == "plain":
            for _ in range(args.sur_eval):
                etics.leapfrog_step(xs, vs, accs, dt, etics.SCF, n_max, l_max)
            st = None
        else:
            st = surrogate.run(xs, vs, accs, args.sur_eval, dt, fc, mode=mode)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.sur_eval
        modes[mode] = {"ms_per_step": ms, "particle_steps_per_s": n / (ms * 1e-3),
                       "energy_drift": abs(energy(vs, accs) / e0 - 1.0)}
        if st is not None:
            modes[mode].update({"recomputes": st.recomputes, "forecast_steps": st.forecasts,
                                "fallback_blocks": st.fallbacks,
                                "checks": len(st.checks),
                                "check_frac_above_median_budget": med([c[1] for c in st.checks])
                                if st.checks else None,
                                "check_frac_above_p99_budget": med([c[2] for c in st.checks])
                                if st.checks else None})
        del xs, vs, accs
    for mode in ("forecast", "fitted", "hold"):
        modes[mode]["speedup_vs_plain"] = modes["plain"]["ms_per_step"] / modes[mode]["ms_per_step"]
    # untimed accuracy pass: every substep against plain SCF at the same positions
    s_n = min(65536, n)
    for mode in ("forecast", "fitted", "hold"):
        xs, vs, accs = x.clone(), v.clone(), acc.clone()
        fc.reset(traj)
        per_sub = {k: [] for k in range(1, S)}
        a_ref = torch.empty((s_n, 4), dtype=torch.float32, device=dev)
        a_use = torch.empty_like(a_ref)

        def hook(t, kind, c_use, hz):
            if kind == "recompute":
                return
            c_true = etics.scf_coeffs(xs, n_max, l_max)
            etics.scf_field(xs[:s_n], c_true, n_max, l_max, out=a_ref)
            etics.scf_field(xs[:s_n], c_use.view(n_max + 1, -1), n_max, l_max, out=a_use)
            a = a_use.double().cpu().numpy()[:, :3]
            r = a_ref.double().cpu().numpy()[:, :3]
            e = np.linalg.norm(a - r, axis=1) / np.linalg.norm(r, axis=1)
            per_sub[hz].append((float(np.median(e)), float(np.quantile(e, 0.99)),
                                float(e.max())))

        surrogate.run(xs, vs, accs, min(args.sur_eval, 200), dt, fc, mode=mode, hook=hook)
        modes[mode]["force_error_by_substep"] = {
            str(k): {"median": med([p[0] for p in v_]), "p99": med([p[1] for p in v_]),
                     "max": float(max(p[2] for p in v_)), "samples": len(v_)}
            for k, v_ in per_sub.items() if v_}
        del xs, vs, accs
    # split of the plain step: coefficient pass vs field pass at the final state
    c_fin = etics.scf_coeffs(x, n_max, l_max)
    for _ in range(2):
        etics.scf_field(x, c_fin, n_max, l_max, out=acc)
    ev0.record()
    for _ in range(5):
        etics.scf_coeffs(x, n_max, l_max, out=c_fin)
    ev1.record()
    torch.cuda.synchronize()
    ms_coef = ev0.elapsed_time(ev1) / 5
    ev0.record()
    for _ in range(5):
        etics.scf_field(x, c_fin, n_max, l_max, out=acc)
    ev1.record()
    torch.cuda.synchronize()
    ms_field = ev0.elapsed_time(ev1) / 5
    # the plain FP64 form for reference (a few steps)
    x64, v64 = x.double(), v.double()
    acc64, _ = etics.scf_force(x64, n_max, l_max)
    k64 = 3
    ev0.record()
    for _ in range(k64):
        etics.leapfrog_step(x64, v64, acc64, dt, etics.SCF, n_max, l_max)
    ev1.record()
    torch.cuda.synchronize()
    ms64 = ev0.elapsed_time(ev1) / k64
    etics.check_error()
    return {"experiment": "surrogate",
            "workload": f"hernquist + 5% l=2 m=2 bar, N={n}, SCF(14,8), KDK dt={dt}",
            "trajectory": {"steps": args.sur_steps, "plain_ms_per_step": ms_traj,
                           "initial_conditions_s": t_ic},
            "training": {"network": f"per-coefficient 8->256->256->{S}, tanh, bf16 x bf16 -> FP32",
                         "train_vectors": n_train, "iters": args.sur_iters,
                         "histories_per_batch": 16, "ms": ms_train, "loss_log": losses},
            "horizon_error_validation": {
                str(k): {"hold": med(d["hold"]), "cubic": med(d["cubic"]),
                         "fitted_linear_predictor": med(d["fitted"]), "fitted_plus_mlp": med(d["net"])}
                for k, d in he.items()} | {"unit": "|c_hat - c_{t+k}| / |c_{t+k} - c_t|, median"},
            "budget": {"median": 1e-5, "p99": 1e-4, "sample": 4096, "stride": S},
            "rollout_steps": args.sur_eval, "modes": modes,
            "plain_fp64": {"ms_per_step": ms64, "steps": k64},
            "plain_mixed_split_ms": {"coefficients": ms_coef, "field": ms_field}}


def run_accuracy(args):
    """Sec. 4.1's study: the relative force error eps_i = |F_i - F_real| / |F_real|
    (eq. 22) of MEX and SCF against the smooth force of the model the
    particles were drawn from, in FP64 as the paper did.  Models: the Ferrers
    n = 1 ellipsoids model1 (10:10:9) and model2 (3:2:1) of the paper, with
    their polynomial potential recomputed from the 1-D index-symbol
    integrals, and the closed-form Hernquist and Plummer spheres.  N from
    10^3 to 10^6; realisations are stacked up to 10^6 particles per point (at
    most 100).  MEX at even l_max = 0..10 (the paper's Figs. 8 and 9); SCF at
    l_max = 6 with n_max = 0..14 and at l_max = 10 with n_max = 6, 10, 14
    (the paper's Fig. 10 sweep, where SCF approaches MEX as n_max grows), and
    SCF in the Clutton-Brock basis (Plummer zeroth term) at l_max = 6.  The
    overlap of the log10(eps) histograms of SCF and MEX at the same l_max (6
    and 10) measures that approach."""
    import torch
    from paper_1406_4254_gb300 import etics, inputs, models
    dev = torch.device("cuda", 0)
    co = {"model1": models.ferrers_coefficients(models.MODEL1),
          "model2": models.ferrers_coefficients(models.MODEL2)}

    def sample(model, n, seed):
        if model in ("model1", "model2"):
            axes = models.MODEL1 if model == "model1" else models.MODEL2
            pm = models.ferrers(n, seed=seed, axes=axes)
            acc, _ = models.ferrers_force(pm[:, :3], axes, co[model])
        elif model == "hernquist":
            pm = inputs.hernquist(n, seed=seed)
            acc, _ = models.hernquist_force(pm[:, :3])
        else:
            pm, _ = inputs.plummer(n, seed=seed)
            acc, _ = models.plummer_force(pm[:, :3])
        return pm, acc

    methods = ([("mex", 0, l) for l in (0, 2, 4, 6, 8, 10)] +
               [("scf", n, 6) for n in (0, 2, 4, 6, 10, 14)] +
               [("scf", n, 10) for n in (6, 10, 14)] +
               [("scfcb", n, 6) for n in (0, 2, 6, 10)])
    bins = np.linspace(-9.0, 1.0, 101)
    out = {}
    for model in ("model1", "model2", "hernquist", "plummer"):
        out[model] = {}
        for n in args.acc_n:
            reps = max(1, min(100, 1000000 // n))
            errs = {m: [] for m in methods}
            for rep in range(reps):
                pm, a_real = sample(model, n, 1000 * rep + 17)
                x = torch.tensor(pm, dtype=torch.float64, device=dev)
                nr = np.linalg.norm(a_real, axis=1)
                for meth in methods:
                    kind, nm, lm = meth
                    if kind == "mex":
                        a = etics.mex_field(x, lm)
                    else:
                        a, _ = etics.scf_force(x, nm, lm, basis=etics.BASIS_CB
                                               if kind == "scfcb" else etics.BASIS_HO)
                    a = a.cpu().numpy()[:, :3]
                    errs[meth].append(np.linalg.norm(a - a_real, axis=1) / nr)
            etics.check_error()
            row = {}
            hist = {}
            for meth, es in errs.items():
                e = np.concatenate(es)
                key = f"mex_l{meth[2]}" if meth[0] == "mex" else f"{meth[0]}_n{meth[1]}_l{meth[2]}"
                row[key] = {"mean": float(e.mean()), "median": float(np.median(e)),
                            "p90": float(np.quantile(e, 0.9))}
                h, _ = np.histogram(np.log10(np.maximum(e, 1e-12)), bins=bins)
                hist[key] = h / max(1, h.sum())
            for lm in (6, 10):
                row[f"overlap_with_mex_l{lm}"] = {
                    k: float(np.minimum(hist[k], hist[f"mex_l{lm}"]).sum())
                    for k in hist if k.startswith("scf_") and k.endswith(f"_l{lm}")}
            row["realisations"] = reps
            out[model][str(n)] = row
    return {"experiment": "accuracy", "precision": "FP64",
            "error": "eps_i = |F_i - F_real| / |F_real| (eq. 22); mean, median and p90 over "
                     "all particles of all realisations",
            "models": {"model1": "Ferrers n=1, axes 10:10:9", "model2": "Ferrers n=1, axes 3:2:1",
                       "hernquist": "Hernquist a=1", "plummer": "Plummer b=1"},
            "results": out}


def run_gemm(args):
    """The MLP's bf16 product on the tcgen05 kernel at a size that fills the
    GPU: one layer K -> N over M rows (M = 16384, N = K = 4096 by default),
    y = x W + b.  The product kernel's time comes from the library's stage
    events around it; achieved = 2 M N K / that time, against the measured
    cuBLAS bf16 peak."""
    import torch
    from paper_1406_4254_gb300 import etics, surrogate
    dev = torch.device("cuda", 0)
    M, N, K = args.gemm_mnk
    net = surrogate.Mlp([K, N], seed=args.seed, device=dev)
    g = torch.Generator(device=dev).manual_seed(args.seed)
    x = torch.randn((M, K), generator=g, device=dev).to(torch.bfloat16)
    y = torch.empty((M, N), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        net.forward(x, y)
    torch.cuda.synchronize()
    rev = RawEvents(3)
    gemm_ms, epi_ms = [], []
    for _ in range(args.steps):
        etics.set_stage_events(rev.handles(0, 3))
        net.forward(x, y)
        etics.set_stage_events(None)
        torch.cuda.synchronize()
        gemm_ms.append(rev.ms(0, 1))
        epi_ms.append(rev.ms(1, 2))
    etics.check_error()
    peaks, src = load_peaks()
    ms = statistics.median(gemm_ms)
    tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
    # spot check against a float32 product of the same bf16 operands
    w = net.params_bf16[:K * N].view(K, N).float()
    idx = torch.randint(0, M, (64,), generator=g, device=dev)
    ref = x[idx].float() @ w + net.params[K * N:].view(1, N)
    err = float(((y[idx] - ref).abs().max() / ref.abs().max()).item())
    return {"experiment": "gemm", "kernel": "tc::gemm_tma_kernel (TMA operand ring, 128-byte swizzle, tcgen05.mma kind::f16, TMEM accumulator)",
            "M": M, "N": N, "K": K, "product_ms": ms, "epilogue_ms": statistics.median(epi_ms),
            "achieved_tflops": tf, "peak_tflops": peaks["bf16_tflops"],
            "frac": tf / peaks["bf16_tflops"], "peak_source": f"bf16_tflops of MEASURED_PEAKS.json ({src})",
            "max_rel_err_vs_fp32_product": err}


def run_sweep(args):
    """Shape sweeps of the paper's scaling study (Sec. 3.4, Fig. 5: time against N,
    l_max and n_max): SCF (coefficients + field) and MEX timed separately,
    mixed precision, on the flattened Hernquist model of the headline
    workload (the first N particles of one 2^24 realisation).  Each point is
    the median of 5 calls timed with CUDA events, L2 flushed before each; the
    SCF coefficient and field passes are also timed on their own.
      N in 2^14 .. 2^24 at (n_max, l_max) = (10, 6);
      l_max in 0..10 at N = 2^20, n_max = 10 (MEX up to its compiled limit 6);
      n_max in 0..16 at N = 2^20, l_max = 6 (SCF only).
    fp32_frac: algorithmic flop per particle (the counts of the headline
    kernels) x N / time, over the derived FP32 peak."""
    import torch
    from paper_1406_4254_gb300 import etics, inputs
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peak = fp32_peak_tflops() * 1e12
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nmax_all = 1 << 24
    xall = torch.tensor(inputs.hernquist(nmax_all, seed=args.seed, axes=(1.0, 0.8, 0.6)),
                        dtype=torch.float32, device=dev)

    def timed(fn, reps=5, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            t0.record()
            fn()
            t1.record()
            torch.cuda.synchronize()
            ts.append(t0.elapsed_time(t1))
        return statistics.median(ts)

    def point(n, n_max, l_max, scf=True, mex=True):
        x = xall[:n]
        out = torch.empty_like(x)
        res = {"N": n, "n_max": n_max, "l_max": l_max}
        if scf:
            coeffs = torch.empty((n_max + 1, (l_max + 1) ** 2), dtype=torch.float64, device=dev)
            ws = etics.workspace(n, n_max, l_max, etics.SCF, etics.MIXED, dev)
            ms = timed(lambda: (etics.scf_coeffs(x, n_max, l_max, out=coeffs, ws=ws),
                                etics.scf_field(x, coeffs, n_max, l_max, out=out)))
            mc = timed(lambda: etics.scf_coeffs(x, n_max, l_max, out=coeffs, ws=ws))
            mf = timed(lambda: etics.scf_field(x, coeffs, n_max, l_max, out=out))
            flop = scf_coeff_flops(n_max, l_max) + scf_field_flops(n_max, l_max)
            res.update(scf_ms=ms, scf_pf_per_s=n / (ms * 1e-3),
                       scf_fp32_frac=flop * n / (ms * 1e-3) / peak,
                       scf_coeff_ms=mc, scf_field_ms=mf)
        if mex and l_max <= MEX_L_LIMIT:
            ws = etics.workspace(n, 0, l_max, etics.MEX, etics.MIXED, dev)
            ms = timed(lambda: etics.mex_field(x, l_max, out=out, ws=ws))
            res.update(mex_ms=ms, mex_pf_per_s=n / (ms * 1e-3),
                       mex_fp32_frac=mex_flops(l_max) * n / (ms * 1e-3) / peak)
        return res

    sweep_n = [point(1 << k, N_MAX, L_MAX) for k in range(14, 25)]
    sweep_l = [point(1 << 20, N_MAX, l) for l in range(0, 11)]
    sweep_nmax = [point(1 << 20, nm, L_MAX, mex=False) for nm in range(0, 17)]
    etics.check_error()
    return {"experiment": "sweep", "workload": "hernquist-1:0.8:0.6, first N of a 2^24 "
            "realisation, mixed precision", "fp32_peak_tflops": peak * 1e-12,
            "fp32_peak_note": FP32_PEAK_NOTE, "N": sweep_n, "l_max": sweep_l, "n_max": sweep_nmax}


def run_coeffprec(args):
    """Precision of the mixed coefficient passes against the FP64 paths
    (Sec. 2.4 eq. 18 coefficients; the mixed path accumulates FP32 products in
    FP64 blocks): max |c_mixed - c_fp64| / max |c_fp64| and the largest
    deviations with their (n, l, m), for the bar-perturbed Hernquist model at
    N = 2^20 .. 2^26 and (n_max, l_max) = (10, 6) and (14, 8), both at the
    same FP32-rounded positions; at N <= 2^22 also both against the FP64
    oracle."""
    import torch
    import oracle
    from paper_1406_4254_gb300 import etics, inputs
    out = {"experiment": "coeffprec", "model": "hernquist + 5% l=2,m=2 bar (seed 3)", "rows": []}
    for k in (20, 22, 24, 26):
        n = 1 << k
        pm, _ = inputs.hernquist_bar(n, seed=3, eps=0.05, velocities=False)
        pm32 = pm.astype(np.float32)
        del pm
        x = torch.tensor(pm32, device="cuda")
        for nm, lm in ((10, 6), (14, 8)):
            c32 = etics.scf_coeffs(x, nm, lm).cpu().numpy()
            c64 = etics.scf_coeffs(x.double(), nm, lm).cpu().numpy()
            scale = float(np.max(np.abs(c64)))
            dev = np.abs(c32 - c64)
            top = []
            for f in np.argsort(dev.ravel())[::-1][:3]:
                nn, j = divmod(int(f), c64.shape[1])
                l = int(np.sqrt(j))
                top.append({"n": nn, "l": l, "m": j - l * l - l, "dev": float(dev[nn, j]),
                            "c_fp64": float(c64[nn, j])})
            row = {"N": n, "n_max": nm, "l_max": lm, "max_dev_over_max_c": float(dev.max()) / scale,
                   "largest": top}
            if k <= 22:
                p64 = pm32.astype(np.float64)
                cor = oracle.scf_coeffs(p64[:, :3], p64[:, 3], nm, lm)
                row["fp64_vs_oracle"] = float(np.max(np.abs(c64 - cor))) / scale
                row["mixed_vs_oracle"] = float(np.max(np.abs(c32 - cor))) / scale
            out["rows"].append(row)
        etics.check_error()
        del x
        torch.cuda.empty_cache()
    return out


def run_peaks(args):
    """FP32 and FP64 FMA rates of the GPU (the roofline denominators of the
    arithmetic-bound kernels), from etics_fma_peak: as a burst (best of 5
    launches of ~5 ms, what a kernel timed inside a short step sees) and
    sustained (back-to-back launches of ~50 ms for ~3 s, median), with the SM
    clocks sampled during each.  Nothing about the GPU's clocks or power
    settings is changed."""
    import torch
    from paper_1406_4254_gb300 import etics
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"experiment": "peaks", "sms": sms, "derived_fp32_tflops": fp32_peak_tflops(),
           "derived_note": FP32_PEAK_NOTE, "burst": {}, "sustained": {}}
    clk = Clocks(0)
    clk.start()
    out["burst"] = measure_fma_peaks(dev)
    out["burst"]["clocks"] = clk.stop()
    blocks = sms * 4
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, kind in (("ffma", etics.PEAK_FFMA), ("ffma2", etics.PEAK_FFMA2),
                       ("dfma", etics.PEAK_DFMA)):
        # calibrate a ~50 ms launch
        iters = 256
        e0.record()
        etics.fma_peak(kind, blocks, iters, sink)
        e1.record()
        torch.cuda.synchronize()
        iters = max(1, int(iters * 50.0 / max(e0.elapsed_time(e1), 1e-3)))
        clk = Clocks(0)
        clk.start()
        rates, t_end = [], time.perf_counter() + 3.0
        while time.perf_counter() < t_end:
            e0.record()
            flops = etics.fma_peak(kind, blocks, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            rates.append(flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out["sustained"][name] = statistics.median(rates)
        out["sustained"][name + "_clocks"] = clk.stop()
    etics.check_error()
    return out


def emit(obj):
    print(json.dumps(obj), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["etics", "reference"], default="etics")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=65536)
    ap.add_argument("--experiment", choices=["leapfrog", "batch", "surrogate", "accuracy", "gemm",
                                             "sweep", "peaks", "coeffprec"],
                    default=None)
    ap.add_argument("--gemm-mnk", type=int, nargs=3, default=[16384, 4096, 4096])
    ap.add_argument("--acc-n", type=int, nargs="+", default=[1000, 10000, 100000, 1000000])
    ap.add_argument("--lf-steps", type=int, default=100)
    ap.add_argument("--sur-n", type=int, default=1 << 26)
    ap.add_argument("--sur-steps", type=int, default=2000)
    ap.add_argument("--sur-eval", type=int, default=400)
    ap.add_argument("--sur-iters", type=int, default=3000)
    ap.add_argument("--sur-stride", type=int, default=3)
    args = ap.parse_args()
    if args.experiment == "surrogate":
        emit(run_surrogate(args))
        return
    if args.experiment == "accuracy":
        emit(run_accuracy(args))
        return
    if args.experiment == "gemm":
        emit(run_gemm(args))
        return
    if args.experiment == "leapfrog":
        emit(run_leapfrog(args))
        return
    if args.experiment == "batch":
        emit(run_batch(args))
        return
    if args.experiment == "sweep":
        emit(run_sweep(args))
        return
    if args.experiment == "peaks":
        emit(run_peaks(args))
        return
    if args.experiment == "coeffprec":
        emit(run_coeffprec(args))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    cfg = {"workload": workload_name(args.n), "N": args.n, "n_max": N_MAX, "l_max": L_MAX,
           "methods": "SCF+MEX per step", "precision": "mixed (FP32 arithmetic, FP64 reductions)",
           "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) between timed steps"}

    if args.impl == "reference":
        if rank != 0:
            return
        n_s = 65536
        from paper_1406_4254_gb300 import inputs
        pm = inputs.hernquist(n_s, seed=0, axes=(1.0, 0.8, 0.6))
        for _ in range(args.warmup):
            oracle_step_time(pm)
        times = [sum(oracle_step_time(pm)) for _ in range(args.steps)]
        import oracle
        t = statistics.mean(times)
        v = 2 * n_s / t
        emit({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
              "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
              "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.default_threads(),
                               "kind": "oracle",
                               "sample": f"{n_s} particles of the workload per step"},
              "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": 0}})
        return

    res = run_etics(args, rank, world)
    if rank != 0:
        return
    peaks, src = load_peaks()
    n = args.n
    st = res["stage"]
    # every timed kernel against the roofline that bounds it; the dominant one
    # (largest share of the step) is the headline roofline.  The FP32 peak is
    # the rate measured in this run (FMA-chain microbenchmark); the figure
    # derived from unit counts and the maximum clock is kept beside it.
    pk = res["peaks"]
    fp32_peak = pk["fp32"]
    fp32_derived = fp32_peak_tflops()
    traffic = kernel_traffic()
    kern = {
        "scf_coeff_pairs_kernel": ("alu", st["coef_kernel"], scf_coeff_flops(N_MAX, L_MAX)),
        "scf_field_kernel": ("alu", st["field_kernel"], scf_field_flops(N_MAX, L_MAX)),
        "mex_pass2_kernel": ("alu", st["mex_pass2"], mex_flops(L_MAX)),
        "mex_sort (keys + 4 radix passes + ties)": ("hbm", st["mex_keys"] + st["mex_sort"],
                                                    16 + 4 + 4 * 16 + 4),
        "mex_pass1_kernel": ("hbm", st["mex_tile_sums"], 4 + 16 + 16),
    }
    table = {}
    for name, (bound, ms_k, work) in kern.items():
        if bound == "alu":
            ach = work * n / (ms_k * 1e-3) / 1e12
            table[name] = {"bound": "alu", "ms": ms_k, "achieved": ach, "peak": fp32_peak,
                           "unit": "TFLOP/s", "frac": ach / fp32_peak,
                           "frac_of_derived": ach / fp32_derived,
                           "work_per_particle": work, "work_unit": "flop"}
        else:
            ach = work * n / (ms_k * 1e-3) / 1e9
            table[name] = {"bound": "hbm", "ms": ms_k, "achieved": ach, "peak": peaks["hbm_gbs"],
                           "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                           "work_per_particle": work, "work_unit": "byte"}
        if name.startswith("mex_sort"):
            # the group's launches: keygen, the 4 radix passes, the tie fix-up
            parts = [traffic.get("keygen_kernel"), traffic.get("onesweep_kernel"),
                     traffic.get("tie_fixup_kernel")]
            table[name]["traffic"] = (None if None in parts
                                      else parts[0] + 4 * parts[1] + parts[2])
        else:
            table[name]["traffic"] = traffic.get(name)
    # the SCF pass as a whole (coefficient kernel + finalize + field kernel),
    # timed as one call
    mt = res["method"]
    scf_work = scf_coeff_flops(N_MAX, L_MAX) + scf_field_flops(N_MAX, L_MAX)
    scf_ach = scf_work * n / (mt["scf"] * 1e-3) / 1e12
    scf_total = {"bound": "alu", "ms": mt["scf"], "achieved": scf_ach, "peak": fp32_peak,
                 "unit": "TFLOP/s", "frac": scf_ach / fp32_peak,
                 "frac_of_derived": scf_ach / fp32_derived, "work_per_particle": scf_work,
                 "work_unit": "flop"}
    dom = max(table, key=lambda k: table[k]["ms"])
    d = table[dom]
    peak_note_alu = (f"of measured: FP32 FMA rate measured in this run by etics_fma_peak "
                     f"(16 independent FMA chains per thread, best of 5 bursts of ~5 ms): "
                     f"FFMA {pk['ffma']:.2f}, paired FFMA2 {pk['ffma2']:.2f} TFLOP/s; "
                     f"derived {FP32_PEAK_NOTE} = {fp32_derived:.2f}")
    roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
            "unit": d["unit"], "frac": d["frac"], "traffic": d["traffic"],
            "peak_note": peak_note_alu if d["bound"] == "alu" else
            f"of {src}: hbm_gbs of MEASURED_PEAKS.json"}
    if d["bound"] == "alu":
        roof["frac_of_derived"] = d["frac_of_derived"]
    other = {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv) for kk, vv in v.items()}
             for k, v in table.items()}
    out = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": cfg, "roofline": roof,
           "e2e": {"value": job_throughput(2 * n, world, res["e2e_ms"]), "unit": UNIT,
                   "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": 2 * n * 16},
           "gpu_launches": res["launches"], "clocks": res["clocks"],
           "step": "MEX on a high-priority CUDA stream concurrent with SCF (coefficients + "
                   "field) on a normal-priority one",
           "serial_ms_per_step": res["serial_ms"],
           "kernel_timing": "CUDA events between the kernels of the same step run serially "
                            "on one stream (K steps after the timed region)",
           "stages_ms": {k: round(v, 5) for k, v in st.items()},
           "method_ms": {k: round(v, 5) for k, v in mt.items()},
           "method_timing": "each method alone as one call (SCF: coefficients + field; MEX), "
                            "L2 flushed before each, no events between its kernels",
           "kernels": other,
           "scf_total": {k: (round(v, 6) if isinstance(v, float) else v)
                         for k, v in scf_total.items()},
           "fma_peaks_tflops": {k: (round(v, 3) if isinstance(v, float) else v)
                                for k, v in pk.items()},
           "fp64_path": {"scf_ms": res["f64"][0], "mex_ms": res["f64"][1],
                         "value": 2 * n / ((res["f64"][0] + res["f64"][1]) * 1e-3),
                         "scf_particle_forces_per_s": n / (res["f64"][0] * 1e-3),
                         "mex_particle_forces_per_s": n / (res["f64"][1] * 1e-3),
                         "scf_roofline": {
                             "bound": "alu", "unit": "TFLOP/s",
                             "achieved": scf_work * n / (res["f64"][0] * 1e-3) / 1e12,
                             "peak": pk["fp64"],
                             "frac": scf_work * n / (res["f64"][0] * 1e-3) / 1e12 / pk["fp64"],
                             "peak_note": "of measured: FP64 FMA rate of etics_fma_peak in "
                                          "this run"},
                         "mixed_over_fp64": {"scf": res["f64"][0] / mt["scf"],
                                             "mex": res["f64"][1] / mt["mex"]}},
           "mixed_per_method": {"scf_particle_forces_per_s": n / (mt["scf"] * 1e-3),
                                "mex_particle_forces_per_s": n / (mt["mex"] * 1e-3)}}
    if not args.no_accuracy:
        acc = accuracy(res["x"], res["out_scf"], res["out_mex"])
        out["accuracy_eps_mixed_vs_oracle"] = acc["vs_oracle"]
        out["accuracy_eps_mixed_vs_fp64_gpu"] = acc["vs_fp64_gpu"]
    if not args.no_cpu_baseline and world >= 1:
        out["cpu_baseline"] = cpu_baseline(n, args.cpu_sample)
    emit(out)


if __name__ == "__main__":
    main()
