"""The remaining workloads at their full sizes, in the launch configuration
the benchmark uses, checked on sampled outputs the oracle computes one by one
or through properties that hold at any size: the 256-system ensemble with
the tuned launch shape, one graph-captured leapfrog step of the 2^20 Plummer
sphere, and the 2^26-particle (14, 8) step that drives the surrogate."""
import numpy as np
import pytest
import torch

import oracle
from helpers import assert_field_close, rounded
from paper_1406_4254_gb300 import autotune, etics, inputs

pytestmark = pytest.mark.gpu


def test_batch_ensemble_full_size_sampled():
    pm, sizes, nm, lm = autotune.ensemble(seed=0)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    plan = etics.BatchPlan(sizes, nm, lm, tuning=autotune.lookup(nm, lm, sizes))
    coeffs, out = etics.scf_batch(x, plan)
    etics.check_error()
    order = np.argsort(sizes)
    rng = np.random.default_rng(1)
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        a, b = plan.particle_offsets[i], plan.particle_offsets[i + 1]
        ref_in = rounded(pm[a:b], "mixed")
        c_ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], nm[i], lm[i])
        got = plan.coeffs_of(coeffs, i).cpu().numpy().reshape(c_ref.shape)
        # FP32 products summed in FP32 tiles: the error grows like sqrt(N)
        # (up to 2.6e5 particles here); the force check below is the criterion
        assert np.max(np.abs(got - c_ref)) <= 1e-5 * np.max(np.abs(c_ref)), i
        idx = rng.choice(b - a, min(2000, b - a), replace=False)
        acc_ref, pot_ref = oracle.scf_field(ref_in[idx, :3], nm[i], lm[i], c_ref)
        assert_field_close(out[a:b].cpu().numpy()[idx], acc_ref, pot_ref, "mixed", f"system {i}")


def test_leapfrog_full_size_graph_step_sampled():
    n, n_max, l_max, dt = 1 << 20, 10, 6, 0.01
    pm, vel = inputs.plummer(n, seed=0)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    v[:, :3] = torch.tensor(vel, dtype=torch.float32)
    acc, _ = etics.scf_force(x, n_max, l_max)
    extra = ((n_max + 1) * (l_max + 1) ** 2 * 8 + 255) // 256 * 256
    ws = torch.empty(etics.workspace_bytes(n, n_max, l_max, etics.SCF, etics.MIXED) + extra + 256,
                     dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    xs, vs, as_ = x.clone(), v.clone(), acc.clone()
    with torch.cuda.stream(side):
        etics.leapfrog_step(xs, vs, as_, dt, etics.SCF, n_max, l_max, ws=ws)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        etics.leapfrog_step(x, v, acc, dt, etics.SCF, n_max, l_max, ws=ws)
    g.replay()
    torch.cuda.synchronize()
    etics.check_error()
    # the force after the step against the oracle at the step's new positions
    xp = x.double().cpu().numpy()
    c = oracle.scf_coeffs(xp[:, :3], xp[:, 3], n_max, l_max)
    idx = np.random.default_rng(2).choice(n, 16384, replace=False)
    acc_ref, pot_ref = oracle.scf_field(xp[idx, :3], n_max, l_max, c)
    assert_field_close(acc.cpu().numpy()[idx], acc_ref, pot_ref, "mixed", "leapfrog 2^20")


def test_surrogate_full_size_step_properties():
    # the 2^26-particle (14, 8) step: the forecast-driven step with the
    # coefficients the plain step computed reproduces the plain step exactly
    n, n_max, l_max, dt = 1 << 26, 14, 8, 0.005
    pm = inputs.hernquist(n, seed=3)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    del pm
    v = torch.zeros_like(x)
    acc, _ = etics.scf_force(x, n_max, l_max)
    x2, v2, a2 = x.clone(), v.clone(), acc.clone()
    c = torch.empty((n_max + 1, (l_max + 1) ** 2), dtype=torch.float64, device="cuda")
    etics.leapfrog_step(x, v, acc, dt, etics.SCF, n_max, l_max, coeffs_out=c)
    etics.leapfrog_step_coeffs(x2, v2, a2, dt, n_max, l_max, c)
    etics.check_error()
    assert torch.equal(x, x2) and torch.equal(v, v2) and torch.equal(acc, a2)
    # and the coefficients of the whole set are the sum over two halves
    h = n // 2
    ca = etics.scf_coeffs(x[:h].contiguous(), n_max, l_max)
    cb = etics.scf_coeffs(x[h:].contiguous(), n_max, l_max)
    cs = etics.scf_coeffs(x, n_max, l_max)
    etics.check_error()
    assert torch.max(torch.abs(ca + cb - cs)) <= 1e-6 * torch.max(torch.abs(cs))


def test_surrogate_config_full_size_coefficients_and_force_vs_fp64():
    """The C5 workload at its full size: 2^26 particles of the bar-perturbed
    Hernquist sphere, (n_max, l_max) = (14, 8).  The mixed coefficients
    (per-warp-bin kernel, FP32 register windows flushed to FP64) are compared
    element by element with the library's FP64 GPU path at the same
    FP32-rounded positions (that path is tied to the oracle to 1e-12 in the
    parity tests), and the mixed force at 4096 sampled particles with the FP64
    oracle's field from those FP64 coefficients (eq. 23 bound: median 1e-5,
    max 1e-4)."""
    n, n_max, l_max = 1 << 26, 14, 8
    pm, _ = inputs.hernquist_bar(n, seed=3, eps=0.05, velocities=False)
    pm32 = pm.astype(np.float32)
    del pm
    x = torch.tensor(pm32, device="cuda")
    c32 = etics.scf_coeffs(x, n_max, l_max)
    x64 = x.double()
    c64 = etics.scf_coeffs(x64, n_max, l_max)
    del x64
    etics.check_error()
    c32n, c64n = c32.cpu().numpy(), c64.cpu().numpy()
    # the mixed coefficient bound of the parity tests (max |dc| / max |c|)
    scale = np.max(np.abs(c64n))
    dev = np.abs(c32n - c64n)
    rows = [float(dev[k].max() / np.max(np.abs(c64n[k]))) for k in range(n_max + 1)]
    assert dev.max() <= 2e-6 * scale, (dev.max() / scale, rows)
    out = etics.scf_field(x, c32, n_max, l_max)
    etics.check_error()
    idx = np.sort(np.random.default_rng(4).choice(n, 4096, replace=False))
    ref = pm32[idx].astype(np.float64)
    acc_ref, pot_ref = oracle.scf_field(ref[:, :3], n_max, l_max, c64n)
    assert_field_close(out.cpu().numpy()[idx], acc_ref, pot_ref, "mixed", "2^26 (14, 8)")
