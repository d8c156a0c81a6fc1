"""Batched SCF over independent systems (etics_scf_batch) against the
single-system path and the FP64 oracle; graph capture; determinism."""
import numpy as np
import pytest
import torch

import oracle
from helpers import assert_field_close, rounded
from paper_1406_4254_gb300 import autotune, etics, inputs

pytestmark = pytest.mark.gpu


def small_batch():
    sizes = [1, 0, 3, 700, 2500, 4096, 9000, 130, 5001]
    n_maxes = [4, 6, 0, 14, 10, 8, 6, 12, 3]
    l_maxes = [2, 3, 0, 8, 6, 2, 8, 5, 1]
    parts = [inputs.hernquist(n, seed=100 + i, axes=(1.0, 0.8, 0.6)) for i, n in enumerate(sizes)]
    return np.concatenate(parts), sizes, n_maxes, l_maxes


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_matches_single_system_calls(dtype):
    pm, sizes, nm, lm = small_batch()
    prec = etics.MIXED if dtype == torch.float32 else etics.FP64
    x = torch.tensor(pm, dtype=dtype, device="cuda")
    plan = etics.BatchPlan(sizes, nm, lm, precision=prec)
    coeffs, out = etics.scf_batch(x, plan)
    etics.check_error()
    ctol = 2e-6 if dtype == torch.float32 else 1e-12
    for i, n in enumerate(sizes):
        a, b = plan.particle_offsets[i], plan.particle_offsets[i + 1]
        cb = plan.coeffs_of(coeffs, i).cpu().numpy()
        if n == 0:
            assert np.all(cb == 0)
            continue
        xi = x[a:b].contiguous()
        cs = etics.scf_coeffs(xi, nm[i], lm[i]).cpu().numpy()
        assert np.max(np.abs(cb - cs)) <= ctol * max(np.max(np.abs(cs)), 1e-300), i
        fs = etics.scf_field(xi, plan.coeffs_of(coeffs, i).contiguous(), nm[i], lm[i])
        # same arithmetic, different kernel instantiation: contraction may differ
        o, f = out[a:b].cpu().numpy(), fs.cpu().numpy()
        ftol = 2e-6 if dtype == torch.float32 else 1e-13
        assert np.max(np.abs(o - f)) <= ftol * np.max(np.abs(f)), i


def test_batch_matches_oracle():
    pm, sizes, nm, lm = small_batch()
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    plan = etics.BatchPlan(sizes, nm, lm)
    coeffs, out = etics.scf_batch(x, plan)
    etics.check_error()
    for i in (3, 4, 6):
        a, b = plan.particle_offsets[i], plan.particle_offsets[i + 1]
        ref_in = rounded(pm[a:b], "mixed")
        c_ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], nm[i], lm[i])
        acc_ref, pot_ref = oracle.scf_field(ref_in[:, :3], nm[i], lm[i], c_ref)
        assert_field_close(out[a:b].cpu().numpy(), acc_ref, pot_ref, "mixed", f"batch {i}")


def test_batch_graph_capture_and_determinism():
    pm, sizes, nm, lm = small_batch()
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    plan = etics.BatchPlan(sizes, nm, lm)
    c1, o1 = etics.scf_batch(x, plan)
    coeffs = torch.empty_like(c1)
    out = torch.empty_like(o1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        etics.scf_batch(x, plan, coeffs=coeffs, out=out)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        etics.scf_batch(x, plan, coeffs=coeffs, out=out)
    coeffs.zero_()
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    etics.check_error()
    assert torch.equal(coeffs, c1) and torch.equal(out, o1)


def test_batch_tunings_agree():
    pm, sizes, nm, lm = small_batch()
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    ref = None
    for vals in [(32, 1, 128, 1024), (64, 2, 256, 4096), (128, 3, 256, 1000)]:
        plan = etics.BatchPlan(sizes, nm, lm, tuning=etics.BatchTuning(*vals))
        c, o = etics.scf_batch(x, plan)
        etics.check_error()
        if ref is None:
            ref = (c.cpu().numpy(), o.cpu().numpy())
            continue
        scale = np.max(np.abs(ref[0]))
        assert np.max(np.abs(c.cpu().numpy() - ref[0])) <= 2e-6 * scale
        err = np.linalg.norm(o.cpu().numpy()[:, :3] - ref[1][:, :3], axis=1) / \
            np.maximum(np.linalg.norm(ref[1][:, :3], axis=1), 1e-30)
        assert np.max(err) < 1e-4


def test_autotune_picks_a_valid_shape(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "TABLE", str(tmp_path / "t.json"))
    monkeypatch.setattr(autotune, "CANDIDATES", {"tile": [32, 64], "blocks_per_sm": [1, 2],
                                                 "field_threads": [256], "field_chunk": [2048]})
    pm, sizes, nm, lm = small_batch()
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    best, res = autotune.tune(x, sizes, nm, lm, reps=2)
    assert len(res) == 4 and res[0][0] <= res[-1][0]
    t = autotune.lookup(nm, lm, sizes)
    assert t is not None and t.tile == best["tile"]
