"""Checkpoint / resume of a leapfrog run and run-to-run determinism.

CPU part: the file format round-trips and rejects damaged files.  GPU part:
a run resumed from a checkpoint continues bit for bit like the uninterrupted
run (every reduction in the library sums in a fixed order), and two runs of
the force passes give bitwise-equal outputs."""
import numpy as np
import pytest
import torch

from paper_1406_4254_gb300 import checkpoint, etics, inputs


def test_format_round_trip_and_damage(tmp_path):
    p = str(tmp_path / "c.bin")
    a = torch.arange(12, dtype=torch.float64).reshape(3, 4)
    b = torch.tensor([3, 1, 4, 1], dtype=torch.int32)
    checkpoint.save(p, posm=a, vel=a * 2, accpot=a * 3, step=7, dt=0.01, seed=5,
                    extra={"order": b, "empty": torch.empty(0, 4)})
    arr, hd = checkpoint.load(p, device="cpu")
    assert hd["step"] == 7 and hd["dt"] == 0.01 and hd["seed"] == 5
    assert torch.equal(arr["posm"], a) and torch.equal(arr["accpot"], a * 3)
    assert torch.equal(arr["order"], b) and arr["empty"].shape == (0, 4)
    raw = bytearray(open(p, "rb").read())
    raw[40] ^= 0xFF
    open(p, "wb").write(bytes(raw))
    with pytest.raises(ValueError):
        checkpoint.load(p, device="cpu")
    open(p, "wb").write(b"garbage")
    with pytest.raises(ValueError):
        checkpoint.load(p, device="cpu")


def _state(n, dtype):
    pm, vel = inputs.plummer(n, seed=9)
    x = torch.tensor(pm, dtype=dtype, device="cuda")
    v = torch.zeros_like(x)
    v[:, :3] = torch.tensor(vel, dtype=dtype)
    return x, v


@pytest.mark.gpu
@pytest.mark.parametrize("method", [etics.SCF, etics.MEX])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_resume_is_bitwise_identical(tmp_path, method, dtype):
    n_max, l_max, dt = 6, 4, 0.01
    x, v = _state(20000, dtype)
    if method == etics.SCF:
        acc, _ = etics.scf_force(x, n_max, l_max)
    else:
        acc = etics.mex_field(x, l_max)
    x2, v2, a2 = x.clone(), v.clone(), acc.clone()
    for _ in range(10):
        etics.leapfrog_step(x, v, acc, dt, method, n_max, l_max)
    p = str(tmp_path / "run.ck")
    for step in range(5):
        etics.leapfrog_step(x2, v2, a2, dt, method, n_max, l_max)
    checkpoint.save(p, posm=x2, vel=v2, accpot=a2, step=5, dt=dt)
    del x2, v2, a2
    arr, hd = checkpoint.load(p)
    x3, v3, a3 = arr["posm"], arr["vel"], arr["accpot"]
    for _ in range(10 - hd["step"]):
        etics.leapfrog_step(x3, v3, a3, hd["dt"], method, n_max, l_max)
    etics.check_error()
    assert torch.equal(x, x3) and torch.equal(v, v3) and torch.equal(acc, a3)


@pytest.mark.gpu
def test_force_passes_are_deterministic():
    pm = inputs.hernquist(300000, seed=10, axes=(1.0, 0.8, 0.6))
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    outs = []
    for _ in range(2):
        s, c = etics.scf_force(x, 10, 6)
        m = etics.mex_field(x, 6)
        outs.append((s.clone(), c.clone(), m.clone()))
    etics.check_error()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
