"""GPU kick-drift-kick step (paper Secs. 3.4 and 5.4) against the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from helpers import assert_field_close, rounded
from paper_1406_4254_gb300 import etics, inputs

pytestmark = pytest.mark.gpu


def as4(v):
    out = np.zeros((len(v), 4))
    out[:, :3] = v
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("method", [etics.SCF, etics.MEX])
def test_one_step_matches_oracle(precision, method):
    pm, vel = inputs.plummer(6000, seed=1)
    dt, n_max, l_max = 0.01, 8, 4
    dtype = torch.float64 if precision == "fp64" else torch.float32
    x = torch.tensor(pm, dtype=dtype, device="cuda")
    v = torch.tensor(as4(vel), dtype=dtype, device="cuda")
    ref_pm = rounded(pm, precision)
    ref_v = rounded(as4(vel), precision)[:, :3].copy()
    ref_x = ref_pm[:, :3].copy()
    # a(x) at the start, from the GPU itself (the step takes it as input)
    if method == etics.SCF:
        acc0, _ = etics.scf_force(x, n_max, l_max)
    else:
        acc0 = etics.mex_field(x, l_max)
    ref_a = acc0.double().cpu().numpy()[:, :3].copy()
    etics.leapfrog_step(x, v, acc0, dt, method, n_max, l_max)
    etics.check_error()
    pot_ref, _ = oracle.leapfrog_step(ref_x, ref_v, ref_pm[:, 3], ref_a, dt, method, n_max, l_max)
    xg = x.double().cpu().numpy()
    vg = v.double().cpu().numpy()
    tol_x = 1e-14 if precision == "fp64" else 1e-6
    np.testing.assert_allclose(xg[:, :3], ref_x, rtol=tol_x, atol=tol_x)
    np.testing.assert_allclose(vg[:, :3], ref_v, rtol=1e-5 if precision == "mixed" else 1e-12,
                               atol=1e-6 if precision == "mixed" else 1e-13)
    if precision == "fp64":
        # the new force is evaluated at bitwise-identical positions
        assert_field_close(acc0.cpu().numpy(), ref_a, pot_ref, precision, "kdk")
    else:
        # FP32 positions drift from the oracle's by rounding, so the new force
        # is judged against the oracle's force at the positions the GPU
        # reached (the same FP32 values, widened)
        pos = xg[:, :3]
        if method == etics.SCF:
            c = oracle.scf_coeffs(pos, ref_pm[:, 3], n_max, l_max)
            a_new, p_new = oracle.scf_field(pos, n_max, l_max, c)
        else:
            a_new, p_new, _ = oracle.mex_field(pos, ref_pm[:, 3], l_max)
        assert_field_close(acc0.cpu().numpy(), a_new, p_new, precision, "kdk new force")


def test_energy_conservation_plummer_scf():
    """A Plummer sphere integrated with the mixed SCF path conserves energy
    to leapfrog accuracy over 50 steps."""
    pm, vel = inputs.plummer(1 << 16, seed=2)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    v = torch.tensor(as4(vel), dtype=torch.float32, device="cuda")
    acc, _ = etics.scf_force(x, 10, 6)
    m = x[:, 3].double()

    def energy():
        kin = 0.5 * (m * (v[:, :3].double() ** 2).sum(1)).sum()
        return float(kin + 0.5 * (m * acc[:, 3].double()).sum())

    e0 = energy()
    for _ in range(50):
        etics.leapfrog_step(x, v, acc, 0.01, etics.SCF, 10, 6)
    etics.check_error()
    assert abs(energy() / e0 - 1) < 2e-4
