"""GPU SCF with the Clutton-Brock radial basis (etics_scf_coeffs_basis /
etics_scf_field_basis, basis 1) against the FP64 oracle's Clutton-Brock
functions: coefficients element by element, forces per particle (eq. 23's
relative error), a Plummer realisation whose (0, 0) expansion reproduces the
closed-form Plummer force, edge cases, and the HO basis through the same
entry points."""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import assert_field_close, device_particles, rounded
from paper_1406_4254_gb300 import etics, inputs

pytestmark = pytest.mark.gpu

CB = etics.BASIS_CB
COEF_TOL = {"fp64": 1e-12, "mixed": 2e-6}   # max |dc| / max |c|


def plummer_pm(n, seed):
    pm, _ = inputs.plummer(n, seed=seed)
    return pm


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nl", [(10, 6), (4, 2), (0, 0), (3, 0), (0, 5), (14, 8), (16, 14)])
def test_coefficients_match_oracle(precision, nl):
    n_max, l_max = nl
    pm = plummer_pm(5003, 1)
    ref_in = rounded(pm, precision)
    ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], n_max, l_max, basis=oracle.CB)
    d = device_particles(pm, precision)
    got = etics.scf_coeffs(d, n_max, l_max, basis=CB).cpu().numpy().reshape(ref.shape)
    etics.check_error()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= COEF_TOL[precision], (err, nl)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nl", [(10, 6), (6, 3), (2, 1), (14, 8)])
def test_force_matches_oracle(precision, nl):
    n_max, l_max = nl
    pm = plummer_pm(7777, 2)
    ref_in = rounded(pm, precision)
    c_ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], n_max, l_max, basis=oracle.CB)
    acc_ref, pot_ref = oracle.scf_field(ref_in[:, :3], n_max, l_max, c_ref, basis=oracle.CB)
    d = device_particles(pm, precision)
    out, _ = etics.scf_force(d, n_max, l_max, basis=CB)
    etics.check_error()
    assert_field_close(out.cpu().numpy(), acc_ref, pot_ref, precision, f"cb{nl}")


def test_plummer_monopole_is_the_plummer_force():
    # c_000 Y_00 = (16/(3 pi)) sum m/sqrt(1+r^2): every particle's force is the
    # Plummer force times that number
    pm = plummer_pm(1 << 16, 3)
    d = device_particles(pm, "fp64")
    out, _ = etics.scf_force(d, 0, 0, basis=CB)
    etics.check_error()
    r2 = np.sum(pm[:, :3] ** 2, axis=1)
    s = 16.0 / (3.0 * math.pi) * np.sum(pm[:, 3] / np.sqrt(1 + r2))
    np.testing.assert_allclose(out.cpu().numpy()[:, :3],
                               s * (-pm[:, :3] / ((1 + r2) ** 1.5)[:, None]),
                               rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out.cpu().numpy()[:, 3], -s / np.sqrt(1 + r2), rtol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_cases(precision):
    """A particle at the origin, particles on the z axis, N = 1."""
    big = plummer_pm(600, 5)
    big[:10, 0] = 0.0
    big[:10, 1] = 0.0
    big[10] = [0.0, 0.0, 0.0, big[10, 3]]
    for pm in (big, np.array([[0.3, -0.2, 0.5, 1.0]])):
        ref_in = rounded(pm, precision)
        c_ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], 6, 4, basis=oracle.CB)
        acc_ref, pot_ref = oracle.scf_field(ref_in[:, :3], 6, 4, c_ref, basis=oracle.CB)
        d = device_particles(pm, precision)
        out, _ = etics.scf_force(d, 6, 4, basis=CB)
        etics.check_error()
        assert_field_close(out.cpu().numpy(), acc_ref, pot_ref, precision, "cb edge")


def test_ho_through_the_basis_entry_points_is_unchanged():
    pm = inputs.hernquist(4000, seed=6)
    d = device_particles(pm, "mixed")
    a = etics.scf_coeffs(d, 10, 6)
    b = torch.empty_like(a)
    lib = etics.load()
    ws = etics.workspace(len(pm), 10, 6, etics.SCF, etics.MIXED)
    wp, wb = etics._aligned_ptr(ws)
    rc = lib.etics_scf_coeffs_basis(d.data_ptr(), len(pm), 10, 6, etics.BASIS_HO, etics.MIXED,
                                    b.data_ptr(), wp, wb, etics._stream(None))
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert lib.etics_scf_coeffs_basis(d.data_ptr(), len(pm), 10, 6, 7, etics.MIXED,
                                      b.data_ptr(), wp, wb, etics._stream(None)) == -1
