"""GPU SCF (CUDA kernels through the C ABI) against the FP64 oracle.

Coefficients (paper Sec. 2.4 eq. 18) element by element; accelerations and
potentials per particle with the relative error of eq. 23, at sizes that span
many tiles with a ragged tail, at the benchmark's full size (N = 2^20,
(n_max, l_max) = (10, 6)), and on edge cases.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import assert_field_close, device_particles, hernquist, rounded
from paper_1406_4254_gb300 import etics, inputs

pytestmark = pytest.mark.gpu

COEF_TOL = {"fp64": 1e-12, "mixed": 2e-6}   # max |dc| / max |c|


def gpu_coeffs(pm, n_max, l_max, precision):
    d = device_particles(pm, precision)
    c = etics.scf_coeffs(d, n_max, l_max)
    etics.check_error()
    return c.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nl", [(10, 6), (4, 2), (0, 0), (3, 0), (0, 5), (14, 8), (16, 14)])
def test_coefficients_match_oracle(precision, nl):
    n_max, l_max = nl
    pm = hernquist(5003, seed=1)
    ref_in = rounded(pm, precision)
    ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], n_max, l_max)
    got = gpu_coeffs(pm, n_max, l_max, precision).reshape(ref.shape)
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref)) / scale
    assert err <= COEF_TOL[precision], (err, nl)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nl", [(10, 6), (6, 3), (2, 1), (14, 8)])
def test_force_matches_oracle(precision, nl):
    """Coefficient pass + field pass end to end against the oracle's."""
    n_max, l_max = nl
    pm = hernquist(7777, seed=2)
    ref_in = rounded(pm, precision)
    c_ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], n_max, l_max)
    acc_ref, pot_ref = oracle.scf_field(ref_in[:, :3], n_max, l_max, c_ref)
    d = device_particles(pm, precision)
    out, _ = etics.scf_force(d, n_max, l_max)
    etics.check_error()
    assert_field_close(out.cpu().numpy(), acc_ref, pot_ref, precision, f"scf{nl}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_field_pass_alone_with_oracle_coefficients(precision):
    pm = hernquist(3001, seed=3)
    ref_in = rounded(pm, precision)
    c = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], 10, 6)
    acc_ref, pot_ref = oracle.scf_field(ref_in[:, :3], 10, 6, c)
    d = device_particles(pm, precision)
    out = etics.scf_field(d, torch.tensor(c, device="cuda"), 10, 6)
    etics.check_error()
    assert_field_close(out.cpu().numpy(), acc_ref, pot_ref, precision, "field")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_cases(precision):
    """N = 1, 2, 3; a particle at the origin; particles on the +-z axis;
    negative 'masses' (quadrature weights)."""
    rng = np.random.default_rng(4)
    cases = [np.array([[0.3, -0.2, 0.5, 1.0]]),
             np.array([[0.0, 0.0, 0.0, 0.5], [1.0, 2.0, -1.0, 0.5]]),
             np.array([[0.0, 0.0, 2.0, 0.3], [0.0, 0.0, -0.7, 0.3], [1e-3, 0.0, 0.0, 0.4]])]
    big = hernquist(600, seed=5)
    big[:10, 0] = 0.0
    big[:10, 1] = 0.0                  # on the z axis
    big[10, :3] = 0.0                  # the origin
    big[20:60, 3] *= -rng.uniform(0.1, 1.0, 40)   # negative weights
    cases.append(big)
    for pm in cases:
        for n_max, l_max in [(6, 4), (0, 0), (3, 1)]:
            ref_in = rounded(pm, precision)
            c_ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], n_max, l_max)
            acc_ref, pot_ref = oracle.scf_field(ref_in[:, :3], n_max, l_max, c_ref)
            d = device_particles(pm, precision)
            c = etics.scf_coeffs(d, n_max, l_max)
            out = etics.scf_field(d, c, n_max, l_max)
            etics.check_error()
            cg = c.cpu().numpy().reshape(c_ref.shape)
            tol = 1e-12 if precision == "fp64" else 2e-6
            assert np.max(np.abs(cg - c_ref)) <= tol * np.max(np.abs(c_ref)), (len(pm), n_max)
            o = out.cpu().numpy()
            # absolute check scaled by the largest force (some forces vanish by symmetry)
            amax = np.max(np.linalg.norm(acc_ref, axis=1))
            tola = 1e-11 if precision == "fp64" else 2e-5
            assert np.max(np.abs(o[:, :3] - acc_ref)) <= tola * amax, (len(pm), n_max, l_max)
            assert np.max(np.abs(o[:, 3] - pot_ref)) <= tola * np.max(np.abs(pot_ref))


def test_output_masks_and_empty_input():
    pm = hernquist(1000, seed=6)
    d = device_particles(pm, "mixed")
    c = etics.scf_coeffs(d, 6, 4)
    both = etics.scf_field(d, c, 6, 4).cpu().numpy()
    pot = etics.scf_field(d, c, 6, 4, out_mask=etics.OUT_POT).cpu().numpy()
    acc = etics.scf_field(d, c, 6, 4, out_mask=etics.OUT_ACC).cpu().numpy()
    assert np.all(pot[:, :3] == 0)
    np.testing.assert_allclose(pot[:, 3], both[:, 3], rtol=1e-6)
    assert np.all(acc[:, 3] == 0) and np.array_equal(acc[:, :3], both[:, :3])
    e = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    ce = etics.scf_coeffs(e, 6, 4)
    assert torch.all(ce == 0)
    etics.check_error()


def test_spherical_monopole_full_size():
    """A_000 = c_000/sqrt(4 pi) of a spherical Hernquist realisation of
    2^20 particles is 1 within 3 sigma, sigma = sqrt(1/(2N))."""
    n = 1 << 20
    pm = inputs.hernquist(n, seed=0)
    c = etics.scf_coeffs(device_particles(pm, "mixed"), 0, 0).cpu().numpy()
    assert c[0, 0] / math.sqrt(4 * math.pi) == pytest.approx(1.0, abs=3 * math.sqrt(0.5 / n))


def test_deterministic():
    pm = hernquist(20000, seed=7)
    d = device_particles(pm, "mixed")
    a1, c1 = etics.scf_force(d, 10, 6)
    a2, c2 = etics.scf_force(d, 10, 6)
    assert torch.equal(c1, c2) and torch.equal(a1, a2)


def test_full_size_bench_config_sampled():
    """N = 2^20, (10, 6), mixed path as the benchmark runs it: coefficients
    element by element, the field on a 4096-particle sample."""
    n = 1 << 20
    pm = hernquist(n, seed=0)
    ref_in = rounded(pm, "mixed")
    c_ref = oracle.scf_coeffs(ref_in[:, :3], ref_in[:, 3], 10, 6)
    d = device_particles(pm, "mixed")
    out, c = etics.scf_force(d, 10, 6)
    etics.check_error()
    cg = c.cpu().numpy().reshape(c_ref.shape)
    assert np.max(np.abs(cg - c_ref)) <= 2e-6 * np.max(np.abs(c_ref))
    idx = np.random.default_rng(0).choice(n, 4096, replace=False)
    acc_ref, pot_ref = oracle.scf_field(ref_in[idx, :3], 10, 6, c_ref)
    assert_field_close(out.cpu().numpy()[idx], acc_ref, pot_ref, "mixed", "scf 2^20")
