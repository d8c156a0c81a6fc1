"""The expansions against the smooth force of the model (Sec. 4.1, eq. 22) on
the GPU FP64 path: properties the paper's accuracy study rests on."""
import numpy as np
import pytest
import torch

from paper_1406_4254_gb300 import etics, inputs, models

pytestmark = pytest.mark.gpu


def _eps(a, a_real):
    a = a.cpu().numpy()[:, :3]
    return np.linalg.norm(a - a_real, axis=1) / np.linalg.norm(a_real, axis=1)


def test_scf_zeroth_order_reproduces_the_hernquist_profile():
    # the Hernquist profile is the basis's zeroth function: SCF (0, 0) has no
    # radial or angular bias, its force is the exact force times the one
    # coefficient's sample estimate, c_000 Y_00 = 3 sum_k m_k / (1 + r_k)
    # (J_00 = -1/(12 pi)), so every particle has the same relative error
    # |3 S - 1|; MEX's monopole instead carries the particle noise of M(<r)
    pm = inputs.hernquist(1 << 17, seed=21)
    a_real, _ = models.hernquist_force(pm[:, :3])
    x = torch.tensor(pm, dtype=torch.float64, device="cuda")
    e_scf = _eps(etics.scf_force(x, 0, 0)[0], a_real)
    s = np.sum(pm[:, 3] / (1.0 + np.linalg.norm(pm[:, :3], axis=1)))
    np.testing.assert_allclose(e_scf, abs(3.0 * s - 1.0), rtol=1e-8, atol=1e-14)
    e_mex = _eps(etics.mex_field(x, 0), a_real)
    assert np.std(e_mex) > 100 * np.std(e_scf)


def test_triaxial_model_needs_multipoles_and_scf_approaches_mex():
    pm = models.ferrers(1 << 18, seed=22, axes=models.MODEL2)
    a_real, _ = models.ferrers_force(pm[:, :3], models.MODEL2)
    x = torch.tensor(pm, dtype=torch.float64, device="cuda")
    mex = {l: np.mean(_eps(etics.mex_field(x, l), a_real)) for l in (0, 2, 6)}
    assert mex[6] < mex[0] and mex[2] < mex[0]
    # MEX is SCF with n_max -> infinity (Sec. 2.4): the SCF error at l_max = 6
    # approaches MEX's as n_max grows
    scf = {n: np.mean(_eps(etics.scf_force(x, n, 6)[0], a_real)) for n in (2, 14)}
    etics.check_error()
    assert abs(scf[14] - mex[6]) < abs(scf[2] - mex[6])
