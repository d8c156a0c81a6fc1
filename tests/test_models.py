"""Pins of the closed-form model forces used by the accuracy study
(paper_1406_4254_gb300/models.py): the Ferrers n = 1 sphere against its
elementary enclosed-mass force, Poisson's equation for the triaxial model,
Hernquist and Plummer against their potentials, and the sampler's profile."""
import math

import numpy as np
import pytest

from paper_1406_4254_gb300 import models


def test_ferrers_sphere_matches_enclosed_mass():
    # rho = rho0 (1 - r^2), rho0 = 15/(8 pi): M(r) = 4 pi rho0 (r^3/3 - r^5/5)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(50, 3))
    x *= (rng.uniform(0.05, 0.99, 50) / np.linalg.norm(x, axis=1))[:, None]
    acc, pot = models.ferrers_force(x, (1.0, 1.0, 1.0))
    r = np.linalg.norm(x, axis=1)
    rho0 = 15.0 / (8.0 * math.pi)
    g = 4.0 * math.pi * rho0 * (r / 3.0 - r ** 3 / 5.0)
    np.testing.assert_allclose(acc, -g[:, None] * x / r[:, None], rtol=1e-12, atol=1e-14)
    # potential: -int_r^inf g dr' = -(pi rho0)(...) in closed form for the sphere
    phi = -4.0 * math.pi * rho0 * (1.0 / 3.0 - 1.0 / 5.0 + (1 - r ** 2) / 6.0
                                   - (1 - r ** 4) / 20.0)
    np.testing.assert_allclose(pot, phi, rtol=1e-12)


@pytest.mark.parametrize("axes", [models.MODEL1, models.MODEL2])
def test_ferrers_poisson(axes):
    # div a = -4 pi rho inside the ellipsoid (4th-order central differences)
    co = models.ferrers_coefficients(axes)
    rng = np.random.default_rng(2)
    pts = models.ferrers(200, seed=3, axes=axes)[:, :3] * 0.9
    h = 1e-3
    div = np.zeros(len(pts))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        f = lambda s: models.ferrers_force(pts + s * e, axes, co)[0][:, k]  # noqa: E731
        div += (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * h)
    np.testing.assert_allclose(div, -4 * math.pi * models.ferrers_density(pts, axes),
                               rtol=1e-8, atol=1e-8)
    # the force is minus the gradient of the potential
    k = 1
    e = np.zeros(3)
    e[k] = h
    p = lambda s: models.ferrers_force(pts + s * e, axes, co)[1]  # noqa: E731
    grad = (-p(2) + 8 * p(1) - 8 * p(-1) + p(-2)) / (12 * h)
    np.testing.assert_allclose(models.ferrers_force(pts, axes, co)[0][:, k], -grad,
                               rtol=1e-8, atol=1e-10)


def test_hernquist_and_plummer_forces_are_gradients():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(40, 3)) * 2.0
    h = 1e-4
    for fn in (models.hernquist_force, models.plummer_force):
        acc, _ = fn(x)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            g = (fn(x + e)[1] - fn(x - e)[1]) / (2 * h)
            np.testing.assert_allclose(acc[:, k], -g, rtol=1e-6, atol=1e-9)


def test_ferrers_sampler_profile():
    # ellipsoidal radius m has density 15/2 (1 - m^2) m^2 on [0, 1]:
    # mean m = 15/2 (1/4 - 1/6) = 5/8
    pm = models.ferrers(200000, seed=5, axes=models.MODEL2)
    m = np.sqrt(np.sum((pm[:, :3] / np.asarray(models.MODEL2)) ** 2, axis=1))
    assert m.max() <= 1.0
    assert abs(m.mean() - 5.0 / 8.0) < 4e-3
    assert abs(pm[:, 3].sum() - 1.0) < 1e-12
