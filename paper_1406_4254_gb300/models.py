"""Closed-form ("real") forces of the synthetic models, for accuracy studies.

Sec. 4.1 measures the expansions against the smooth force of the model the
particles were drawn from (eq. 22).  This module gives that force for:

* the Hernquist sphere (M = a = 1): Phi = -1/(1+r), a = -x / (r (1+r)^2);
* the Plummer sphere (M = b = 1): Phi = -1/sqrt(1+r^2), a = -x / (1+r^2)^(3/2);
* Ferrers ellipsoids of index 1 (the paper's model1, axes 10:10:9, and
  model2, axes 3:2:1), rho = rho0 (1 - m^2) inside m^2 = sum x_i^2/a_i^2 <= 1,
  total mass 1.  Their interior potential is the classical heterogeneous-
  ellipsoid integral (Chandrasekhar 1969; Binney & Tremaine Sec. 2.5)
      Phi(x) = -pi G a1 a2 a3 rho0 / 2 * int_0^inf du / Delta(u) (1 - m^2(u))^2,
  Delta(u) = sqrt(prod (a_i^2 + u)), m^2(u) = sum x_i^2 / (a_i^2 + u), a
  polynomial in x^2, y^2, z^2 whose coefficients are the 1-D integrals
  W0 = int du/Delta, W_i = int du/(Delta (a_i^2+u)),
  W_ij = int du/(Delta (a_i^2+u)(a_j^2+u)); with rho0 = 15 / (8 pi a1 a2 a3):
      Phi = -(15/16) [W0 - 2 sum_i W_i x_i^2 + sum_ij W_ij x_i^2 x_j^2],
      a_k = (15/4) x_k (sum_j W_kj x_j^2 - W_k).
  The paper computed these coefficients with Sage; here scipy's adaptive
  quadrature gives them to ~1e-13.

Plus the sampler of the Ferrers models (the other samplers are in inputs.py).
Host-side numpy only; none of the expansion method's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

MODEL1 = (1.0, 1.0, 0.9)          # Sec. 4.1 model1: mildly oblate, 10:10:9
MODEL2 = (1.0, 2.0 / 3.0, 1.0 / 3.0)   # model2: triaxial, 3:2:1


def hernquist_force(x: np.ndarray):
    r = np.linalg.norm(x, axis=1)
    pot = -1.0 / (1.0 + r)
    acc = -x / (np.where(r > 0, r, 1.0) * (1.0 + r) ** 2)[:, None]
    acc[r == 0] = 0.0
    return acc, pot


def plummer_force(x: np.ndarray):
    r2 = np.sum(x * x, axis=1)
    pot = -1.0 / np.sqrt(1.0 + r2)
    acc = -x / ((1.0 + r2) ** 1.5)[:, None]
    return acc, pot


def ferrers_coefficients(axes):
    """(W0, W[3], W[3][3]) index-symbol integrals of a Ferrers ellipsoid."""
    from scipy.integrate import quad
    a2 = np.asarray(axes, dtype=np.float64) ** 2

    def integral(f):
        # u = t / (1 - t) maps [0, 1) onto [0, inf)
        g = lambda t: f(t / (1.0 - t)) / (1.0 - t) ** 2  # noqa: E731
        v, _ = quad(g, 0.0, 1.0, epsabs=0.0, epsrel=1e-13, limit=400)
        return v

    delta = lambda u: math.sqrt((a2[0] + u) * (a2[1] + u) * (a2[2] + u))  # noqa: E731
    w0 = integral(lambda u: 1.0 / delta(u))
    w1 = np.array([integral(lambda u, i=i: 1.0 / (delta(u) * (a2[i] + u))) for i in range(3)])
    w2 = np.zeros((3, 3))
    for i in range(3):
        for j in range(i, 3):
            w2[i, j] = w2[j, i] = integral(
                lambda u, i=i, j=j: 1.0 / (delta(u) * (a2[i] + u) * (a2[j] + u)))
    return w0, w1, w2


def ferrers_force(x: np.ndarray, axes, coeffs=None):
    """Acceleration (N, 3) and potential (N,) of the unit-mass Ferrers n = 1
    ellipsoid at interior points x (N, 3)."""
    w0, w1, w2 = coeffs if coeffs is not None else ferrers_coefficients(axes)
    x2 = x * x
    pot = -(15.0 / 16.0) * (w0 - 2.0 * x2 @ w1 + np.einsum("ni,ij,nj->n", x2, w2, x2))
    acc = (15.0 / 4.0) * x * (x2 @ w2 - w1[None, :])
    return acc, pot


def ferrers_density(x: np.ndarray, axes) -> np.ndarray:
    a = np.asarray(axes, dtype=np.float64)
    m2 = np.sum((x / a) ** 2, axis=1)
    rho0 = 15.0 / (8.0 * math.pi * np.prod(a))
    return np.where(m2 <= 1.0, rho0 * (1.0 - m2), 0.0)


def ferrers(n: int, seed: int = 0, axes=MODEL2) -> np.ndarray:
    """Equal-mass (1/N) realisation of the Ferrers n = 1 ellipsoid: the
    ellipsoidal radius m has density (1 - m^2) m^2 on [0, 1] (drawn by
    rejection), directions are isotropic, then the axes scale x, y, z."""
    rng = np.random.Generator(np.random.Philox(key=[int(seed), 7]))
    m = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        t = rng.uniform(0.0, 1.0, todo.size)
        ok = rng.uniform(0.0, 0.25, todo.size) < (1.0 - t * t) * t * t
        m[todo[ok]] = t[ok]
        todo = todo[~ok]
    ct = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    u = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    out = np.empty((n, 4))
    out[:, :3] = u * m[:, None] * np.asarray(axes, dtype=np.float64)[None, :]
    out[:, 3] = 1.0 / n
    return out
