"""Seeded synthetic particle models (the workloads of the paper's tests).

This module draws particle realisations only; it contains none of the
expansion method's arithmetic and is shared by the CUDA path's tests, the
benchmark and the oracle tests as their common input source.  All randomness
comes from numpy's counter-based Philox generator, so a (model, N, seed)
triple always gives the same particles on any machine.

Models (G = M = 1):

* ``hernquist``: the Hernquist (1990) sphere with scale a = 1, radii by the
  inverse cumulative mass r = sqrt(u)/(1 - sqrt(u)) and isotropic directions
  (the model of the paper's single-precision test, Sec. 4.2).  ``axes``
  stretches it to a triaxial shape, e.g. (1, 0.8, 0.6).
* ``plummer``: Plummer sphere with b = 1, r = 1/sqrt(u^(-2/3) - 1), and
  isotropic equilibrium velocities by the Aarseth-Henon-Wielen (1974)
  rejection sampler.
* ``hernquist_bar``: Hernquist radii with the angular density
  1 + eps sin^2(theta) cos(2 phi) (an l = 2, m = 2 bar perturbation) drawn by
  rejection, and isotropic velocities from the Hernquist (1990)
  distribution function by rejection.
* ``mlp_params``: seeded initial weights of the coefficient-forecasting MLP.

Arrays are float64 with shape (N, 4) = (x, y, z, m) and velocities (N, 3).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    ct = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)


def hernquist(n: int, seed: int = 0, axes=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Equal-mass (1/N) Hernquist sphere, optionally stretched by ``axes``."""
    rng = _rng(seed, 1)
    u = rng.uniform(0.0, 1.0, n)
    su = np.sqrt(u)
    r = su / (1.0 - su)
    x = _isotropic(rng, n) * r[:, None]
    x = x * np.asarray(axes, dtype=np.float64)[None, :]
    out = np.empty((n, 4))
    out[:, :3] = x
    out[:, 3] = 1.0 / max(n, 1)
    return out


def plummer(n: int, seed: int = 0):
    """Plummer sphere (b = 1) with AHW74 isotropic velocities: (posm, vel)."""
    rng = _rng(seed, 2)
    u = rng.uniform(0.0, 1.0, n)
    u = np.maximum(u, 1e-300)
    r = 1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    x = _isotropic(rng, n) * r[:, None]
    # speed fraction q = v / v_esc from g(q) = q^2 (1 - q^2)^(7/2) (max < 0.1)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.uniform(0.0, 1.0, todo.size)
        yy = rng.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    v = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vel = _isotropic(rng, n) * v[:, None]
    out = np.empty((n, 4))
    out[:, :3] = x
    out[:, 3] = 1.0 / n
    return out, vel


def _hernquist_df(e: np.ndarray) -> np.ndarray:
    """Isotropic Hernquist (1990) distribution function f(E) for 0 < E < 1
    (binding energy E = -Phi - v^2/2, G = M = a = 1), up to a constant.  Below
    E = 1e-4 the closed form cancels to O(E^(5/2)); there its leading term
    (128/5) E^(5/2) (1 - E)^(-5/2) (the series of the closed form) is used."""
    e = np.asarray(e, dtype=np.float64)
    q = np.sqrt(e)
    s = np.sqrt(np.maximum(1.0 - e, 1e-300))
    full = (3.0 * np.arcsin(q) + q * s * (1.0 - 2.0 * e) * (8.0 * e * e - 8.0 * e - 3.0)) \
        / np.maximum(1.0 - e, 1e-300) ** 2.5
    small = 25.6 * e ** 2.5 / np.maximum(1.0 - e, 1e-300) ** 2.5
    return np.where(e < 1e-4, small, full)


def hernquist_bar(n: int, seed: int = 0, eps: float = 0.05, velocities: bool = True):
    """Hernquist sphere with density 1 + eps sin^2(theta) cos(2 phi) in angle."""
    rng = _rng(seed, 3)
    u = rng.uniform(0.0, 1.0, n)
    su = np.sqrt(u)
    r = su / (1.0 - su)
    d = np.empty((n, 3))
    todo = np.arange(n)
    while todo.size:
        c = _isotropic(rng, todo.size)
        w = 1.0 + eps * (c[:, 0] ** 2 - c[:, 1] ** 2)  # sin^2 t cos 2p = x^2 - y^2
        ok = rng.uniform(0.0, 1.0 + eps, todo.size) < w
        d[todo[ok]] = c[ok]
        todo = todo[~ok]
    out = np.empty((n, 4))
    out[:, :3] = d * r[:, None]
    out[:, 3] = 1.0 / n
    if not velocities:
        return out, None
    # speeds at each radius from f(E) v^2 by rejection.  The bound
    # max_x f(psi (1 - x^2)) x^2 (x = v / v_esc) grows with psi because f
    # grows with E, so its value at the grid point just above psi bounds it;
    # the grid is geometric in psi below 1/2 and in 1 - psi above (ratio
    # 1.02), and particles above the top grid point get their own bound.
    psi = 1.0 / (1.0 + r)                         # -Phi of the spherical model
    vesc = np.sqrt(2.0 * psi)
    xs = np.linspace(0.0, 1.0, 513)[1:-1]

    def bound(ps):
        e = np.maximum(ps[:, None] * (1.0 - xs[None, :] ** 2), 1e-300)
        return np.max(_hernquist_df(e) * xs[None, :] ** 2, axis=1) * 1.5

    lo = 0.5 * 1.02 ** -np.arange(2100.0)         # 0.5 down to ~4e-19
    hi = 1.0 - 0.5 * 1.02 ** -np.arange(1, 1400.0)  # up to 1 - ~5e-13
    grid = np.concatenate([lo[::-1], hi])
    table = bound(grid)
    cell = np.searchsorted(grid, psi)             # first grid point >= psi
    fmax = table[np.minimum(cell, grid.size - 1)]
    top = np.nonzero(cell >= grid.size)[0]
    if top.size:
        fmax[top] = bound(psi[top])
    v = np.empty(n)
    for c0 in range(0, n, 1 << 20):
        todo = np.arange(c0, min(n, c0 + (1 << 20)))
        for _ in range(100000):
            if not todo.size:
                break
            x = rng.uniform(0.0, 1.0, todo.size)      # v / v_esc
            e = np.maximum(psi[todo] * (1.0 - x * x), 1e-12)
            g = _hernquist_df(e) * x * x
            ok = rng.uniform(0.0, 1.0, todo.size) * fmax[todo] < g
            v[todo[ok]] = x[ok] * vesc[todo[ok]]
            todo = todo[~ok]
        if todo.size:
            raise RuntimeError("hernquist_bar: velocity rejection did not converge")
    vel = _isotropic(rng, n) * v[:, None]
    return out, vel


def rotation(seed: int) -> np.ndarray:
    """A random proper rotation matrix (QR of a Gaussian matrix)."""
    rng = _rng(seed, 4)
    a = rng.normal(size=(3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def mlp_params(dims, seed: int = 0) -> np.ndarray:
    """Initial parameters of an MLP with layer widths ``dims``, flat FP64 in
    the layout W_0, b_0, W_1, b_1, ... (W_i: dims[i] x dims[i+1], row-major):
    weights uniform in +-1/sqrt(fan_in), the last layer's scaled by 0.1 so
    that the untrained network's output starts near zero; biases zero."""
    rng = _rng(seed, 5)
    n = sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))
    p = np.zeros(n)
    o = 0
    for i in range(len(dims) - 1):
        a, b = dims[i], dims[i + 1]
        lim = 1.0 / math.sqrt(a) * (0.1 if i == len(dims) - 2 else 1.0)
        p[o:o + a * b] = rng.uniform(-lim, lim, a * b)
        o += a * b + b
    return p
