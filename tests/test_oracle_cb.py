"""Pins of the oracle's Clutton-Brock radial basis (the Plummer model as the
zeroth term; the alternative basis Sec. 2.5 names) against mathematics that
does not come from the oracle: scipy's Gegenbauer polynomials, the radial
Poisson equation, quadrature of the normalisation, exact-quadrature
biorthogonality and the closed-form Plummer potential."""
import math

import numpy as np
import pytest
from scipy.special import eval_gegenbauer, roots_legendre, sph_harm_y

import oracle
from paper_1406_4254_gb300 import inputs

CB = oracle.CB


def k_nl(n, l):
    return 4 * n * (n + 2 * l + 2) + (2 * l + 1) * (2 * l + 3)


def rho_nl(n, l, r):
    """Density partner: (K_nl/4pi) r^l (1+r^2)^-(l+5/2) C_n^(l+1)(xi)."""
    xi = (r * r - 1.0) / (r * r + 1.0)
    return k_nl(n, l) / (4 * math.pi) * r ** l * (1 + r * r) ** (-(l + 2.5)) \
        * eval_gegenbauer(n, l + 1.0, xi)


def phi_nl_scipy(n, l, r):
    xi = (r * r - 1.0) / (r * r + 1.0)
    return -r ** l * (1 + r * r) ** (-(l + 0.5)) * eval_gegenbauer(n, l + 1.0, xi)


def real_ylm_scipy(l, m, theta, phi):
    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    y = sph_harm_y(l, abs(m), theta, phi) * (-1) ** abs(m)
    return math.sqrt(2) * (np.real(y) if m > 0 else np.imag(y))


def quadrature(nx, nt, nphi):
    """Nodes and weights for int f d^3x: in xi = (r^2-1)/(r^2+1) the radial
    products rho_nl phi_n'l' r^2 dr are (1-xi^2)^(l+1/2) times a polynomial;
    Gauss-Legendre nodes in the angle acos(xi) integrate these smooth
    integrands to rounding."""
    th, wth = roots_legendre(nx)
    ang = (th + 1.0) * math.pi / 2.0                      # xi = cos(ang), ang in (0, pi)
    xi = np.cos(ang)
    r = np.sqrt((1 + xi) / (1 - xi))
    dr = (math.pi / 2.0) * np.sin(ang) / ((1 - xi) ** 2 * r)   # dr/dang * dang/dth
    t, wt = roots_legendre(nt)
    ph = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    R, T, P = np.meshgrid(r, t, ph, indexing="ij")
    W = (wth * dr * r * r)[:, None, None] * wt[None, :, None] * (2 * math.pi / nphi)
    W = np.broadcast_to(W, R.shape)
    st = np.sqrt(1 - T * T)
    pos = np.stack([R * st * np.cos(P), R * st * np.sin(P), R * T], axis=-1).reshape(-1, 3)
    return pos, R.ravel(), np.arccos(T).ravel(), P.ravel(), W.ravel()


def test_jnl_closed_form_and_quadrature():
    """J_00 = -3/64 (the Plummer pair); J_nl equals int rho_nl phi_nl r^2 dr."""
    from scipy.integrate import quad
    assert oracle.jnl(0, 0, CB) == pytest.approx(-3.0 / 64.0, rel=1e-14)
    for n, l in [(0, 0), (1, 0), (3, 2), (5, 1), (10, 6), (14, 8)]:
        f = lambda r: rho_nl(n, l, r) * phi_nl_scipy(n, l, r) * r * r  # noqa: E731
        val = quad(f, 0, 1, limit=200, epsabs=0)[0] + quad(f, 1, np.inf, limit=400, epsabs=0)[0]
        assert oracle.jnl(n, l, CB) == pytest.approx(val, rel=1e-9), (n, l)


@pytest.mark.parametrize("n,l", [(0, 0), (1, 0), (4, 1), (7, 3), (10, 6), (14, 8)])
def test_phi_nl_matches_scipy_and_poisson(n, l):
    """phi_nl against scipy's Gegenbauer, its derivative against finite
    differences, and phi'' + 2 phi'/r - l(l+1) phi / r^2 = 4 pi rho_nl."""
    for r in [0.03, 0.3, 1.0, 2.7, 11.0]:
        p, dp = oracle.phi_nl(n, l, r, CB)
        assert p == pytest.approx(phi_nl_scipy(n, l, r), rel=1e-12, abs=1e-300)
        h = 1e-5 * max(r, 0.1)
        fd = (oracle.phi_nl(n, l, r + h, CB)[0] - oracle.phi_nl(n, l, r - h, CB)[0]) / (2 * h)
        assert dp == pytest.approx(fd, rel=1e-7, abs=1e-12 * abs(p) + 1e-14)
        h = 1e-3 * max(r, 0.1)
        g = lambda x: oracle.phi_nl(n, l, x, CB)[1]  # noqa: E731
        d2 = (8 * (g(r + h) - g(r - h)) - (g(r + 2 * h) - g(r - 2 * h))) / (12 * h)
        lap = d2 + 2 * dp / r - l * (l + 1) * p / r ** 2
        ref = 4 * math.pi * rho_nl(n, l, r)
        scale = abs(d2) + abs(2 * dp / r) + abs(l * (l + 1) * p / r ** 2)
        assert lap == pytest.approx(ref, rel=1e-6, abs=1e-7 * scale), (r,)


@pytest.mark.parametrize("target", [(0, 0, 0), (3, 2, -1), (5, 1, 1), (10, 6, 6),
                                    (2, 6, 0), (9, 5, -5)])
def test_biorthogonality_by_quadrature(target):
    """Quadrature 'particles' whose masses sample rho_n'l' Y_l'm' (scipy) give
    c_nlm = delta_nn' delta_ll' delta_mm'."""
    n1, l1, m1 = target
    pos, R, TH, PH, W = quadrature(120, 16, 32)
    mass = W * rho_nl(n1, l1, R) * real_ylm_scipy(l1, m1, TH, PH)
    c = oracle.scf_coeffs(pos, mass, 10, 6, basis=CB)
    ref = np.zeros_like(c)
    ref[n1, l1 * l1 + l1 + m1] = 1.0
    np.testing.assert_allclose(c, ref, atol=1e-9, rtol=0)


def test_plummer_density_recovers_closed_form_potential():
    """The Plummer density is the n = l = 0 pair of this basis: quadrature
    gives c_000 Y_00 = 16/(3 pi) * (3 pi/16) = 1 and all other c = 0, and the
    field is Phi = -1/sqrt(1+r^2), a = -x/(1+r^2)^(3/2)."""
    pos, R, TH, PH, W = quadrature(120, 12, 24)
    mass = W * 3.0 / (4.0 * math.pi) * (1 + R * R) ** -2.5
    c = oracle.scf_coeffs(pos, mass, 6, 4, basis=CB)
    assert c[0, 0] / math.sqrt(4 * math.pi) == pytest.approx(1.0, rel=1e-12)
    rest = c.copy()
    rest[0, 0] = 0
    assert np.max(np.abs(rest)) < 1e-10
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(200, 3)) * rng.lognormal(0, 1.5, size=(200, 1))
    acc, pot = oracle.scf_field(pts, 6, 4, c, basis=CB)
    r2 = np.sum(pts * pts, axis=1)
    np.testing.assert_allclose(pot, -1 / np.sqrt(1 + r2), rtol=1e-10)
    np.testing.assert_allclose(acc, -pts / ((1 + r2) ** 1.5)[:, None], rtol=1e-9, atol=1e-12)


def test_plummer_particles_monopole():
    """At n_max = l_max = 0 on Plummer particles: c_000 Y_00 = (16/(3 pi)) sum_k
    m_k/sqrt(1+r_k^2) exactly, so every particle's force is the Plummer force
    times that one number; for a realisation it is 1 within a few sigma."""
    N = 16384
    pm, _ = inputs.plummer(N, seed=3)
    c = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 0, 0, basis=CB)
    r2 = np.sum(pm[:, :3] ** 2, axis=1)
    s = 16.0 / (3.0 * math.pi) * np.sum(pm[:, 3] / np.sqrt(1 + r2))
    assert c[0, 0] / math.sqrt(4 * math.pi) == pytest.approx(s, rel=1e-13)
    acc, _ = oracle.scf_field(pm[:, :3], 0, 0, c, basis=CB)
    np.testing.assert_allclose(acc, s * (-pm[:, :3] / ((1 + r2) ** 1.5)[:, None]),
                               rtol=1e-12, atol=1e-15)
    assert abs(s - 1) < 0.02


def test_bases_differ_and_origin_is_regular():
    """The two bases are different functions; at the origin the Clutton-Brock
    field is finite and its l = 0 gradient vanishes (the basis is smooth)."""
    assert oracle.phi_nl(2, 1, 0.7, CB)[0] != oracle.phi_nl(2, 1, 0.7)[0]
    rng = np.random.default_rng(5)
    c = rng.normal(size=(5, 9))
    acc, pot = oracle.scf_field(np.zeros((1, 3)), 4, 2, c, basis=CB)
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(pot))
    e = 1e-7
    acc_e, _ = oracle.scf_field(np.array([[e, 0, 0]]), 4, 2, c, basis=CB)
    np.testing.assert_allclose(acc, acc_e, rtol=1e-5, atol=1e-9)
