"""Pins of the FP64 oracle's SCF functions against mathematics that does not
come from the oracle itself (scipy's Gegenbauer polynomials and spherical
harmonics, closed-form Hernquist and Plummer potentials, exact quadrature,
rotation invariance, finite differences).

SCF is Sec. 2.4 eq. 18 of the paper with the Hernquist-Ostriker radial basis
it adopts in Sec. 2.5.
"""
import math

import numpy as np
import pytest
from scipy.special import eval_gegenbauer, roots_legendre, sph_harm_y

import oracle
from paper_1406_4254_gb300 import inputs


# ---------------------------------------------------------------------------
# independent reference pieces (scipy)
# ---------------------------------------------------------------------------

def k_nl(n, l):
    return 0.5 * n * (n + 4 * l + 3) + (l + 1) * (2 * l + 1)


def rho_nl(n, l, r):
    """Density partner of phi_nl: (K_nl/2pi) r^(l-1) (1+r)^-(2l+3) C_n^(2l+3/2)(xi)."""
    xi = (r - 1.0) / (r + 1.0)
    return k_nl(n, l) / (2 * math.pi) * r ** (l - 1) * (1 + r) ** (-(2 * l + 3)) \
        * eval_gegenbauer(n, 2 * l + 1.5, xi)


def phi_nl_scipy(n, l, r):
    xi = (r - 1.0) / (r + 1.0)
    return -r ** l * (1 + r) ** (-(2 * l + 1)) * eval_gegenbauer(n, 2 * l + 1.5, xi)


def real_ylm_scipy(l, m, theta, phi):
    """Real orthonormal Y_lm without the Condon-Shortley phase from scipy's
    complex harmonics (which include it)."""
    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    y = sph_harm_y(l, abs(m), theta, phi) * (-1) ** abs(m)
    return math.sqrt(2) * (np.real(y) if m > 0 else np.imag(y))


def quadrature(nr, nt, nphi):
    """Nodes and weights that integrate sum_k w_k f(x_k) = int f d^3x exactly
    for the polynomial-in-xi radial integrands of this basis."""
    xi, wxi = roots_legendre(nr)
    r = (1 + xi) / (1 - xi)
    dr = 2.0 / (1 - xi) ** 2
    t, wt = roots_legendre(nt)
    ph = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    R, T, P = np.meshgrid(r, t, ph, indexing="ij")
    W = (wxi * dr * r * r)[:, None, None] * wt[None, :, None] * (2 * math.pi / nphi)
    W = np.broadcast_to(W, R.shape)
    st = np.sqrt(1 - T * T)
    pos = np.stack([R * st * np.cos(P), R * st * np.sin(P), R * T], axis=-1).reshape(-1, 3)
    return pos, R.ravel(), np.arccos(T).ravel(), P.ravel(), W.ravel()


# ---------------------------------------------------------------------------

def test_jnl_closed_form_and_quadrature():
    """J_00 = -1/(12 pi); J_nl equals int rho_nl phi_nl r^2 dr (scipy quad)."""
    from scipy.integrate import quad
    assert oracle.jnl(0, 0) == pytest.approx(-1 / (12 * math.pi), rel=1e-14)
    for n, l in [(0, 0), (1, 0), (3, 2), (5, 1), (10, 6), (14, 8)]:
        f = lambda r: rho_nl(n, l, r) * phi_nl_scipy(n, l, r) * r * r
        val = quad(f, 0, 1, limit=200, epsabs=0)[0] + quad(f, 1, np.inf, limit=400, epsabs=0)[0]
        assert oracle.jnl(n, l) == pytest.approx(val, rel=1e-9), (n, l)


@pytest.mark.parametrize("n,l", [(0, 0), (1, 0), (4, 1), (7, 3), (10, 6), (14, 8)])
def test_phi_nl_matches_scipy_and_poisson(n, l):
    """phi_nl against scipy's Gegenbauer, its derivative against finite
    differences, and the radial Poisson equation
    phi'' + 2 phi'/r - l(l+1) phi / r^2 = 4 pi rho_nl (Sec. 2.5)."""
    for r in [0.03, 0.3, 1.0, 2.7, 11.0]:
        p, dp = oracle.phi_nl(n, l, r)
        assert p == pytest.approx(phi_nl_scipy(n, l, r), rel=1e-12, abs=1e-300)
        h = 1e-5 * max(r, 0.1)
        fd = (oracle.phi_nl(n, l, r + h)[0] - oracle.phi_nl(n, l, r - h)[0]) / (2 * h)
        assert dp == pytest.approx(fd, rel=1e-7, abs=1e-12 * abs(p) + 1e-14)
        h = 1e-3 * max(r, 0.1)
        g = lambda x: oracle.phi_nl(n, l, x)[1]
        d2 = (8 * (g(r + h) - g(r - h)) - (g(r + 2 * h) - g(r - 2 * h))) / (12 * h)
        lap = d2 + 2 * dp / r - l * (l + 1) * p / r ** 2
        ref = 4 * math.pi * rho_nl(n, l, r)
        scale = abs(d2) + abs(2 * dp / r) + abs(l * (l + 1) * p / r ** 2)
        assert lap == pytest.approx(ref, rel=1e-6, abs=1e-7 * scale), (r,)


def test_ylm_matches_scipy_real_harmonics():
    rng = np.random.default_rng(5)
    L = 9
    for _ in range(20):
        v = rng.normal(size=3)
        y = oracle.ylm(L, *v)
        r = np.linalg.norm(v)
        th, ph = math.acos(v[2] / r), math.atan2(v[1], v[0])
        for l in range(L + 1):
            for m in range(-l, l + 1):
                assert y[l * l + l + m] == pytest.approx(real_ylm_scipy(l, m, th, ph),
                                                         rel=1e-12, abs=1e-13)
    # poles: only m = 0 survives; Y_l0(0) = sqrt((2l+1)/4pi), Y_l0(pi) = (-1)^l of it
    for sgn in (1, -1):
        y = oracle.ylm(L, 0.0, 0.0, sgn * 2.0)
        for l in range(L + 1):
            for m in range(-l, l + 1):
                ref = math.sqrt((2 * l + 1) / (4 * math.pi)) * sgn ** l if m == 0 else 0.0
                assert y[l * l + l + m] == pytest.approx(ref, abs=1e-14)


@pytest.mark.parametrize("target", [(0, 0, 0), (3, 2, -1), (5, 1, 1), (10, 6, 6),
                                    (7, 4, -3), (2, 6, 0), (9, 5, -5)])
def test_biorthogonality_by_exact_quadrature(target):
    """Quadrature 'particles' whose masses sample rho_n'l' Y_l'm' (scipy) give
    c_nlm = delta_nn' delta_ll' delta_mm' (Sec. 2.5: coefficients are the
    projections of the density on the biorthogonal basis)."""
    n1, l1, m1 = target
    pos, R, TH, PH, W = quadrature(40, 16, 32)
    mass = W * rho_nl(n1, l1, R) * real_ylm_scipy(l1, m1, TH, PH)
    c = oracle.scf_coeffs(pos, mass, 10, 6)
    ref = np.zeros_like(c)
    ref[n1, l1 * l1 + l1 + m1] = 1.0
    # the quadrature is exact; 1e-10 covers FP64 rounding of the large, mutually
    # cancelling high-n terms (|C_10^13.5| reaches 2.5e8 at the interval ends)
    np.testing.assert_allclose(c, ref, atol=1e-10, rtol=0)


def test_hernquist_density_recovers_closed_form_potential():
    """The Hernquist density is the n=l=0 basis pair: quadrature gives
    A_000 = c_000/sqrt(4 pi) = 1 and all other c = 0, and the field is
    Phi = -1/(1+r), a = -x/(r (1+r)^2) (Hernquist 1990)."""
    pos, R, TH, PH, W = quadrature(40, 12, 24)
    mass = W / (2 * math.pi * R * (1 + R) ** 3)
    c = oracle.scf_coeffs(pos, mass, 6, 4)
    assert c[0, 0] / math.sqrt(4 * math.pi) == pytest.approx(1.0, rel=1e-13)
    rest = c.copy()
    rest[0, 0] = 0
    assert np.max(np.abs(rest)) < 1e-12
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(200, 3)) * rng.lognormal(0, 1.5, size=(200, 1))
    acc, pot = oracle.scf_field(pts, 6, 4, c)
    r = np.linalg.norm(pts, axis=1)
    np.testing.assert_allclose(pot, -1 / (1 + r), rtol=1e-12)
    np.testing.assert_allclose(acc, -pts / (r * (1 + r) ** 2)[:, None], rtol=1e-11,
                               atol=1e-13)


def test_hernquist_particles_monopole():
    """At n_max = l_max = 0, A_000 = 3 sum_k m_k/(1+r_k) exactly and, for a
    Hernquist realisation, A_000 = 1 within 3 sigma, sigma = sqrt(1/(2N))."""
    N = 16384
    pm = inputs.hernquist(N, seed=0)
    c = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 0, 0)
    a000 = c[0, 0] / math.sqrt(4 * math.pi)
    r = np.linalg.norm(pm[:, :3], axis=1)
    assert a000 == pytest.approx(3 * np.sum(pm[:, 3] / (1 + r)), rel=1e-13)
    assert abs(a000 - 1) < 3 * math.sqrt(0.5 / N)


def test_plummer_bias_decreases_with_nmax():
    """Plummer's density expanded in the Hernquist basis (Sec. 4.1: radial
    bias of SCF).  The force error against -r/(1+r^2)^(3/2) falls as n_max
    grows."""
    pos, R, TH, PH, W = quadrature(300, 4, 8)
    mass = W * 3 / (4 * math.pi) * (1 + R * R) ** -2.5
    radii = np.geomspace(0.05, 20, 40)
    pts = np.stack([radii * 0.6, radii * 0.0, radii * 0.8], axis=1)
    errs = []
    for n_max in [0, 2, 4, 8, 12, 16]:
        c = oracle.scf_coeffs(pos, mass, n_max, 0)
        acc, pot = oracle.scf_field(pts, n_max, 0, c)
        ar = -radii / (1 + radii ** 2) ** 1.5
        errs.append(np.max(np.abs(np.linalg.norm(acc, axis=1) - np.abs(ar)) / np.abs(ar)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.02


def test_rotation_invariance():
    """sum_m c_nlm^2 is invariant under a rotation of all particles, and the
    field rotates with them."""
    pm = inputs.hernquist(400, seed=3, axes=(1.0, 0.7, 0.4))
    Rm = inputs.rotation(11)
    x = pm[:, :3]
    xr = x @ Rm.T
    c1 = oracle.scf_coeffs(x, pm[:, 3], 6, 5)
    c2 = oracle.scf_coeffs(xr, pm[:, 3], 6, 5)
    for l in range(6):
        sl = slice(l * l, (l + 1) ** 2)
        p1 = np.sum(c1[:, sl] ** 2, axis=1)
        p2 = np.sum(c2[:, sl] ** 2, axis=1)
        np.testing.assert_allclose(p2, p1, rtol=1e-11, atol=1e-14 * np.max(p1))
    a1, f1 = oracle.scf_field(x, 6, 5, c1)
    a2, f2 = oracle.scf_field(xr, 6, 5, c2)
    np.testing.assert_allclose(f2, f1, rtol=1e-11)
    np.testing.assert_allclose(a2, a1 @ Rm.T, rtol=1e-9, atol=1e-11 * np.max(np.abs(a1)))


def test_gradient_is_minus_grad_potential():
    pm = inputs.hernquist(300, seed=4, axes=(1.0, 0.8, 0.6))
    c = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 8, 6)
    rng = np.random.default_rng(2)
    pts = rng.normal(size=(40, 3)) * 1.5
    pts[0] = [0.0, 0.0, 0.7]          # on the z axis
    pts[1] = [0.0, 0.0, -0.3]
    pts[2] = [1e-3, -2e-3, 5e-4]      # near the origin
    acc, _ = oracle.scf_field(pts, 8, 6, c)
    h = 1e-5 * np.minimum(1.0, np.linalg.norm(pts, axis=1) / 10)   # step below the local scale
    for d in range(3):
        e = np.zeros_like(pts)
        e[:, d] = h
        _, fp = oracle.scf_field(pts + e, 8, 6, c)
        _, fm = oracle.scf_field(pts - e, 8, 6, c)
        np.testing.assert_allclose(acc[:, d], -(fp - fm) / (2 * h), rtol=1e-6,
                                   atol=1e-7 * np.max(np.abs(acc)))


def test_origin_limit():
    """At r = 0 the potential is the l = 0 part and the acceleration the
    constant l = 1 gradient; both are the limits of the field at tiny r."""
    pm = inputs.hernquist(200, seed=6, axes=(1.0, 0.9, 0.5))
    pm[:, 0] += 0.05                  # a dipole, so the l = 1 gradient is non-zero
    c = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 5, 4)
    a0, p0 = oracle.scf_field(np.zeros((1, 3)), 5, 4, c)
    # the l = 0 radial term has a cusp; compare with the average of +x and -x limits
    eps = 1e-9
    acc_l1 = []
    for s in (1, -1):
        for d in range(3):
            pt = np.zeros((1, 3))
            pt[0, d] = s * eps
            a, p = oracle.scf_field(pt, 5, 4, c)
            assert p[0] == pytest.approx(p0[0], rel=1e-7)
            acc_l1.append(a[0])
    mean = np.mean(acc_l1, axis=0)
    np.testing.assert_allclose(a0[0], mean, rtol=1e-6, atol=1e-8)


def test_linearity_and_permutation():
    pm = inputs.hernquist(500, seed=8, axes=(1.0, 0.8, 0.6))
    c1 = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 10, 6)
    c2 = oracle.scf_coeffs(pm[:, :3], 2.5 * pm[:, 3], 10, 6)
    np.testing.assert_allclose(c2, 2.5 * c1, rtol=1e-13, atol=1e-15)
    perm = np.random.default_rng(0).permutation(len(pm))
    c3 = oracle.scf_coeffs(pm[perm, :3], pm[perm, 3], 10, 6)
    np.testing.assert_allclose(c3, c1, rtol=1e-11, atol=1e-14 * np.max(np.abs(c1)))


def test_sharded_coefficients_sum_to_full():
    """Data-parallel SCF (Sec. 3.1): partial coefficients of contiguous
    particle shards add up to those of the whole set."""
    pm = inputs.hernquist(900, seed=9)
    full = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 6, 4)
    parts = sum(oracle.scf_coeffs(pm[a:b, :3], pm[a:b, 3], 6, 4)
                for a, b in [(0, 300), (300, 620), (620, 900)])
    np.testing.assert_allclose(parts, full, rtol=1e-12, atol=1e-15)


def test_threaded_coefficients_match_exact_sum_of_particle_terms():
    """The coefficient sum runs in fixed particle chunks over threads: its
    result is bitwise the same for any thread count, and equals the exactly
    rounded sum (math.fsum) of the single-particle coefficients (Sec. 2.4
    eq. 18 is a plain sum over particles) to rounding, so no chunk boundary
    drops or repeats a particle."""
    n = 9000 + 17                           # three chunks of 4096 and a ragged tail
    pm = inputs.hernquist(n, seed=12, axes=(1.0, 0.8, 0.6))
    c1 = oracle.scf_coeffs(pm[:, :3], pm[:, 3], 4, 2, nthreads=1)
    for nt in (2, 3, 0):
        assert np.array_equal(oracle.scf_coeffs(pm[:, :3], pm[:, 3], 4, 2, nthreads=nt), c1)
    terms = np.stack([oracle.scf_coeffs(pm[k:k + 1, :3], pm[k:k + 1, 3], 4, 2, nthreads=1)
                      for k in range(n)])
    exact = np.array([[math.fsum(terms[:, i, j]) for j in range(terms.shape[2])]
                      for i in range(terms.shape[1])])
    np.testing.assert_allclose(c1, exact, rtol=1e-13, atol=1e-15 * np.max(np.abs(exact)))
