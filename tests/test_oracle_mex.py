"""Pins of the FP64 oracle's MEX, direct-summation and leapfrog functions, and
of the input samplers.

MEX is Sec. 2.4 eqs. 15-17 of the paper (with the sorted exclusive cumulative
sums of Sec. 2.2); direct summation is Sec. 2.1 eq. 4.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1406_4254_gb300 import inputs


def random_dirs(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


def test_direct_summation_matches_numpy_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(60, 3))
    m = rng.uniform(0.5, 1.5, 60)
    acc, pot = oracle.direct(x, m)
    d = x[:, None, :] - x[None, :, :]
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    np.testing.assert_allclose(pot, -np.sum(m[None, :] / r, axis=1), rtol=1e-13)
    np.testing.assert_allclose(acc, -np.sum(m[None, :, None] * d / r[:, :, None] ** 3, axis=1),
                               rtol=1e-11, atol=1e-13)


def test_mex_monopole_is_shell_theorem():
    """l_max = 0: Phi_i = -[M_in(i)/r_i + sum_out m_j/r_j] and a_i = -M_in x_i/r_i^3
    (Sec. 1: the spherical-shell method is MEX of order zero)."""
    pm = inputs.hernquist(700, seed=1, axes=(1.0, 0.8, 0.6))
    x, m = pm[:, :3], pm[:, 3] * np.random.default_rng(3).uniform(0.5, 1.5, 700)
    acc, pot, order = oracle.mex_field(x, m, 0)
    r2 = (x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2]
    srt = np.lexsort((np.arange(len(x)), r2))
    np.testing.assert_array_equal(order, srt)
    r = np.sqrt(r2)
    for k, i in enumerate(srt):
        m_in = m[srt[:k]].sum()
        outer = (m[srt[k + 1:]] / r[srt[k + 1:]]).sum()
        assert pot[i] == pytest.approx(-(m_in / r[i] + outer), rel=1e-13)
        np.testing.assert_allclose(acc[i], -m_in * x[i] / r[i] ** 3, rtol=1e-12, atol=1e-300)


def test_mex_converges_to_direct_summation_geometric_radii():
    """For radii r_j = 2^(j-16) every pair has r_</r_> <= 1/2, so the
    multipole series of 1/|x-x'| converges like 2^-l: at l_max = 40 MEX equals
    direct summation (Sec. 2.4: the MEX potential at a particle is built from the
    individual inner and outer particles, as in direct summation)."""
    rng = np.random.default_rng(7)
    n = 33
    r = 2.0 ** (np.arange(n) - 16.0)
    x = random_dirs(rng, n) * r[:, None]
    m = rng.uniform(0.5, 1.5, n)
    acc_d, pot_d = oracle.direct(x, m)
    acc_m, pot_m, _ = oracle.mex_field(x, m, 40)
    np.testing.assert_allclose(pot_m, pot_d, rtol=1e-10)
    rel = np.linalg.norm(acc_m - acc_d, axis=1) / np.linalg.norm(acc_d, axis=1)
    assert rel.max() < 1e-10, rel.max()
    errs = []
    for L in [0, 4, 8, 16, 24]:
        a, p, _ = oracle.mex_field(x, m, L)
        errs.append(np.max(np.abs(p - pot_d) / np.abs(pot_d)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_mex_error_vs_direct_falls_with_lmax_random():
    pm = inputs.hernquist(512, seed=2)
    x, m = pm[:, :3], pm[:, 3]
    acc_d, _ = oracle.direct(x, m)
    errs = []
    for L in [0, 2, 4, 8, 12, 16]:
        a, _, _ = oracle.mex_field(x, m, L)
        e = np.linalg.norm(a - acc_d, axis=1) / np.linalg.norm(acc_d, axis=1)
        errs.append(np.median(e))
    assert all(b <= a * 1.05 for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.6 * errs[0], errs


def test_mex_gradient_is_minus_grad_of_own_potential():
    """Moving particle i does not change q(i), p(i) (they exclude i), so a_i is
    minus the gradient of Phi_i in its own position while the order is kept."""
    pm = inputs.hernquist(300, seed=5, axes=(1.0, 0.8, 0.6))
    x, m = pm[:, :3].copy(), pm[:, 3]
    acc, pot, order = oracle.mex_field(x, m, 6)
    r = np.linalg.norm(x, axis=1)
    rs = np.sort(r)
    for i in np.random.default_rng(1).choice(len(x), 25, replace=False):
        gap = np.min(np.abs(rs[rs != r[i]] - r[i]))
        h = min(1e-6 * r[i], 0.1 * gap)
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            _, pp, op = oracle.mex_field(xp, m, 6)
            _, pmm, om = oracle.mex_field(xm, m, 6)
            assert np.array_equal(op, order) and np.array_equal(om, order)
            fd = -(pp[i] - pmm[i]) / (2 * h)
            assert acc[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.linalg.norm(acc[i]))


def test_mex_rotation_and_permutation_invariance():
    pm = inputs.hernquist(400, seed=4, axes=(1.0, 0.7, 0.5))
    x, m = pm[:, :3], pm[:, 3]
    acc, pot, order = oracle.mex_field(x, m, 6)
    R = inputs.rotation(3)
    acc_r, pot_r, order_r = oracle.mex_field(x @ R.T, m, 6)
    assert np.array_equal(order, order_r)
    np.testing.assert_allclose(pot_r, pot, rtol=1e-11)
    np.testing.assert_allclose(acc_r, acc @ R.T, rtol=1e-9, atol=1e-11 * np.abs(acc).max())
    perm = np.random.default_rng(2).permutation(len(x))
    acc_p, pot_p, _ = oracle.mex_field(x[perm], m[perm], 6)
    np.testing.assert_allclose(pot_p, pot[perm], rtol=1e-12)
    np.testing.assert_allclose(acc_p, acc[perm], rtol=1e-11, atol=1e-13 * np.abs(acc).max())
    acc_s, pot_s, _ = oracle.mex_field(x, 3.0 * m, 6)
    np.testing.assert_allclose(pot_s, 3.0 * pot, rtol=1e-13)


def test_mex_origin_particle_and_ties():
    """A particle at the origin sorts first and feels only the outer l <= 1
    field; equal radii are ordered by index."""
    rng = np.random.default_rng(9)
    x = random_dirs(rng, 40) * rng.uniform(0.5, 2.0, (40, 1))
    x[0] = 0.0
    x[5] = x[7] * np.array([-1, 1, 1])      # same radius as particle 7
    m = rng.uniform(0.5, 1.5, 40)
    acc, pot, order = oracle.mex_field(x, m, 5)
    assert order[0] == 0
    assert list(order).index(5) < list(order).index(7)
    r = np.linalg.norm(x, axis=1)
    # potential at the origin = -sum_{j>0} m_j / r_j (l = 0 term)
    assert pot[0] == pytest.approx(-np.sum(m[1:] / r[1:]), rel=1e-13)
    # dipole term: a = sum_j m_j x_j / r_j^3 (the l = 1 part of direct summation)
    np.testing.assert_allclose(acc[0], np.sum(m[1:, None] * x[1:] / r[1:, None] ** 3, axis=0),
                               rtol=1e-12)
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(pot))


def test_leapfrog_kdk_and_energy():
    """One KDK step equals its definition; a Plummer sphere integrated with
    SCF conserves energy to the expected leapfrog order."""
    pm, vel = inputs.plummer(2000, seed=0)
    x, m = pm[:, :3].copy(), pm[:, 3]
    v = vel.copy()
    c = oracle.scf_coeffs(x, m, 6, 2)
    a0, p0 = oracle.scf_field(x, 6, 2, c)
    acc = a0.copy()
    x1, v1 = x.copy(), v.copy()
    pot, c1 = oracle.leapfrog_step(x1, v1, m, acc, 0.01, 0, 6, 2)
    vh = v + 0.005 * a0
    xe = x + 0.01 * vh
    np.testing.assert_allclose(x1, xe, rtol=1e-15, atol=1e-15)
    ce = oracle.scf_coeffs(xe, m, 6, 2)
    np.testing.assert_allclose(c1, ce, rtol=1e-14, atol=1e-15)
    ae, pe = oracle.scf_field(xe, 6, 2, ce)
    np.testing.assert_allclose(acc, ae, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(v1, vh + 0.005 * ae, rtol=1e-15, atol=1e-16)

    def energy(x, v, pot):
        return 0.5 * np.sum(m * np.sum(v * v, axis=1)) + 0.5 * np.sum(m * pot)

    xs, vs, acs = x.copy(), v.copy(), a0.copy()
    e0 = energy(xs, vs, p0)
    for _ in range(20):
        pot, _ = oracle.leapfrog_step(xs, vs, m, acs, 0.02, 0, 6, 2)
    assert abs(energy(xs, vs, pot) / e0 - 1) < 1e-3


def test_hernquist_sampler_cumulative_mass():
    """Radii follow M(<r) = r^2/(1+r)^2 (Kolmogorov-Smirnov at 99.9%)."""
    pm = inputs.hernquist(20000, seed=0)
    r = np.sort(np.linalg.norm(pm[:, :3], axis=1))
    cdf = r * r / (1 + r) ** 2
    ks = np.max(np.abs(cdf - (np.arange(1, len(r) + 1) - 0.5) / len(r)))
    assert ks < 1.95 / math.sqrt(len(r))
    assert np.all(pm[:, 3] == 1.0 / len(pm))
    st = inputs.hernquist(1000, seed=0, axes=(1.0, 0.8, 0.6))
    sp = inputs.hernquist(1000, seed=0)
    np.testing.assert_allclose(st[:, :3], sp[:, :3] * [1.0, 0.8, 0.6])


def test_plummer_sampler_virial():
    """Plummer (b = 1): W = -3 pi/32, K = 3 pi/64, so 2K/|W| = 1."""
    n = 40000
    pm, vel = inputs.plummer(n, seed=1)
    r = np.linalg.norm(pm[:, :3], axis=1)
    K = 0.5 * np.sum(pm[:, 3] * np.sum(vel * vel, axis=1))
    W = 0.5 * np.sum(pm[:, 3] * (-1.0 / np.sqrt(1 + r * r)))
    assert K == pytest.approx(3 * math.pi / 64, rel=0.03)
    assert W == pytest.approx(-3 * math.pi / 32, rel=0.03)
    assert 2 * K / abs(W) == pytest.approx(1.0, abs=0.04)


def test_bar_sampler_quadrupole():
    """The angular density 1 + eps sin^2(t) cos(2p) gives <x^2 - y^2>/<r^2> =
    (4/15) eps / (1/1) ... checked against its exact mean 4 eps/15."""
    pm, vel = inputs.hernquist_bar(60000, seed=2, eps=0.3, velocities=False)
    u = pm[:, :3] / np.linalg.norm(pm[:, :3], axis=1)[:, None]
    q = np.mean(u[:, 0] ** 2 - u[:, 1] ** 2)
    assert q == pytest.approx(4 * 0.3 / 15, abs=4 * math.sqrt(0.2 / 60000))


def test_mex_threaded_blocks_match_serial_and_shell_theorem():
    """The oracle's MEX takes the sorted list in blocks of 65536 with the
    per-particle work over threads: for several blocks and a ragged tail the
    result is bitwise the same for any thread count, and at l_max = 0 it
    equals the shell theorem counted independently here (numpy sort and
    cumulative sums), so the running sums cross block boundaries intact."""
    n = 2 * 65536 + 1001
    pm = inputs.hernquist(n, seed=21)
    pm[7, :3] = 0.0                        # a particle at the origin
    x, m = pm[:, :3], pm[:, 3]
    a1, p1, o1 = oracle.mex_field(x, m, 3, nthreads=1)
    a4, p4, o4 = oracle.mex_field(x, m, 3, nthreads=4)
    assert np.array_equal(a1, a4) and np.array_equal(p1, p4) and np.array_equal(o1, o4)
    a0, p0, order = oracle.mex_field(x, m, 0)
    r2 = (x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2]
    assert np.array_equal(order, np.lexsort((np.arange(n), r2)))
    r = np.sqrt(r2[order])
    ms = m[order]
    inner = np.concatenate([[0.0], np.cumsum(ms)[:-1]])           # mass strictly inside
    w = np.where(r > 0, ms / np.where(r > 0, r, 1.0), 0.0)
    outer = np.concatenate([np.cumsum(w[::-1])[::-1][1:], [0.0]])  # sum over j outside
    pot = -(np.where(r > 0, inner / np.where(r > 0, r, 1.0), 0.0) + outer)
    np.testing.assert_allclose(p0[order], pot, rtol=1e-11, atol=0)
