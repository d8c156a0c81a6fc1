"""GPU MEX (radix sort + scans + field through the C ABI) against the FP64
oracle (paper Sec. 2.4 eqs. 15-17 with the sort of Sec. 2.2).

The radial order is integer work and must match bit for bit; fields are
compared per particle with eq. 23's relative error."""
import numpy as np
import pytest
import torch

import oracle
from helpers import assert_field_close, device_particles, hernquist, rounded
from paper_1406_4254_gb300 import etics

pytestmark = pytest.mark.gpu


def oracle_order(pm):
    x = pm[:, :3]
    r2 = (x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2]
    return np.lexsort((np.arange(len(x)), r2))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [1, 2, 3, 4095, 4096, 4097, 12345, 100003])
def test_radial_order_is_exact(precision, n):
    pm = hernquist(n, seed=n)
    if n > 10:
        # exact ties (mirror images) and tiny-gap near ties
        pm[5, :3] = pm[3, :3] * np.array([-1.0, 1.0, -1.0])
        pm[8, :3] = pm[3, :3][[1, 0, 2]]
        pm[9, :3] = pm[3, :3] * (1 + 1e-15)
    ref_in = rounded(pm, precision)
    got = etics.radial_order(device_particles(pm, precision)).cpu().numpy()
    etics.check_error()
    ref = oracle_order(ref_in)
    assert np.array_equal(got, ref)
    _, _, o_or = oracle.mex_field(ref_in[:, :3], ref_in[:, 3], 0)
    assert np.array_equal(o_or, ref)


def near_boundary_particles(n, seed):
    """FP32 particles whose r^2 lies within a few FP64 ulps of a boundary of
    the 20-bit mantissa buckets of the sort key (and exact squares, zeros,
    tiny and huge radii)."""
    rng = np.random.default_rng(seed)
    e = rng.integers(-40, 40, n)
    m = rng.integers(1 << 20, 1 << 21, n).astype(np.float64)
    b = m * 2.0 ** (e - 20)                       # a bucket boundary
    x = np.sqrt(b).astype(np.float32)
    pm = np.zeros((n, 4), dtype=np.float32)
    pm[:, 0] = x
    k = n // 2
    pm[:k, 1] = (np.sqrt(b[:k]) * rng.uniform(1e-5, 1e-3, k)).astype(np.float32)
    pm[:k, 2] = (np.sqrt(b[:k]) * rng.uniform(1e-5, 1e-3, k)).astype(np.float32)
    pm[:10, :3] = 0.0
    pm[10:20, 0] = np.float32(1e-30)
    pm[20:25, 0] = np.float32(3e18)
    pm[25:30, 0] = np.float32(1e20)           # r^2 overflows FP32
    pm[30:40, :3] = [3.0, 4.0, 12.0]
    pm[:, 3] = 1.0
    return pm.astype(np.float64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_radial_keys_are_fp64_bits(precision):
    """The sort key equals the high word of the CPU's FP64 (x*x+y*y)+z*z."""
    for pm in (near_boundary_particles(200000, 1), hernquist(100000, seed=3)):
        ref_in = rounded(pm, precision)
        x = ref_in[:, :3]
        r2 = (x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2]
        ref = (r2.view(np.uint64) >> np.uint64(32)).astype(np.int64)
        got = etics.radial_keys(device_particles(pm, precision)).cpu().numpy()
        etics.check_error()
        bad = np.nonzero(got != ref)[0]
        assert bad.size == 0, (bad[:5], got[bad[:5]], ref[bad[:5]])


def long_tie_particles(n_shell, n_copies, n_background, seed):
    """Degenerate radial orders: a thin shell (unit vectors, r^2 within a few
    ulps of 1: every member shares one of two sort keys, so each half is one
    run of equal keys), copies of one point (identical r^2: a run ordered by
    index alone), runs of 17..300 members whose r^2 differ in the low bits
    only, inside a Hernquist background; rows shuffled."""
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(n_shell, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    parts = [np.hstack([u, np.full((n_shell, 1), 1.0 / max(n_shell, 1))])]
    parts.append(np.tile([0.3, -0.4, 0.5, 1e-3], (n_copies, 1)))
    for m in (17, 18, 33, 100, 300):
        p0 = rng.normal(size=3) * 0.7
        k = np.arange(m)[:, None]
        parts.append(np.hstack([p0[None, :] * (1.0 + k * 1e-12), np.full((m, 1), 1e-4)]))
    parts.append(hernquist(n_background, seed=seed))
    pm = np.vstack(parts)
    return pm[rng.permutation(len(pm))]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_radial_order_long_runs(precision):
    """Runs of equal sort keys of any length (two shell halves of ~20000, a
    run of 3000 identical points, runs of 17..300): the order is still the
    exact (FP64 r^2, index) order, bit for bit."""
    pm = long_tie_particles(40000, 3000, 60000, seed=31)
    got = etics.radial_order(device_particles(pm, precision)).cpu().numpy()
    etics.check_error()
    assert np.array_equal(got, oracle_order(rounded(pm, precision)))
    # every particle at the same point: one run holding all of them
    same = np.tile([0.25, 0.5, -1.0, 1.0], (5000, 1))
    got = etics.radial_order(device_particles(same, precision)).cpu().numpy()
    etics.check_error()
    assert np.array_equal(got, np.arange(5000))


def test_radial_order_full_shell():
    """2^20 particles on the unit sphere (FP32): two runs of ~2^19 equal keys,
    each ordered by one block."""
    pm = long_tie_particles(1 << 20, 0, 0, seed=32)
    got = etics.radial_order(device_particles(pm, "mixed")).cpu().numpy()
    etics.check_error()
    assert np.array_equal(got, oracle_order(rounded(pm, "mixed")))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_field_with_long_runs(precision):
    """The MEX field of the degenerate set above against the oracle (the
    shell's members are summed in the tie order, the same on both sides)."""
    pm = long_tie_particles(3000, 500, 4000, seed=33)
    ref_in = rounded(pm, precision)
    acc_ref, pot_ref, _ = oracle.mex_field(ref_in[:, :3], ref_in[:, 3], 6)
    out = etics.mex_field(device_particles(pm, precision), 6)
    etics.check_error()
    assert_field_close(out.cpu().numpy(), acc_ref, pot_ref, precision, "mex long runs")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_radial_order_near_boundaries(precision):
    pm = near_boundary_particles(50000, 2)
    got = etics.radial_order(device_particles(pm, precision)).cpu().numpy()
    etics.check_error()
    assert np.array_equal(got, oracle_order(rounded(pm, precision)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_radial_order_full_size(precision):
    n = 1 << 20
    pm = hernquist(n, seed=0)
    got = etics.radial_order(device_particles(pm, precision)).cpu().numpy()
    etics.check_error()
    assert np.array_equal(got, oracle_order(rounded(pm, precision)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("l_max", [10, 9, 8, 7, 6, 4, 2, 1, 0])
def test_field_matches_oracle(precision, l_max):
    pm = hernquist(12345, seed=11)
    ref_in = rounded(pm, precision)
    acc_ref, pot_ref, _ = oracle.mex_field(ref_in[:, :3], ref_in[:, 3], l_max)
    out = etics.mex_field(device_particles(pm, precision), l_max)
    etics.check_error()
    o = out.cpu().numpy()
    # the innermost particle has no inner mass: its force is pure noise of the
    # outer moments; compare all particles with the eq. 23 metric
    assert_field_close(o, acc_ref, pot_ref, precision, f"mex l={l_max}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_cases(precision):
    rng = np.random.default_rng(12)
    cases = [np.array([[0.3, -0.2, 0.5, 1.0]]),
             np.array([[0.0, 0.0, 0.0, 0.5], [1.0, 2.0, -1.0, 0.5]]),
             np.array([[0.0, 0.0, 2.0, 0.3], [0.0, 0.0, -0.7, 0.3], [1e-3, 0.0, 0.0, 0.4]])]
    big = hernquist(3000, seed=13)
    big[:10, :2] = 0.0                 # on the z axis
    big[10, :3] = 0.0                  # the origin
    big[11, :3] = big[12, :3] * [-1, -1, 1]   # tie
    big[100:140, 3] *= rng.uniform(0.5, 2.0, 40)
    cases.append(big)
    for pm in cases:
        for l_max in [10, 7, 6, 3, 0]:
            ref_in = rounded(pm, precision)
            acc_ref, pot_ref, _ = oracle.mex_field(ref_in[:, :3], ref_in[:, 3], l_max)
            o = etics.mex_field(device_particles(pm, precision), l_max).cpu().numpy()
            etics.check_error()
            amax = max(np.max(np.linalg.norm(acc_ref, axis=1)), 1e-300)
            tol = 1e-11 if precision == "fp64" else 2e-5
            assert np.max(np.abs(o[:, :3] - acc_ref)) <= tol * amax, (len(pm), l_max)
            pmax = max(np.max(np.abs(pot_ref)), 1e-300)
            assert np.max(np.abs(o[:, 3] - pot_ref)) <= tol * pmax, (len(pm), l_max)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sparse_radii_within_a_thread(precision):
    """Consecutive particles whose radii grow by 2x each (r^6 moments spanning
    many decades inside one thread's run and one tile): the inner sums must be
    accumulated forward, never recovered by subtraction."""
    rng = np.random.default_rng(21)
    n = 3000
    r = np.concatenate([2.0 ** np.arange(-20, 20, 1.0), rng.uniform(0.5, 2.0, n - 40)])
    v = rng.normal(size=(n, 3))
    pm = np.zeros((n, 4))
    pm[:, :3] = v / np.linalg.norm(v, axis=1)[:, None] * r[:, None]
    pm[:, 3] = rng.uniform(0.5, 1.5, n) / n
    ref_in = rounded(pm, precision)
    acc_ref, pot_ref, _ = oracle.mex_field(ref_in[:, :3], ref_in[:, 3], 6)
    o = etics.mex_field(device_particles(pm, precision), 6).cpu().numpy()
    etics.check_error()
    assert_field_close(o, acc_ref, pot_ref, precision, "sparse")


def test_output_masks_and_empty():
    pm = hernquist(5000, seed=14)
    d = device_particles(pm, "mixed")
    both = etics.mex_field(d, 6).cpu().numpy()
    pot = etics.mex_field(d, 6, out_mask=etics.OUT_POT).cpu().numpy()
    acc = etics.mex_field(d, 6, out_mask=etics.OUT_ACC).cpu().numpy()
    # the potential-only kernel is a separate instantiation: equal up to FP32 rounding
    assert np.all(pot[:, :3] == 0)
    np.testing.assert_allclose(pot[:, 3], both[:, 3], rtol=1e-6)
    assert np.all(acc[:, 3] == 0) and np.array_equal(acc[:, :3], both[:, :3])
    e = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    etics.mex_field(e, 6)
    etics.check_error()


def test_deterministic():
    d = device_particles(hernquist(50000, seed=15), "mixed")
    a = etics.mex_field(d, 6)
    b = etics.mex_field(d, 6)
    assert torch.equal(a, b)


@pytest.mark.parametrize("l_max", [6, 10])
def test_full_size_bench_config(l_max):
    """N = 2^20 flattened Hernquist (1 : 0.8 : 0.6), mixed path, every
    particle against the oracle: l_max = 6 (the benchmark) and 10 (all three
    level groups)."""
    n = 1 << 20
    pm = hernquist(n, seed=0)
    ref_in = rounded(pm, "mixed")
    acc_ref, pot_ref, _ = oracle.mex_field(ref_in[:, :3], ref_in[:, 3], l_max)
    o = etics.mex_field(device_particles(pm, "mixed"), l_max).cpu().numpy()
    etics.check_error()
    assert_field_close(o, acc_ref, pot_ref, "mixed", f"mex 2^20 l={l_max}")


def test_workspace_by_l_max():
    """The MEX workspace holds 49 components per side up to l_max = 6 and
    (l_max + 1)^2 above; l_max beyond the compiled limit has no workspace and
    the call is refused."""
    n = 100000
    sizes = [etics.workspace_bytes(n, 0, l, etics.MEX, etics.MIXED) for l in range(11)]
    assert all(s > 0 for s in sizes)
    assert len(set(sizes[:7])) == 1                     # l_max <= 6: one layout
    assert all(b > a for a, b in zip(sizes[6:], sizes[7:]))
    assert etics.workspace_bytes(n, 0, 11, etics.MEX, etics.MIXED) == 0
    d = device_particles(hernquist(1000, seed=41), "mixed")
    with pytest.raises(etics.EticsError):
        etics.mex_field(d, 11)
