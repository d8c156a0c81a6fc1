"""The coefficient-forecasting MLP on the GPU against the FP64 MLP oracle
(oracle/mlp.py): forward pass, loss and gradients (exact and with the
kernels' bf16 rounding points), Adam, the feature / update glue (bit-exact),
the force-error statistic, the given-coefficient leapfrog step, training, and
the gain of the forecast over plain coefficient reuse."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_1406_4254_gb300 import etics, inputs, surrogate

pytestmark = pytest.mark.gpu


def _bits(t: torch.Tensor) -> np.ndarray:
    return t.view(torch.int16).cpu().numpy().view(np.uint16)


def _net(dims, seed):
    net = surrogate.Mlp(dims, seed=seed)
    p64 = net.params.double().cpu().numpy()       # the FP32 master values, exactly
    return net, p64


def _data(dims, batch, seed):
    rng = np.random.default_rng(seed)
    xbits = omlp.bf16_bits(rng.normal(size=(batch, dims[0])))
    x = torch.from_numpy(xbits.view(np.int16)).cuda().view(torch.bfloat16)
    tgt = rng.normal(size=(batch, dims[-1])).astype(np.float32)
    return x, omlp.bf16_value(xbits), torch.from_numpy(tgt).cuda(), tgt.astype(np.float64)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# products with an output side below 64 run on the mma.sync kernel, the
# others on the tcgen05 kernel (128 x 128 tiles)
SHAPES = [([40, 24, 13], 5),                # one tile, ragged everything (mma.sync)
          ([96, 72, 40, 19], 37),           # several tiles, odd widths (mma.sync)
          ([512, 384, 200], 300),           # tcgen05: 3 x 3 tiles, ragged, split-K
          ([8, 256, 256, 1], 2000),         # the shared per-coefficient network
          ([1080, 256, 256, 135], 100),     # split-K in the first layer
          ([9720, 256, 256, 1215], 64)]     # the joint (14, 8) forecaster's shape


@pytest.mark.parametrize("dims,batch", SHAPES)
def test_forward_matches_oracle(dims, batch):
    net, p64 = _net(dims, seed=1)
    x, xv, _, _ = _data(dims, batch, seed=2)
    y = net.forward(x).double().cpu().numpy()
    yq, _ = omlp.forward(p64, dims, xv, quantize=True)
    y0, _ = omlp.forward(p64, dims, xv, quantize=False)
    # same rounding points: FP32 vs FP64 accumulation only (and a rare bf16 flip)
    assert _rel(y, yq) < 1e-4
    # against the all-FP64 network: bf16 operands (2^-9 relative each)
    assert _rel(y, y0) < 3e-2


@pytest.mark.parametrize("dims,batch", SHAPES)
def test_gradient_matches_oracle(dims, batch):
    net, p64 = _net(dims, seed=3)
    x, xv, tg, tv = _data(dims, batch, seed=4)
    loss = net.loss_grad(x, tg).item()
    g = net.grads.double().cpu().numpy()
    lq, gq = omlp.loss_grad(p64, dims, xv, tv, quantize=True)
    l0, g0 = omlp.loss_grad(p64, dims, xv, tv, quantize=False)
    assert abs(loss - lq) <= 1e-5 * lq
    o = 0
    for i in range(len(dims) - 1):
        nw, nb = dims[i] * dims[i + 1], dims[i + 1]
        for lo, hi in ((o, o + nw), (o + nw, o + nw + nb)):
            assert _rel(g[lo:hi], gq[lo:hi]) < 2e-3, (i, lo)
            assert _rel(g[lo:hi], g0[lo:hi]) < 5e-2, (i, lo)
        o += nw + nb


def test_adam_matches_oracle():
    dims = [96, 72, 40, 19]
    net, p64 = _net(dims, seed=5)
    x, _, tg, _ = _data(dims, 16, seed=6)
    m = np.zeros(net.n)
    v = np.zeros(net.n)
    p = p64.copy()
    for t in range(1, 4):
        net.loss_grad(x, tg)
        g = net.grads.double().cpu().numpy()
        net.adam_step(1e-2)
        p, m, v = omlp.adam(p, g, m, v, t, 1e-2)
        got = net.params.double().cpu().numpy()
        step = np.abs(p - p64).max()
        assert np.max(np.abs(got - p)) <= 1e-4 * step + 1e-6 * np.abs(p).max()
        p = got                                   # continue from the device state
        assert np.array_equal(_bits(net.params_bf16), omlp.bf16_bits(got))


def test_training_lowers_the_loss():
    dims = [64, 48, 48, 8]
    net = surrogate.Mlp(dims, seed=7)
    rng = np.random.default_rng(8)
    xv = omlp.bf16_round(rng.normal(size=(256, 64)))
    w = rng.normal(size=(64, 8)) / 8.0
    tv = np.tanh(xv @ w).astype(np.float32)      # a smooth target the net can fit
    x = torch.from_numpy(omlp.bf16_bits(xv).view(np.int16)).cuda().view(torch.bfloat16)
    tg = torch.from_numpy(tv).cuda()
    first = net.loss_grad(x, tg).item()
    for it in range(300):
        net.loss_grad(x, tg)
        net.adam_step(3e-3)
    last = net.loss_grad(x, tg).item()
    assert last < 0.05 * first


# ---- feature / update glue (bit-exact: same FP64 operations in the same order)
def _traj(T, D, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(T)[:, None]
    return (rng.normal(size=(1, D)) + rng.normal(size=(1, D)) * 0.01 * t
            + rng.normal(size=(1, D)) * 1e-4 * t * t + rng.normal(size=(T, D)) * 1e-6)


def test_stats_match_oracle():
    traj = _traj(50, 77, 9)
    traj[:, 5] = 1.25                             # a constant coefficient: zero scales
    norm = etics.coeff_stats(torch.tensor(traj, device="cuda")).cpu().numpy()
    ref = omlp.stats(traj)
    np.testing.assert_allclose(norm, ref, rtol=1e-12, atol=1e-300)
    assert np.all(norm[1:, 5] == 0)


@pytest.mark.parametrize("per_coeff", [False, True])
def test_features_bit_exact(per_coeff):
    traj = _traj(40, 131, 10)
    norm = omlp.stats(traj)
    rng = np.random.default_rng(11)
    last = rng.integers(7, 39, size=23)
    rows = last[:, None] + np.arange(-7, 1)[None, :]
    rows[3] = rows[3][::-1]                       # any slot order is allowed
    x, tg = etics.coeff_features(torch.tensor(traj, device="cuda"),
                                 torch.tensor(rows, dtype=torch.int32, device="cuda"),
                                 torch.tensor(norm, device="cuda"),
                                 torch.tensor(last + 1, dtype=torch.int32, device="cuda"),
                                 per_coeff=per_coeff)
    xr, tr = omlp.features(traj, rows, norm, next_rows=last + 1, per_coeff=per_coeff)
    assert np.array_equal(_bits(x).reshape(xr.shape), xr)
    assert np.array_equal(tg.cpu().numpy(), tr)


def test_advance_bit_exact_and_ring_order():
    D = 53
    traj = _traj(12, D, 12)
    nr = omlp.stats(traj)
    norm = torch.tensor(nr, device="cuda")
    ring = torch.tensor(traj[:8], device="cuda")
    start = [3, 4, 5, 6, 7, 0, 1, 2]
    order = torch.tensor(start, dtype=torch.int32, device="cuda")
    y = np.random.default_rng(13).normal(size=D).astype(np.float32)
    out = torch.empty(D, dtype=torch.float64, device="cuda")
    # a dry forecast changes nothing
    etics.coeff_advance(ring, order, norm, y=torch.tensor(y, device="cuda"), coeffs_out=out,
                        commit=False)
    r_ring, r_order, r_new = omlp.advance(traj[:8], start, nr, y=y)
    assert np.array_equal(out.cpu().numpy(), r_new)
    assert np.array_equal(ring.cpu().numpy(), traj[:8])
    assert order.cpu().tolist() == start
    # committed forecast, then a pushed vector
    etics.coeff_advance(ring, order, norm, y=torch.tensor(y, device="cuda"), coeffs_out=out)
    assert np.array_equal(ring.cpu().numpy(), r_ring) and order.cpu().tolist() == r_order
    push = torch.tensor(traj[9], device="cuda")
    etics.coeff_advance(ring, order, coeffs_in=push)
    r_ring, r_order, _ = omlp.advance(r_ring, r_order, nr, coeffs=traj[9])
    assert np.array_equal(ring.cpu().numpy(), r_ring) and order.cpu().tolist() == r_order


def test_force_error_statistic():
    rng = np.random.default_rng(14)
    n = 10007
    r = rng.normal(size=(n, 4))
    a = r * (1.0 + rng.normal(size=(n, 1)) * 10.0 ** rng.uniform(-8, -3, size=(n, 1)))
    r[5, :3] = 0.0                                # zero reference: infinite error
    for dt in (torch.float32, torch.float64):
        ad = torch.tensor(a, dtype=dt, device="cuda")
        rd = torch.tensor(r, dtype=dt, device="cuda")
        out = etics.force_error(ad, rd, 1e-5, 1e-4).cpu().numpy()
        av, rv = ad.double().cpu().numpy(), rd.double().cpu().numpy()
        nr = np.linalg.norm(rv[:, :3], axis=1)
        e = np.linalg.norm(av[:, :3] - rv[:, :3], axis=1) / np.where(nr > 0, nr, 1.0)
        e[nr == 0] = np.inf
        assert out[0] == np.sum(e > 1e-5) and out[1] == np.sum(e > 1e-4)
        assert np.isinf(np.array([out[2]]).view(np.float64)[0])
        e[5] = 0.0
        rd[5, :3] = torch.tensor(a[5, :3], dtype=dt)
        out = etics.force_error(ad, rd, 1e-5, 1e-4).cpu().numpy()
        assert abs(np.array([out[2]]).view(np.float64)[0] - e.max()) <= 1e-12 * e.max()


def test_leapfrog_step_coeffs_equals_plain_step():
    pm, vel = inputs.plummer(3000, seed=15)
    n_max, l_max = 6, 4
    for dt in (torch.float32, torch.float64):
        x1 = torch.tensor(pm, dtype=dt, device="cuda")
        v1 = torch.zeros_like(x1)
        v1[:, :3] = torch.tensor(vel, dtype=dt)
        a1, _ = etics.scf_force(x1, n_max, l_max)
        x2, v2, a2 = x1.clone(), v1.clone(), a1.clone()
        c = torch.empty((n_max + 1, (l_max + 1) ** 2), dtype=torch.float64, device="cuda")
        etics.leapfrog_step(x1, v1, a1, 0.01, etics.SCF, n_max, l_max, coeffs_out=c)
        etics.leapfrog_step_coeffs(x2, v2, a2, 0.01, n_max, l_max, c)
        etics.check_error()
        assert torch.equal(x1, x2) and torch.equal(v1, v2) and torch.equal(a1, a2)


# ---- end to end: the forecast's gain over plain reuse ------------------------
def test_forecast_beats_coefficient_reuse():
    n_max, l_max = 6, 4
    pm, vel = inputs.hernquist_bar(1 << 14, seed=16, eps=0.05)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    v[:, :3] = torch.tensor(vel, dtype=torch.float32)
    dt = 0.005
    traj, acc = surrogate.coefficient_trajectory(x, v, 160, dt, n_max, l_max)
    fc = surrogate.Forecaster(n_max, l_max, hidden=64, seed=17)
    losses = fc.fit(traj[:121], iters=400, batch=16, lr=2e-3, seed=18, log_every=100)
    assert losses[-1] < losses[0]
    hold, lin, cubic, net = fc.one_step_errors(traj, 120)
    assert np.median(hold) == pytest.approx(1.0)
    # the forecast beats plain reuse by orders of magnitude and the trained
    # correction does not lose against its cubic base
    assert np.median(net) < 1e-2 * np.median(hold)
    assert np.median(net) <= 1.05 * np.median(cubic)
    # rollout: 3 of 4 steps forecast, every 4th judged by plain SCF
    state = (x.clone(), v.clone(), acc.clone())
    fc.reset(traj)
    st_f = surrogate.run(*state, 40, dt, fc, period=4, tol_med=1e-3, tol_p99=1e-2)
    state = (x.clone(), v.clone(), acc.clone())
    fc.reset(traj)
    st_h = surrogate.run(*state, 40, dt, fc, period=4, tol_med=1e-3, tol_p99=1e-2, mode="hold")
    etics.check_error()
    assert st_f.recomputes + st_f.forecasts == 40
    mf = np.median([c[3] for c in st_f.checks[1:]])
    mh = np.median([c[3] for c in st_h.checks[1:]])
    assert mf < 0.5 * mh, (mf, mh)
