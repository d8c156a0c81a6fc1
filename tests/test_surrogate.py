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


@pytest.mark.parametrize("stride", [1, 3])
def test_stats_match_oracle(stride):
    traj = _traj(50, 77, 9)
    traj[:, 5] = 1.25                             # a constant coefficient: zero scales
    norm = etics.coeff_stats(torch.tensor(traj, device="cuda"), stride).cpu().numpy()
    ref = omlp.stats(traj, stride=stride)
    assert norm.shape == ref.shape == (omlp.norm_rows(stride), 77)
    np.testing.assert_allclose(norm[:7], ref[:7], rtol=1e-12, atol=1e-300)
    # the fitted predictors: the GPU's Cholesky against the oracle's LU solve
    # of the same normal equations (Gram matrices of differences are
    # ill-conditioned), then the residual RMS they imply
    for k in range(1, stride + 1):
        b = omlp._beta_row(k)
        scale = np.abs(ref[b:b + 7]).max(axis=0) + 1e-300
        assert np.all(np.abs(norm[b:b + 7] - ref[b:b + 7]) <= 1e-6 * scale), k
        np.testing.assert_allclose(norm[b + 7], ref[b + 7], rtol=1e-6)
    assert np.all(norm[1:, 5] == 0)


@pytest.mark.parametrize("per_coeff,stride", [(False, 1), (True, 1), (False, 3), (True, 3)])
def test_features_bit_exact(per_coeff, stride):
    traj = _traj(60, 131, 10)
    norm = omlp.stats(traj, stride=stride)
    rng = np.random.default_rng(11)
    last = rng.integers(7 * stride, 59 - stride, size=23)
    rows = last[:, None] + stride * np.arange(-7, 1)[None, :]
    rows[3] = rows[3][::-1]                       # any slot order is allowed
    nxt = last[:, None] + np.arange(1, stride + 1)[None, :]
    x, tg = etics.coeff_features(torch.tensor(traj, device="cuda"),
                                 torch.tensor(rows, dtype=torch.int32, device="cuda"),
                                 torch.tensor(norm, device="cuda"),
                                 torch.tensor(nxt, dtype=torch.int32, device="cuda"),
                                 per_coeff=per_coeff, stride=stride)
    xr, tr = omlp.features(traj, rows, norm, next_rows=nxt, per_coeff=per_coeff, stride=stride)
    assert np.array_equal(_bits(x).reshape(xr.shape), xr)
    assert tg.shape == tr.shape
    assert np.array_equal(tg.cpu().numpy(), tr)


@pytest.mark.parametrize("stride", [1, 3])
def test_advance_bit_exact_and_ring_order(stride):
    D = 53
    traj = _traj(40, D, 12)
    nr = omlp.stats(traj, stride=stride)
    norm = torch.tensor(nr, device="cuda")
    ring0 = traj[:8 * stride:stride]
    ring = torch.tensor(ring0, device="cuda")
    start = [3, 4, 5, 6, 7, 0, 1, 2]
    order = torch.tensor(start, dtype=torch.int32, device="cuda")
    y = np.random.default_rng(13).normal(size=(D, stride)).astype(np.float32)
    yd = torch.tensor(y, device="cuda")
    out = torch.empty(D, dtype=torch.float64, device="cuda")
    # forecasts at every horizon change nothing; y read with its stride
    for k in range(1, stride + 1):
        etics.coeff_advance(ring, order, norm, y=yd.view(-1)[k - 1:], coeffs_out=out,
                            commit=False, stride=stride, horizon=k, y_stride=stride)
        _, _, r_new = omlp.advance(ring0, start, nr, y=y[:, k - 1], stride=stride, horizon=k,
                                   commit=False)
        assert np.array_equal(out.cpu().numpy(), r_new), k
        assert np.array_equal(ring.cpu().numpy(), ring0)
        assert order.cpu().tolist() == start
    # a committed forecast, then a pushed vector
    etics.coeff_advance(ring, order, norm, y=yd.view(-1), coeffs_out=out, stride=stride,
                        horizon=1, y_stride=stride)
    r_ring, r_order, _ = omlp.advance(ring0, start, nr, y=y[:, 0], stride=stride, horizon=1)
    assert np.array_equal(ring.cpu().numpy(), r_ring) and order.cpu().tolist() == r_order
    push = torch.tensor(traj[39], device="cuda")
    etics.coeff_advance(ring, order, coeffs_in=push)
    r_ring, r_order, _ = omlp.advance(r_ring, r_order, nr, coeffs=traj[39])
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
    n_max, l_max, S = 6, 4, 3
    pm, vel = inputs.hernquist_bar(1 << 14, seed=16, eps=0.05)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    v[:, :3] = torch.tensor(vel, dtype=torch.float32)
    dt = 0.005
    traj, acc = surrogate.coefficient_trajectory(x, v, 200, dt, n_max, l_max)
    fc = surrogate.Forecaster(n_max, l_max, stride=S, hidden=64, seed=17)
    losses = fc.fit(traj[:161], iters=400, batch=16, lr=2e-3, seed=18, log_every=100)
    # the network's target is what the fitted predictors miss, normalised to
    # unit RMS; its minibatch loss stays of order 1 rather than falling
    assert all(np.isfinite(losses)) and max(losses) < 3.0
    he = fc.horizon_errors(traj, 160)
    for k in range(1, S + 1):
        med = {n: np.median(a) for n, a in he[k].items()}
        # forecasts beat holding the last vector by orders of magnitude and
        # the fitted predictor beats its cubic base; the network, trained on
        # 161 vectors of a small system, may overfit a little
        assert med["net"] < 1e-2 * med["hold"], (k, med)
        assert med["fitted"] < med["cubic"], (k, med)
        assert med["net"] <= 1.5 * med["fitted"], (k, med)
    # rollout with a recomputation every third step, judged by plain SCF.
    # The force error of any forecast grows with the particle noise of the
    # coefficients (~N^-1/2); the stated budget is met at 2^26 particles
    # (test_forecast_meets_the_stated_budget), so this 2^14 system is judged
    # at a budget 100 times looser: the forecast passes checks that plain
    # reuse fails, so it forecasts more steps, and its errors at the checks
    # are smaller
    runs = {}
    for mode in ("forecast", "hold"):
        state = (x.clone(), v.clone(), acc.clone())
        fc.reset(traj)
        runs[mode] = surrogate.run(*state, 42, dt, fc, mode=mode, tol_med=1e-3, tol_p99=1e-2)
    etics.check_error()
    st_f, st_h = runs["forecast"], runs["hold"]
    assert st_f.recomputes + st_f.forecasts == 42
    assert st_f.forecasts >= st_h.forecasts + 6, (st_f.forecasts, st_h.forecasts)
    mf = np.median([c[3] for c in st_f.checks])
    mh = np.median([c[3] for c in st_h.checks])
    assert mf < 0.5 * mh, (mf, mh)


def test_forecast_meets_the_stated_budget():
    # the experiment's system (Hernquist + 5% bar, 2^26 particles, SCF (14, 8),
    # dt = 0.005) on a shorter trajectory: with a recomputation every third
    # step the forecast meets the stated budget (median <= 1e-5, 99th
    # percentile <= 1e-4 on 4096 particles) at most checks, plain reuse at
    # almost none
    n_max, l_max, S, dt = 14, 8, 3, 0.005
    pm, vel = inputs.hernquist_bar(1 << 26, seed=0, eps=0.05)
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(x)
    v[:, :3] = torch.tensor(vel, dtype=torch.float32, device="cuda")
    del pm, vel
    traj, acc = surrogate.coefficient_trajectory(x, v, 500, dt, n_max, l_max)
    fc = surrogate.Forecaster(n_max, l_max, stride=S, hidden=256, seed=0)
    fc.fit(traj, iters=1000, batch=16, lr=1e-3, seed=0)
    runs = {}
    for mode in ("forecast", "hold"):
        state = (x.clone(), v.clone(), acc.clone())
        fc.reset(traj)
        runs[mode] = surrogate.run(*state, 60, dt, fc, mode=mode)
        del state
    etics.check_error()
    st_f, st_h = runs["forecast"], runs["hold"]
    passed_f = len(st_f.checks) - st_f.fallbacks
    passed_h = len(st_h.checks) - st_h.fallbacks
    assert len(st_f.checks) == 20
    assert passed_f >= 14, st_f.checks
    assert passed_h <= 2, st_h.checks
    assert st_f.forecasts >= 28, st_f.forecasts
